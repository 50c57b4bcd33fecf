"""Chebyshev spectral-integration boundary value solver (oracle), Appendix A.

Per transverse mode k = |k_par| the far-field potential solves Eq. (BVP) on
[a, b]:  eps (psi'' - k^2 psi) = -f,  psi' - k psi = 0 at a,  psi' + k psi = 0
at b (the Dirichlet-to-Neumann conditions Eq. (BCs1)). In the scaled variable
s = 2 (z - a)/Hbar - 1 this reads (Eq. (BVPH), (BVPBCH) with the overall
factors written out)

    y_ss - K^2 y = F,          K = k Hbar / 2,  F = -(Hbar/2)^2 f / eps,
    y_s + K y = 0 at s = 1,    y_s - K y = 0 at s = -1.

The unknowns are the Chebyshev coefficients of y'' (n = 0..N-1) and the two
integration constants y_0, y'_0. The coefficients of y' and y follow from
the indefinite integrals of T_n, Eq. (ds) and Eq. (cs):

    y'_1 = y''_0 - y''_2 / 2,    y'_n = (y''_{n-1} - y''_{n+1}) / (2n), n >= 2,
    y_1  = y'_0  - y'_2  / 2,    y_n  = (y'_{n-1}  - y'_{n+1})  / (2n), n >= 2,

with y''_n = y'_n = 0 for n > N-1 (the truncation stated after Eq. (cs)).
Matching modes gives Eq. (modes) y''_n - K^2 y_n = F_n and the two boundary
rows Eq. (BCs). For k = 0 the rows become y''_n = F_n with the homogeneous
Dirichlet rows Eq. (BCs0) (Sec. 5.2.2 steps 2-3 use them for the k = 0 mode).

The oracle assembles the full (N+2) x (N+2) system Eq. (blocksys) and solves
it with a dense LU; it does not use the banded/Schur structure the paper
uses for speed.
"""
import numpy as np


def integration_matrix(n):
    """J with (coefficients of the integral) = J @ (coefficients), the
    integration constant excluded: rows follow Eq. (ds)/(cs)."""
    J = np.zeros((n, n))
    if n > 1:
        J[1, 0] = 1.0
        if n > 2:
            J[1, 2] = -0.5
    for m in range(2, n):
        J[m, m - 1] = 1.0 / (2.0 * m)
        if m + 1 < n:
            J[m, m + 1] = -1.0 / (2.0 * m)
    return J


def system_matrix(K, n):
    """Eq. (blocksys): unknown vector (y''_0..y''_{N-1}, y_0, y'_0)."""
    J = integration_matrix(n)
    J2 = J @ J
    e0 = np.zeros(n)
    e0[0] = 1.0
    Je0 = J @ e0                     # y_1 picks up y'_0 with coefficient 1
    ones = np.ones(n)
    alt = (-1.0) ** np.arange(n)
    M = np.zeros((n + 2, n + 2))
    if K == 0.0:
        M[:n, :n] = np.eye(n)
        # Eq. (BCs0): sum y_n = 0, sum (-1)^n y_n = 0
        M[n, :n] = ones @ J2
        M[n, n] = ones @ e0
        M[n, n + 1] = ones @ Je0
        M[n + 1, :n] = alt @ J2
        M[n + 1, n] = alt @ e0
        M[n + 1, n + 1] = alt @ Je0
        return M
    # Eq. (modes): y''_n - K^2 y_n = F_n, y = J^2 y'' + y_0 e0 + y'_0 J e0
    M[:n, :n] = np.eye(n) - K * K * J2
    M[:n, n] = -K * K * e0
    M[:n, n + 1] = -K * K * Je0
    # Eq. (BCs) at s = 1: sum (y'_n + K y_n) = 0, y' = J y'' + y'_0 e0
    M[n, :n] = ones @ (J + K * J2)
    M[n, n] = K * (ones @ e0)
    M[n, n + 1] = ones @ e0 + K * (ones @ Je0)
    # Eq. (BCs) at s = -1: sum (-1)^n (y'_n - K y_n) = 0
    M[n + 1, :n] = alt @ (J - K * J2)
    M[n + 1, n] = -K * (alt @ e0)
    M[n + 1, n + 1] = alt @ e0 - K * (alt @ Je0)
    return M


def solve(K, F):
    """Solve for all columns of F (shape (N, m)) sharing the scaled wavenumber
    K. Returns (y, yp): coefficients of y and of y' = dy/ds, each (N, m)."""
    n = F.shape[0]
    M = system_matrix(K, n)
    rhs = np.zeros((n + 2,) + F.shape[1:], dtype=np.result_type(F, np.float64))
    rhs[:n] = F
    sol = np.linalg.solve(M, rhs)
    ypp, y0, yp0 = sol[:n], sol[n], sol[n + 1]
    J = integration_matrix(n)
    yp = J @ ypp
    yp[0] = yp0
    y = J @ yp
    y[0] = y0
    return y, yp
