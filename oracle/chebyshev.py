"""Chebyshev grid and interpolant in z (oracle).

Sec. 5.2.2 (opening paragraph): one second-kind Chebyshev grid on
z in [a, b] = [-3 H_E, H + 3 H_E]. With Hbar = b - a and the scaled variable
s = 2 (z - a)/Hbar - 1 in [-1, 1] (Appendix A maps [0, H] to [-1, 1] the same
way), the nodes are the extrema s_j = cos(pi j/(N-1)), j = 0..N-1, so z_0 = b
and z_{N-1} = a.

A column of N values is represented by its interpolating polynomial
f(s) = sum_{n<N} fhat_n T_n(s), Eq. (chebexp), with no factor 1/2 on fhat_0
(Appendix A, remark after Eq. (cs)). The oracle obtains fhat by solving the
interpolation conditions directly (the definition), not by a fast transform.
"""
import numpy as np


def scaled(z, a, b):
    """s = 2 (z - a)/(b - a) - 1."""
    return 2.0 * (np.asarray(z, dtype=np.float64) - a) / (b - a) - 1.0


def nodes(nz, a, b):
    """z_j = a + (Hbar/2)(1 + cos(pi j/(N-1))), j = 0..N-1 (descending)."""
    j = np.arange(nz, dtype=np.float64)
    return a + 0.5 * (b - a) * (1.0 + np.cos(np.pi * j / (nz - 1)))


def cheb_T(n_terms, s):
    """Matrix T[i, n] = T_n(s_i) = cos(n arccos s_i), |s_i| <= 1."""
    s = np.clip(np.atleast_1d(np.asarray(s, dtype=np.float64)), -1.0, 1.0)
    n = np.arange(n_terms, dtype=np.float64)
    return np.cos(np.outer(np.arccos(s), n))


def values_to_coeffs(values, nz):
    """Coefficients of the interpolant through the node values (axis 0 = nodes)."""
    s = np.cos(np.pi * np.arange(nz) / (nz - 1))
    V = cheb_T(nz, s)
    return np.linalg.solve(V, values)


def coeffs_to_values(coeffs, nz):
    """Values at the nodes of sum_n coeffs_n T_n (axis 0 = coefficients)."""
    s = np.cos(np.pi * np.arange(nz) / (nz - 1))
    return cheb_T(coeffs.shape[0], s) @ coeffs


def evaluate(coeffs, s):
    """sum_n coeffs_n T_n(s) at arbitrary points s (axis 0 = coefficients)."""
    return cheb_T(coeffs.shape[0], s) @ coeffs


def quadrature_weights(nz, a, b):
    """Weights w_j with sum_j w_j f(z_j) = integral over [a, b] of the
    interpolant of f, i.e. w = V^{-T} m (Hbar/2), m_n = int_{-1}^{1} T_n ds
    = 2/(1 - n^2) for even n and 0 for odd n. These are the Clenshaw-Curtis
    weights on the extrema grid."""
    n = np.arange(nz, dtype=np.float64)
    m = np.zeros(nz)
    even = (np.arange(nz) % 2) == 0
    m[even] = 2.0 / (1.0 - n[even] ** 2)
    s = np.cos(np.pi * np.arange(nz) / (nz - 1))
    V = cheb_T(nz, s)
    return np.linalg.solve(V.T, m) * (0.5 * (b - a))
