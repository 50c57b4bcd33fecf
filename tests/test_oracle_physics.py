"""The full oracle solve pinned to method-independent truth (CPU).

Reference: direct Fourier sums over the periodic lattice and the complete
dielectric image series (oracle.brute), no grid and no splitting. The oracle
is run with a wider Gaussian truncation (n_sigma = 7, Sec. 5.1 notes that
accuracy is then limited only by roundoff) on a grid that resolves the
charges, so it must agree to ~1e-7 or better; a dropped term, a wrong sign or
a swapped wall in any step shows up far above that."""
import numpy as np
import pytest

from oracle import brute, params, solver

L, H, GW = 24.0, 24.0, 1.0


def _charges(n=6, seed=0, zlo=1.0):
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.uniform(0, L, n), rng.uniform(0, L, n), rng.uniform(zlo, H - zlo, n)], 1)
    q = np.array([1.0, -1.0] * (n // 2))
    return pos, q


def _params(eb, et, xi, rcut, nz=0, nx=48):
    return params.derive(L, L, H, GW, 1e-4, nx, nx, nz=nz, xi=xi, r_cut=rcut,
                         eps_b=eb, eps_t=et, n_sigma=7.0)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


CASES = [
    ("uniform", 1.0, 1.0, np.inf, 0.0, 1e-7),
    ("uniform-split", 1.0, 1.0, 1.2, 10.0, 1e-7),
    ("jumps", 1 / 80, 1 / 80, np.inf, 0.0, 3e-7),
    ("jumps-split", 1 / 80, 1 / 80, 1.2, 10.0, 3e-7),
    ("unequal-split", 0.5, 5.0, 1.2, 10.0, 3e-7),
    ("metal-bottom-split", np.inf, 1 / 80, 1.2, 10.0, 3e-7),
    ("metal-top", 1 / 80, np.inf, np.inf, 0.0, 3e-7),
]


@pytest.fixture(scope="module")
def charges():
    return _charges()


@pytest.mark.parametrize("name,eb,et,xi,rcut,tol", CASES, ids=[c[0] for c in CASES])
def test_against_image_series(charges, name, eb, et, xi, rcut, tol):
    pos, q = charges
    ref = brute.solve(pos, q, L, L, H, GW, 1.0, eb, et)
    out = solver.solve(pos, q, _params(eb, et, xi, rcut))
    assert _rel(out["force"], ref["force"]) < tol
    assert out["U"] == pytest.approx(ref["U"], rel=tol)
    dphi = (out["phi"] - out["phi"].mean()) - (ref["phi"] - ref["phi"].mean())
    assert np.max(np.abs(dphi)) < tol * np.max(np.abs(ref["phi"]))


def test_convergence_in_nz(charges):
    """Spectral convergence of the force error under N_z refinement."""
    pos, q = charges
    ref = brute.solve(pos, q, L, L, H, GW, 1.0, 1 / 80, 1 / 80)
    errs = [_rel(solver.solve(pos, q, _params(1 / 80, 1 / 80, np.inf, 0.0, nz=nz))["force"], ref["force"])
            for nz in (60, 100, 140, 180)]
    assert all(e2 < e1 / 5 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-8


def test_mirror_symmetry():
    """z -> H - z with eps_b <-> eps_t: F_z flips, F_x, F_y and U unchanged.
    The grid is symmetric about H/2, so this holds to roundoff."""
    pos, q = _charges(8, seed=3)
    P1 = params.derive(L, L, H, GW, 1e-4, 48, 48, nz=80, r_cut=4.0, eps_b=0.05, eps_t=0.4)
    P2 = params.derive(L, L, H, GW, 1e-4, 48, 48, nz=80, r_cut=4.0, eps_b=0.4, eps_t=0.05)
    a = solver.solve(pos, q, P1)
    mpos = pos.copy()
    mpos[:, 2] = H - pos[:, 2]
    b = solver.solve(mpos, q, P2)
    s = np.max(np.abs(a["force"]))
    assert np.max(np.abs(a["force"][:, :2] - b["force"][:, :2])) < 1e-11 * s
    assert np.max(np.abs(a["force"][:, 2] + b["force"][:, 2])) < 1e-11 * s
    # U only to the truncation level: the k = 0 linear mode A_i z is anchored
    # at z = 0, the mirrored solve anchors it at the other wall, and the
    # truncated-Gaussian quadrature of a constant is 1 only to ~e^{-n_sigma^2/2}
    assert a["U"] == pytest.approx(b["U"], rel=1e-6)


def test_metal_bottom_matches_huge_permittivity():
    """eps_b = inf follows from eps_b -> inf of every formula except A_i, where a
    metal wall drops its own displacement equation (Eq. (ai1)); that changes
    A_i only by the discrete mismatch of Eq. (ai1) and (ai2)."""
    pos, q = _charges(6, seed=5)
    Pm = _params(np.inf, 1 / 80, 1.2, 10.0)
    Pb = _params(1e12, 1 / 80, 1.2, 10.0)
    a, b = solver.solve(pos, q, Pm), solver.solve(pos, q, Pb)
    assert _rel(a["force"], b["force"]) < 1e-7


def test_translation_invariance_and_zero_net_lateral_force():
    pos, q = _charges(8, seed=11)
    P = _params(1 / 80, 0.3, 1.2, 10.0)
    a = solver.solve(pos, q, P)
    sh = pos.copy()
    sh[:, 0] += 0.37
    sh[:, 1] += 5.11
    b = solver.solve(sh, q, P)
    assert _rel(b["force"], a["force"]) < 1e-7
    assert b["U"] == pytest.approx(a["U"], rel=1e-8)
    s = np.sum(np.abs(a["force"][:, :2]))
    assert abs(np.sum(a["force"][:, 0])) < 1e-7 * s
    assert abs(np.sum(a["force"][:, 1])) < 1e-7 * s


def test_force_is_minus_energy_gradient():
    """Rate-of-work check of Sec. 6.3 (Eq. (w1), (w2)) at high accuracy."""
    pos, q = _charges(6, seed=2, zlo=2.0)
    P = _params(1 / 20, 1 / 50, 1.2, 10.0)
    rng = np.random.default_rng(4)
    dX = rng.standard_normal(pos.shape)
    dX /= np.linalg.norm(dX, axis=1, keepdims=True)
    d0 = 1e-4
    Up = solver.solve(pos + 0.5 * d0 * dX, q, P)["U"]
    Um = solver.solve(pos - 0.5 * d0 * dX, q, P)["U"]
    W1 = -(Up - Um) / d0
    W2 = float(np.sum(solver.solve(pos, q, P)["force"] * dX))
    assert abs(W1 - W2) < 1e-6 * abs(W2)


def test_uniform_permittivity_needs_no_correction():
    """With eps_b = eps_t = eps the images vanish and the harmonic correction
    of Sec. 4.3.3 is zero up to discretisation: the mismatch of psi_i* and
    psi_o* at a wall is the potential of the far charges C_nover, which
    already decays like e^{k z} below them. Charges are put mid-slab (in
    C_nover) of a taller slab so the mismatches are not trivially zero."""
    Ht = 40.0
    rng = np.random.default_rng(9)
    n = 6
    pos = np.stack([rng.uniform(0, L, n), rng.uniform(0, L, n), rng.uniform(16.0, 24.0, n)], 1)
    q = np.array([1.0, -1.0] * 3)

    def run(eb, et):
        P = params.derive(L, L, Ht, GW, 1e-4, 48, 48, nz=220, xi=np.inf, eps_b=eb, eps_t=et,
                          n_sigma=7.0)
        out = solver.solve(pos, q, P)
        nz0 = np.abs(out["psi0"]) > 0
        nz0[0] = False                         # k = 0 has no correction
        return np.max(np.abs(out["corr0"])), np.max(np.abs(out["psi0"][nz0]))
    c_u, p_u = run(1.0, 1.0)
    c_j, p_j = run(1 / 80, 1 / 80)
    assert c_u < 1e-6 * p_u
    assert c_j > 0.5 * p_j


def test_near_field_tree_matches_pairs():
    pos, q = _charges(40, seed=13)
    P = params.derive(L, L, H, GW, 1e-4, 48, 48, nz=64, r_cut=4.0, eps_b=0.1, eps_t=np.inf)
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    a = solver.near_field(x, y, z, q, P, "pairs")
    b = solver.near_field(x, y, z, q, P, "tree")
    assert np.allclose(a[0], b[0], rtol=1e-13, atol=1e-16)
    assert np.allclose(a[1], b[1], rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("name,eb,et,xi,rcut,tol", CASES, ids=[c[0] for c in CASES])
def test_gauge_against_pointwise_image_series(charges, name, eb, et, xi, rcut, tol):
    """The gauge phi(0) = 0 (Eq. (phi00); the gauge paragraph of Sec. 5.2.2)
    without mean subtraction: the oracle's phibar_k must be the brute-force
    averaged potential minus the brute-force pointwise potential of the
    Gaussian charges and their image series at the origin. This fixes
    B = -(phi^(n)(0) + phi^(f)(0)): the pointwise kernel Eq. (Gnear) at the
    origin, the gamma^{1/2} average of the far series there (xy factor and z
    weights), and the sign of B."""
    pos, q = charges
    ref = brute.solve(pos, q, L, L, H, GW, 1.0, eb, et)
    phi0 = brute.pointwise_potential([[0.0, 0.0, 0.0]], pos, q, L, L, H, GW, 1.0, eb, et)[0]
    out = solver.solve(pos, q, _params(eb, et, xi, rcut))
    scale = np.max(np.abs(ref["phi"]))
    assert np.max(np.abs(out["phi"] - (ref["phi"] - phi0))) < tol * scale
    if np.isinf(eb):
        # a metal bottom is grounded by its images: phi = 0 on all of it
        assert abs(phi0) < tol * scale
    else:
        # the constant is not trivially small: a solve without the gauge fails
        assert abs(phi0) > 100 * tol * scale


def test_gauge_at_another_point():
    """The same identity with the origin of the box moved: shifting every charge
    by -c in x and y and wrapping puts the point c at the origin, so the
    shifted solve's phibar_k equals the brute-force phibar_k minus phi(c).
    Exercises the far-field gauge sum at nonzero phases of every mode."""
    pos, q = _charges(6, seed=7)
    c = np.array([7.3, 15.9])
    sh = pos.copy()
    sh[:, :2] = np.mod(pos[:, :2] - c, L)
    eb, et = 1 / 80, 0.5
    ref = brute.solve(pos, q, L, L, H, GW, 1.0, eb, et)
    phic = brute.pointwise_potential([[c[0], c[1], 0.0]], pos, q, L, L, H, GW, 1.0, eb, et)[0]
    out = solver.solve(sh, q, _params(eb, et, 1.2, 10.0))
    assert np.max(np.abs(out["phi"] - (ref["phi"] - phic))) < 3e-7 * np.max(np.abs(ref["phi"]))


@pytest.mark.parametrize("xi,nz", [(1.2, 60), (0.6, 90), (3.0, 41)])
def test_gauge_weights_by_quadrature(xi, nz):
    """gauge_weights: w_n = int G_sigma(z) T_n(s(z)) dz with sigma = 1/(2 xi)
    (the z part of gamma^{1/2}, Eq. (gt)), against adaptive quadrature of the
    same integral, with T_n(s) = cos(n arccos s) inside [-1, 1] and
    cosh(n arccosh |s|) sgn(s)^n outside."""
    from scipy.integrate import quad
    P = params.derive(L, L, H, GW, 1e-4, 48, 48, nz=nz, xi=xi, r_cut=10.0,
                      eps_b=1 / 80, eps_t=1 / 80, n_sigma=7.0)
    w = solver.gauge_weights(P)
    sigma = 1.0 / (2.0 * xi)
    a, b = P["a"], P["b"]

    def T(n, s):
        if abs(s) <= 1.0:
            return np.cos(n * np.arccos(s))
        return np.cosh(n * np.arccosh(abs(s))) * (np.sign(s) ** n)

    for n in (0, 1, 2, 5, nz // 2, nz - 1):
        f = lambda z: np.exp(-z * z / (2 * sigma * sigma)) / np.sqrt(2 * np.pi * sigma * sigma) \
            * T(n, 2.0 * (z - a) / (b - a) - 1.0)
        ref, _ = quad(f, -12 * sigma, 12 * sigma, epsabs=1e-14, epsrel=1e-12, limit=200)
        assert abs(w[n] - ref) < 1e-11 * max(1.0, abs(ref))
    # without smearing (xi = inf) the weights are T_n at the origin
    P2 = params.derive(L, L, H, GW, 1e-4, 48, 48, nz=nz, xi=np.inf, eps_b=1 / 80, eps_t=1 / 80)
    s0 = 2.0 * (0.0 - P2["a"]) / (P2["b"] - P2["a"]) - 1.0
    assert np.allclose(solver.gauge_weights(P2), np.cos(np.arange(nz) * np.arccos(s0)), atol=1e-14)
