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
