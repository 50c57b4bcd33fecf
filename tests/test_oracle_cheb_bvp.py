"""Oracle building blocks pinned to closed forms (CPU): Chebyshev interpolant,
quadrature, the Appendix-A BVP solver and the harmonic correction."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from scipy.special import erf, erfc

from oracle import bvp, chebyshev as cheb
from oracle.correction import correction, wall_factors, zero_mode_slope


def test_interpolant_recovers_polynomial():
    rng = np.random.default_rng(1)
    for nz in (5, 17, 64, 129):
        c = rng.standard_normal(nz)
        s = np.cos(np.pi * np.arange(nz) / (nz - 1))
        vals = npcheb.chebval(s, c)              # library evaluation
        assert np.allclose(cheb.values_to_coeffs(vals, nz), c, atol=1e-12 * nz)
        assert np.allclose(cheb.coeffs_to_values(c, nz), vals, atol=1e-12 * nz)


def test_nodes_are_extrema_grid():
    z = cheb.nodes(9, -2.0, 6.0)
    assert z[0] == pytest.approx(6.0) and z[-1] == pytest.approx(-2.0)
    assert np.all(np.diff(z) < 0)
    assert z[4] == pytest.approx(2.0)


def test_quadrature_integrates_polynomials():
    a, b = -1.5, 4.0
    for nz in (8, 33, 64):
        z = cheb.nodes(nz, a, b)
        w = cheb.quadrature_weights(nz, a, b)
        for m in range(nz):
            exact = (b ** (m + 1) - a ** (m + 1)) / (m + 1)
            assert np.dot(w, z ** m) == pytest.approx(exact, rel=1e-11, abs=1e-11)


def _gauss_mode_solution(z, z0, sig, k, eps):
    """(1/(2 eps k)) int e^{-k|z-z'|} G(z'-z0) dz' and its z-derivative (closed
    form with erfc; G the normalised Gaussian of std sig)."""
    d = z - z0
    c = np.exp(0.5 * k * k * sig * sig) / 2.0
    lo = np.exp(-k * d) * erfc((k * sig * sig - d) / (sig * np.sqrt(2)))
    hi = np.exp(k * d) * erfc((k * sig * sig + d) / (sig * np.sqrt(2)))
    return c * (lo + hi) / (2 * eps * k), c * k * (hi - lo) / (2 * eps * k)


@pytest.mark.parametrize("k", [0.2, 1.0, 4.0, 20.0])
def test_bvp_matches_free_space_mode(k):
    """A Gaussian source well inside [a, b]: the DtN problem's exact solution is
    the free-space mode solution, which satisfies both Robin conditions."""
    a, b, z0, sig, eps, nz = -6.0, 7.0, 0.4, 0.6, 2.0, 96
    Hbar = b - a
    z = cheb.nodes(nz, a, b)
    f = np.exp(-(z - z0) ** 2 / (2 * sig * sig)) / (sig * np.sqrt(2 * np.pi))
    fh = cheb.values_to_coeffs(f, nz)
    y, yp = bvp.solve(k * Hbar / 2, (-(Hbar / 2) ** 2 / eps * fh)[:, None])
    psi = cheb.coeffs_to_values(y[:, 0], nz)
    dpsi = (2 / Hbar) * cheb.coeffs_to_values(yp[:, 0], nz)
    ex, dex = _gauss_mode_solution(z, z0, sig, k, eps)
    assert np.max(np.abs(psi - ex)) < 1e-11 * np.max(np.abs(ex))
    assert np.max(np.abs(dpsi - dex)) < 1e-10 * np.max(np.abs(dex))


def test_bvp_k0_dirichlet_double_integral():
    """k = 0 with the homogeneous Dirichlet rows, Eq. (BCs0): psi'' = -f/eps,
    psi(a) = psi(b) = 0, against the closed-form double integral of a Gaussian."""
    a, b, z0, sig, eps, nz = -3.0, 5.0, 1.1, 0.5, 1.0, 80
    Hbar = b - a
    z = cheb.nodes(nz, a, b)
    f = np.exp(-(z - z0) ** 2 / (2 * sig * sig)) / (sig * np.sqrt(2 * np.pi))
    y, _ = bvp.solve(0.0, (-(Hbar / 2) ** 2 / eps * cheb.values_to_coeffs(f, nz))[:, None])
    psi = cheb.coeffs_to_values(y[:, 0], nz)

    def I2(t):   # int_a^t int_a^t' G, up to a linear function of t
        d = t - z0
        return d * 0.5 * (1 + erf(d / (sig * np.sqrt(2)))) + sig ** 2 * np.exp(-d * d / (2 * sig * sig)) / (sig * np.sqrt(2 * np.pi))
    ex = -I2(z) / eps
    ex -= ex[-1] + (ex[0] - ex[-1]) * (z - a) / (b - a)     # enforce psi(a) = psi(b) = 0
    assert np.max(np.abs(psi - ex)) < 1e-12 * np.max(np.abs(ex))


def test_bvp_spectral_convergence():
    a, b, z0, sig, k = -4.0, 4.0, 0.0, 0.35, 2.0
    errs = []
    for nz in (16, 24, 32, 48, 64, 80):
        Hbar = b - a
        z = cheb.nodes(nz, a, b)
        f = np.exp(-(z - z0) ** 2 / (2 * sig * sig)) / (sig * np.sqrt(2 * np.pi))
        y, _ = bvp.solve(k * Hbar / 2, (-(Hbar / 2) ** 2 * cheb.values_to_coeffs(f, nz))[:, None])
        ex, _ = _gauss_mode_solution(z, z0, sig, k, 1.0)
        errs.append(np.max(np.abs(cheb.coeffs_to_values(y[:, 0], nz) - ex)))
    assert errs[0] > 1e-3 and errs[-1] < 1e-12
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))


def _jump_solve(k, H, eps, eb, et, m):
    """Solve the jump conditions Eq. (harmbc1)-(harmbc4) directly for
    (A_i, B_i, A_b, B_t): psi_i = A e^{kz} + B e^{-kz}, psi_b = A_b e^{kz},
    psi_t = B_t e^{-kz}; m = (m_phi_b, m_E_b, m_phi_t, m_E_t) (m_E not scaled)."""
    eH, emH = np.exp(k * H), np.exp(-k * H)
    M = np.array([[1.0, 1.0, -1.0, 0.0],
                  [eps * k, -eps * k, -eb * k, 0.0],
                  [eH, emH, 0.0, -emH],
                  [eps * k * eH, -eps * k * emH, 0.0, et * k * emH]])
    rhs = -np.array([m[0], m[1], m[2], m[3]])
    return np.linalg.solve(M, rhs)


@pytest.mark.parametrize("eps,eb,et", [(1.0, 0.5, 0.2), (1.0, 1 / 80, 1 / 80), (2.0, 7.0, 0.3), (1.0, 1.0, 1.0)])
@pytest.mark.parametrize("k", [0.3, 1.7, 6.0])
def test_correction_solves_jump_conditions(eps, eb, et, k):
    H = 2.5
    rng = np.random.default_rng(7)
    m = rng.standard_normal(4)
    A, B, _, _ = _jump_solve(k, H, eps, eb, et, m)
    z = np.linspace(-0.5, H + 0.5, 11)
    val, der = correction(np.array([k]), z, m[0], m[1] / eps, m[2], m[3] / eps, H, eps, eb, et)
    ex = A * np.exp(k * z) + B * np.exp(-k * z)
    dex = k * (A * np.exp(k * z) - B * np.exp(-k * z))
    assert np.allclose(val[0], ex, rtol=1e-12, atol=1e-13 * np.max(np.abs(ex)))
    assert np.allclose(der[0], dex, rtol=1e-12, atol=1e-13 * np.max(np.abs(dex)))


def test_correction_metal_limit_is_continuous():
    H, k, z = 3.0, 1.3, np.linspace(0.0, 3.0, 7)
    m = (0.3, -1.1, 0.7, 0.4)
    v_inf, d_inf = correction(np.array([k]), z, *m, H, 1.0, np.inf, 0.25)
    v_big, d_big = correction(np.array([k]), z, *m, H, 1.0, 1e13, 0.25)
    assert np.allclose(v_inf, v_big, rtol=1e-11) and np.allclose(d_inf, d_big, rtol=1e-11)
    # a grounded metal wall: psi_i*(0) + psi^(c)(0) = 0 when psi_b* = 0
    v0, _ = correction(np.array([k]), np.array([0.0]), m[0], m[1], m[2], m[3], H, 1.0, np.inf, 0.25)
    assert v0[0, 0] == pytest.approx(-m[0], rel=1e-13)


def test_wall_factors():
    G, c, d, tau, rtau = wall_factors(1.0, 1.0 / 80)
    assert G == pytest.approx((1 / 80 - 1) / (1 / 80 + 1))
    assert tau == pytest.approx(2 / (1 + 1 / 80))      # Eq. (phibst): 2 eps/(eps_b + eps)
    assert wall_factors(1.0, np.inf) == (1.0, 1.0, 0.0, 0.0, 2.0)


def test_zero_mode_uniform_neutral_agree():
    """For eps_b = eps_t = eps, Eq. (ai1) and Eq. (ai2) differ by the total
    charge / eps (divergence theorem, Sec. 3.1.3); check with the exact
    derivatives of a smooth k = 0 problem."""
    # psi_i*' and psi_o*' satisfy psi' (x2) - psi'(x1) = -(1/eps) int f
    Qi_slab, Qo_slab, Qo_all, Q = 0.4, 0.25, 0.3, 0.0
    d_i0, d_o0, d_oa = 0.7, -0.2, 0.1
    d_iH = d_i0 - Qi_slab
    d_oH = d_o0 - Qo_slab
    d_ob = d_oa - Qo_all
    ai = zero_mode_slope(d_i0, d_iH, d_oa, d_o0, d_oH, d_ob, 0.0, 0.0, 1.0, 1.0, 1.0, 1.0)
    ai1 = (d_o0 - d_oa) - d_i0
    ai2 = (d_oH - d_ob) - d_iH
    assert ai == pytest.approx(0.5 * (ai1 + ai2))
    # neutral: Qi_slab = Qo_slab + (Q - Qo_all)... the two agree when
    # int_0^H f_i = int_0^H f_o + Q_nover and Q_nover + Q_o = 0
    Qn = Q - Qo_all
    d_iH = d_i0 - (Qo_slab + Qn)
    ai1 = (d_o0 - d_oa) - d_i0
    ai2 = (d_oH - d_ob) - d_iH
    assert ai1 == pytest.approx(ai2, abs=1e-15)
