"""The doubly-periodic slab solve, step by step (oracle).

Problem (Sec. 2): N Gaussian charges (Eq. (gcharge)) at z_k = (x_k, y_k, z_k)
with 0 < z_k < H, periodic on [0, Lx) x [0, Ly), permittivity eps in the
slab, eps_b below z = 0, eps_t above z = H. Outputs: the averaged potential
phibar_k (Eq. (pbar)), the force F_k = q_k Ebar(z_k) (Eq. (fqE)) and the
energy U = 1/2 sum q_k phibar_k plus, with wall charges sigma_b, sigma_t,
1/2 int (sigma_b phi(x, y, 0) + sigma_t phi(x, y, H)) (Eq. (Ufinal); see
wall_charge_energy). The gauge is phi(0) = 0 (Eq. (phi00)). This module is
test infrastructure: only tests and the benchmark's CPU baseline use it.

Far field, Sec. 5.2.2 steps 1-7 (figure "ffsolve"):
 1. C_over = charges within 2 H_E of a wall (z <= 2H_E or z >= H - 2H_E),
    C_nover = the rest; one image per near wall for C_over (Eq. (ims)).
 2. rho_o = spread of C_over with the kernel S (Eq. (spreadkernelEw)),
    truncated to the box |dx|, |dy|, |dz| <= H_E; solve eps Lap psi_o* = -rho_o
    (Eq. (phiost); the printed right-hand side lacks the minus sign that
    Eq. (phio0bvp) has) with the DtN solver; k=0 with Dirichlet BCs.
 3. rho_i = rho_o + spread of C_nover and of the images; solve for psi_i*.
 4. mismatches Eq. (mm1)-(mm4) at z = 0, H -> psi^(c) (Eq. (inphisc)) at the
    nodes with -H_E <= z_j <= H + H_E, only for 0 < |k| <= pi/h_xy.
 5. k = 0: add A_i z (Sec. 4.3.4, A_i from Eq. (ai1)/(ai2)).
 6. psi_i = psi_i* + psi^(c); E = -grad psi_i with i k_x, i k_y in xy and the
    Chebyshev derivative in z for psi_i*, the analytic one for psi^(c)
    (paragraph after step 7); inverse transforms to the grid.
 7. interpolate phi and E at the charges with S and the grid quadrature.
Near field (Sec. 4.2, Sec. 5.2.2 first paragraph): pairs closer than r_cut,
every charge plus one image per wall, the averaged kernels Eq. (GnearK),
(EnearK), nearest periodic image in xy.
Gauge (paragraph after the E-field one in Sec. 5.2.2): B_i(0) such that
phi^(n)(0) + phi^(f)(0) = 0.

Transform conventions: xy forward DFT sum_x f e^{-i k.x} (numpy rfft2,
unnormalised), inverse with 1/(Nx Ny). At an even-size Nyquist index the
wavenumber magnitude uses |k| = pi/h but the derivative multiplier i k is 0,
so the differentiated fields stay real.
"""
import numpy as np

from . import bvp, chebyshev as cheb
from .correction import correction, mismatches, wall_factors, zero_mode_slope
from .kernels import near_kernel, near_kernel_dr_over_r, spread_kernel_1d


# ----------------------------------------------------------------------------
# particle <-> grid
# ----------------------------------------------------------------------------

def support_1d(c, HE, h, n):
    """Grid indices i with |i h - c| <= H_E (unwrapped) and their offsets."""
    lo = int(np.ceil((c - HE) / h))
    hi = int(np.floor((c + HE) / h))
    idx = np.arange(lo, hi + 1)
    return np.mod(idx, n), idx * h - c


def support_z(c, HE, zn):
    j = np.nonzero(np.abs(zn - c) <= HE)[0]
    return j, zn[j] - c


def spread(xs, ys, zs, qs, P, zn):
    """rho(x_i, y_l, z_j) = sum_k q_k S(x_i - x_k, y_l - y_k, z_j - z_k) over the
    truncated box (Sec. 5.2.2 steps 2-3, Sec. 5.1 on truncation)."""
    rho = np.zeros((P["nz"], P["ny"], P["nx"]))
    gt, HE = P["gt"], P["HE"]
    for x, y, z, q in zip(xs, ys, zs, qs):
        ix, dx = support_1d(x, HE, P["hx"], P["nx"])
        iy, dy = support_1d(y, HE, P["hy"], P["ny"])
        jz, dz = support_z(z, HE, zn)
        w = (q * spread_kernel_1d(dz, gt)[:, None, None]
             * spread_kernel_1d(dy, gt)[None, :, None]
             * spread_kernel_1d(dx, gt)[None, None, :])
        np.add.at(rho, np.ix_(jz, iy, ix), w)
    return rho


def interpolate(fields, xs, ys, zs, P, zn, wz):
    """phibar(z_k) = sum_grid h_x h_y w_j f(x_i, y_l, z_j) S(x_i - x_k, ...):
    the integral of Eq. (compGfar) by the grid quadrature (uniform in xy,
    Clenshaw-Curtis in z). fields: (..., nz, ny, nx); returns (n, ...)."""
    gt, HE = P["gt"], P["HE"]
    out = np.zeros((len(xs),) + fields.shape[:-3])
    wxy = P["hx"] * P["hy"]
    for k, (x, y, z) in enumerate(zip(xs, ys, zs)):
        ix, dx = support_1d(x, HE, P["hx"], P["nx"])
        iy, dy = support_1d(y, HE, P["hy"], P["ny"])
        jz, dz = support_z(z, HE, zn)
        w = (wxy * (wz[jz] * spread_kernel_1d(dz, gt))[:, None, None]
             * spread_kernel_1d(dy, gt)[None, :, None]
             * spread_kernel_1d(dx, gt)[None, None, :])
        sub = fields[..., jz[:, None, None], iy[None, :, None], ix[None, None, :]]
        out[k] = np.sum(sub * w, axis=(-3, -2, -1))
    return out


# ----------------------------------------------------------------------------
# near field
# ----------------------------------------------------------------------------

def _min_image(d, L):
    return d - L * np.round(d / L)


def near_sources(x, y, z, q, P):
    """Every charge and its first image across each wall (Sec. 4.2, one image
    per wall): (x, y, z, strength) arrays of length 3N."""
    Gb = wall_factors(P["eps"], P["eps_b"])[0]
    Gt = wall_factors(P["eps"], P["eps_t"])[0]
    H = P["H"]
    return (np.concatenate([x, x, x]), np.concatenate([y, y, y]),
            np.concatenate([z, -z, 2.0 * H - z]),
            np.concatenate([q, -Gb * q, -Gt * q]))


def near_field(x, y, z, q, P, method="auto"):
    """phibar^(n) and Ebar^(n) at every charge: sum over sources (charges and
    images) with |r| < r_cut of q Gbar(r) and -q (1/r) dGbar/dr r_vec.
    method 'pairs' is the plain double loop over all pairs; 'tree' takes the
    candidate pairs from a k-d tree, then applies the same formulas."""
    n = len(q)
    phi = np.zeros(n)
    E = np.zeros((n, 3))
    if P["r_cut"] <= 0.0:
        return phi, E
    sx, sy, sz, sq = near_sources(x, y, z, q, P)
    if method == "auto":
        method = "pairs" if n <= 2048 else "tree"
    if method == "pairs":
        for t in range(n):
            dx = _min_image(x[t] - sx, P["Lx"])
            dy = _min_image(y[t] - sy, P["Ly"])
            dz = z[t] - sz
            r = np.sqrt(dx * dx + dy * dy + dz * dz)
            m = r < P["r_cut"]
            _accumulate(phi, E, t, r[m], dx[m], dy[m], dz[m], sq[m], P)
        return phi, E
    from scipy.spatial import cKDTree
    H = P["H"]
    box = [P["Lx"], P["Ly"], 20.0 * (H + P["r_cut"])]
    shift = 2.0 * (H + P["r_cut"])   # keeps every source z in [0, box_z)
    tree = cKDTree(np.stack([np.mod(sx, P["Lx"]), np.mod(sy, P["Ly"]), sz + shift], 1),
                   boxsize=box)
    cand = tree.query_ball_point(np.stack([x, y, z + shift], 1), P["r_cut"] * (1 + 1e-9))
    for t in range(n):
        s = np.asarray(cand[t], dtype=np.int64)
        if s.size == 0:
            continue
        dx = _min_image(x[t] - sx[s], P["Lx"])
        dy = _min_image(y[t] - sy[s], P["Ly"])
        dz = z[t] - sz[s]
        r = np.sqrt(dx * dx + dy * dy + dz * dz)
        m = r < P["r_cut"]
        _accumulate(phi, E, t, r[m], dx[m], dy[m], dz[m], sq[s][m], P)
    return phi, E


def _accumulate(phi, E, t, r, dx, dy, dz, qs, P):
    g = near_kernel(r, P["gw"], P["xi"], P["eps"], averaged=True)
    d = near_kernel_dr_over_r(r, P["gw"], P["xi"], P["eps"], averaged=True)
    phi[t] += np.sum(qs * g)
    E[t, 0] += np.sum(-qs * d * dx)
    E[t, 1] += np.sum(-qs * d * dy)
    E[t, 2] += np.sum(-qs * d * dz)


def near_potential_at_origin(x, y, z, q, P):
    """phi^(n)(0): the pointwise kernel Eq. (Gnearsum) at x = 0 summed over the
    charges and one image per wall, truncated at r_cut (gauge paragraph of
    Sec. 5.2.2)."""
    if P["r_cut"] <= 0.0:
        return 0.0
    sx, sy, sz, sq = near_sources(x, y, z, q, P)
    dx = _min_image(0.0 - sx, P["Lx"])
    dy = _min_image(0.0 - sy, P["Ly"])
    dz = 0.0 - sz
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    m = r < P["r_cut"]
    return float(np.sum(sq[m] * near_kernel(r[m], P["gw"], P["xi"], P["eps"], averaged=False)))


# ----------------------------------------------------------------------------
# the solve
# ----------------------------------------------------------------------------

def wavenumbers(P):
    kx = 2.0 * np.pi * np.fft.rfftfreq(P["nx"], d=P["hx"])
    ky = 2.0 * np.pi * np.fft.fftfreq(P["ny"], d=P["hy"])
    KX, KY = np.meshgrid(kx, ky)                       # (ny, nx//2+1)
    kmag = np.sqrt(KX * KX + KY * KY)
    dkx, dky = KX.copy(), KY.copy()
    if P["nx"] % 2 == 0:
        dkx[:, P["nx"] // 2] = 0.0
    if P["ny"] % 2 == 0:
        dky[P["ny"] // 2, :] = 0.0
    return kmag, dkx, dky


def gauge_weights(P):
    """w_n = int G_sigma(z) T_n(s(z)) dz, sigma = 1/(2 xi): the z part of the
    average of the Chebyshev series with gamma^{1/2} at z = 0 (Gauss-Hermite,
    exact for polynomials of degree < 2M)."""
    nz = P["nz"]
    s0 = cheb.scaled(0.0, P["a"], P["b"])
    if np.isinf(P["xi"]):
        return cheb.cheb_T(nz, s0)[0]
    sigma = 1.0 / (2.0 * P["xi"])
    t, w = np.polynomial.hermite.hermgauss(nz + 2)
    s = s0 + (2.0 / P["Hbar"]) * np.sqrt(2.0) * sigma * t
    # T_n(s) for |s| possibly slightly > 1: three-term recurrence
    T = np.zeros((len(s), nz))
    T[:, 0] = 1.0
    if nz > 1:
        T[:, 1] = s
    for m in range(2, nz):
        T[:, m] = 2.0 * s * T[:, m - 1] - T[:, m - 2]
    return (w @ T) / np.sqrt(np.pi)


def gauge_weights_at(P, z0):
    """gauge_weights at height z0 instead of 0: the z part of the average of
    the Chebyshev series with gamma^{1/2} at z = z0."""
    Q = dict(P)
    Q["a"], Q["b"] = P["a"] - z0, P["b"] - z0
    return gauge_weights(Q)


def wall_near_planar(d, P):
    """Integral over the wall plane of the pointwise near-field kernel
    Eq. (Gnear) of a unit charge at distance d from it, truncated at r_cut
    like the near field: (1/(2 eps)) int_d^{r_cut} [erf(r/a1) - erf(r/a2)] dr
    with a1 = sqrt2 g_w, a2 = sqrt(2 g_w^2 + xi^-2), written with
    I(x, a) = int_x^inf erfc(r/a) dr = a (e^{-(x/a)^2}/sqrt(pi) - (x/a) erfc(x/a))."""
    from scipy.special import erfc
    d = np.abs(np.asarray(d, dtype=np.float64))
    if P["r_cut"] <= 0.0 or np.isinf(P["xi"]):
        return np.zeros_like(d)
    a1 = np.sqrt(2.0) * P["gw"]
    a2 = np.sqrt(2.0 * P["gw"] ** 2 + (1.0 / P["xi"] ** 2 if P["xi"] > 0 else np.inf))

    def I(x, a):
        if np.isinf(a):
            return np.zeros_like(x)
        u = x / a
        return a * (np.exp(-u * u) / np.sqrt(np.pi) - u * erfc(u))

    rc = P["r_cut"]
    val = (I(d, a2) - I(d, a1)) - (I(np.full_like(d, rc), a2) - I(np.full_like(d, rc), a1))
    return np.where(d < rc, val, 0.0) / (2.0 * P["eps"])


def solve(pos, q, P, near_method="auto", sigma_b=None, sigma_t=None):
    """Full solve. pos (n, 3), q (n,). sigma_b, sigma_t: wall charge
    densities sampled on the xy grid, arrays (ny, nx) with [j, i] at
    (i h_x, j h_y), or None. Returns a dict with U, phi, force and the
    intermediate quantities the GPU path is compared with stage by stage."""
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    Lx, Ly, H, HE = P["Lx"], P["Ly"], P["H"], P["HE"]
    eps, eps_b, eps_t = P["eps"], P["eps_b"], P["eps_t"]
    nx, ny, nz, Hbar = P["nx"], P["ny"], P["nz"], P["Hbar"]
    x = np.mod(pos[:, 0], Lx)
    y = np.mod(pos[:, 1], Ly)
    z = pos[:, 2].copy()
    zn = cheb.nodes(nz, P["a"], P["b"])
    wz = cheb.quadrature_weights(nz, P["a"], P["b"])
    Gb = wall_factors(eps, eps_b)[0]
    Gt = wall_factors(eps, eps_t)[0]

    # step 1: classification and first images (Eq. (ims))
    near_b = z <= 2.0 * HE
    near_t = z >= H - 2.0 * HE
    over = near_b | near_t
    img_x = np.concatenate([x[near_b], x[near_t]])
    img_y = np.concatenate([y[near_b], y[near_t]])
    img_z = np.concatenate([-z[near_b], 2.0 * H - z[near_t]])
    img_q = np.concatenate([-Gb * q[near_b], -Gt * q[near_t]])

    # steps 2-3: spreading
    rho_o = spread(x[over], y[over], z[over], q[over], P, zn)
    rho_i = (rho_o + spread(x[~over], y[~over], z[~over], q[~over], P, zn)
             + spread(img_x, img_y, img_z, img_q, P, zn))

    # FFCT: xy FFT per plane, then Chebyshev coefficients per column
    kmag, dkx, dky = wavenumbers(P)
    M = kmag.size
    fi = cheb.values_to_coeffs(np.fft.rfft2(rho_i, axes=(1, 2)).reshape(nz, M), nz)
    fo = cheb.values_to_coeffs(np.fft.rfft2(rho_o, axes=(1, 2)).reshape(nz, M), nz)

    # BVP per mode (Appendix A); F = -(Hbar/2)^2 f / eps
    Kflat = kmag.reshape(M) * Hbar / 2.0
    yi = np.zeros((nz, M), complex)
    ypi = np.zeros((nz, M), complex)
    yo = np.zeros((nz, M), complex)
    ypo = np.zeros((nz, M), complex)
    scale = -(Hbar / 2.0) ** 2 / eps
    for K in np.unique(Kflat):
        cols = np.nonzero(Kflat == K)[0]
        rhs = np.concatenate([fi[:, cols], fo[:, cols]], axis=1) * scale
        y_, yp_ = bvp.solve(K, rhs)
        m = len(cols)
        yi[:, cols], yo[:, cols] = y_[:, :m], y_[:, m:]
        ypi[:, cols], ypo[:, cols] = yp_[:, :m], yp_[:, m:]

    # values at z = a, 0, H, b (derivatives d/dz = (2/Hbar) d/ds)
    sa, s0, sH, sb = (cheb.scaled(v, P["a"], P["b"]) for v in (P["a"], 0.0, H, P["b"]))
    T4 = cheb.cheb_T(nz, np.array([sa, s0, sH, sb]))
    dz_ = 2.0 / Hbar
    psi_i_at = T4 @ yi
    dpsi_i_at = dz_ * (T4 @ ypi)
    psi_o_at = T4 @ yo
    dpsi_o_at = dz_ * (T4 @ ypo)

    # step 4: correction for 0 < |k| <= pi/h_xy at nodes in [-H_E, H + H_E]
    kf = kmag.reshape(M)
    kmax = np.pi / P["h"]
    cmask = (kf > 0.0) & (kf <= kmax)
    zsel = (zn >= -HE) & (zn <= H + HE)
    corr = np.zeros((nz, M), complex)
    dcorr = np.zeros((nz, M), complex)
    corr0 = np.zeros(M, complex)
    # wall charges (Eq. (rho)): their xy transforms, unnormalised like rho's
    with_sigma = sigma_b is not None or sigma_t is not None
    zero = np.zeros((ny, nx))
    sb_hat = np.fft.rfft2(np.asarray(sigma_b if sigma_b is not None else zero, np.float64)).reshape(M)
    st_hat = np.fft.rfft2(np.asarray(sigma_t if sigma_t is not None else zero, np.float64)).reshape(M)
    if with_sigma and ((np.isinf(eps_b) and np.any(sb_hat != 0)) or (np.isinf(eps_t) and np.any(st_hat != 0))):
        raise ValueError("a wall charge on a metallic wall is not part of the method")
    mm = mismatches(psi_i_at[1], dpsi_i_at[1], psi_i_at[2], dpsi_i_at[2],
                    psi_o_at[1], dpsi_o_at[1], psi_o_at[2], dpsi_o_at[2], eps, eps_b, eps_t,
                    sb_hat, st_hat)
    if np.any(cmask):
        c = np.nonzero(cmask)[0]
        args = [m_[c] for m_ in mm]
        v, d = correction(kf[c], zn[zsel], *args, H, eps, eps_b, eps_t)
        corr[np.ix_(zsel, c)] = v.T
        dcorr[np.ix_(zsel, c)] = d.T
        v0, _ = correction(kf[c], np.array([0.0]), *args, H, eps, eps_b, eps_t)
        corr0[c] = v0[:, 0]

    # step 5: k = 0 linear mode
    k0 = int(np.nonzero(kf == 0.0)[0][0])
    Ai = zero_mode_slope(dpsi_i_at[1, k0].real, dpsi_i_at[2, k0].real,
                         dpsi_o_at[0, k0].real, dpsi_o_at[1, k0].real,
                         dpsi_o_at[2, k0].real, dpsi_o_at[3, k0].real,
                         psi_i_at[1, k0].real, psi_i_at[2, k0].real, H, eps, eps_b, eps_t,
                         sb_hat[k0].real, st_hat[k0].real)

    # step 6: values at the nodes, derivatives, inverse transforms
    psi = cheb.coeffs_to_values(yi, nz) + corr
    dpsi = dz_ * cheb.coeffs_to_values(ypi, nz) + dcorr
    psi[:, k0] += Ai * zn
    dpsi[:, k0] += Ai
    psi = psi.reshape(nz, ny, nx // 2 + 1)
    dpsi = dpsi.reshape(nz, ny, nx // 2 + 1)

    def inv(a):
        return np.fft.irfft2(a, s=(ny, nx), axes=(1, 2))
    phi_g = inv(psi)
    Ex_g = inv(-1j * dkx[None] * psi)
    Ey_g = inv(-1j * dky[None] * psi)
    Ez_g = inv(-dpsi)
    fields = np.stack([phi_g, Ex_g, Ey_g, Ez_g])

    # step 7: interpolation
    far = interpolate(fields, x, y, z, P, zn, wz)          # (n, 4)

    # near field
    phin, En = near_field(x, y, z, q, P, near_method)

    # gauge phi(0) = 0
    wg = gauge_weights(P)
    sigma2 = 0.0 if np.isinf(P["xi"]) else (1.0 / (2.0 * P["xi"])) ** 2
    smooth = np.exp(-0.5 * sigma2 * kf * kf)
    per_k = smooth * (wg @ yi) + corr0                      # half spectrum
    full = np.full(M, 2.0)
    full = full.reshape(ny, nx // 2 + 1)
    full[:, 0] = 1.0
    if nx % 2 == 0:
        full[:, nx // 2] = 1.0
    phi_f0 = float(np.sum(full.reshape(M) * per_k.real)) / (nx * ny)
    phi_n0 = near_potential_at_origin(x, y, z, q, P)
    B = -(phi_f0 + phi_n0)

    phibar = far[:, 0] + phin + B
    Ebar = far[:, 1:4] + En
    force = q[:, None] * Ebar
    U = 0.5 * float(np.sum(q * phibar))
    wall = {}
    if with_sigma:
        wall = wall_charge_energy(x, y, z, q, P, sb_hat, st_hat, yi[:, k0].real, Ai, B, kf, cmask, zn, wz, full)
        U += wall["U_wall"]
    return dict(U=U, phi=phibar, force=force, B=B, Ai=Ai, phi_f0=phi_f0, phi_n0=phi_n0, wall=wall,
                corr0=corr0, psi0=psi_i_at[1],
                rho_i=rho_i, rho_o=rho_o, fields=fields, far=far, phin=phin, En=En,
                psi=psi, dpsi=dpsi, over=over, zn=zn, wz=wz)


def wall_charge_energy(x, y, z, q, P, sb_hat, st_hat, y0, Ai, B, kf, cmask, zn, wz, full):
    """The wall term of Eq. (Ufinal), 1/2 int (sigma_b phi(x, y, 0) + sigma_t phi(x, y, H)) dx dy,
    split by xy mode.

    k_par = 0: the mean wall charge times the plane average of the pointwise
    potential at the wall. Its far part is the k=0 column averaged with
    gamma^{1/2} in z (the series with the weights of gauge_weights at z = 0 or
    H) plus A_i z, plus the gauge B; its near part is wall_near_planar summed
    over the charges and their images (the near field's sources).

    k_par != 0: by Green's reciprocity int sigma phi_q = sum_k q_k phibar_sigma(z_k),
    with phi_sigma the correction driven by the wall charges alone (Eq. (mm2),
    (mm4) with psi* = 0), interpolated at the charges like the far field; plus
    the wall charges' own term int sigma phi_sigma by Parseval. On these modes
    the correction is the exact per-mode solution of the jump conditions, so
    the energy's derivative is the force the solve returns. (A direct
    quadrature of the charges' near potential on the wall would need the scale
    g_w there; the reciprocity form needs none.)"""
    Lx, Ly, H = P["Lx"], P["Ly"], P["H"]
    eps, eps_b, eps_t = P["eps"], P["eps_b"], P["eps_t"]
    nx, ny, nz = P["nx"], P["ny"], P["nz"]
    M = kf.size
    k0 = int(np.nonzero(kf == 0.0)[0][0])
    hxhy = P["hx"] * P["hy"]
    # k_par = 0
    far0 = float(gauge_weights_at(P, 0.0) @ y0) / (nx * ny) + B
    farH = float(gauge_weights_at(P, H) @ y0 + Ai * H) / (nx * ny) + B
    sx, sy, sz, sq = near_sources(x, y, z, q, P)
    area = Lx * Ly
    near0 = float(np.sum(sq * wall_near_planar(sz, P))) / area
    nearH = float(np.sum(sq * wall_near_planar(H - sz, P))) / area
    Qb, Qt = hxhy * sb_hat[k0].real, hxhy * st_hat[k0].real
    U0 = 0.5 * (Qb * (far0 + near0) + Qt * (farH + nearH))
    # k_par != 0: the wall charges' own correction
    sb = np.where(cmask, sb_hat, 0.0)
    st = np.where(cmask, st_hat, 0.0)
    corr = np.zeros((nz, M), complex)
    wall0 = np.zeros(M, complex)
    wallH = np.zeros(M, complex)
    if np.any(cmask):
        c = np.nonzero(cmask)[0]
        zsel = (zn >= -P["HE"]) & (zn <= H + P["HE"])
        zero = np.zeros(c.size)
        args = (zero, sb[c] / eps, zero, -st[c] / eps)
        v, _ = correction(kf[c], zn[zsel], *args, H, eps, eps_b, eps_t)
        corr[np.ix_(zsel, c)] = v.T
        v0, _ = correction(kf[c], np.array([0.0, H]), *args, H, eps, eps_b, eps_t)
        wall0[c], wallH[c] = v0[:, 0], v0[:, 1]
    grid = np.fft.irfft2(corr.reshape(nz, ny, nx // 2 + 1), s=(ny, nx), axes=(1, 2))
    zeros = np.zeros_like(grid)
    phis = interpolate(np.stack([grid, zeros, zeros, zeros]), x, y, z, P, zn, wz)[:, 0]
    cross = float(np.sum(q * phis))
    fullv = full.reshape(M)
    self_ = hxhy / (nx * ny) * float(np.sum(fullv * (np.conj(sb) * wall0 + np.conj(st) * wallH).real))
    Uk = 0.5 * (cross + self_)
    return dict(U_wall=U0 + Uk, U_wall0=U0, U_wall_cross=0.5 * cross, U_wall_self=0.5 * self_,
                phi_wall0=far0 + near0, phi_wallH=farH + nearH, phi_sigma=phis)
