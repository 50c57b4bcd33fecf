"""Harmonic correction and the k=0 mode (oracle).

k_par != 0 -- Sec. 3.1.2, Eq. (harmeq)-(harmbc4), solution Eq. (inphisc);
mismatches Eq. (mm1)-(mm4) of Sec. 4.3.3.

The correction psi^(c) is A e^{kz} + B e^{-kz} in the slab, A_b e^{kz} below
and B_t e^{-kz} above, with the four jump conditions

  psi_i(0) - psi_b(0) = -m_phi^b,   eps psi_i'(0) - eps_b psi_b'(0) = -m_E^b,
  psi_i(H) - psi_t(H) = -m_phi^t,   eps psi_i'(H) - eps_t psi_t'(H) = -m_E^t.

Solving them gives Eq. (inphisc) with the numerators as printed (in units
eps = 1) but with the denominator

  k [ (eps_b + 1)(eps_t + 1) - (eps_b - 1)(eps_t - 1) e^{-2Hk} ];

the printed k (eps_b+1)(eps_t+1) - (eps_b eps_t + eps_b + eps_t - 1) e^{-2Hk}
is garbled (its two terms do not even carry the same power of k). For a
general slab permittivity eps, replace eps_b -> eps_b/eps, eps_t -> eps_t/eps
and m_E -> m_E/eps. Dividing numerator and denominator by
(eps_b + eps)(eps_t + eps) gives the form used below, which is finite for a
metallic wall (eps_w -> inf) and only ever multiplies decaying exponentials
on -H_E <= z <= H + H_E:

  psi^(c)(z) = [ -P_b (e^{-kz} - G_t e^{k(z-2H)}) + Q_t (e^{k(z-H)} - G_b e^{-k(z+H)}) ]
               / (1 - G_b G_t e^{-2kH}),
  P_b = c_b m_phi^b - d_b m_E^b/(eps k),   Q_t = -c_t m_phi^t - d_t m_E^t/(eps k),

with r_w = eps_w/eps, G_w = (r_w - 1)/(r_w + 1), c_w = r_w/(1 + r_w),
d_w = 1/(1 + r_w) (metal: G_w = c_w = 1, d_w = 0).

k_par = 0 -- Sec. 4.3.4, Eq. (CE), (ai1), (ai2) and Sec. 5.2.2 step 5 (A_i is
the mean of the two expressions).

Wall charges sigma_b, sigma_t (Eq. (rho), Sec. 4.3.1) enter only here: through
the displacement mismatches Eq. (mm2), (mm4) for k_par != 0 and the sigma
terms of Eq. (ai1), (ai2) for k_par = 0.
"""
import numpy as np


def wall_factors(eps, eps_w):
    """(G_w, c_w, d_w, tau_w, r_w tau_w) for one wall.

    tau_w = 2 eps/(eps_w + eps) is the factor of Eq. (phibst)/(phitst) and
    -G_w q is the image strength of Eq. (ims)."""
    if np.isinf(eps_w):
        return 1.0, 1.0, 0.0, 0.0, 2.0
    r = eps_w / eps
    return (r - 1.0) / (r + 1.0), r / (1.0 + r), 1.0 / (1.0 + r), 2.0 / (1.0 + r), 2.0 * r / (1.0 + r)


def mismatches(psi_i0, dpsi_i0, psi_iH, dpsi_iH, psi_o0, dpsi_o0, psi_oH, dpsi_oH,
               eps, eps_b, eps_t, sigma_b=0.0, sigma_t=0.0):
    """Eq. (mm1)-(mm4) with psi_b* = tau_b psi_o*, psi_t* = tau_t psi_o*
    (Eq. (phibst), (phitst)) and the wall charges' transforms sigma_b, sigma_t
    (+sigma_b in m_E^b, -sigma_t in m_E^t). Returned m_E are divided by eps:
    (m_phi^b, m_E^b/eps, m_phi^t, m_E^t/eps)."""
    _, _, _, tb, rtb = wall_factors(eps, eps_b)
    _, _, _, tt, rtt = wall_factors(eps, eps_t)
    m_phi_b = psi_i0 - tb * psi_o0
    m_E_b = dpsi_i0 - rtb * dpsi_o0 + sigma_b / eps
    m_phi_t = psi_iH - tt * psi_oH
    m_E_t = dpsi_iH - rtt * dpsi_oH - sigma_t / eps
    return m_phi_b, m_E_b, m_phi_t, m_E_t


def correction(k, z, m_phi_b, m_E_b, m_phi_t, m_E_t, H, eps, eps_b, eps_t):
    """psi^(c)(k, z) and d psi^(c)/dz for k > 0 (m_E already divided by eps).
    k and the mismatches broadcast against each other; z is the last axis."""
    Gb, cb, db, _, _ = wall_factors(eps, eps_b)
    Gt, ct, dt, _, _ = wall_factors(eps, eps_t)
    k = np.asarray(k, dtype=np.float64)[..., None]
    P = (cb * np.asarray(m_phi_b) - db * np.asarray(m_E_b) / k[..., 0])[..., None]
    Q = (-ct * np.asarray(m_phi_t) - dt * np.asarray(m_E_t) / k[..., 0])[..., None]
    den = 1.0 - Gb * Gt * np.exp(-2.0 * k * H)
    e1 = np.exp(-k * z)
    e2 = np.exp(k * (z - 2.0 * H))
    e3 = np.exp(k * (z - H))
    e4 = np.exp(-k * (z + H))
    val = (-P * (e1 - Gt * e2) + Q * (e3 - Gb * e4)) / den
    der = k * (P * (e1 + Gt * e2) + Q * (e3 + Gb * e4)) / den
    return val, der


def zero_mode_slope(dpsi_i0, dpsi_iH, dpsi_o_a, dpsi_o0, dpsi_oH, dpsi_o_b,
                    psi_i0, psi_iH, H, eps, eps_b, eps_t, sigma_b0=0.0, sigma_t0=0.0):
    """A_i(0) of Sec. 4.3.4, from the k=0 Dirichlet solutions psi_i*, psi_o*
    (derivatives d/dz at a, 0, H, b) and the k=0 transforms of the wall
    charges sigma_b0, sigma_t0.

    Eq. (CE): A_b = -d psi_b*/dz (a), A_t = -d psi_t*/dz (b);
    Eq. (ai1): A_i = (eps_b/eps) tau_b (psi_o*'(0) - psi_o*'(a)) - psi_i*'(0) - sigma_b0/eps;
    Eq. (ai2): A_i = (eps_t/eps) tau_t (psi_o*'(H) - psi_o*'(b)) - psi_i*'(H) + sigma_t0/eps.
    Both dielectric: the mean (Sec. 5.2.2 step 5). A metallic wall only enters
    through the other wall's equation; two metallic walls are held at equal
    potential, A_i = -(psi_i*(H) - psi_i*(0))/H."""
    _, _, _, _, rtb = wall_factors(eps, eps_b)
    _, _, _, _, rtt = wall_factors(eps, eps_t)
    ai1 = rtb * (dpsi_o0 - dpsi_o_a) - dpsi_i0 - sigma_b0 / eps
    ai2 = rtt * (dpsi_oH - dpsi_o_b) - dpsi_iH + sigma_t0 / eps
    mb, mt = np.isinf(eps_b), np.isinf(eps_t)
    if mb and mt:
        return -(psi_iH - psi_i0) / H
    if mb:
        return ai2
    if mt:
        return ai1
    return 0.5 * (ai1 + ai2)
