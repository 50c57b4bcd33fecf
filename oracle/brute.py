"""Method-independent reference for tiny inputs (used only to pin the oracle).

It evaluates the exact model the paper solves: Gaussian charges of width g_w
(Eq. (gcharge)) in a slab with permittivity eps, periodic in x and y, with
dielectric jumps at z = 0 and z = H represented by the classical image series
(Sec. 4.1: reflecting across z = 0 multiplies the strength by
-(eps_b - eps)/(eps_b + eps), Eq. (ims), and across z = H by the same factor
with eps_t; the images of images continue alternately). Within the slab the
potential of the charges plus all images in a uniform medium eps satisfies
the jump conditions (Sec. 4.1 shows this holds for isotropic clouds too).

The Gaussian-averaged potential at a charge (Eq. (pbar)) is the potential of
a Gaussian with variance sigma^2 = 2 g_w^2 per direction (g * g), so each
source-target term is the doubly-periodic Green's function of that Gaussian:

  Phi(dr, dz) = 1/(eps Lx Ly) [ sum_{k != 0} cos(k.dr) e^{-sigma^2 k^2/2} m_k(dz)
                                - (1/2) (dz erf(dz/(sigma sqrt2)) + sigma sqrt(2/pi) e^{-dz^2/(2 sigma^2)}) ]

with m_k(dz) = [h_k(dz) + h_k(-dz)]/(4k), h_k(z) = e^{-z^2/(2 sigma^2)} erfcx((k sigma^2 - z)/(sigma sqrt2)),
i.e. (1/(2k)) times e^{-k|z|} convolved with the z Gaussian. The k = 0 term is
the 1D potential -|z|/2 convolved with the Gaussian (defined up to a
constant, which cancels for neutral systems). Fields are the analytic
derivatives. No grid, no splitting, no truncated Gaussian.
"""
import numpy as np
from scipy.special import erf, erfcx


def _h(k, z, sigma):
    """e^{-z^2/(2 s^2)} erfcx((k s^2 - z)/(s sqrt2)), evaluated without overflow."""
    x = (k * sigma * sigma - z) / (sigma * np.sqrt(2.0))
    out = np.empty(np.broadcast(k, z).shape)
    k_b, z_b, x_b = np.broadcast_arrays(k, z, x)
    pos = x_b >= 0.0
    out[pos] = np.exp(-z_b[pos] ** 2 / (2 * sigma ** 2)) * erfcx(x_b[pos])
    neg = ~pos
    # erfcx(x) = 2 e^{x^2} - erfcx(-x); e^{x^2 - z^2/(2 s^2)} = e^{k^2 s^2/2 - k z}
    kk, zz, xx = k_b[neg], z_b[neg], x_b[neg]
    out[neg] = (2.0 * np.exp(0.5 * kk * kk * sigma * sigma - kk * zz)
                - np.exp(-zz ** 2 / (2 * sigma ** 2)) * erfcx(-xx))
    return out


def image_series(z0, H, Gb, Gt, tol=1e-18, max_terms=200000):
    """Positions and relative strengths of a unit charge at z0 and all of its
    images (both alternating reflection sequences)."""
    pos, stren = [z0], [1.0]
    for first in ("b", "t"):
        p, s, wall = z0, 1.0, first
        for _ in range(max_terms):
            if wall == "b":
                p, s, wall = -p, -Gb * s, "t"
            else:
                p, s, wall = 2.0 * H - p, -Gt * s, "b"
            if abs(s) < tol:
                break
            pos.append(p)
            stren.append(s)
    return np.array(pos), np.array(stren)


def solve(pos, q, Lx, Ly, H, gw, eps=1.0, eps_b=1.0, eps_t=1.0, kcut_exp=40.0, tol=1e-18):
    """Averaged potential phibar_t and field Ebar_t at every charge, and
    U = 1/2 sum q phibar (up to the gauge constant, which drops out for a
    neutral system)."""
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    sigma = np.sqrt(2.0) * gw
    kcut = np.sqrt(2.0 * kcut_exp) / sigma
    mx = int(np.ceil(kcut * Lx / (2 * np.pi)))
    my = int(np.ceil(kcut * Ly / (2 * np.pi)))
    m = np.arange(-mx, mx + 1)
    n = np.arange(-my, my + 1)
    KX, KY = np.meshgrid(2 * np.pi * m / Lx, 2 * np.pi * n / Ly, indexing="ij")
    KX, KY = KX.ravel(), KY.ravel()
    K = np.sqrt(KX ** 2 + KY ** 2)
    keep = (K > 0) & (K <= kcut)
    KX, KY, K = KX[keep], KY[keep], K[keep]
    damp = np.exp(-0.5 * sigma ** 2 * K ** 2)
    kmin = K.min()

    def gam(e):
        return 1.0 if np.isinf(e) else (e - eps) / (e + eps)
    Gb, Gt = gam(eps_b), gam(eps_t)
    area = eps * Lx * Ly
    nq = len(q)
    phi = np.zeros(nq)
    E = np.zeros((nq, 3))
    for s in range(nq):
        zi, si = image_series(pos[s, 2], H, Gb, Gt, tol)
        for t in range(nq):
            dx = pos[t, 0] - pos[s, 0]
            dy = pos[t, 1] - pos[s, 1]
            dz = pos[t, 2] - zi                              # all images
            st = q[s] * si
            # k = 0 part (every image)
            a = sigma * np.sqrt(2.0)
            phi[t] += np.sum(st * (-0.5) * (dz * erf(dz / a) + sigma * np.sqrt(2 / np.pi)
                                           * np.exp(-dz ** 2 / (2 * sigma ** 2)))) / area
            E[t, 2] += np.sum(st * 0.5 * erf(dz / a)) / area
            # k != 0 part (images close enough for e^{-k |dz|} to matter)
            close = kmin * np.abs(dz) < 60.0
            for dzc, stc in zip(dz[close], st[close]):
                ph = KX * dx + KY * dy
                hp, hm = _h(K, dzc, sigma), _h(K, -dzc, sigma)
                mk = (hp + hm) / (4.0 * K)
                mkz = (hm - hp) / 4.0
                c, sn = np.cos(ph), np.sin(ph)
                phi[t] += stc * np.sum(c * damp * mk) / area
                E[t, 0] += stc * np.sum(KX * sn * damp * mk) / area
                E[t, 1] += stc * np.sum(KY * sn * damp * mk) / area
                E[t, 2] += -stc * np.sum(c * damp * mkz) / area
    U = 0.5 * float(np.sum(q * phi))
    return dict(U=U, phi=phi, force=q[:, None] * E)


def pointwise_potential(points, pos, q, Lx, Ly, H, gw, eps=1.0, eps_b=1.0, eps_t=1.0,
                        kcut_exp=40.0, tol=1e-18):
    """The potential phi(x) of the Gaussian charges (Eq. (gcharge), std g_w per
    direction) plus their full image series, at arbitrary points x with
    0 <= z <= H. This is the field whose value at the origin the gauge
    Eq. (phi00) sets to zero (Sec. 2).

    Same sums as solve(), with the kernel of one Gaussian (variance g_w^2)
    instead of the pair average (2 g_w^2): the k = 0 part is -|z|/2
    convolved with that Gaussian, whose constant is the one solve() uses, so
    differences phibar_k - phi(x) carry no undetermined constant for a neutral
    system."""
    points = np.atleast_2d(np.asarray(points, dtype=np.float64))
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    sigma = float(gw)
    kcut = np.sqrt(2.0 * kcut_exp) / sigma
    mx = int(np.ceil(kcut * Lx / (2 * np.pi)))
    my = int(np.ceil(kcut * Ly / (2 * np.pi)))
    KX, KY = np.meshgrid(2 * np.pi * np.arange(-mx, mx + 1) / Lx,
                         2 * np.pi * np.arange(-my, my + 1) / Ly, indexing="ij")
    KX, KY = KX.ravel(), KY.ravel()
    K = np.sqrt(KX ** 2 + KY ** 2)
    keep = (K > 0) & (K <= kcut)
    KX, KY, K = KX[keep], KY[keep], K[keep]
    damp = np.exp(-0.5 * sigma ** 2 * K ** 2)
    kmin = K.min()

    def gam(e):
        return 1.0 if np.isinf(e) else (e - eps) / (e + eps)
    Gb, Gt = gam(eps_b), gam(eps_t)
    area = eps * Lx * Ly
    a = sigma * np.sqrt(2.0)
    out = np.zeros(len(points))
    for s in range(len(q)):
        zi, si = image_series(pos[s, 2], H, Gb, Gt, tol)
        st = q[s] * si
        for t, (px, py, pz) in enumerate(points):
            dx, dy = px - pos[s, 0], py - pos[s, 1]
            dz = pz - zi
            out[t] += np.sum(st * (-0.5) * (dz * erf(dz / a) + sigma * np.sqrt(2 / np.pi)
                                           * np.exp(-dz ** 2 / (2 * sigma ** 2)))) / area
            close = kmin * np.abs(dz) < 60.0
            c = np.cos(KX * dx + KY * dy) * damp
            for dzc, stc in zip(dz[close], st[close]):
                mk = (_h(K, dzc, sigma) + _h(K, -dzc, sigma)) / (4.0 * K)
                out[t] += stc * np.sum(c * mk) / area
    return out
