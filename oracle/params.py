"""Parameter selection (oracle): Sec. 5.1 "Cutoffs and grid spacing",
Sec. 5.3 "Constraints on the splitting parameter" and Table (ewconstraints).

Paper rule (Sec. 5.1), with the xy grid size N_x, N_y given:
  h_xy = L/N;  g_t = c_h h_xy  (c_h = 1.4 for delta = 1e-4, 1.2 for 5e-4);
  xi from Eq. (gt): xi = 1 / (2 sqrt(g_t^2 - g_w^2));
  H_E = n_g h_xy / 2 = n_sigma g_t (Eq. (He); n_g = 12 or 10);
  N_z = ceil(pi * Hbar / (2 h_xy)), Hbar = H + 6 H_E (domain [-3H_E, H+3H_E]);
  r_nf = smallest r with |dG(r; g_w, xi)/dr / dG(r; g_w, 0)/dr| < delta
  (Eq. (rnf), pointwise kernel Eq. (Gnear)); r_cut = r_nf + n_sigma g_w.

Grid that resolves g_w itself (g_t = c_h h_xy would be below g_w, so the paper
rule has no real xi): the near-field cutoff r_cut is given and xi is the
smallest value with |dGbar(r_cut; g_w, xi)/dr / dGbar(r_cut; g_w, 0)/dr| < delta
for the averaged kernel Eq. (GnearK); then H_E = n_sigma g_t.

Explicit overrides (xi, r_cut, N_z) win over both rules.
"""
import math

import numpy as np
from scipy.optimize import brentq

from .kernels import near_kernel_dr, total_width

# Table (ewconstraints): tolerance -> (h factor c_h, Gaussian support n_g)
TOL_TABLE = {1e-4: (1.4, 12), 5e-4: (1.2, 10)}


def tolerance_constants(tol):
    """(c_h, n_g, n_sigma) of Table (ewconstraints); n_sigma = n_g / (2 c_h)."""
    key = min(TOL_TABLE, key=lambda t: abs(math.log(t / tol)))
    if abs(key - tol) > 1e-12:
        raise ValueError("tolerance must be 1e-4 or 5e-4 (Table ewconstraints)")
    c_h, n_g = TOL_TABLE[key]
    return c_h, n_g, n_g / (2.0 * c_h)


def _first_crossing(f, lo, hi, n=4000):
    """Smallest root of the decreasing-through-zero function f on [lo, hi]:
    scan on a uniform grid, then bisect the first sign change."""
    xs = np.linspace(lo, hi, n + 1)
    prev = f(xs[0])
    for i in range(1, n + 1):
        cur = f(xs[i])
        if prev >= 0.0 > cur:
            return brentq(f, xs[i - 1], xs[i], xtol=1e-300, rtol=1e-15, maxiter=500)
        prev = cur
    raise ValueError("no crossing found")


def near_field_radius(gw, xi, delta):
    """Eq. (rnf): r_nf for the pointwise kernel (Eq. (Gnear), (Enear))."""
    def f(r):
        return abs(near_kernel_dr(r, gw, xi, averaged=False)
                   / near_kernel_dr(r, gw, 0.0, averaged=False)) - delta
    return _first_crossing(f, 1e-6 / xi, 40.0 / xi)


def alpha_estimate(delta):
    """Eq. (alphest): alpha solving the near-field constraint when g_t = 2 g_w,
    i.e. g_w = 1/(sqrt12 xi); independent of xi (take xi = 1)."""
    gw = 1.0 / math.sqrt(12.0)

    def f(a):
        return abs(near_kernel_dr(a, gw, 1.0, averaged=False)
                   / near_kernel_dr(a, gw, 0.0, averaged=False)) - delta
    return _first_crossing(f, 1e-3, 20.0)


def xi_from_cutoff(r_cut, gw, delta):
    """Smallest xi with |dGbar(r_cut; g_w, xi)/dr / dGbar(r_cut; g_w, 0)/dr| < delta
    (averaged kernel Eq. (GnearK)); used when the grid resolves g_w."""
    ref = near_kernel_dr(r_cut, gw, 0.0, averaged=True)

    def f(xi):
        return abs(near_kernel_dr(r_cut, gw, xi, averaged=True) / ref) - delta
    return _first_crossing(f, 0.05 / gw, 400.0 / gw, n=8000)


def derive(Lx, Ly, H, gw, tol, nx, ny, nz=0, xi=0.0, r_cut=0.0,
           eps=1.0, eps_b=1.0, eps_t=1.0, n_sigma=0.0):
    """All derived quantities of the solve, as a plain dict. n_sigma > 0
    overrides the Gaussian truncation of Table (ewconstraints) (Sec. 5.1 notes
    that wider truncation gives arbitrarily high accuracy)."""
    c_h, n_g, n_sig_tab = tolerance_constants(tol)
    n_sigma = n_sigma if n_sigma > 0.0 else n_sig_tab
    hx, hy = Lx / nx, Ly / ny
    h = max(hx, hy)
    if xi == 0.0:
        if r_cut > 0.0:
            xi = xi_from_cutoff(r_cut, gw, tol)
        else:
            gt_rule = c_h * h
            if gt_rule <= gw:
                raise ValueError("paper rule infeasible (c_h h <= g_w): give r_cut or xi")
            xi = 1.0 / (2.0 * math.sqrt(gt_rule * gt_rule - gw * gw))
    gt = total_width(gw, xi)
    HE = n_sigma * gt
    r_nf = None
    if r_cut == 0.0 and not math.isinf(xi):
        r_nf = near_field_radius(gw, xi, tol)
        r_cut = r_nf + n_sigma * gw
    if math.isinf(xi):
        r_cut = 0.0
    if nz == 0:
        nz = int(math.ceil(math.pi * (H + 6.0 * HE) / (2.0 * h)))
    a, b = -3.0 * HE, H + 3.0 * HE
    return dict(Lx=float(Lx), Ly=float(Ly), H=float(H), gw=float(gw), tol=float(tol),
                nx=int(nx), ny=int(ny), nz=int(nz), hx=hx, hy=hy, h=h,
                xi=float(xi), gt=gt, n_sigma=n_sigma, n_g=n_g, c_h=c_h, HE=HE,
                r_cut=float(r_cut), r_nf=r_nf, a=a, b=b, Hbar=b - a,
                eps=float(eps), eps_b=float(eps_b), eps_t=float(eps_t))
