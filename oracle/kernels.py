"""Charge, spreading and near-field kernels (oracle).

* Eq. (gcharge), Sec. 2: the Gaussian charge g(r), standard deviation g_w.
* Eq. (spreadkernelEw) and Eq. (gt), Sec. 3.2: the spreading/interpolation
  kernel S = g * gamma^{1/2}, a Gaussian of standard deviation
  g_t = sqrt(1/(4 xi^2) + g_w^2).
* Eq. (Gnear), Sec. 3.2: the pointwise near-field kernel
  G^(n)(r; g_w, xi) = [erf(r/(sqrt2 g_w)) - erf(r/sqrt(2 g_w^2 + xi^-2))] / (4 pi eps r).
* Eq. (GnearK): the Gaussian-averaged kernel Gbar^(n)(r; g_w, xi) =
  G^(n)(r; sqrt2 g_w, xi), i.e. widths 2 g_w and sqrt(4 g_w^2 + xi^-2).
* Eq. (EnearK): Ebar^(n) = -q dGbar^(n)/dr rhat. Below r = 1e-3 g_w the
  paper switches to the Taylor series of the kernel (end of Sec. 3.2); the
  same switch is used here for the value and for the derivative.

Both kernels have the form [erf(r/a1) - erf(r/a2)] / (4 pi eps r) with
a1 = sqrt2 g_w (pointwise) or 2 g_w (averaged) and a2 = sqrt(a1^2 + xi^-2).
xi = 0 means "no smearing" (a2 = inf, the second erf vanishes); xi = inf
means the smearing width 1/(2 xi) is zero, so the kernel is identically 0.
"""
import numpy as np
from scipy.special import erf

SQRT_PI = np.sqrt(np.pi)
TAYLOR_RATIO = 1e-3   # r < 1e-3 g_w uses the series (end of Sec. 3.2)


def gaussian_charge(r, gw):
    """Eq. (gcharge): g(r) = (2 pi g_w^2)^{-3/2} exp(-r^2 / (2 g_w^2))."""
    return (2.0 * np.pi * gw * gw) ** -1.5 * np.exp(-r * r / (2.0 * gw * gw))


def total_width(gw, xi):
    """Eq. (gt): g_t = sqrt(1/(4 xi^2) + g_w^2); xi = inf gives g_t = g_w."""
    if np.isinf(xi):
        return float(gw)
    return float(np.sqrt(1.0 / (4.0 * xi * xi) + gw * gw))


def spread_kernel_1d(d, gt):
    """One Cartesian factor of Eq. (spreadkernelEw):
    S(r) = (2 pi g_t^2)^{-3/2} exp(-r^2/(2 g_t^2)) is the product over x, y, z
    of (2 pi g_t^2)^{-1/2} exp(-d^2/(2 g_t^2))."""
    return (2.0 * np.pi * gt * gt) ** -0.5 * np.exp(-d * d / (2.0 * gt * gt))


def _widths(gw, xi, averaged):
    a1 = (2.0 if averaged else np.sqrt(2.0)) * gw
    if xi == 0:
        a2 = np.inf
    elif np.isinf(xi):
        a2 = a1
    else:
        a2 = np.sqrt(a1 * a1 + 1.0 / (xi * xi))
    return a1, a2


def _series_val(r, a):
    """erf(r/a)/r = (2/(sqrt(pi) a)) (1 - x^2/3 + x^4/10 - x^6/42 + ...), x = r/a."""
    if np.isinf(a):
        return np.zeros_like(r)
    x = r / a
    return (2.0 / (SQRT_PI * a)) * (1.0 - x * x / 3.0 + x ** 4 / 10.0 - x ** 6 / 42.0)


def _direct_val(r, a):
    if np.isinf(a):
        return np.zeros_like(r)
    with np.errstate(divide="ignore", invalid="ignore"):
        return erf(r / a) / r


def _series_der(r, a):
    """(1/r) d/dr of the series above."""
    if np.isinf(a):
        return np.zeros_like(r)
    x = r / a
    return (2.0 / (SQRT_PI * a)) * (-2.0 / (3.0 * a * a) + 4.0 * x * x / (10.0 * a * a)
                                    - 6.0 * x ** 4 / (42.0 * a * a))


def _direct_der(r, a):
    """(1/r) d/dr [erf(r/a)/r] = (1/r) [-erf(r/a)/r^2 + 2 exp(-r^2/a^2)/(sqrt(pi) a r)]."""
    if np.isinf(a):
        return np.zeros_like(r)
    with np.errstate(divide="ignore", invalid="ignore"):
        return (-erf(r / a) / (r * r) + (2.0 / (SQRT_PI * a)) * np.exp(-(r / a) ** 2) / r) / r


def near_kernel(r, gw, xi, eps=1.0, averaged=True):
    """Eq. (GnearK) (averaged=True) or Eq. (Gnear) (averaged=False)."""
    r = np.asarray(r, dtype=np.float64)
    a1, a2 = _widths(gw, xi, averaged)
    if a1 == a2:
        return np.zeros_like(r)
    small = r < TAYLOR_RATIO * gw
    t1 = np.where(small, _series_val(r, a1), _direct_val(r, a1))
    t2 = np.where(small, _series_val(r, a2), _direct_val(r, a2))
    return (t1 - t2) / (4.0 * np.pi * eps)


def near_kernel_dr_over_r(r, gw, xi, eps=1.0, averaged=True):
    """(1/r) dG/dr of Eq. (GnearK)/(Gnear). The field of a unit source is
    E = -(1/r) dG/dr * r_vec with r_vec = target - source (Eq. (EnearK))."""
    r = np.asarray(r, dtype=np.float64)
    a1, a2 = _widths(gw, xi, averaged)
    if a1 == a2:
        return np.zeros_like(r)
    small = r < TAYLOR_RATIO * gw
    t1 = np.where(small, _series_der(r, a1), _direct_der(r, a1))
    t2 = np.where(small, _series_der(r, a2), _direct_der(r, a2))
    return (t1 - t2) / (4.0 * np.pi * eps)


def near_kernel_dr(r, gw, xi, eps=1.0, averaged=True):
    """dG/dr itself (used by the cutoff rules of Sec. 5.1 and Sec. 5.3.2)."""
    r = np.asarray(r, dtype=np.float64)
    return near_kernel_dr_over_r(r, gw, xi, eps, averaged) * r


def self_potential(gw, eps=1.0):
    """Gbar^(n)(0; g_w, xi=0) = 1/(4 pi^{3/2} eps g_w): the averaged potential a
    unit Gaussian charge creates at its own centre. The paper subtracts
    q_i times this from phibar_i in the rate-of-work test (Sec. 6.3)."""
    return 1.0 / (4.0 * np.pi ** 1.5 * eps * gw)
