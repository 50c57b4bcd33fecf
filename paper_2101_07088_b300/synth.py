"""Seeded synthetic inputs shaped like the paper's workloads.

Binary +-1 electrolytes (Sec. 6.2, 6.3 and 7 use charges of alternating or
random sign placed uniformly in the slab): exactly N/2 charges +1 and N/2
charges -1 assigned by a random permutation, positions uniform in
[0, Lx) x [0, Ly) x [z_lo, z_hi]. numpy's PCG64 generator; nothing here
depends on the solver. Both the CUDA path's tests and the oracle's take
their inputs from this module.
"""
import math

import numpy as np


def electrolyte(n, Lx, Ly, z_lo, z_hi, seed):
    """(pos [n, 3], q [n]) as float64 numpy arrays; n must be even."""
    if n % 2:
        raise ValueError("n must be even for an exactly neutral +-1 electrolyte")
    rng = np.random.default_rng(seed)
    q = np.concatenate([np.ones(n // 2), -np.ones(n // 2)])
    q = q[rng.permutation(n)]
    pos = np.stack([rng.uniform(0.0, Lx, n), rng.uniform(0.0, Ly, n), rng.uniform(z_lo, z_hi, n)], axis=1)
    return np.ascontiguousarray(pos), np.ascontiguousarray(q)


# The workloads of the benchmark configurations (box, grid, permittivity
# ratio eps_wall/eps_slab, charge width 1, near-field cutoff 4 widths).
WORKLOADS = {
    "c1_uniform_n128": dict(n=128, Lx=32.0, Ly=32.0, H=32.0, nx=64, ny=64, nz=64, eps_b=1.0, eps_t=1.0, seed=0),
    "c2_jumps_n16384": dict(n=16384, Lx=128.0, Ly=128.0, H=64.0, nx=256, ny=256, nz=128,
                            eps_b=1.0 / 80, eps_t=1.0 / 80, seed=1),
    "c2_metal_bottom_n16384": dict(n=16384, Lx=128.0, Ly=128.0, H=64.0, nx=256, ny=256, nz=128,
                                   eps_b=float("inf"), eps_t=1.0 / 80, seed=1),
    "c3_jumps_n1048576": dict(n=1 << 20, Lx=512.0, Ly=512.0, H=128.0, nx=1024, ny=1024, nz=128,
                              eps_b=1.0 / 80, eps_t=1.0 / 80, seed=2),
    # 1/64 of the 2^20-charge box at the same slab, density and grid spacing
    # (a bounded sample of that workload for the CPU oracle)
    "c3s_jumps_n16384": dict(n=16384, Lx=64.0, Ly=64.0, H=128.0, nx=128, ny=128, nz=128,
                             eps_b=1.0 / 80, eps_t=1.0 / 80, seed=7),
    # a quarter of the 2^20-charge box at the same density and grid spacing
    # (for profiler captures that must stay a few GB)
    "c3q_jumps_n262144": dict(n=1 << 18, Lx=256.0, Ly=256.0, H=128.0, nx=512, ny=512, nz=128,
                              eps_b=1.0 / 80, eps_t=1.0 / 80, seed=6),
}


def workload(name):
    """Inputs and parameter dict (for dpslab_params) of a named workload:
    g_w = 1, r_cut = 4 g_w, tolerance 1e-4, charges in [1, H - 1]."""
    w = dict(WORKLOADS[name])
    pos, q = electrolyte(w["n"], w["Lx"], w["Ly"], 1.0, w["H"] - 1.0, w["seed"])
    params = dict(Lx=w["Lx"], Ly=w["Ly"], H=w["H"], eps=1.0, eps_b=w["eps_b"], eps_t=w["eps_t"],
                  gw=1.0, tol=1e-4, nx=w["nx"], ny=w["ny"], nz=w["nz"], r_cut=4.0)
    return pos, q, params


def smooth7(v):
    """Smallest integer >= v whose prime factors are 2, 3, 5, 7."""
    v = max(1, int(math.ceil(v)))
    while True:
        r = v
        for f in (2, 3, 5, 7):
            while r % f == 0:
                r //= f
        if r == 1:
            return v
        v += 1


def batch_systems(count, seed, n_range=(256, 65536), l_range=(32.0, 256.0), h_range=(16.0, 128.0),
                  ratios=(1.0 / 80.0, 1.0, math.inf), h=0.5, gw=1.0, tol=1e-4, r_cut=4.0):
    """Independent slab systems of the batched workload: N log-uniform in
    n_range (even), Lx = Ly log-uniform in l_range, H uniform in h_range, each
    wall's eps_w/eps drawn from `ratios`, grid spacing h (2 points per width
    at g_w = 1; nx rounded up to a 7-smooth size and Lx = nx h), N_z from the
    paper's rule (0 here). Returns a list of (pos, q, params) with the same
    params keys as workload(); system i uses seed + i for its charges."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))) // 2 * 2)
        L = math.exp(rng.uniform(math.log(l_range[0]), math.log(l_range[1])))
        H = float(rng.uniform(*h_range))
        eb, et = (float(ratios[j]) for j in rng.integers(0, len(ratios), 2))
        nx = smooth7(L / h)
        L = nx * h
        pos, q = electrolyte(n, L, L, 1.0, H - 1.0, seed + i)
        params = dict(Lx=L, Ly=L, H=H, eps=1.0, eps_b=eb, eps_t=et, gw=gw, tol=tol, nx=nx, ny=nx, nz=0,
                      r_cut=r_cut)
        out.append((pos, q, params))
    return out


# Smallest box side of the served workload: twice the larger of the cutoff
# (4) and the Gaussian support half-width (about 4.3 at g_w = 1, tolerance
# 1e-4), plus one grid spacing, rounded up.
SERVE_L_MIN = 10.0


def serve_replicas(count, seed, n_range=(512, 262144), h_range=(16.0, 128.0), ratio=1.0 / 80.0,
                   rho=1.0 / 32.0, h=0.5, gw=1.0, tol=1e-4, r_cut=4.0):
    """Replicas of the served workload: N log-uniform in n_range (even), H
    uniform in h_range, both walls at eps_w/eps = ratio, square box side
    L = sqrt(N / (rho H)) (the charge density of the 2^20-charge workload,
    2^20 / (512^2 128) = 1/32 per unit volume) but at least SERVE_L_MIN, grid
    spacing h (nx 7-smooth, Lx = nx h), N_z from the paper's rule. Returns a
    list of params dicts (the keys of workload()) with "n" added."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))) // 2 * 2)
        H = float(rng.uniform(*h_range))
        L = max(SERVE_L_MIN, math.sqrt(n / (rho * H)))
        nx = smooth7(L / h)
        L = nx * h
        out.append(dict(n=n, Lx=L, Ly=L, H=H, eps=1.0, eps_b=ratio, eps_t=ratio, gw=gw, tol=tol, nx=nx, ny=nx,
                        nz=0, r_cut=r_cut))
    return out


def serve_arrivals(count, n_replicas, rate, seed):
    """Request stream of the served workload: `count` requests, each for a
    replica drawn uniformly, Poisson arrivals at `rate` per second. Returns
    (replica ids, arrival times in seconds from the start); request k's
    charges come from electrolyte(..., seed + 1 + k)."""
    rng = np.random.default_rng(seed)
    rep = rng.integers(0, n_replicas, count)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    return rep, t
