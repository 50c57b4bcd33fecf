"""Brownian dynamics of the ions (oracle), Sec. 7.1.

TEST INFRASTRUCTURE, like the rest of this package.

* Steric repulsion, Eq. (steric) with the Lennard-Jones form Eq. (lj):
  U_LJ(r) = 4 U0 ((2a/r)^{2p} - (2a/r)^p) + U0, F_LJ = -dU_LJ/dr; the force is
  F_LJ(r_m) for r <= r_m, F_LJ(r) up to 2^{1/p} 2a and 0 beyond. Pairs use
  the nearest periodic image in x and y. The walls repel each ion through the
  steric force with its own mirror image (at -z and at 2H - z).
* One step, Eq. (leimkuhler):
  z^{n+1} = z^n + mu (F_steric(z^n) + F(z^n)) dt + sqrt(kT mu dt / 2) (W^n + W^{n+1}),
  with F the electrostatic force of the solve (Eq. (fqE)). The displacement
  of an ion may be capped at a length (the paper reports larger stable steps
  with such a cap). x and y are wrapped into the box.
* Domain check: if any ion leaves 0 < z < H the step is discarded and
  retried with a new W^{n+1}; after the last allowed retry the configuration
  is declared unrecoverable.
* Noise: the random numbers of a step are drawn from Philox4x32-10 (Salmon,
  Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3",
  SC 2011), a counter-based generator, so the CUDA path can draw the same
  ones: key = the 64-bit seed, counter = (ion i, step (low, high 32 bits),
  retry); the four 32-bit words become uniforms (w + 1/2) 2^-32 and two
  Box-Muller pairs, the first three numbers giving W_i = (W_x, W_y, W_z).
  W^{n+1} of step n is drawn with step index n + 1, W^0 with 0.
"""
import numpy as np

from . import solver

M0, M1 = 0xD2511F53, 0xCD9E8D57          # Philox4x32 multipliers
W0, W1 = 0x9E3779B9, 0xBB67AE85          # key increments (Weyl sequence)
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds. ctr: (..., 4) uint32-valued ints, key:
    (..., 2). Returns (..., 4) as uint64 arrays holding 32-bit words."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) & MASK for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64) & MASK
    k1 = np.asarray(key[..., 1], dtype=np.uint64) & MASK
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = c[0] * np.uint64(M0)            # < 2^64: exact in uint64
        p1 = c[2] * np.uint64(M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1)


def normals(n, step, retry, seed):
    """W for ions 0..n-1 at (step, retry): (n, 3) standard normals."""
    i = np.arange(n, dtype=np.uint64)
    step = int(step)
    ctr = np.stack([i, np.full(n, step & MASK, np.uint64), np.full(n, (step >> 32) & MASK, np.uint64),
                    np.full(n, int(retry) & MASK, np.uint64)], axis=-1)
    key = np.array([int(seed) & MASK, (int(seed) >> 32) & MASK], dtype=np.uint64)
    w = philox4x32_10(ctr, np.broadcast_to(key, (n, 2))).astype(np.float64)
    u = (w + 0.5) * 2.0 ** -32
    r1 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r2 = np.sqrt(-2.0 * np.log(u[:, 2]))
    return np.stack([r1 * np.cos(2.0 * np.pi * u[:, 1]), r1 * np.sin(2.0 * np.pi * u[:, 1]),
                     r2 * np.cos(2.0 * np.pi * u[:, 3])], axis=-1)


def lj_force(r, a, U0, p):
    """F_LJ(r) = -dU_LJ/dr of Eq. (lj)."""
    s = (2.0 * a / r) ** p
    return 4.0 * U0 * p / r * (2.0 * s * s - s)


def steric_force_mag(r, a, U0, p, r_m):
    """Eq. (steric): capped below r_m, zero beyond 2^{1/p} 2a."""
    r = np.asarray(r, dtype=np.float64)
    rs = 2.0 ** (1.0 / p) * 2.0 * a
    f = lj_force(np.maximum(r, r_m), a, U0, p)
    return np.where(r <= rs, f, 0.0)


def steric_forces(pos, P, bp):
    """Steric force on every ion: all pairs (nearest periodic image in x, y)
    plus each ion's own mirror image in both walls."""
    Lx, Ly, H = P["Lx"], P["Ly"], P["H"]
    a, U0, p, r_m = bp["a"], bp["U0"], bp["p"], bp["r_m"]
    d = pos[:, None, :] - pos[None, :, :]
    d[..., 0] -= Lx * np.round(d[..., 0] / Lx)
    d[..., 1] -= Ly * np.round(d[..., 1] / Ly)
    r = np.sqrt(np.sum(d * d, axis=-1))
    np.fill_diagonal(r, np.inf)
    f = steric_force_mag(r, a, U0, p, r_m) / r
    F = np.sum(f[..., None] * d, axis=1)
    z = pos[:, 2]
    F[:, 2] += steric_force_mag(2.0 * z, a, U0, p, r_m)
    F[:, 2] -= steric_force_mag(2.0 * (H - z), a, U0, p, r_m)
    return F


def step(pos, q, W, n_step, P, bp, force=None, sigma_b=None, sigma_t=None):
    """One step of Eq. (leimkuhler) from step n_step. pos (n, 3), W = W^n
    (n, 3). bp: dict with dt, mu, kT, a, U0, p, r_m, max_disp (<= 0: none),
    max_retries (>= 1), seed. force: the electrostatic force at pos, or None
    to compute it with the oracle solve (with the wall charges sigma_b,
    sigma_t if given). Returns (pos', W', retries used, ok); on failure pos
    and W unchanged."""
    pos = np.asarray(pos, dtype=np.float64)
    if force is None:
        force = solver.solve(pos, q, P, sigma_b=sigma_b, sigma_t=sigma_t)["force"]
    drift = bp["mu"] * (force + steric_forces(pos, P, bp)) * bp["dt"]
    amp = np.sqrt(bp["kT"] * bp["mu"] * bp["dt"] / 2.0)
    for r in range(bp["max_retries"]):
        Wn = normals(len(q), n_step + 1, r, bp["seed"])
        dz = drift + amp * (W + Wn)
        if bp["max_disp"] > 0.0:
            norm = np.sqrt(np.sum(dz * dz, axis=1))
            scale = np.where(norm > bp["max_disp"], bp["max_disp"] / np.where(norm > 0, norm, 1.0), 1.0)
            dz = dz * scale[:, None]
        new = pos + dz
        if np.all((new[:, 2] > 0.0) & (new[:, 2] < P["H"])):
            new[:, 0] = np.mod(new[:, 0], P["Lx"])
            new[:, 1] = np.mod(new[:, 1], P["Ly"])
            return new, Wn, r, True
    return pos, W, bp["max_retries"], False
