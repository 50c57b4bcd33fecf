"""Brownian dynamics oracle (Sec. 7.1) pinned on CPU.

* Philox4x32-10 against the known-answer vectors published with the
  generator (Random123's kat_vectors): counter/key all zeros, all ones, and
  the digits of pi.
* Its normals: mean, variance and lack of correlation on many draws, and
  distinct streams per step and retry.
* Eq. (lj)/(steric): F_LJ = -dU_LJ/dr by finite differences, zero at
  2^{1/p} 2a, constant below r_m; the pair sum against an explicit loop over
  periodic images with the walls' mirror images; Newton's third law.
* Eq. (leimkuhler): with kT = 0 a step is explicit Euler; a free ion's
  displacement after N steps has variance kT mu dt (4N - 2) / 2 per
  component (the scheme's W^n + W^{n+1} telescopes), which is 2 D t - D dt
  with D = kT mu; the displacement cap holds; a step that leaves the slab is
  retried and, past the last retry, reported without moving anything."""
import numpy as np
import pytest

from oracle import bd, params


def test_philox_known_answers():
    ctr = np.array([[0, 0, 0, 0], [0xFFFFFFFF] * 4, [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]], dtype=np.uint64)
    key = np.array([[0, 0], [0xFFFFFFFF] * 2, [0xA4093822, 0x299F31D0]], dtype=np.uint64)
    want = np.array([[0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8],
                     [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD],
                     [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]], dtype=np.uint64)
    assert np.array_equal(bd.philox4x32_10(ctr, key), want)


def test_normals_statistics_and_streams():
    W = bd.normals(200000, 7, 0, seed=12345)
    n = W.size
    assert abs(W.mean()) < 5.0 / np.sqrt(n)
    assert abs(W.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    c = np.corrcoef(W.T)
    assert np.max(np.abs(c - np.eye(3))) < 5.0 / np.sqrt(W.shape[0])
    assert abs(np.mean(W[:, 0] ** 4) - 3.0) < 0.05                 # Gaussian kurtosis
    a, b, c2 = bd.normals(1000, 7, 0, 1), bd.normals(1000, 7, 1, 1), bd.normals(1000, 8, 0, 1)
    assert not np.allclose(a, b) and not np.allclose(a, c2)
    assert np.array_equal(a, bd.normals(1000, 7, 0, 1))
    # the high word of the step index is part of the counter
    assert not np.allclose(bd.normals(10, 5, 0, 1), bd.normals(10, 5 + (1 << 32), 0, 1))


BP = dict(dt=1e-3, mu=1.0, kT=1.0, a=0.5, U0=1.0, p=6, r_m=0.7, max_disp=0.0, max_retries=8, seed=99)


def test_lj_force_is_minus_derivative_and_capped():
    a, U0, p = 0.5, 1.3, 4
    r = np.linspace(0.75, 1.2, 50)

    def U(r):
        s = (2 * a / r) ** p
        return 4 * U0 * (s * s - s) + U0
    h = 1e-6
    fd = -(U(r + h) - U(r - h)) / (2 * h)
    assert np.max(np.abs(bd.lj_force(r, a, U0, p) - fd)) < 1e-6 * np.max(np.abs(fd))
    rs = 2 ** (1 / p) * 2 * a
    assert abs(bd.lj_force(rs, a, U0, p)) < 1e-12 * U0
    assert abs(U(rs)) < 1e-12                                    # shifted: U = 0 at the cutoff
    f = bd.steric_force_mag(np.array([0.1, 0.5, 0.7, rs * 1.0001]), a, U0, p, 0.7)
    assert f[0] == f[1] == f[2] == bd.lj_force(0.7, a, U0, p) and f[3] == 0.0


def test_steric_pair_sum_against_image_loop():
    rng = np.random.default_rng(3)
    P = params.derive(3.0, 2.5, 2.0, 0.2, 1e-4, 16, 16, r_cut=1.0)
    n = 40
    pos = np.stack([rng.uniform(0, 3.0, n), rng.uniform(0, 2.5, n), rng.uniform(0.05, 1.95, n)], 1)
    bp = dict(BP, a=0.3, p=2, r_m=0.3)
    F = bd.steric_forces(pos, P, bp)
    ref = np.zeros_like(pos)
    for i in range(n):
        for j in range(n):
            for ix in (-1, 0, 1):
                for iy in (-1, 0, 1):
                    if i == j and ix == 0 and iy == 0:
                        continue
                    d = pos[i] - (pos[j] + np.array([ix * 3.0, iy * 2.5, 0.0]))
                    r = np.linalg.norm(d)
                    ref[i] += bd.steric_force_mag(r, 0.3, 1.0, 2, 0.3) / r * d
        for zimg in (-pos[i, 2], 4.0 - pos[i, 2]):
            d = pos[i] - np.array([pos[i, 0], pos[i, 1], zimg])
            r = np.linalg.norm(d)
            ref[i] += bd.steric_force_mag(r, 0.3, 1.0, 2, 0.3) / r * d
    assert np.max(np.abs(F - ref)) < 1e-12 * np.max(np.abs(ref))
    walls = np.zeros_like(pos)
    z = pos[:, 2]
    walls[:, 2] = bd.steric_force_mag(2 * z, 0.3, 1.0, 2, 0.3) - bd.steric_force_mag(2 * (2.0 - z), 0.3, 1.0, 2, 0.3)
    assert np.max(np.abs(np.sum(F - walls, axis=0))) < 1e-12 * np.max(np.abs(F))


def test_noise_free_step_is_euler():
    rng = np.random.default_rng(4)
    P = params.derive(3.0, 3.0, 2.0, 0.2, 1e-4, 16, 16, r_cut=1.0)
    pos = np.stack([rng.uniform(0, 3, 6), rng.uniform(0, 3, 6), rng.uniform(0.5, 1.5, 6)], 1)
    q = np.zeros(6)
    Fel = rng.standard_normal((6, 3))
    bp = dict(BP, kT=0.0, a=0.4, r_m=0.6, U0=0.01)
    new, Wn, r, ok = bd.step(pos, q, np.zeros((6, 3)), 0, P, bp, force=Fel)
    want = pos + bp["mu"] * bp["dt"] * (Fel + bd.steric_forces(pos, P, bp))
    want[:, :2] = np.mod(want[:, :2], 3.0)
    assert ok and r == 0 and np.allclose(new, want, rtol=0, atol=1e-15)


def test_free_diffusion_variance():
    # no forces: z_N - z_0 = sqrt(kT mu dt/2) (W^0 + 2 W^1 + ... + 2 W^{N-1} + W^N)
    P = params.derive(1e4, 1e4, 1e4, 0.2, 1e-4, 16, 16, r_cut=1.0)
    n, N = 2000, 6
    bp = dict(BP, a=1e-3, dt=0.01, kT=2.0, mu=0.5)
    rng = np.random.default_rng(8)
    pos0 = rng.uniform(1e3, 9e3, (n, 3))          # far apart: no steric contact
    pos, W = pos0.copy(), bd.normals(n, 0, 0, bp["seed"])
    zero = np.zeros((n, 3))
    for k in range(N):
        pos, W, r, ok = bd.step(pos, np.zeros(n), W, k, P, bp, force=zero)
        assert ok
    d = pos - pos0
    var = bp["kT"] * bp["mu"] * bp["dt"] * (4 * N - 2) / 2
    assert abs(np.mean(d * d) / var - 1.0) < 5 * np.sqrt(2.0 / d.size)


def test_displacement_cap_and_retries():
    P = params.derive(3.0, 3.0, 2.0, 0.2, 1e-4, 16, 16, r_cut=1.0)
    rng = np.random.default_rng(5)
    n = 50
    pos = np.stack([rng.uniform(0, 3, n), rng.uniform(0, 3, n), rng.uniform(0.5, 1.5, n)], 1)
    zero = np.zeros((n, 3))
    bp = dict(BP, a=1e-3, dt=1.0, max_disp=0.05)
    new, _, r, ok = bd.step(pos, np.zeros(n), zero, 0, P, bp, force=zero)
    d = new - pos
    d[:, :2] -= 3.0 * np.round(d[:, :2] / 3.0)
    assert ok and np.max(np.linalg.norm(d, axis=1)) <= 0.05 * (1 + 1e-12)
    # an ion next to the wall with a large step: some proposals leave the slab
    pos[0, 2] = 0.01
    bp = dict(BP, a=1e-3, dt=2e-3, max_retries=200)
    used = []
    for k in range(20):
        new, _, r, ok = bd.step(pos, np.zeros(n), zero, k, P, bp, force=zero)
        assert ok and 0 < new[0, 2] < 2.0
        used.append(r)
    assert max(used) > 0
    # every proposal leaves: nothing moves
    bp = dict(BP, a=1e-3, dt=10.0, max_retries=3)
    new, W, r, ok = bd.step(pos, np.zeros(n), zero, 3, P, bp, force=zero)
    assert not ok and r == 3 and np.array_equal(new, pos) and np.array_equal(W, zero)


def test_harmonic_stationary_variance_is_exact():
    # Eq. (leimkuhler) with F = -k z: z_{n+1} = c z_n + a (W_n + W_{n+1}),
    # c = 1 - mu k dt, a^2 = kT mu dt / 2, whose stationary variance is
    # a^2 (1 + (1 + c)^2 / (1 - c^2)) = kT / k for every dt; Euler-Maruyama
    # (noise sqrt(2 kT mu dt) W_n) would give kT / (k (1 - mu k dt / 2)),
    # 33% more at mu k dt = 0.5
    P = params.derive(1e4, 1e4, 1e4, 0.2, 1e-4, 16, 16, r_cut=1.0)
    n, steps, kspring = 1000, 100, 2.0
    bp = dict(BP, a=1e-3, dt=0.25, kT=1.5, mu=1.0, seed=77)
    rng = np.random.default_rng(10)
    centre = rng.uniform(1e3, 9e3, (n, 3))             # ions far apart: no steric contact
    pos, W = centre.copy(), bd.normals(n, 0, 0, bp["seed"])
    samples = []
    for k in range(steps):
        force = -kspring * (pos - centre)
        pos, W, r, ok = bd.step(pos, np.zeros(n), W, k, P, bp, force=force)
        assert ok
        if k >= 40:                                     # relaxation time 1/(mu k dt) = 2 steps
            samples.append((pos - centre).ravel())
    var = np.var(np.concatenate(samples))
    want = bp["kT"] / kspring
    # 60 x 3000 correlated samples (relaxation in two steps): about 1e5
    # effective ones, a 0.5% standard error
    assert abs(var / want - 1.0) < 0.02
    em = want / (1.0 - bp["mu"] * kspring * bp["dt"] / 2.0)
    assert abs(var / em - 1.0) > 0.2
