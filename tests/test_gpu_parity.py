"""CUDA path vs the FP64 oracle, element by element (needs a B300).

Every case runs the oracle and the C-ABI library on the same seeded inputs
with identical derived parameters and requires relative errors below 1e-10
(forces: relative L2; energy: relative; potentials: max error over max
value). Stage outputs (densities, grid fields, far and near parts) are
compared too, so a failure names the stage."""
import math

import numpy as np
import pytest

from gpu_helpers import TOL_FP64, compare, gpu_solve, oracle_params, plan_for, rel_l2, rel_max
from oracle import solver as osolver
from paper_2101_07088_b300 import build, dpslab, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _charges(n, Lx, Ly, H, seed, zlo=1.0):
    return synth.electrolyte(n, Lx, Ly, zlo, H - zlo, seed)


GRID_TOL = 1e-8


def _stages(plan, ref, n, pos, HE, tol=TOL_FP64):
    """Stage outputs, to say which stage a failure comes from.

    The grid fields are compared on the z nodes the interpolation reads
    (within H_E of a charge) with GRID_TOL: at the outermost of these nodes
    the correction of a mode with |k| near k_max is its boundary mismatch
    (a short, strongly cancelling Chebyshev sum, accurate only to ~1e-16 of
    the largest coefficient) times e^{k |z|} ~ 1e9, so the two
    implementations differ there by ~1e-9 of the field's maximum. Those
    nodes reach the outputs with weight below e^{-n_sigma^2/2} and those
    modes are damped by the Gaussian, so the outputs still agree to 1e-14;
    the outputs are held to TOL_FP64."""
    rho = plan.debug_fetch(0, n)
    assert rel_max(rho[0], ref["rho_i"]) < 1e-13
    if np.max(np.abs(ref["rho_o"])) > 0:
        assert rel_max(rho[1], ref["rho_o"]) < 1e-13
    f = plan.debug_fetch(1, n)
    zn = ref["zn"]
    used = (zn >= pos[:, 2].min() - HE) & (zn <= pos[:, 2].max() + HE)
    for c in range(4):
        assert rel_max(f[used][..., c], ref["fields"][c][used]) < GRID_TOL, c
    far = plan.debug_fetch(2, n)
    assert rel_max(far, ref["far"]) < tol
    near = plan.debug_fetch(3, n)
    if np.max(np.abs(ref["phin"])) > 0:
        assert rel_max(near[:, 0], ref["phin"]) < tol
        assert rel_max(near[:, 1:], ref["En"]) < tol


SMALL = [
    # name, box (Lx, Ly, H), grid (nx, ny, nz), eps_b, eps_t, n, extra params
    ("uniform-c1", (32.0, 32.0, 32.0), (64, 64, 64), 1.0, 1.0, 128, {}),
    ("ragged-jumps", (24.0, 20.0, 20.0), (48, 40, 37), 1 / 80, 0.5, 102, {}),
    ("metal-bottom", (16.0, 16.0, 16.0), (32, 32, 40), math.inf, 1 / 80, 64, {}),
    ("metal-top", (16.0, 16.0, 16.0), (32, 32, 40), 0.3, math.inf, 64, {}),
    ("two-metal", (16.0, 16.0, 16.0), (30, 36, 41), math.inf, math.inf, 64, {}),
    ("no-split", (16.0, 16.0, 16.0), (32, 32, 48), 1 / 80, 1 / 20, 40, dict(xi=math.inf)),
    ("tol5e-4", (20.0, 20.0, 14.0), (40, 40, 33), 1 / 20, 1 / 50, 80, dict(tol=5e-4)),
    ("radix-3-7", (21.0, 28.0, 16.0), (42, 56, 33), 1 / 80, 1 / 10, 90, {}),
]


@pytest.mark.parametrize("name,box,grid,eb,et,n,extra", SMALL, ids=[c[0] for c in SMALL])
def test_small_cases(name, box, grid, eb, et, n, extra):
    Lx, Ly, H = box
    pos, q = _charges(n, Lx, Ly, H, seed=sum(map(ord, name)))
    kw = dict(r_cut=4.0) if "xi" not in extra else {}
    kw.update(extra)
    tol = kw.pop("tol", 1e-4)
    P = oracle_params(Lx, Ly, H, 1.0, tol, grid[0], grid[1], nz=grid[2], eps_b=eb, eps_t=et, **kw)
    ref = osolver.solve(pos, q, P)
    plan = plan_for(P, n)
    out = gpu_solve(plan, pos, q)
    assert out["rc"] == 0
    _stages(plan, ref, n, pos, P["HE"])
    compare(ref, out)
    s = plan.debug_fetch(4, n)
    assert s[1] == pytest.approx(ref["Ai"], rel=1e-10, abs=1e-12 * abs(ref["Ai"]) + 1e-300)
    assert s[0] == pytest.approx(ref["B"], rel=1e-9)


def test_paper_rule_regime():
    """Sec. 6.3 set-up (paper rule, g_w = 0.01, near field dominating, radix-19
    FFT of the 38-point grid)."""
    P = oracle_params(2.0, 2.0, 1.0, 0.01, 1e-4, 38, 38, eps_b=0.05, eps_t=0.02)
    pos, q = synth.electrolyte(40, 2.0, 2.0, 4.5 * 0.01, 1.0 - 4.5 * 0.01, seed=5)
    ref = osolver.solve(pos, q, P)
    plan = plan_for(P, 40)
    out = gpu_solve(plan, pos, q)
    _stages(plan, ref, 40, pos, P["HE"])
    compare(ref, out)


def test_free_space_grid_radix59():
    """Sec. 6.1 set-up: the 236 x 236 x 84 grid (236 = 4 x 59)."""
    P = oracle_params(28.0, 28.0, 2.0, 0.01, 1e-4, 236, 236, eps_b=0.5, eps_t=0.2)
    pos = np.array([[-0.17, -0.71, 0.01], [0.44, -0.82, 0.30], [-1.00, -0.63, 1.00], [-0.40, -0.31, 1.95]])
    q = np.array([1.0, -1.0, 1.0, -1.0])
    ref = osolver.solve(pos, q, P)
    plan = plan_for(P, 4)
    out = gpu_solve(plan, pos, q)
    compare(ref, out)


@pytest.mark.parametrize("name", ["c2_jumps_n16384", "c2_metal_bottom_n16384"])
def test_full_size_benchmark_workload(name):
    """The 16384-charge, 256 x 256 x 128 workload at full size, every output."""
    pos, q, p = synth.workload(name)
    P = oracle_params(p["Lx"], p["Ly"], p["H"], p["gw"], p["tol"], p["nx"], p["ny"], nz=p["nz"],
                      eps_b=p["eps_b"], eps_t=p["eps_t"], r_cut=p["r_cut"])
    ref = osolver.solve(pos, q, P)
    plan = plan_for(P, len(q))
    out = gpu_solve(plan, pos, q)
    _stages(plan, ref, len(q), pos, P["HE"])
    compare(ref, out)


def test_edge_charges():
    """Two charges; charges on top of each other (r = 0 between different
    charges, Taylor branch); charges a hair from the walls and from the
    periodic boundary; negative and out-of-box x, y (wrapped)."""
    Lx, Ly, H = 16.0, 16.0, 16.0
    P = oracle_params(Lx, Ly, H, 1.0, 1e-4, 32, 32, nz=40, eps_b=1 / 80, eps_t=0.25, r_cut=4.0)
    pos = np.array([[1e-12, 3.0, 1e-9], [16.0 - 1e-12, 3.0, 16.0 - 1e-9],
                    [5.0, 5.0, 8.0], [5.0, 5.0, 8.0],
                    [-3.0, 20.0, 2.0], [7.5, -0.25, 14.0]])
    q = np.array([1.0, -1.0, 1.0, -1.0, 1.0, -1.0])
    ref = osolver.solve(pos, q, P)
    plan = plan_for(P, 16)
    compare(ref, gpu_solve(plan, pos, q))
    # two opposite charges at one point: every force and the energy vanish
    ref2 = osolver.solve(pos[2:4], q[2:4], P)
    out2 = gpu_solve(plan, pos[2:4], q[2:4])
    assert np.max(np.abs(ref2["force"])) < 1e-14 and abs(ref2["U"]) < 1e-14
    assert np.max(np.abs(out2["force"])) < 1e-14 and abs(out2["U"]) < 1e-14
    assert np.max(np.abs(out2["phi"] - ref2["phi"])) <= 1e-10 * max(np.max(np.abs(ref2["phi"])), 1e-3)


def test_errors_do_not_fault_and_plan_recovers():
    Lx = H = 16.0
    P = oracle_params(Lx, Lx, H, 1.0, 1e-4, 32, 32, nz=40, eps_b=1 / 80, eps_t=1 / 80, r_cut=4.0)
    plan = plan_for(P, 8)
    pos, q = _charges(8, Lx, Lx, H, seed=3)
    bad = pos.copy()
    bad[2, 2] = H + 1.0
    assert gpu_solve(plan, bad, q, check=False)["rc"] == -3
    bad[2, 2] = float("nan")
    assert gpu_solve(plan, bad, q, check=False)["rc"] == -3
    qq = q.copy()
    qq[0] += 0.5
    assert gpu_solve(plan, pos, qq, check=False)["rc"] == -2
    with pytest.raises(dpslab.DpslabError) as e:
        gpu_solve(plan, np.zeros((9, 3)) + 1.0, np.zeros(9))
    assert e.value.code == -6
    ref = osolver.solve(pos, q, P)
    compare(ref, gpu_solve(plan, pos, q))


def test_host_entry_point_matches_device_one():
    pos, q, p = synth.workload("c1_uniform_n128")
    P = oracle_params(p["Lx"], p["Ly"], p["H"], p["gw"], p["tol"], p["nx"], p["ny"], nz=p["nz"],
                      eps_b=p["eps_b"], eps_t=p["eps_t"], r_cut=p["r_cut"])
    plan = plan_for(P, len(q))
    a = gpu_solve(plan, pos, q)
    U, phi, force, rc = plan.solve_host(pos, q)
    assert rc == 0
    assert abs(U - a["U"]) <= 1e-13 * abs(a["U"])
    assert np.allclose(phi, a["phi"], rtol=0, atol=1e-13 * np.max(np.abs(a["phi"])))
    assert np.allclose(force, a["force"], rtol=0, atol=1e-13 * np.max(np.abs(a["force"])))
    assert plan.last_launch_count() >= 10
    # caller-owned (pinned) output buffers give the same result; a wrongly
    # shaped buffer is refused before any copy
    pin_phi = torch.empty(len(q), dtype=torch.float64, pin_memory=True).numpy()
    pin_force = torch.empty((len(q), 3), dtype=torch.float64, pin_memory=True).numpy()
    U2, phi2, force2, rc = plan.solve_host(pos, q, phi=pin_phi, force=pin_force)
    assert rc == 0 and phi2 is pin_phi and force2 is pin_force
    assert abs(U2 - U) <= 1e-13 * abs(U)
    assert np.allclose(phi2, phi, rtol=0, atol=1e-13 * np.max(np.abs(phi)))
    assert np.allclose(force2, force, rtol=0, atol=1e-13 * np.max(np.abs(force)))
    with pytest.raises(ValueError):
        plan.solve_host(pos, q, force=np.empty((len(q), 2)))


@pytest.mark.parametrize("prec", [dpslab.FP64, dpslab.MIXED], ids=["fp64", "mixed"])
def test_concurrent_near_field_matches_in_line(prec):
    # unprofiled solves run the near field on the plan's second stream
    # (forked after the cell list, joined before the assembly); profiled
    # solves run it in line. Both give the oracle's result, and each other's
    # to rounding (the spreading's summation order may differ between runs).
    pos, q, p = synth.workload("c1_uniform_n128")
    P = oracle_params(p["Lx"], p["Ly"], p["H"], p["gw"], p["tol"], p["nx"], p["ny"], nz=p["nz"],
                      eps_b=p["eps_b"], eps_t=p["eps_t"], r_cut=p["r_cut"])
    plan = plan_for(P, len(q), precision=prec)
    plan.profile(True, near_in_line=True)
    a = gpu_solve(plan, pos, q)
    plan.profile(False)
    b = gpu_solve(plan, pos, q)
    plan.profile(True)        # stage timing of the concurrent form: same results
    c = gpu_solve(plan, pos, q)
    assert plan.stage_times()["near"] > 0.0
    plan.profile(False)
    assert rel_max(c["force"], b["force"]) < (1e-13 if prec == dpslab.FP64 else 1e-6)
    tol = 1e-13 if prec == dpslab.FP64 else 1e-6
    assert abs(a["U"] - b["U"]) <= tol * abs(a["U"])
    assert rel_max(b["phi"], a["phi"]) < tol and rel_max(b["force"], a["force"]) < tol
    if prec == dpslab.FP64:
        compare(osolver.solve(pos, q, P), b, TOL_FP64)


# The power-of-two FFT kernels are compiled once per size (n = 32 .. 4096):
# thin boxes reach the sizes the other cases do not (128, 512, 1024, 2048,
# 4096 in x and in y, with 32 at the other extreme), in both precisions.
# n = 1024 is the size of the 2^20-charge workload's 1024 x 1024 grid.
P2_SIZES = [
    ("x4096-y32", (2048.0, 16.0, 12.0), (4096, 32, 33)),
    ("x32-y4096", (16.0, 2048.0, 12.0), (32, 4096, 33)),
    ("x2048-y128", (1024.0, 64.0, 12.0), (2048, 128, 33)),
    ("x128-y512", (64.0, 256.0, 12.0), (128, 512, 33)),
    ("x1024-y32", (512.0, 16.0, 12.0), (1024, 32, 33)),
    ("x32-y1024", (16.0, 512.0, 12.0), (32, 1024, 33)),
    ("x1024-y64", (512.0, 32.0, 12.0), (1024, 64, 33)),
]


@pytest.mark.parametrize("name,box,grid", P2_SIZES, ids=[c[0] for c in P2_SIZES])
def test_fft_size_instances(name, box, grid):
    from gpu_helpers import TOL_MIXED_FORCE, mixed_energy_tol
    Lx, Ly, H = box
    n = 64
    pos, q = _charges(n, Lx, Ly, H, seed=sum(map(ord, name)))
    P = oracle_params(Lx, Ly, H, 1.0, 1e-4, grid[0], grid[1], nz=grid[2], eps_b=1 / 80, eps_t=1 / 40, r_cut=4.0)
    ref = osolver.solve(pos, q, P)
    compare(ref, gpu_solve(plan_for(P, n), pos, q))
    out = gpu_solve(plan_for(P, n, precision=dpslab.MIXED), pos, q)
    assert rel_l2(out["force"], ref["force"]) < TOL_MIXED_FORCE
    assert abs(out["U"] - ref["U"]) < mixed_energy_tol(P, n) * abs(ref["U"])
