"""Properties of the full-size (2^20-charge, 1024 x 1024 x 128) mixed solve
that hold at any size, where the oracle cannot follow (Sec. 2: the
problem's symmetries):
* a shift of every charge by whole grid spacings in x and y moves the
  spreading, the grid and the interpolation with it, so forces and energy
  are unchanged up to the FP32 rounding of the mixed path (the cell list,
  whose cells are 8 spacings wide, regroups the near-field pairs, and every
  grid value rounds differently); each of the two solves is within the
  mixed bar of the exact result, so they agree within twice the bar;
* with equal walls, mirroring z -> H - z maps the problem onto itself with
  F_z reversed and phi, F_x, F_y, U unchanged (again within twice the
  mixed bar: z and H - z round differently in float)."""
import numpy as np
import pytest

from gpu_helpers import TOL_MIXED_ENERGY, TOL_MIXED_FORCE, gpu_solve, oracle_params, plan_for, rel_l2
from paper_2101_07088_b300 import build, dpslab, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


@pytest.fixture(scope="module")
def c3():
    pos, q, p = synth.workload("c3_jumps_n1048576")
    P = oracle_params(p["Lx"], p["Ly"], p["H"], p["gw"], p["tol"], p["nx"], p["ny"], nz=p["nz"],
                      eps_b=p["eps_b"], eps_t=p["eps_t"], r_cut=p["r_cut"])
    plan = plan_for(P, len(q), precision=dpslab.MIXED)
    return plan, pos, q, P, gpu_solve(plan, pos, q)


def test_grid_aligned_shift(c3):
    plan, pos, q, P, base = c3
    sh = pos.copy()
    sh[:, 0] = np.mod(sh[:, 0] + 3 * P["hx"], P["Lx"])
    sh[:, 1] = np.mod(sh[:, 1] + 5 * P["hy"], P["Ly"])
    out = gpu_solve(plan, sh, q)
    assert rel_l2(out["force"], base["force"]) < 2 * TOL_MIXED_FORCE
    assert abs(out["U"] - base["U"]) < 2 * TOL_MIXED_ENERGY * abs(base["U"])


def test_mirror_between_equal_walls(c3):
    plan, pos, q, P, base = c3
    assert P["eps_b"] == P["eps_t"]
    mi = pos.copy()
    mi[:, 2] = P["H"] - mi[:, 2]
    out = gpu_solve(plan, mi, q)
    flipped = base["force"] * np.array([1.0, 1.0, -1.0])
    assert rel_l2(out["force"], flipped) < 2 * TOL_MIXED_FORCE
    assert abs(out["U"] - base["U"]) < 2 * TOL_MIXED_ENERGY * abs(base["U"])
