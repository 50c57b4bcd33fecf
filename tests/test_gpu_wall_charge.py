"""Wall charge densities on the device (dpslab_plan_set_wall_charge) against
the oracle: the FP64 path to 1e-10, the mixed path within its bar against
FP64, on the oracle's pinned cases (capacitor, single Fourier modes, the
charged walls of Sec. 6.3) plus a ragged grid; setting and clearing,
the electroneutrality check with wall charges, metal walls refused."""
import numpy as np
import pytest

from gpu_helpers import (TOL_FP64, TOL_MIXED_ENERGY, TOL_MIXED_FORCE, compare, gpu_solve, mixed_energy_tol,
                         oracle_params, plan_for, rel_l2)
from oracle import solver as osolver
from paper_2101_07088_b300 import build, dpslab, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _gauss_walls(P, s, xc=0.0, yc=0.0):
    # +/- a periodic Gaussian of width s at (xc, yc), total +-1/2 (Sec. 6.3)
    x = np.arange(P["nx"]) * P["hx"] - xc
    y = np.arange(P["ny"]) * P["hy"] - yc
    x = x - P["Lx"] * np.round(x / P["Lx"])
    y = y - P["Ly"] * np.round(y / P["Ly"])
    X, Y = np.meshgrid(x, y)
    g = np.exp(-(X * X + Y * Y) / (2 * s * s)) / (2.0 * np.sqrt(4.0 * np.pi ** 2 * s ** 4))
    return g, -g


def _cases():
    out = []
    # charged walls of Sec. 6.3 (2 x 2 box, 38 x 38 x 87)
    P = oracle_params(2.0, 2.0, 1.0, 0.01, 1e-4, 38, 38, nz=87, xi=6.8, eps_b=1 / 20, eps_t=1 / 50)
    rng = np.random.default_rng(6)
    pos = np.stack([rng.uniform(0, 2, 10), rng.uniform(0, 2, 10), rng.uniform(0.045, 0.955, 10)], 1)
    q = np.array([1.0, -1.0] * 5)
    out.append(("sec63", P, pos, q, *_gauss_walls(P, 0.2)))
    # capacitor and a Fourier mode on a jump slab, ragged (non power-of-two) grid
    P = oracle_params(24.0, 20.0, 20.0, 1.0, 1e-4, 48, 40, nz=37, eps_b=1 / 80, eps_t=0.5, r_cut=4.0)
    pos, q = synth.electrolyte(102, 24.0, 20.0, 1.0, 19.0, seed=3)
    X, Y = np.meshgrid(np.arange(48) * P["hx"], np.arange(40) * P["hy"])
    s = 0.004
    out.append(("capacitor", P, pos, q, np.full((40, 48), s), np.full((40, 48), -s)))
    out.append(("modes", P, pos, q, s * np.cos(2 * np.pi * X / 24.0), 0.6 * s * np.cos(2 * np.pi * Y / 10.0 + 0.3)))
    # the 16384-charge jump workload with Gaussian walls
    pos, q, p = synth.workload("c2_jumps_n16384")
    P = oracle_params(p["Lx"], p["Ly"], p["H"], p["gw"], p["tol"], p["nx"], p["ny"], nz=p["nz"],
                      eps_b=p["eps_b"], eps_t=p["eps_t"], r_cut=p["r_cut"])
    sb, st = _gauss_walls(P, 6.0, 40.0, 70.0)
    out.append(("c2", P, pos, q, 60.0 * sb, 60.0 * st))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp64_wall_charges_match_oracle(case):
    name, P, pos, q, sb, st = case
    ref = osolver.solve(pos, q, P, sigma_b=sb, sigma_t=st)
    plan = plan_for(P, len(q))
    plan.set_wall_charge(sb, st)
    out = gpu_solve(plan, pos, q)
    compare(ref, out, TOL_FP64)
    # the wall term is a real part of the energy here
    assert abs(ref["wall"]["U_wall"]) > 1e-3 * abs(ref["U"])


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_mixed_wall_charges_match_fp64(case):
    name, P, pos, q, sb, st = case
    p64 = plan_for(P, len(q))
    p64.set_wall_charge(sb, st)
    ref = gpu_solve(p64, pos, q)
    p32 = plan_for(P, len(q), precision=dpslab.MIXED)
    p32.set_wall_charge(sb, st)
    out = gpu_solve(p32, pos, q)
    ef = rel_l2(out["force"], ref["force"])
    eu = abs(out["U"] - ref["U"]) / abs(ref["U"])
    print(name, f"mixed vs fp64: force {ef:.2e} energy {eu:.2e}")
    assert ef < TOL_MIXED_FORCE
    # few charges or few xy modes: the FP32 rounding level (mixed_energy_tol)
    assert eu < mixed_energy_tol(P, len(q))


def test_set_clear_launches_and_checks():
    name, P, pos, q, sb, st = CASES[1]
    plan = plan_for(P, len(q))
    base = gpu_solve(plan, pos, q)
    n0 = plan.last_launch_count()
    plan.set_wall_charge(sb, st)
    withs = gpu_solve(plan, pos, q)
    assert plan.last_launch_count() == n0 + 1               # one gather kernel per solve
    assert abs(withs["U"] - base["U"]) > 1e-3 * abs(base["U"])
    plan.set_wall_charge(None, None)
    again = gpu_solve(plan, pos, q)
    assert abs(again["U"] - base["U"]) <= 1e-13 * abs(base["U"]) and rel_l2(again["force"], base["force"]) < 1e-13
    # wall charges that break electroneutrality are reported
    plan.set_wall_charge(sb, None)
    assert gpu_solve(plan, pos, q, check=False)["rc"] == dpslab.ERR_NOT_NEUTRAL
    # a charge density on a metallic wall is not part of the method
    Pm = oracle_params(24.0, 20.0, 20.0, 1.0, 1e-4, 48, 40, nz=37, eps_b=np.inf, eps_t=0.5, r_cut=4.0)
    pm = plan_for(Pm, len(q))
    with pytest.raises(dpslab.DpslabError):
        pm.set_wall_charge(sb, st)
    pm.set_wall_charge(None, st * 0)                        # the dielectric wall may carry one
