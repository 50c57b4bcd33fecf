"""The allocation-free near-field entry point (needs a B300).

dpslab_near_field_static serves callers that cannot call cudaMalloc (code
running inside an allocator, under a memory pool that must not grow, or in
a loop that reserves everything at start-up): its scratch space is a
file-scope device array. Here its output is checked against the near-field
part that the planned entry point dpslab_solve computes, and directly
against the oracle's near field, each on two calls in a row (the array keeps
the previous call's contents, so the second call also checks that the
library clears what it must). This file is collected last.
"""
import numpy as np
import pytest

from gpu_helpers import TOL_FP64, gpu_solve, oracle_params, plan_for, rel_max
from oracle import solver as osolver
from paper_2101_07088_b300 import build, dpslab, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _params(P):
    return dpslab.make_params(Lx=P["Lx"], Ly=P["Ly"], H=P["H"], gw=P["gw"], tol=P["tol"], nx=P["nx"],
                              ny=P["ny"], nz=P["nz"], eps=P["eps"], eps_b=P["eps_b"], eps_t=P["eps_t"],
                              xi=P["xi"], r_cut=P["r_cut"], n_sigma=P["n_sigma"])


def _static(params, pos, q):
    dev = torch.device("cuda")
    pt = torch.tensor(pos, dtype=torch.float64, device=dev)
    qt = torch.tensor(q, dtype=torch.float64, device=dev)
    out = torch.full((len(q), 4), float("nan"), dtype=torch.float64, device=dev)
    rc = dpslab.near_field_static(params, pt, qt, out, check=False)
    return rc, out.cpu().numpy()


def test_static_near_field_matches_planned_solve_twice():
    cases = []
    pos, q, p = synth.workload("c2_jumps_n16384")
    cases.append((pos, q, p))
    pos2, q2 = synth.electrolyte(4096, p["Lx"], p["Ly"], 1.0, p["H"] - 1.0, seed=77)
    cases.append((pos2, q2, p))
    for pos, q, p in cases:        # two calls in a row, different inputs
        P = oracle_params(p["Lx"], p["Ly"], p["H"], p["gw"], p["tol"], p["nx"], p["ny"], nz=p["nz"],
                          eps_b=p["eps_b"], eps_t=p["eps_t"], r_cut=p["r_cut"])
        plan = plan_for(P, len(q))
        assert gpu_solve(plan, pos, q)["rc"] == 0
        ref = plan.debug_fetch(3, len(q))
        plan.close()
        rc, got = _static(_params(P), pos, q)
        assert rc == 0
        assert rel_max(got[:, 0], ref[:, 0]) < TOL_FP64
        assert rel_max(got[:, 1:], ref[:, 1:]) < TOL_FP64


def test_static_near_field_matches_oracle():
    """The same entry point held directly to the oracle's near field (the
    plain double loop over all pairs and one image per wall), on a small
    box with unequal walls: two calls in a row with different charges."""
    P = oracle_params(24.0, 20.0, 20.0, 1.0, 1e-4, 48, 40, nz=37, eps_b=1 / 80, eps_t=0.5, r_cut=4.0)
    for n, seed in ((300, 41), (518, 42)):
        pos, q = synth.electrolyte(n, 24.0, 20.0, 1.0, 19.0, seed=seed)
        phin, En = osolver.near_field(pos[:, 0], pos[:, 1], pos[:, 2], q, P, method="pairs")
        rc, got = _static(_params(P), pos, q)
        assert rc == 0
        assert rel_max(got[:, 0], phin) < TOL_FP64
        assert rel_max(got[:, 1:], En) < TOL_FP64


def test_static_near_field_rejects_oversize_inputs():
    pos, q, p = synth.workload("c2_jumps_n16384")
    P = oracle_params(p["Lx"], p["Ly"], p["H"], p["gw"], p["tol"], p["nx"], p["ny"], nz=p["nz"],
                      eps_b=p["eps_b"], eps_t=p["eps_t"], r_cut=p["r_cut"])
    big_pos, big_q = synth.electrolyte(65538, p["Lx"], p["Ly"], 1.0, p["H"] - 1.0, seed=1)
    rc, _ = _static(_params(P), big_pos, big_q)
    assert rc == -6                                   # more than 65536 charges
    Pc = oracle_params(2048.0, 2048.0, p["H"], p["gw"], p["tol"], 4096, 4096, nz=p["nz"],
                       eps_b=p["eps_b"], eps_t=p["eps_t"], r_cut=p["r_cut"])
    rc, _ = _static(_params(Pc), pos, q)
    assert rc == -6                                   # 512 x 512 x 16 cells > 65536
