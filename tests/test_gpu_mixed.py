"""Mixed-precision path (DPSLAB_MIXED) vs the FP64 oracle and the FP64 GPU
path (needs a B300).

Targets: relative L2 force error <= 1e-5 and relative energy error <= 1e-7
against FP64 at the same discretisation; potentials are reported."""
import math

import numpy as np
import pytest

from gpu_helpers import (TOL_MIXED_ENERGY, TOL_MIXED_FORCE, gpu_solve, mixed_energy_tol, oracle_params, plan_for,
                         rel_l2, rel_max, rho_o_pair_launch)
from oracle import chebyshev as cheb
from oracle import solver as osolver
from paper_2101_07088_b300 import build, dpslab, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _check(ref, out, label, energy_tol=TOL_MIXED_ENERGY):
    errs = dict(force=rel_l2(out["force"], ref["force"]), U=abs(out["U"] - ref["U"]) / abs(ref["U"]),
                phi=rel_max(out["phi"], ref["phi"]))
    print(label, "mixed errors:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert errs["force"] < TOL_MIXED_FORCE, errs
    assert errs["U"] < energy_tol, errs
    return errs


CASES = [
    ("c1_uniform_n128", None),
    ("c2_jumps_n16384", None),
    ("c2_metal_bottom_n16384", None),
]


PRECISIONS = [(dpslab.MIXED, "tensor-z"), (dpslab.MIXED_SIMT, "simt-z")]


@pytest.mark.parametrize("prec,plabel", PRECISIONS, ids=[p[1] for p in PRECISIONS])
@pytest.mark.parametrize("name,_", CASES, ids=[c[0] for c in CASES])
def test_mixed_against_oracle(name, _, prec, plabel):
    pos, q, p = synth.workload(name)
    P = oracle_params(p["Lx"], p["Ly"], p["H"], p["gw"], p["tol"], p["nx"], p["ny"], nz=p["nz"],
                      eps_b=p["eps_b"], eps_t=p["eps_t"], r_cut=p["r_cut"])
    ref = osolver.solve(pos, q, P)
    out = gpu_solve(plan_for(P, len(q), precision=prec), pos, q)
    _check(ref, out, f"{name} {plabel}", mixed_energy_tol(P, len(q)))


def test_tensor_z_transform_runs():
    # Nz <= 128 with ny (nx/2+1) even: the z transforms run as two tensor-core
    # GEMM launches around the BVP kernel, and rho_o's coefficients (20 node
    # pairs here) as one CUDA-core launch: three launches more than the SIMT
    # form
    pos, q, p = synth.workload("c2_jumps_n16384")
    P = oracle_params(p["Lx"], p["Ly"], p["H"], p["gw"], p["tol"], p["nx"], p["ny"], nz=p["nz"],
                      eps_b=p["eps_b"], eps_t=p["eps_t"], r_cut=p["r_cut"])
    counts = {}
    for prec in (dpslab.MIXED, dpslab.MIXED_SIMT):
        plan = plan_for(P, len(q), precision=prec)
        gpu_solve(plan, pos, q)
        counts[prec] = plan.last_launch_count()
    assert counts[dpslab.MIXED] == counts[dpslab.MIXED_SIMT] + 3, counts


def test_mixed_small_ragged_and_paper_rule():
    P = oracle_params(24.0, 20.0, 20.0, 1.0, 1e-4, 48, 40, nz=37, eps_b=1 / 80, eps_t=0.5, r_cut=4.0)
    pos, q = synth.electrolyte(102, 24.0, 20.0, 1.0, 19.0, seed=3)
    _check(osolver.solve(pos, q, P), gpu_solve(plan_for(P, 102, precision=dpslab.MIXED), pos, q), "ragged",
           mixed_energy_tol(P, 102))
    P = oracle_params(2.0, 2.0, 1.0, 0.01, 1e-4, 38, 38, eps_b=0.05, eps_t=0.02)
    pos, q = synth.electrolyte(40, 2.0, 2.0, 0.045, 0.955, seed=5)
    _check(osolver.solve(pos, q, P), gpu_solve(plan_for(P, 40, precision=dpslab.MIXED), pos, q), "paper-rule",
           mixed_energy_tol(P, 40))


def test_mixed_without_split():
    # xi = inf: no near field, so no cell list; the sources and the
    # interpolation windows then follow the charges' own order
    P = oracle_params(16.0, 16.0, 16.0, 1.0, 1e-4, 32, 32, nz=48, eps_b=1 / 80, eps_t=1 / 20, xi=math.inf)
    pos, q = synth.electrolyte(40, 16.0, 16.0, 1.0, 15.0, seed=7)
    _check(osolver.solve(pos, q, P), gpu_solve(plan_for(P, 40, precision=dpslab.MIXED), pos, q), "no-split",
           mixed_energy_tol(P, 40))


@pytest.mark.parametrize("case", ["ragged", "c2"])
def test_interpolation_stage_against_oracle_quadrature(case):
    """The interpolation stage of the mixed form on its own (Sec. 5.2.2
    step 7): the far parts a solve returns (the warp-per-charge gather, with
    one and with eight warps per block) against the oracle's quadrature of
    the very grid fields that solve produced, widened to FP64. The ragged
    grid (48 x 40 x 37) has supports that wrap around the period; two
    charges of each sign get zero strength, whose potential still needs the
    far part."""
    if case == "ragged":
        P = oracle_params(24.0, 20.0, 20.0, 1.0, 1e-4, 48, 40, nz=37, eps_b=1 / 80, eps_t=0.5, r_cut=4.0)
        pos, q = synth.electrolyte(102, 24.0, 20.0, 1.0, 19.0, seed=3)
    else:
        pos, q, p = synth.workload("c2_jumps_n16384")
        P = oracle_params(p["Lx"], p["Ly"], p["H"], p["gw"], p["tol"], p["nx"], p["ny"], nz=p["nz"],
                          eps_b=p["eps_b"], eps_t=p["eps_t"], r_cut=p["r_cut"])
    q = np.array(q, dtype=float)
    zero = np.concatenate([np.nonzero(q > 0)[0][:2], np.nonzero(q < 0)[0][:2]])
    q[zero] = 0.0
    n = len(q)
    zn = cheb.nodes(P["nz"], P["a"], P["b"])
    wz = cheb.quadrature_weights(P["nz"], P["a"], P["b"])
    plan = plan_for(P, n, precision=dpslab.MIXED)
    k0 = plan.tuning()
    for knob in (1, 8):
        plan.set_tuning(k0[:4] + [knob] + k0[5:])
        out = gpu_solve(plan, pos, q)
        far = plan.debug_fetch(2, n)
        fields = np.moveaxis(plan.debug_fetch(1, n), -1, 0)
        ref = osolver.interpolate(fields, pos[:, 0], pos[:, 1], pos[:, 2], P, zn, wz)
        errs = [rel_max(far[:, c], ref[:, c]) for c in range(4)]
        print(case, "knob", knob, "far-part errors (phi, E):", [f"{e:.1e}" for e in errs])
        # FP32 fields and an FP32 quadrature: a few FP32 roundoff units of
        # the largest value
        assert max(errs) < 1e-6, (knob, errs)
        assert np.all(out["force"][zero] == 0.0)
    plan.close()


def test_mixed_against_fp64_gpu_at_one_million_charges():
    """2^20 charges, 1024 x 1024 x 128: the oracle would take hours, so the
    mixed path is compared with the FP64 GPU path (itself held to 1e-10
    against the oracle on every smaller case)."""
    pos, q, p = synth.workload("c3_jumps_n1048576")
    P = oracle_params(p["Lx"], p["Ly"], p["H"], p["gw"], p["tol"], p["nx"], p["ny"], nz=p["nz"],
                      eps_b=p["eps_b"], eps_t=p["eps_t"], r_cut=p["r_cut"])
    plan64 = plan_for(P, len(q))
    ref = gpu_solve(plan64, pos, q)
    plan64.close()
    plan32 = plan_for(P, len(q), precision=dpslab.MIXED)
    out = gpu_solve(plan32, pos, q)
    _check(ref, out, "c3")
    # zero net lateral force (walls push only along z) holds at any size
    s = np.sum(np.abs(out["force"][:, :2]))
    assert abs(np.sum(out["force"][:, 0])) < 1e-6 * s and abs(np.sum(out["force"][:, 1])) < 1e-6 * s


@pytest.mark.parametrize("ny,nz", [(39, 37), (40, 272)], ids=["odd-columns", "nz-272"])
def test_mixed_fallback_to_cuda_core_z_transform(ny, nz):
    # ny (nx/2+1) odd, or Nz > 256: DPSLAB_MIXED runs the z transforms on the
    # CUDA cores (same launch count as DPSLAB_MIXED_SIMT) and meets the same bar
    P = oracle_params(24.0, 20.0, 20.0, 1.0, 1e-4, 48, ny, nz=nz, eps_b=1 / 80, eps_t=0.5, r_cut=4.0)
    pos, q = synth.electrolyte(102, 24.0, 20.0, 1.0, 19.0, seed=4)
    ref = osolver.solve(pos, q, P)
    counts = {}
    for prec in (dpslab.MIXED, dpslab.MIXED_SIMT):
        plan = plan_for(P, 102, precision=prec)
        out = gpu_solve(plan, pos, q)
        counts[prec] = plan.last_launch_count()
        _check(ref, out, f"fallback ny={ny} nz={nz} prec={prec}", mixed_energy_tol(P, 102))
    assert counts[dpslab.MIXED] == counts[dpslab.MIXED_SIMT], counts


@pytest.mark.parametrize("nz", [136, 200, 256])
def test_tensor_z_transform_in_two_blocks(nz):
    # 128 < Nz <= 256: the z transforms run on the tensor cores in 2 x 2
    # blocks of 128 (two or three launches more than the CUDA-core form), within the
    # bar against the oracle and close to the CUDA-core form
    P = oracle_params(24.0, 20.0, 20.0, 1.0, 1e-4, 48, 40, nz=nz, eps_b=1 / 80, eps_t=0.5, r_cut=4.0)
    pos, q = synth.electrolyte(800, 24.0, 20.0, 1.0, 19.0, seed=8)
    ref = osolver.solve(pos, q, P)
    out, counts = {}, {}
    for prec in (dpslab.MIXED, dpslab.MIXED_SIMT):
        plan = plan_for(P, 800, precision=prec)
        out[prec] = gpu_solve(plan, pos, q)
        counts[prec] = plan.last_launch_count()
        _check(ref, out[prec], f"two blocks nz={nz} prec={prec}", mixed_energy_tol(P, 800))
    # plus rho_o's coefficients by their own launch when it reaches few nodes
    assert counts[dpslab.MIXED] == counts[dpslab.MIXED_SIMT] + 2 + rho_o_pair_launch(P), counts
    assert rel_l2(out[dpslab.MIXED]["force"], out[dpslab.MIXED_SIMT]["force"]) < TOL_MIXED_FORCE


@pytest.mark.parametrize("nz", [64, 200], ids=["one-block", "two-block"])
def test_bounded_wait_reports_timeout(nz):
    """The bounded waits of the tensor-core z transforms: with a limit of 0
    polls every wait gives up at once; the kernels then wait for their work in
    flight, free their tensor memory and return, and the solve reports
    DPSLAB_ERR_TIMEOUT. With the default limit the same plan solves again and
    matches a fresh plan."""
    P = oracle_params(24.0, 20.0, 20.0, 1.0, 1e-4, 48, 40, nz=nz, eps_b=1 / 80, eps_t=0.5, r_cut=4.0)
    pos, q = synth.electrolyte(200, 24.0, 20.0, 1.0, 19.0, seed=12)
    plan = plan_for(P, 200, precision=dpslab.MIXED)
    ref = gpu_solve(plan, pos, q)
    plan.set_wait_limit(0)
    with pytest.raises(dpslab.DpslabError) as e:
        gpu_solve(plan, pos, q)
    assert e.value.code == dpslab.ERR_TIMEOUT
    plan.set_wait_limit()
    again = gpu_solve(plan, pos, q)
    assert rel_l2(again["force"], ref["force"]) < 1e-6
    with pytest.raises(dpslab.DpslabError):
        plan.set_wait_limit(-1)
