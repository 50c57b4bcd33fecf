"""Launch-shape autotuning (dpslab_plan_autotune / set_tuning / tuning):
the knobs change block shapes only, so results are unchanged; invalid knobs
are refused without changing anything; the cache serves a second plan of
the same grid."""
import os

import numpy as np
import pytest

from gpu_helpers import rel_l2
from paper_2101_07088_b300 import build, dpslab, synth, tuning

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _solve(plan, pt, qt):
    phi = torch.empty(qt.shape[0], dtype=torch.float64, device="cuda")
    f = torch.empty((qt.shape[0], 3), dtype=torch.float64, device="cuda")
    U, _ = plan.solve(pt, qt, phi, f)
    return U, f.cpu().numpy()


@pytest.mark.parametrize("prec", [dpslab.FP64, dpslab.MIXED], ids=["fp64", "mixed"])
def test_autotune_keeps_results(prec, tmp_path):
    pos, q, p = synth.workload("c2_jumps_n16384")
    plan = dpslab.Plan(dpslab.make_params(precision=prec, **p), len(q))
    pt = torch.tensor(pos, dtype=torch.float64, device="cuda")
    qt = torch.tensor(q, dtype=torch.float64, device="cuda")
    U0, f0 = _solve(plan, pt, qt)
    k0 = plan.tuning()
    knobs = plan.autotune(pt, qt, reps=2)
    assert all(v >= 1 for v in knobs)
    U1, f1 = _solve(plan, pt, qt)
    # mixed: the sources are bucketed by atomics, so the spreading's FP32
    # summation order (and the forces, by about 1e-6) differs between any two
    # solves; the bar is half the mixed force bar
    tol = 1e-12 if prec == dpslab.FP64 else 5e-6
    assert abs(U1 - U0) <= tol * abs(U0) and rel_l2(f1, f0) <= tol
    with pytest.raises(dpslab.DpslabError):
        plan.set_tuning([1 << 20, 1, 1, 1])
    assert plan.tuning() == knobs
    plan.set_tuning(k0)
    assert plan.tuning() == k0
    # the cache: a second plan of the same grid takes the stored knobs
    path = os.path.join(str(tmp_path), "tuning.json")
    kn, cached = tuning.tuned(plan, pt, qt, path, reps=2)
    assert not cached
    plan2 = dpslab.Plan(dpslab.make_params(precision=prec, **p), len(q))
    kn2, cached2 = tuning.tuned(plan2, pt, qt, path)
    assert cached2 and kn2 == kn and plan2.tuning() == kn


@pytest.mark.parametrize("prec", [dpslab.FP64, dpslab.MIXED], ids=["fp64", "mixed"])
def test_kernel_knobs_keep_results(prec):
    """Knobs 4-6 (interpolation warps per block, column-kernel modes per
    block, spreading columns per thread): every allowed value gives the same
    solve; values outside the kernels' shapes are refused with nothing
    changed."""
    pos, q = synth.electrolyte(600, 24.0, 20.0, 1.0, 19.0, seed=31)
    p = dict(Lx=24.0, Ly=20.0, H=20.0, gw=1.0, tol=1e-4, nx=48, ny=40, nz=37, eps_b=1 / 80, eps_t=0.5, r_cut=4.0)
    plan = dpslab.Plan(dpslab.make_params(precision=prec, **p), len(q))
    pt = torch.tensor(pos, dtype=torch.float64, device="cuda")
    qt = torch.tensor(q, dtype=torch.float64, device="cuda")
    k0 = plan.tuning()
    assert len(k0) == dpslab.NKNOBS
    U0, f0 = _solve(plan, pt, qt)
    tol = 1e-12 if prec == dpslab.FP64 else 5e-6
    # column kernel modes per block: the tensor-core form (this grid: Nz 37,
    # ny (nx/2+1) = 1000 even) 8, 16, 32; FP64 2, 4
    cols = (8, 16, 32) if prec == dpslab.MIXED else (2, 4)
    cpts = (1, 2, 4) if prec == dpslab.MIXED else (1,)
    for w in (1, 2, 4, 8):
        for cb in cols:
            for cpt in cpts:
                plan.set_tuning(k0[:4] + [w, cb, cpt])
                assert plan.tuning()[4:] == [w, cb, cpt]
                U1, f1 = _solve(plan, pt, qt)
                assert abs(U1 - U0) <= tol * abs(U0) and rel_l2(f1, f0) <= tol, (w, cb, cpt)
    plan.set_tuning(k0)
    for bad in ([3, k0[5], k0[6]], [k0[4], 64, k0[6]], [k0[4], k0[5], 3], [k0[4], k0[5], 8]) + (
            ([k0[4], k0[5], 2],) if prec == dpslab.FP64 else ()):
        with pytest.raises(dpslab.DpslabError):
            plan.set_tuning(k0[:4] + bad)
        assert plan.tuning() == k0
    # four knobs (the FFT shapes) are still accepted and leave the others
    plan.set_tuning(k0[:4])
    assert plan.tuning() == k0
    plan.close()


@pytest.mark.parametrize("prec", [dpslab.FP64, dpslab.MIXED], ids=["fp64", "mixed"])
def test_fft_knobs_on_ragged_rows_keep_results(prec):
    """Knobs 0-3 (rows or columns per block of the four power-of-two xy
    transforms) at 1, 2 and 4 on a 64 x 45 x 37 grid: 1665 rows, so the last
    block of 2 or 4 rows is partial (the inverse x transform pairs each
    row's two sequences on neighbouring lanes), and 33 columns along y; the
    solve is unchanged."""
    pos, q = synth.electrolyte(300, 32.0, 22.5, 1.0, 19.0, seed=41)
    p = dict(Lx=32.0, Ly=22.5, H=20.0, gw=1.0, tol=1e-4, nx=64, ny=45, nz=37, eps_b=1 / 80, eps_t=0.5, r_cut=4.0)
    plan = dpslab.Plan(dpslab.make_params(precision=prec, **p), len(q))
    pt = torch.tensor(pos, dtype=torch.float64, device="cuda")
    qt = torch.tensor(q, dtype=torch.float64, device="cuda")
    k0 = plan.tuning()
    U0, f0 = _solve(plan, pt, qt)
    tol = 1e-12 if prec == dpslab.FP64 else 5e-6
    for which in range(4):
        for v in (1, 2, 4):
            k = list(k0)
            k[which] = v
            plan.set_tuning(k)
            U1, f1 = _solve(plan, pt, qt)
            assert abs(U1 - U0) <= tol * abs(U0) and rel_l2(f1, f0) <= tol, (which, v)
    plan.set_tuning(k0)
    plan.close()
