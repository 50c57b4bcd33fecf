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
