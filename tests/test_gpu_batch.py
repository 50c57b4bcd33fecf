"""Batches of independent systems (dpslab_batch_*): every system's result in
the batch equals its result alone (the same kernels; only the order of
floating-point additions inside the spreading buckets may differ), also when
the captured graph is replayed with new values in the same buffers, and a
bad system reports its own status without affecting the others."""
import numpy as np
import pytest

from gpu_helpers import TOL_MIXED_ENERGY, TOL_MIXED_FORCE, rel_l2
from paper_2101_07088_b300 import build, dpslab, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _systems(count, seed):
    # the batched workload's recipe at small sizes (N_z from the paper's rule)
    return synth.batch_systems(count, seed, n_range=(64, 2048), l_range=(16.0, 40.0), h_range=(12.0, 30.0))


def _tensors(pos, q):
    dev = torch.device("cuda:0")
    return (torch.tensor(pos, dtype=torch.float64, device=dev), torch.tensor(q, dtype=torch.float64, device=dev),
            torch.empty(len(q), dtype=torch.float64, device=dev),
            torch.empty((len(q), 3), dtype=torch.float64, device=dev))


def _alone(pos, q, p, prec):
    plan = dpslab.Plan(dpslab.make_params(precision=prec, **p), len(q))
    pt, qt, phi, f = _tensors(pos, q)
    U, _ = plan.solve(pt, qt, phi, f)
    plan.close()
    return U, phi.cpu().numpy(), f.cpu().numpy()


@pytest.mark.parametrize("schedule", [dpslab.BATCH_STREAMS, dpslab.BATCH_WAVES], ids=["streams", "waves"])
@pytest.mark.parametrize("prec,ftol,utol", [(dpslab.FP64, 1e-12, 1e-12), (dpslab.MIXED, TOL_MIXED_FORCE, TOL_MIXED_ENERGY)],
                         ids=["fp64", "mixed"])
def test_batch_equals_alone_and_replays(prec, ftol, utol, schedule):
    systems = _systems(7, 11)
    params = [dpslab.make_params(precision=prec, **p) for _, _, p in systems]
    batch = dpslab.Batch(params, [len(q) for _, q, _ in systems], nstreams=3)
    batch.set_schedule(schedule)
    bufs = [_tensors(pos, q) for pos, q, _ in systems]
    for rnd in range(2):
        if rnd == 1:
            # new charges in the same buffers: the captured graph is replayed
            systems = [(synth.electrolyte(len(q), p["Lx"], p["Ly"], 1.0, p["H"] - 1.0, 100 + i)[0], q, p)
                       for i, (_, q, p) in enumerate(systems)]
            for (pos, _, _), (pt, _, _, _) in zip(systems, bufs):
                pt.copy_(torch.tensor(pos, dtype=torch.float64))
        U, status = batch.solve([b[0] for b in bufs], [b[1] for b in bufs], [b[2] for b in bufs],
                                [b[3] for b in bufs])
        assert (status == 0).all(), status
        for i, (pos, q, p) in enumerate(systems):
            U1, phi1, f1 = _alone(pos, q, p, prec)
            assert abs(U[i] - U1) <= utol * abs(U1), (rnd, i, U[i], U1)
            assert rel_l2(bufs[i][3].cpu().numpy(), f1) <= ftol, (rnd, i)
            assert np.max(np.abs(bufs[i][2].cpu().numpy() - phi1)) <= max(ftol, 1e-6) * np.max(np.abs(phi1)), (rnd, i)
    batch.close()


def test_batch_reports_each_systems_status():
    systems = _systems(3, 5)
    params = [dpslab.make_params(precision=dpslab.MIXED, **p) for _, _, p in systems]
    batch = dpslab.Batch(params, [len(q) for _, q, _ in systems], nstreams=2)
    bufs = [_tensors(pos, q) for pos, q, _ in systems]
    bufs[1][0][0, 2] = -1.0                       # system 1: a charge below the slab
    U, status = batch.solve([b[0] for b in bufs], [b[1] for b in bufs], [b[2] for b in bufs],
                            [b[3] for b in bufs], check=False)
    assert status[0] == dpslab.OK and status[2] == dpslab.OK
    assert status[1] == dpslab.ERR_OUT_OF_SLAB, status
    assert np.isfinite(U[0]) and np.isfinite(U[2])
    batch.close()


def test_batch_shares_workspaces_by_stream():
    systems = _systems(8, 7)
    params = [dpslab.make_params(precision=dpslab.MIXED, **p) for _, _, p in systems]
    mx = [len(q) for _, q, _ in systems]
    one = sum(dpslab.Plan(pp, m).device_bytes for pp, m in zip(params, mx))
    b2 = dpslab.Batch(params, mx, nstreams=2)
    b8 = dpslab.Batch(params, mx, nstreams=8)
    # two shared workspaces need less than eight, and eight (one per system)
    # need about what eight separate plans do
    assert b2.device_bytes < b8.device_bytes <= one * 1.01 + 1
    b2.close()
    b8.close()


def _column_kind(plan_params, prec):
    """The column kernel of one system solved alone (one launch): FP64; mixed
    with CUDA-core z transforms; or mixed with tensor-core z transforms
    (Nz <= 256 and ny (nx/2 + 1) even), whose kernel shape is 8 W modes per
    block and R rows per lane, W the largest of 4, 2, 1 whose shared memory
    lets two blocks share an SM. A wave launches once per distinct kind."""
    if prec == dpslab.FP64:
        return ("fp64",)
    d = dpslab.derive(plan_params)
    nz = d["nz"]
    if not (nz <= 256 and (d["ny"] * (d["nx"] // 2 + 1)) % 2 == 0):
        return ("simt",)
    smem = lambda w: 8 * w * (nz | 1) * 24 + 15 * nz * 4
    w = next((w for w in (4, 2, 1) if 2 * (smem(w) + 1024) <= 228 * 1024), 1)
    return ("tensor", w, 4 if nz <= 128 else 8)


@pytest.mark.parametrize("prec,ftol,utol", [(dpslab.FP64, 1e-12, 1e-12), (dpslab.MIXED, TOL_MIXED_FORCE, TOL_MIXED_ENERGY)],
                         ids=["fp64", "mixed"])
@pytest.mark.parametrize("nstreams", [2, 9])
def test_batch_column_stage_is_one_launch_per_wave(prec, ftol, utol, nstreams):
    """The per-mode column stage (BVP and correction) of every system of a
    wave runs as one launch per kind of column kernel: the batch launches
    the per-system kernels of the systems solved alone, less their column
    launches, plus one column launch per kind and wave. Results equal the
    systems solved alone."""
    systems = _systems(9, 21)
    params = [dpslab.make_params(precision=prec, **p) for _, _, p in systems]
    batch = dpslab.Batch(params, [len(q) for _, q, _ in systems], nstreams=nstreams)
    batch.set_schedule(dpslab.BATCH_WAVES)
    bufs = [_tensors(pos, q) for pos, q, _ in systems]
    U, status = batch.solve([b[0] for b in bufs], [b[1] for b in bufs], [b[2] for b in bufs], [b[3] for b in bufs])
    assert (status == 0).all(), status
    alone_launches, kinds = 0, []
    for i, (pos, q, p) in enumerate(systems):
        plan = dpslab.Plan(params[i], len(q))
        pt, qt, phi, f = _tensors(pos, q)
        U1, _ = plan.solve(pt, qt, phi, f)
        alone_launches += plan.last_launch_count()
        plan.close()
        kinds.append((i // nstreams,) + _column_kind(params[i], prec))
        assert abs(U[i] - U1) <= utol * abs(U1), (i, U[i], U1)
        assert rel_l2(bufs[i][3].cpu().numpy(), f.cpu().numpy()) <= ftol, i
    col_alone, per_wave = len(systems), len(set(kinds))
    assert batch.last_launch_count() == alone_launches - col_alone + per_wave, \
        (batch.last_launch_count(), alone_launches, col_alone, per_wave)
    batch.close()


def test_batch_autotune_picks_a_schedule():
    """dpslab_batch_autotune times both schedules and keeps one; the batch
    then still equals its systems solved alone. Unknown schedules are
    refused."""
    systems = _systems(5, 17)
    params = [dpslab.make_params(precision=dpslab.MIXED, **p) for _, _, p in systems]
    batch = dpslab.Batch(params, [len(q) for _, q, _ in systems], nstreams=5)
    bufs = [_tensors(pos, q) for pos, q, _ in systems]
    assert batch.schedule() == dpslab.BATCH_STREAMS
    kept = batch.autotune([b[0] for b in bufs], [b[1] for b in bufs], reps=2)
    assert kept in (dpslab.BATCH_STREAMS, dpslab.BATCH_WAVES) and batch.schedule() == kept
    U, status = batch.solve([b[0] for b in bufs], [b[1] for b in bufs], [b[2] for b in bufs], [b[3] for b in bufs])
    assert (status == 0).all()
    for i, (pos, q, p) in enumerate(systems):
        U1, _, f1 = _alone(pos, q, p, dpslab.MIXED)
        assert abs(U[i] - U1) <= TOL_MIXED_ENERGY * abs(U1)
        assert rel_l2(bufs[i][3].cpu().numpy(), f1) <= TOL_MIXED_FORCE
    with pytest.raises(dpslab.DpslabError):
        batch.set_schedule(7)
    assert batch.schedule() == kept
    batch.close()
