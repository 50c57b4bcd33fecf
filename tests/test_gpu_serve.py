"""Serving loop on the device: every request's result in the mix (other
replicas' solves overlapping on several streams, workspaces evicted and
re-admitted under a tight memory budget) equals the same request solved
alone, within the tolerance of its precision; the same kernels run, and only
the order of floating-point additions inside the spreading buckets may
differ."""
import numpy as np
import pytest

from gpu_helpers import TOL_MIXED_ENERGY, TOL_MIXED_FORCE, rel_l2
from paper_2101_07088_b300 import build, dpslab, synth
from paper_2101_07088_b300.serve import Request, Server, latency_stats

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _replicas(count, seed):
    # the served workload's recipe at small sizes
    return synth.serve_replicas(count, seed, n_range=(64, 3000), h_range=(12.0, 30.0))


def _inputs(rep, seed):
    dev = torch.device("cuda:0")
    pos, q = synth.electrolyte(rep["n"], rep["Lx"], rep["Ly"], 1.0, rep["H"] - 1.0, seed)
    n = rep["n"]
    return (torch.tensor(pos, dtype=torch.float64, device=dev), torch.tensor(q, dtype=torch.float64, device=dev),
            torch.empty(n, dtype=torch.float64, device=dev), torch.empty((n, 3), dtype=torch.float64, device=dev))


def _params(rep):
    return {k: v for k, v in rep.items() if k != "n"}


# the mixed path's sums over spreading buckets run in a different order from
# run to run; for these small systems (N <= 3000) that moves the energy at the
# FP32 noise level, 3e-7 (the larger workloads are held to 1e-7)
@pytest.mark.parametrize("prec,ftol,utol", [(dpslab.FP64, 1e-12, 1e-12), (dpslab.MIXED, TOL_MIXED_FORCE, 3e-7)],
                         ids=["fp64", "mixed"])
def test_each_result_is_the_same_alone_and_in_the_mix(prec, ftol, utol):
    reps = _replicas(9, 21)
    work = []
    for r in reps:
        pl = dpslab.Plan(dpslab.make_params(precision=prec, **_params(r)), r["n"], own_work=False)
        work.append(pl.work_bytes)
        pl.close()
    # room for about three workspaces: admissions wait and idle ones are evicted
    budget = int(sorted(work)[-1] + sorted(work)[-2] + sorted(work)[0])
    srv = Server(budget, nstreams=4, max_inflight=4, precision=prec)
    for i, r in enumerate(reps):
        srv.register(i, _params(r), r["n"])
    rng = np.random.default_rng(5)
    reqs = []
    for k, i in enumerate(rng.integers(0, len(reps), 30)):
        pos, q, phi, f = _inputs(reps[i], 1000 + k)
        reqs.append(Request(int(i), pos, q, phi, f, t_arrival=0.002 * k))
    done = srv.run(reqs, realtime=True, timeout_s=300)
    assert len(done) == 30 and all(r.code == dpslab.OK for r in done), [r.code for r in done]
    assert srv.stats["evictions"] > 0 and srv.peak_ws_bytes <= budget
    print(latency_stats(done), dict(srv.stats))
    for req in done:
        r = reps[req.replica]
        plan = dpslab.Plan(dpslab.make_params(precision=prec, **_params(r)), r["n"])
        phi1 = torch.empty_like(req.phi)
        f1 = torch.empty_like(req.force)
        U1, _ = plan.solve(req.pos, req.q, phi1, f1)
        plan.close()
        assert abs(req.U - U1) <= utol * abs(U1), (req.replica, req.U, U1)
        assert rel_l2(req.force.cpu().numpy(), f1.cpu().numpy()) <= ftol
        p0, p1 = req.phi.cpu().numpy(), phi1.cpu().numpy()
        assert np.max(np.abs(p0 - p1)) <= max(ftol, 1e-6) * np.max(np.abs(p1))
    srv.close()


def test_unbound_plan_refuses_to_solve_and_checks_its_workspace():
    r = _replicas(1, 3)[0]
    plan = dpslab.Plan(dpslab.make_params(precision=dpslab.MIXED, **_params(r)), r["n"], own_work=False)
    pos, q, phi, f = _inputs(r, 7)
    with pytest.raises(dpslab.DpslabError):
        plan.solve(pos, q, phi, f)                       # nothing bound
    small = torch.empty(plan.work_bytes - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(dpslab.DpslabError):
        plan.bind_work(small)
    plan.bind_work(torch.empty(plan.work_bytes, dtype=torch.uint8, device="cuda"))
    U, _ = plan.solve(pos, q, phi, f)
    own = dpslab.Plan(dpslab.make_params(precision=dpslab.MIXED, **_params(r)), r["n"])
    U1, _ = own.solve(pos, q, torch.empty_like(phi), torch.empty_like(f))
    assert abs(U - U1) <= 3e-7 * abs(U1)                # FP32 noise of a small system, as above
    with pytest.raises(dpslab.DpslabError):
        own.bind_work(None)                              # owns its workspace
    # the host-side footprint matches what a plan takes
    assert dpslab.plan_bytes(own.params, r["n"]) == own.device_bytes
    plan.close()
    own.close()


def test_enqueue_poll_matches_solve():
    r = _replicas(1, 4)[0]
    plan = dpslab.Plan(dpslab.make_params(precision=dpslab.FP64, **_params(r)), r["n"])
    pos, q, phi, f = _inputs(r, 9)
    st = torch.cuda.Stream()
    plan.enqueue(pos, q, phi, f, stream=st)
    with pytest.raises(dpslab.DpslabError):
        plan.enqueue(pos, q, phi, f, stream=st)          # one solve in flight per plan
    code = dpslab.PENDING
    for _ in range(10 ** 7):
        code, U = plan.poll()
        if code != dpslab.PENDING:
            break
    assert code == dpslab.OK
    U1, _ = plan.solve(pos, q, torch.empty_like(phi), torch.empty_like(f))
    assert abs(U - U1) <= 1e-12 * abs(U1)
    plan.close()


def test_bd_steps_same_alone_and_in_the_mix():
    # each request one Brownian-dynamics step of its replica; replicas advance
    # in the mix exactly as they do alone
    reps = _replicas(4, 31)
    bp = dpslab.bd_params(0.01, 1.0, 1.0, 0.5, 1.0, 1.0, 6, max_retries=8, seed=5)
    srv = Server(1 << 40, nstreams=3, max_inflight=3, precision=dpslab.FP64)
    state, init = [], []
    for i, r in enumerate(reps):
        srv.register(i, _params(r), r["n"])
        pos, q, _, f = _inputs(r, 300 + i)
        W = torch.empty((r["n"], 3), dtype=torch.float64, device="cuda")
        dpslab.bd_init_noise(11 + i, W)
        init.append((pos.clone(), W.clone()))
        state.append((pos, q, W, f))
    reqs, steps = [], [0] * len(reps)
    for k in range(12):
        i = k % len(reps)
        pos, q, W, f = state[i]
        reqs.append(Request(i, pos, q, None, f, t_arrival=0.0, bd=bp, W=W, step=steps[i]))
        steps[i] += 1
    done = srv.run(reqs, realtime=False, timeout_s=300)
    assert all(r.code == dpslab.OK for r in done)
    for i, r in enumerate(reps):
        plan = dpslab.Plan(dpslab.make_params(precision=dpslab.FP64, **_params(r)), r["n"])
        pos, W = init[i][0].clone(), init[i][1].clone()
        for k in range(steps[i]):
            plan.bd_step(bp, pos, state[i][1], W, k)
        assert torch.max(torch.abs(pos - state[i][0])).item() < 1e-12
        assert torch.equal(W, state[i][2])
        plan.close()
    srv.close()
