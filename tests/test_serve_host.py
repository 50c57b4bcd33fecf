"""Host logic of the serving loop (admission by memory footprint, workspace
eviction, slots, per-replica ordering), with fake plans and a fake device:
no GPU and no CUDA library calls."""
import random

from paper_2101_07088_b300 import dpslab
from paper_2101_07088_b300.serve import Request, Server, latency_stats


class FakeQ:
    def __init__(self, n):
        self.shape = (n,)


class FakeDevice:
    """Solves finish when complete() says so."""

    def __init__(self):
        self.running = []


class FakePlan:
    def __init__(self, dev, work_bytes, log):
        self.dev, self.work_bytes, self.device_bytes, self.log = dev, work_bytes, 1000, log
        self.work, self.pending = None, None

    def bind_work(self, w):
        self.log.append(("bind", id(self), w is not None))
        self.work = w

    def enqueue(self, pos, q, phi, force, stream=None):
        assert self.work is not None and self.pending is None
        self.pending = [False, pos]
        self.dev.running.append(self)

    def poll(self):
        if not self.pending[0]:
            return dpslab.PENDING, None
        U = float(self.pending[1])
        self.pending = None
        return dpslab.OK, U

    def close(self):
        pass


def _server(budget, sizes, max_inflight=4):
    dev, log, allocs = FakeDevice(), [], []

    def alloc(nbytes):
        allocs.append(nbytes)
        return bytearray(1)

    srv = Server(budget, max_inflight=max_inflight, plan_factory=lambda params, n: FakePlan(dev, params["w"], log),
                 alloc=alloc, streams=["s0", "s1"])
    for r, w in enumerate(sizes):
        srv.register(r, dict(w=w), 100)
    return srv, dev, allocs


def _finish_all(srv, dev):
    for p in dev.running:
        p.pending[0] = True
    dev.running.clear()


def test_budget_is_never_exceeded_and_idle_workspaces_are_evicted_lru():
    srv, dev, allocs = _server(budget=100, sizes=[40, 40, 40, 30])
    for r in (0, 1):
        srv.submit(Request(r, pos=r, q=FakeQ(10)))
    srv.step()
    assert set(srv.busy) == {0, 1} and srv.ws_bytes == 80
    srv.submit(Request(2, pos=2, q=FakeQ(10)))
    srv.step()                                 # 0 and 1 busy: no room for 2
    assert 2 not in srv.busy and srv.ws_bytes == 80
    _finish_all(srv, dev)
    srv.step()                                 # 0 and 1 done; 0 (least recent) evicted for 2
    assert set(srv.busy) == {2} and list(srv.ws) == [1, 2] and srv.ws_bytes == 80
    assert srv.stats["evictions"] == 1 and srv.peak_ws_bytes <= 100
    _finish_all(srv, dev)
    srv.step()
    srv.submit(Request(1, pos=5, q=FakeQ(10)))  # resident: no new workspace
    srv.step()
    assert srv.stats["resident_hits"] == 1 and allocs == [40, 40, 40]
    _finish_all(srv, dev)
    srv.step()
    assert [(r.replica, r.U) for r in srv.done] == [(0, 0.0), (1, 1.0), (2, 2.0), (1, 5.0)]


def test_one_solve_per_replica_in_arrival_order_and_slot_limit():
    srv, dev, _ = _server(budget=1000, sizes=[10] * 6, max_inflight=3)
    for k in range(4):
        srv.submit(Request(0, pos=k, q=FakeQ(1)))
    for r in range(1, 6):
        srv.submit(Request(r, pos=10 + r, q=FakeQ(1)))
    srv.step()
    assert len(srv.busy) == 3 and 0 in srv.busy       # three slots
    order = []
    for _ in range(20):
        _finish_all(srv, dev)
        srv.step()
        order = [r.U for r in srv.done if r.replica == 0]
        if srv.idle():
            break
    assert srv.idle() and order == [0.0, 1.0, 2.0, 3.0] and len(srv.done) == 9


def test_too_large_replica_is_rejected_and_large_one_is_not_starved():
    srv, dev, _ = _server(budget=100, sizes=[150, 60, 30, 30, 30])
    srv.submit(Request(0, pos=0, q=FakeQ(1)))
    srv.step()
    assert srv.done[0].code == dpslab.ERR_CAPACITY and srv.stats["rejected"] == 1
    srv.submit(Request(2, pos=2, q=FakeQ(1)))
    srv.submit(Request(3, pos=3, q=FakeQ(1)))
    srv.step()                                   # 60 bytes busy
    srv.submit(Request(1, pos=1, q=FakeQ(1)))    # needs 60: waits
    srv.submit(Request(4, pos=4, q=FakeQ(1)))    # would fit (30) but queues behind 1
    srv.step()
    assert 1 not in srv.busy and 4 not in srv.busy
    _finish_all(srv, dev)
    srv.step()
    assert 1 in srv.busy                         # the large one went first
    for _ in range(5):
        _finish_all(srv, dev)
        srv.step()
    assert srv.idle() and sorted(r.replica for r in srv.done if r.code == dpslab.OK) == [1, 2, 3, 4]


def test_random_traffic_keeps_invariants():
    rng = random.Random(1)
    sizes = [rng.randint(5, 60) for _ in range(12)]
    srv, dev, _ = _server(budget=120, sizes=sizes, max_inflight=5)
    sent = 0
    for tick in range(400):
        if sent < 150 and rng.random() < 0.6:
            srv.submit(Request(rng.randrange(12), pos=sent, q=FakeQ(rng.randint(1, 9))))
            sent += 1
        for p in list(dev.running):
            if rng.random() < 0.3:
                p.pending[0] = True
                dev.running.remove(p)
        srv.step()
        assert srv.ws_bytes <= 120 and len(srv.busy) <= 5
        assert srv.ws_bytes == sum(srv.plans[r].work_bytes for r in srv.ws)
        assert all(r in srv.ws for r in srv.busy)
    while not srv.idle():
        _finish_all(srv, dev)
        srv.step()
    assert len(srv.done) == 150 and sorted(r.U for r in srv.done) == list(range(150))
    for r in srv.done:
        r.t_arrival_abs = r.t_start
    s = latency_stats(srv.done)
    assert s["requests"] == 150 and s["p50_ms"] <= s["p99_ms"]


def test_injected_faults_malformed_cancel_and_allocator_refusal():
    from paper_2101_07088_b300.serve import CANCELLED
    srv, dev, allocs = _server(budget=100, sizes=[40, 40, 40], max_inflight=1)
    srv.plans[0].max_n = 5
    # malformed: unregistered replica, too many charges for the plan
    srv.submit(Request(7, pos=0, q=FakeQ(1)))
    srv.submit(Request(0, pos=0, q=FakeQ(9)))
    assert [r.code for r in srv.done] == [dpslab.ERR_INVALID_ARG, dpslab.ERR_CAPACITY]
    # cancellation: a waiting request can be withdrawn, one in flight cannot
    a, b = Request(1, pos=1, q=FakeQ(1)), Request(2, pos=2, q=FakeQ(1))
    srv.submit(a)
    srv.submit(b)
    srv.step()                                       # a starts (one slot), b waits
    assert not srv.cancel(a) and srv.cancel(b)
    assert b.code == CANCELLED and 2 not in srv.busy
    _finish_all(srv, dev)
    srv.step()
    assert a.code == dpslab.OK
    # the device allocator refuses once: idle workspaces are given back and
    # the admission retried
    fails = [1]

    def flaky(nbytes):
        if fails[0]:
            fails[0] -= 1
            raise RuntimeError("out of memory")
        allocs.append(nbytes)
        return bytearray(1)
    srv.alloc = flaky
    c = Request(0, pos=3, q=FakeQ(1))
    srv.submit(c)
    srv.step()
    assert 0 in srv.busy and srv.stats["alloc_failures"] == 1 and list(srv.ws) == [0]
    _finish_all(srv, dev)
    srv.step()
    assert c.code == dpslab.OK
    # it refuses for good with nothing in flight: the request fails, the loop goes on
    srv.alloc = lambda nbytes: (_ for _ in ()).throw(RuntimeError("out of memory"))
    d = Request(2, pos=4, q=FakeQ(1))
    srv.submit(d)
    srv.step()
    assert d.code == dpslab.ERR_CUDA and srv.idle()


def test_snapshot_roundtrip(tmp_path):
    torch = __import__("pytest").importorskip("torch")
    from paper_2101_07088_b300.serve import load_snapshot, save_snapshot, snapshot
    pos = torch.rand(10, 3, dtype=torch.float64)
    q = torch.tensor([1.0, -1.0] * 5, dtype=torch.float64)
    W = torch.randn(10, 3, dtype=torch.float64)
    path = str(tmp_path / "rep.npz")
    save_snapshot(path, snapshot(pos, q, W, step=17))
    back = load_snapshot(path, device="cpu")
    assert back["step"] == 17 and torch.equal(back["pos"], pos) and torch.equal(back["W"], W)
    assert torch.equal(back["q"], q)
