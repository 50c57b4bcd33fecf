"""Serving loop for force/energy requests of many independent systems
(Brownian-dynamics replicas): continuous batching over CUDA streams with
admission by device-memory footprint.

A replica's plan (derived parameters, Chebyshev and FFT tables: a few MB) is
created once and stays resident. The large per-solve arrays (grids, spectra,
field grids, cell list, charge arrays: the plan's workspace, about 9 grid
copies of 4 bytes plus ~10 KB per charge) are admitted separately: a
replica's workspace stays bound and resident between its requests while the
memory budget allows, and idle replicas' workspaces are evicted, least
recently used first, when a new replica needs room. Workspaces come from the
device allocator of the process (PyTorch's caching allocator), so evicting
one and admitting another reuses the memory without a device-wide
synchronisation.

Requests wait in arrival order. Each pass of the loop polls the solves in
flight without blocking (dpslab_solve_poll) and starts every waiting request
that can start: its replica has no solve in flight, a slot is free (at most
`max_inflight` solves at once), and its workspace is resident or fits the
budget after evictions; it is enqueued (dpslab_solve_enqueue) on the next of
S streams. Requests that arrive while others run therefore join as slots and
memory free up, and their kernels overlap on the device. A request that
needs a new workspace and cannot get one holds back later requests that need
new workspaces too (no starvation of large systems); requests of replicas
with a resident workspace pass it. A replica whose workspace alone exceeds
the budget is rejected with DPSLAB_ERR_CAPACITY.

Requests may be Brownian-dynamics steps of their replica (the solve, the
steric forces and the update of Eq. (leimkuhler) in stream order): a
replica's steps then run in order and its positions advance in place.

Latency is arrival to completion on the host's clock; throughput is charges
solved per second of the run.
"""
import collections
import time

from . import dpslab

CANCELLED = -100     # Request.code of a request withdrawn before it started


class Request:
    """One force/energy solve for `replica`: device tensors pos [n, 3] and
    q [n] (float64), outputs phi [n] and force [n, 3] (float64, device, or
    None). t_arrival is in seconds from the start of Server.run. The server
    fills in U, code (DPSLAB_OK or an error), t_start and t_done.

    With bd (a dpslab.BdParams), W (device [n, 3]) and step, the request is
    one Brownian-dynamics step (dpslab_bd_step_enqueue): the solve at pos,
    then pos and W advanced in place; retries reports the discarded
    proposals."""

    def __init__(self, replica, pos, q, phi=None, force=None, t_arrival=0.0, bd=None, W=None, step=0):
        self.replica = replica
        self.pos, self.q, self.phi, self.force = pos, q, phi, force
        self.bd, self.W, self.step = bd, W, step
        self.n = int(q.shape[0])
        self.t_arrival = t_arrival
        self.t_arrival_abs = None
        self.t_start = self.t_done = None
        self.U = None
        self.code = None
        self.retries = None


def _torch_backend(nstreams):
    import torch

    def alloc(nbytes):
        return torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")

    return alloc, [torch.cuda.Stream() for _ in range(nstreams)]


class Server:
    """budget_bytes: device memory for resident workspaces. Replicas are
    registered with their params (a dict of dpslab.make_params keywords) and
    largest charge count; plans are created at registration.

    plan_factory(params, max_n), alloc(nbytes) and streams replace the CUDA
    pieces in host-only tests."""

    def __init__(self, budget_bytes, nstreams=8, max_inflight=None, precision=dpslab.MIXED,
                 plan_factory=None, alloc=None, streams=None):
        self.budget = int(budget_bytes)
        self.precision = precision
        if alloc is None or streams is None:
            a, s = _torch_backend(max(1, nstreams))
            alloc = alloc or a
            streams = streams or s
        self.alloc, self.streams = alloc, list(streams)
        self.plan_factory = plan_factory or (
            lambda params, max_n: dpslab.Plan(dpslab.make_params(precision=precision, **params), max_n,
                                              own_work=False))
        self.max_inflight = max_inflight or 2 * len(self.streams)
        self.next_stream = 0
        self.plans = {}                              # replica -> plan (resident)
        self.ws = collections.OrderedDict()          # replica -> workspace (resident, LRU order)
        self.ws_bytes = 0
        self.busy = {}                               # replica -> request in flight
        self.waiting = collections.deque()
        self.done = []
        self.stats = collections.Counter()
        self.peak_ws_bytes = 0

    # replicas ---------------------------------------------------------------
    def register(self, replica, params, max_n):
        if replica in self.plans:
            raise ValueError(f"replica {replica} is already registered")
        self.plans[replica] = self.plan_factory(params, max_n)
        self.stats["plans"] += 1

    def unregister(self, replica):
        if replica in self.busy:
            raise ValueError(f"replica {replica} has a solve in flight")
        self._evict(replica)
        self.plans.pop(replica).close()

    def plan_bytes(self):
        return sum(p.device_bytes for p in self.plans.values())

    # workspaces -------------------------------------------------------------
    def _evict(self, replica):
        w = self.ws.pop(replica, None)
        if w is None:
            return
        plan = self.plans[replica]
        plan.bind_work(None)
        self.ws_bytes -= plan.work_bytes
        self.stats["evictions"] += 1

    def _make_room(self, need):
        """Evict idle workspaces (least recently used first) until `need`
        more bytes fit the budget; False if they cannot."""
        while self.ws_bytes + need > self.budget:
            victim = next((r for r in self.ws if r not in self.busy), None)
            if victim is None:
                return False
            self._evict(victim)
        return True

    # the loop ---------------------------------------------------------------
    def submit(self, req):
        """Queue a request. A request for an unregistered replica, or one
        whose charge count exceeds the replica's plan, finishes at once with
        DPSLAB_ERR_INVALID_ARG / DPSLAB_ERR_CAPACITY (it never reaches the
        device)."""
        if req.replica not in self.plans:
            self._finish(req, dpslab.ERR_INVALID_ARG)
            self.stats["malformed"] += 1
            return
        if req.n > getattr(self.plans[req.replica], "max_n", req.n):
            self._finish(req, dpslab.ERR_CAPACITY)
            self.stats["malformed"] += 1
            return
        self.waiting.append(req)

    def cancel(self, req):
        """Withdraw a waiting request (it finishes with code CANCELLED);
        False if it is already on the device or done (a solve in flight runs
        to completion: kernels are not interrupted)."""
        try:
            self.waiting.remove(req)
        except ValueError:
            return False
        self._finish(req, CANCELLED)
        self.stats["cancelled"] += 1
        return True

    def _finish(self, req, code, U=None):
        req.code, req.U, req.t_done = code, U, time.perf_counter()
        self.done.append(req)

    def _start(self, req, plan):
        st = self.streams[self.next_stream]
        self.next_stream = (self.next_stream + 1) % len(self.streams)
        req.t_start = time.perf_counter()
        try:
            if req.bd is not None:
                plan.bd_enqueue(req.bd, req.pos, req.q, req.W, req.step, req.force, stream=st)
            else:
                plan.enqueue(req.pos, req.q, req.phi, req.force, stream=st)
        except dpslab.DpslabError as e:
            self._finish(req, e.code)
            return
        self.busy[req.replica] = req

    def step(self):
        """One pass: poll the solves in flight, then start what can start.
        Returns the number of requests that finished in this pass."""
        finished = 0
        for r in list(self.busy):
            code, U = self.plans[r].poll()
            if code == dpslab.PENDING:
                continue
            req = self.busy.pop(r)
            if req.bd is not None:
                req.retries = self.plans[r].last_bd_retries()
            self._finish(req, code, U)
            finished += 1
        blocked = False
        keep = collections.deque()
        while self.waiting:
            req = self.waiting.popleft()
            r = req.replica
            if r in self.busy or len(self.busy) >= self.max_inflight:
                keep.append(req)
                continue
            plan = self.plans[r]
            if r in self.ws:
                self.ws.move_to_end(r)
                self.stats["resident_hits"] += 1
                self._start(req, plan)
                continue
            if plan.work_bytes > self.budget:
                self._finish(req, dpslab.ERR_CAPACITY)
                self.stats["rejected"] += 1
                continue
            if blocked or not self._make_room(plan.work_bytes):
                blocked = True
                keep.append(req)
                continue
            try:
                work = self.alloc(plan.work_bytes)
            except (MemoryError, RuntimeError):
                # the device allocator refused (memory held outside the
                # budget): give back every idle workspace and retry once; if
                # that fails too, wait for solves in flight to free theirs,
                # or fail the request when nothing is in flight
                self.stats["alloc_failures"] += 1
                for v in [k for k in self.ws if k not in self.busy]:
                    self._evict(v)
                try:
                    work = self.alloc(plan.work_bytes)
                except (MemoryError, RuntimeError):
                    if self.busy:
                        blocked = True
                        keep.append(req)
                    else:
                        self._finish(req, dpslab.ERR_CUDA)
                    continue
            plan.bind_work(work)
            self.ws[r] = True
            self.ws_bytes += plan.work_bytes
            self.peak_ws_bytes = max(self.peak_ws_bytes, self.ws_bytes)
            self.stats["admissions"] += 1
            self._start(req, plan)
        self.waiting = keep
        return finished

    def idle(self):
        return not self.busy and not self.waiting

    def run(self, requests, realtime=True, timeout_s=600.0):
        """Serve `requests` (t_arrival in seconds from the start): with
        realtime each is submitted once the clock reaches its arrival, else
        all at once. Returns the requests finished in this run."""
        t0 = time.perf_counter()
        first = len(self.done)
        pending = collections.deque(sorted(requests, key=lambda q: q.t_arrival))
        for req in pending:
            req.t_arrival_abs = t0 + (req.t_arrival if realtime else 0.0)
        while pending or not self.idle():
            now = time.perf_counter()
            while pending and pending[0].t_arrival_abs <= now:
                self.submit(pending.popleft())
            self.step()
            if now - t0 > timeout_s:
                raise TimeoutError("the serving run exceeded its time limit")
        return self.done[first:]

    def close(self):
        for r in list(self.plans):
            if r not in self.busy:
                self.unregister(r)


def latency_stats(done):
    """p50 / p99 latency (ms, arrival to completion) and charges solved per
    second between the first arrival and the last completion."""
    ok = [r for r in done if r.code == dpslab.OK]
    lat = sorted((r.t_done - r.t_arrival_abs) * 1e3 for r in ok)
    if not lat:
        return dict(requests=0)
    t_first = min(r.t_arrival_abs for r in ok)
    t_last = max(r.t_done for r in ok)
    charges = sum(r.n for r in ok)

    def pick(f):
        return lat[min(len(lat) - 1, int(f * len(lat)))]

    return dict(requests=len(ok), failed=len(done) - len(ok), p50_ms=pick(0.5), p99_ms=pick(0.99),
                charges=charges, wall_s=t_last - t_first, charges_per_s=charges / max(t_last - t_first, 1e-9))


def snapshot(pos, q, W=None, step=0):
    """Host copy of a replica's state (positions, charges, noise W^n and the
    step index of a Brownian-dynamics replica): everything a plan needs to
    resume it, since plans and workspaces are re-creatable from parameters."""
    import numpy as np
    out = dict(pos=np.asarray(pos.detach().cpu()), q=np.asarray(q.detach().cpu()), step=int(step))
    if W is not None:
        out["W"] = np.asarray(W.detach().cpu())
    return out


def save_snapshot(path, snap):
    import numpy as np
    np.savez(path, **snap)


def load_snapshot(path, device="cuda"):
    """The state saved by save_snapshot, as tensors on `device`."""
    import numpy as np
    import torch
    with np.load(path) as z:
        out = {k: (torch.tensor(z[k], device=device) if k != "step" else int(z[k])) for k in z.files}
    return out
