#!/usr/bin/env python
"""Benchmark: charges/s of the doubly-periodic slab spectral Ewald solve.

One step = one full solve (far field, near field, gauge, energy, forces) of
the named workload with the inputs resident in HBM. Default workload:
2^20 Gaussian charges (width 1, +-1, neutral) in a 512 x 512 x 128 slab
with eps_wall/eps = 1/80 on both walls, grid 1024 x 1024 x 128, mixed
precision (FP32 grids, FP64 correction, k = 0 mode and energy); its error
against the FP64 path is measured on the same inputs and reported.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--precision mixed|fp64] [--impl ours|reference]
                  [--no-cpu-baseline]

Timing: W untimed solves, then K solves each bracketed by CUDA events on the
solve's stream, with a 512 MiB memset between steps to flush the 126 MB L2
(outside the events); barrier + synchronize around the timed region, max
over ranks. Under torchrun every rank solves its own independent system
(replicas: the solve has no exchange step), so value = total charges / time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "charges/s force+energy at ≤1e-5 rel err, mixed vs FP64 plain; p50/p99 ms"
UNIT = "charges/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)   # p50/p99 from >= 50 timed solves
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="c3_jumps_n1048576")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "mixed_simt"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=150.0)
    ap.add_argument("--streams", type=int, default=0,
                    help="batched workload: streams (systems per wave) of the mixed batch; 0 = the workload's")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# roofline bookkeeping: algorithmic work per launch of each stage
# ---------------------------------------------------------------------------
def node_fractions(params, d):
    """Fractions of the z nodes where rho_o can be non-zero (within H_E of a
    charge within 2 H_E of a wall: z_j in [-H_E, 3 H_E] or [H - 3 H_E, H + H_E])
    and where the interpolation reads the fields (z_j in [-H_E, H + H_E]):
    the mixed form's tensor-core path moves those planes only."""
    import numpy as np
    from paper_2101_07088_b300 import dpslab
    zn = dpslab.table(params, 0)
    he, H = d["HE"], params.H
    fo = np.mean(((zn >= -he) & (zn <= 3 * he)) | ((zn >= H - 3 * he) & (zn <= H + he)))
    ff = np.mean((zn >= -he) & (zn <= H + he))
    return float(fo), float(ff)


def stage_work(d, n, n_over, wbytes=8, fo=1.0, ff=1.0):
    """Algorithmic bytes (HBM-bound stages) or flops (ALU-bound stages) of
    one launch of each stage, for the grid and charge counts of the solve.
    G = nx ny nz grid points, S = nz ny (nx/2+1) complex modes, M = ny (nx/2+1)
    columns; fo, ff the fractions of the nodes where rho_o can be non-zero
    and where the interpolation reads the fields (1 when every plane moves).
    Bytes count every grid array read or written once where the path needs
    it; flops count the operations the stage's algorithm cannot avoid."""
    nx, ny, nz = d["nx"], d["ny"], d["nz"]
    G, S = nx * ny * nz, nz * ny * (nx // 2 + 1)
    M = ny * (nx // 2 + 1)
    c = 2 * wbytes                     # complex
    lg = lambda v: math.log2(v)
    out = {
        # rho_i over the whole grid, rho_o over its planes, charges read once
        "spread": ("hbm", (G + G * fo) * wbytes + n * 4 * wbytes),
        "fft_x_fwd": ("hbm", (1 + fo) * (G * wbytes + S * c)),
        "fft_y_fwd": ("hbm", 2 * (1 + fo) * S * c),
        # z transforms (tensor cores; FP32 storage): node values of both
        # densities in, coefficients out; coefficients in, psi and dpsi/dz
        # out at the planes the interpolation reads
        "z_fwd": ("hbm", (1 + fo) * S * c + 2 * S * c),
        "z_inv": ("hbm", 2 * S * c + 2 * ff * S * c),
        # per-mode BVP: coefficients of both densities in, psi and dpsi/dz
        # coefficients out (mixed); the FP64 form also transforms in z, dense
        # N/2 x N/2 blocks, even/odd, real x complex = 4 flops per entry
        "bvp": ("hbm", 4 * S * c) if wbytes == 4 else ("alu", M * 4 * (2 * (nz // 2 + 1) ** 2) * 4.0),
        "fft_y_inv": ("hbm", ff * (2 * S * c + 3 * S * c)),
        "fft_x_inv": ("hbm", ff * (3 * S * c + 4 * G * wbytes)),
        # the fields once over the planes the supports reach, the charges' windows
        "interp": ("hbm", ff * 4 * G * wbytes + n * 8 * wbytes),
        "near": ("hbm", n * 12 * wbytes),
        "prepare": ("hbm", n * 8 * wbytes),
        "finish": ("hbm", n * 12 * wbytes),
    }
    # FFT flop counts (5 n log2 n per complex transform) for reference
    fft_flops = {
        "fft_x_fwd": nz * ny * 5 * nx * lg(nx),               # 2 nz ny real rows packed in pairs
        "fft_y_fwd": 2 * nz * (nx // 2 + 1) * 5 * ny * lg(ny),
        "fft_y_inv": 3 * nz * (nx // 2 + 1) * 5 * ny * lg(ny),
        "fft_x_inv": 2 * nz * ny * 5 * nx * lg(nx),
    }
    return out, fft_flops


# Stages that are one kernel each (the roofline names one kernel)
SINGLE_KERNEL_STAGES = ("fft_x_fwd", "fft_y_fwd", "bvp", "z_inv", "fft_y_inv", "fft_x_inv", "interp", "near")

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch,
# from one ncu capture of the mixed path on the 262144-charge quarter box
# (512 x 512 x 128 grid, 131584 columns); scaled to another grid by its column
# count. Only kernels unchanged since their capture are listed.
NCU_TRAFFIC_C3Q = {"interp": 379663360 + 9702144}
NCU_TRAFFIC_COLUMNS = 512 * 257


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return dict(hbm_gbs=p.get("hbm_gbs", 6400.0), bf16=p.get("bf16_tflops", 1800.0),
                    bf16_sus=p.get("bf16_tflops_sustained", 1400.0), source="measured")
    return dict(hbm_gbs=6400.0, bf16=1800.0, bf16_sus=1400.0, source="fallback")


def measure_fp64_tflops(dev, n=8192, reps=5):
    """FP64 arithmetic peak of this GPU, measured like the BF16 one of
    MEASURED_PEAKS.json: a cuBLAS GEMM (2 n^3 flops), best of `reps`."""
    import torch
    a = torch.randn((n, n), dtype=torch.float64, device=dev)
    b = torch.randn((n, n), dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    return 2.0 * n ** 3 / best / 1e12


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        """Start sampling (every 100 ms) and wait for the first sample, so
        that the sampler is running when the timed region begins."""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
            return
        t0 = time.monotonic()
        while not self.lines and time.monotonic() - t0 < 5.0:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def begin(self):
        self.t_begin = time.monotonic()

    def end(self):
        self.t_end = time.monotonic()

    def stop(self):
        """Samples taken during [begin, end] (the nearest one after begin if
        none fell inside)."""
        if not self.proc:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        t0, t1 = getattr(self, "t_begin", 0.0), getattr(self, "t_end", float("inf"))
        inside = [ln for (t, ln) in self.lines if t0 <= t <= t1 + 0.1]
        if not inside:
            after = [ln for (t, ln) in self.lines if t >= t0]
            inside = after[:1]
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in inside:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names[1:], parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


# ---------------------------------------------------------------------------
# CPU baseline: the oracle, as it stands, on the host cores, on a bounded
# sample of the workload (same slab, grid spacing and charge density on a
# smaller periodic patch; the method's work is proportional to the patch)
# ---------------------------------------------------------------------------
CPU_SAMPLE = {"c3_jumps_n1048576": "c3s_jumps_n16384", "c3q_jumps_n262144": "c3s_jumps_n16384"}
def oracle_rate(pos, q, p, budget_s, max_steps):
    from oracle import params as oparams
    from oracle import solver as osolver
    P = oparams.derive(p["Lx"], p["Ly"], p["H"], p["gw"], p["tol"], p["nx"], p["ny"], nz=p["nz"],
                       r_cut=p["r_cut"], eps_b=p["eps_b"], eps_t=p["eps_t"])
    times = []
    t_start = time.perf_counter()
    while len(times) < max_steps:
        t0 = time.perf_counter()
        osolver.solve(pos, q, P)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start + times[-1] > budget_s:
            break
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        threads = max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        threads = os.cpu_count()
    return times, threads


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ---------------------------------------------------------------------------
BATCH_WORKLOADS = {"c4_batch256": dict(count=256, seed=3, nstreams=8)}


def bench_batch(args):
    """The batched workload: 256 independent systems (N log-uniform in
    [256, 65536], L in [32, 256], H in [16, 128], walls from {1/80, 1, metal},
    2 grid points per width, N_z from the paper's rule) solved by one
    dpslab_batch_solve call (a replayed CUDA graph). Reports total charges/s
    of the mixed form, the FP64 batch beside it, and the same mixed plans
    solved one system after another (no graph, one stream)."""
    import numpy as np
    import torch
    from paper_2101_07088_b300 import build, dpslab, synth
    cfg = BATCH_WORKLOADS[args.workload]
    build.build()
    dev = torch.device("cuda:0")
    systems = synth.batch_systems(cfg["count"], cfg["seed"])
    total = sum(len(q) for _, q, _ in systems)
    bufs = [(torch.tensor(pos, dtype=torch.float64, device=dev), torch.tensor(q, dtype=torch.float64, device=dev),
             torch.empty(len(q), dtype=torch.float64, device=dev),
             torch.empty((len(q), 3), dtype=torch.float64, device=dev)) for pos, q, _ in systems]
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    out = {}
    streams = dict(mixed=args.streams or cfg["nstreams"], fp64=cfg["nstreams"])
    args_ = ([b[0] for b in bufs], [b[1] for b in bufs], [b[2] for b in bufs], [b[3] for b in bufs])
    schedules = {}
    for name, prec in (("mixed", dpslab.MIXED), ("fp64", dpslab.FP64)):
        params = [dpslab.make_params(precision=prec, **p) for _, _, p in systems]
        batch = dpslab.Batch(params, [len(q) for _, q, _ in systems], nstreams=streams[name])
        if name == "mixed":
            # both schedules timed as the bench times steps, then the
            # library's batch autotuner picks one (outside the timed region)
            for sched, label in ((dpslab.BATCH_STREAMS, "streams"), (dpslab.BATCH_WAVES, "waves")):
                batch.set_schedule(sched)
                sms = timed(lambda: batch.solve(*args_), max(1, min(args.steps, 3)), 2)
                schedules[label] = dict(ms_per_step=sum(sms) / len(sms), gpu_launches=batch.last_launch_count())
            batch.set_schedule(dpslab.BATCH_STREAMS)
            schedules["autotuned"] = "waves" if batch.autotune(args_[0], args_[1], reps=2) == dpslab.BATCH_WAVES \
                else "streams"
        ms = timed(lambda: batch.solve(*args_), max(1, args.steps), max(3, args.warmup))
        U, _ = batch.solve(*args_)
        out[name] = dict(ms=ms, U=U.copy(), bytes=batch.device_bytes, launches=batch.last_launch_count())
        batch.close()
    # the mixed plans one after another (no graph, no concurrency)
    plans = [dpslab.Plan(dpslab.make_params(precision=dpslab.MIXED, **p), len(q)) for _, q, p in systems]
    seq = timed(lambda: [pl.solve(b[0], b[1], b[2], b[3]) for pl, b in zip(plans, bufs)], 3, 1)
    for pl in plans:
        pl.close()
    ms = sorted(out["mixed"]["ms"])
    mean = sum(ms) / len(ms)
    f64 = sum(out["fp64"]["ms"]) / len(out["fp64"]["ms"])
    uerr = float(np.max(np.abs(out["mixed"]["U"] - out["fp64"]["U"]) / np.abs(out["fp64"]["U"])))
    line = dict(metric=METRIC, value=total / (mean * 1e-3), unit=UNIT, n_gpus=1, steps=len(ms),
                warmup=max(3, args.warmup), ms_per_step=mean, p50_ms=ms[len(ms) // 2],
                p99_ms=ms[min(len(ms) - 1, int(math.ceil(0.99 * len(ms))) - 1)], higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f32+f64", data="synthetic (seeded +-1 electrolytes)",
                config=dict(workload=args.workload, systems=cfg["count"], charges=total, streams=streams,
                            form="one dpslab_batch_solve call (CUDA graph replay); mixed schedule chosen by "
                                 "dpslab_batch_autotune (per-system streams, or waves of `streams` systems with one "
                                 "column-stage launch per kind over all their modes); FP64 per-system streams",
                            l2="512 MiB memset between timed steps"),
                gpu_launches=dict(mixed=out["mixed"]["launches"], fp64=out["fp64"]["launches"]),
                mixed_schedules=schedules,
                fp64_value=total / (f64 * 1e-3), fp64_ms_per_step=f64,
                mixed_over_fp64=f64 / mean, sequential_ms_per_step=sum(seq) / len(seq),
                max_energy_rel_vs_fp64=uerr, device_bytes=dict(mixed=out["mixed"]["bytes"], fp64=out["fp64"]["bytes"]))
    print(json.dumps(line))
    return 0


SERVE_WORKLOADS = {"c5_serve1000": dict(replicas=1000, seed=4, rate=20000.0, per_step=100, nstreams=8,
                                         budget_frac=0.6, bd=True)}
# Brownian dynamics of the served replicas (Sec. 7.1): ions of radius 1/2 in
# units of the Gaussian width, soft cap at r_m = 2a, one hundredth of the
# diffusive time per step
SERVE_BD = dict(dt=0.01, mu=1.0, kT=1.0, a=0.5, U0=1.0, r_m=1.0, p=6, max_retries=8)


def bench_serve(args):
    """The served workload: 1000 Brownian-dynamics replicas (N log-uniform in
    [512, 262144], H in [16, 128], both walls at 1/80, the charge density of
    the 2^20-charge workload, 2 grid points per width, N_z from the paper's
    rule), requests for uniformly drawn replicas arriving as a Poisson stream
    of 20,000 per second (far above what one device serves: the run is in
    overload and shows queueing and admission). Each request is one
    Brownian-dynamics step of its replica (Eq. (leimkuhler): the solve, the
    steric forces, the update), so replicas move. Replica plans are registered
    up front; workspaces are admitted under a budget of 60% of the free
    device memory. `warmup` x 100 requests are served first (filling the
    resident set), then `steps` x 100 requests are timed. Reports charges/s,
    p50/p99 latency (arrival to completion) and service time (start to
    completion), admission counters, the first 100 timed requests solved
    one after another on one stream for comparison, and 200 requests at half
    the measured capacity (latency without the overload's queue)."""
    os.environ.setdefault("PYTORCH_CUDA_ALLOC_CONF", "expandable_segments:True")
    import numpy as np
    import torch
    from paper_2101_07088_b300 import build, dpslab, synth
    from paper_2101_07088_b300.serve import Request, Server, latency_stats
    cfg = SERVE_WORKLOADS[args.workload]
    build.build()
    dev = torch.device("cuda:0")
    reps = synth.serve_replicas(cfg["replicas"], cfg["seed"])
    # one state per replica (a replica has one solve in flight at a time)
    bufs, noise = [], []
    for i, r in enumerate(reps):
        pos, q = synth.electrolyte(r["n"], r["Lx"], r["Ly"], 1.0, r["H"] - 1.0, cfg["seed"] + 1 + i)
        bufs.append((torch.tensor(pos, dtype=torch.float64, device=dev), torch.tensor(q, dtype=torch.float64, device=dev),
                     torch.empty(r["n"], dtype=torch.float64, device=dev),
                     torch.empty((r["n"], 3), dtype=torch.float64, device=dev)))
        if cfg["bd"]:
            W = torch.empty((r["n"], 3), dtype=torch.float64, device=dev)
            dpslab.bd_init_noise(cfg["seed"] * 100003 + i, W)
            noise.append(W)
    bdp = dpslab.bd_params(seed=cfg["seed"], **SERVE_BD) if cfg["bd"] else None
    steps_of = [0] * len(reps)
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    budget = int(cfg["budget_frac"] * free)
    prec = {"fp64": dpslab.FP64, "mixed": dpslab.MIXED, "mixed_simt": dpslab.MIXED_SIMT}[args.precision]
    srv = Server(budget, nstreams=cfg["nstreams"], precision=prec)
    t0 = time.perf_counter()
    for i, r in enumerate(reps):
        srv.register(i, {k: v for k, v in r.items() if k != "n"}, r["n"])
    t_register = time.perf_counter() - t0
    warm, steps = max(3, args.warmup), max(1, args.steps)
    rep_ids, t_arr = synth.serve_arrivals((warm + steps) * cfg["per_step"], len(reps), cfg["rate"], cfg["seed"])

    def requests(lo, hi):
        t_base = t_arr[lo]
        out = []
        for k in range(lo, hi):
            i = int(rep_ids[k])
            if cfg["bd"]:
                out.append(Request(i, bufs[i][0], bufs[i][1], None, bufs[i][3], t_arrival=float(t_arr[k] - t_base),
                                   bd=bdp, W=noise[i], step=steps_of[i]))
                steps_of[i] += 1
            else:
                out.append(Request(i, *bufs[i], t_arrival=float(t_arr[k] - t_base)))
        return out

    nw = warm * cfg["per_step"]
    srv.run(requests(0, nw))
    torch.cuda.synchronize()
    stats0 = dict(srv.stats)
    clocks = Clocks(0)
    clocks.start()
    clocks.begin()
    t0 = time.perf_counter()
    done = srv.run(requests(nw, len(rep_ids)))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks.end()
    ck = clocks.stop()
    st = latency_stats(done)
    svc = sorted((r.t_done - r.t_start) * 1e3 for r in done)
    counters = {k: srv.stats[k] - stats0.get(k, 0) for k in ("admissions", "evictions", "resident_hits", "rejected")}
    # the first 100 timed requests again, one after another on one stream
    subset = done[:cfg["per_step"]]
    for r in list(srv.ws):
        srv._evict(r)
    one = srv.alloc(max(srv.plans[r.replica].work_bytes for r in subset))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    seq_charges = 0
    for r in subset:
        pl = srv.plans[r.replica]
        pl.bind_work(one)
        if r.bd is not None:
            pl.bd_step(r.bd, r.pos, r.q, r.W, steps_of[r.replica], r.force)
            steps_of[r.replica] += 1
        else:
            pl.solve(r.pos, r.q, r.phi, r.force)
        pl.bind_work(None)
        seq_charges += r.n
    torch.cuda.synchronize()
    seq_rate = seq_charges / (time.perf_counter() - t1)
    del one
    # the same replicas at half the measured capacity (Poisson arrivals at
    # 0.5 x requests/s served above): latency without the overload's queue
    half_rate = 0.5 * st["requests"] / wall
    nh = 2 * cfg["per_step"]
    h_ids, h_t = synth.serve_arrivals(nh, len(reps), half_rate, cfg["seed"] + 1)
    h_reqs = []
    for k in range(nh):
        i = int(h_ids[k])
        if cfg["bd"]:
            h_reqs.append(Request(i, bufs[i][0], bufs[i][1], None, bufs[i][3], t_arrival=float(h_t[k] - h_t[0]),
                                  bd=bdp, W=noise[i], step=steps_of[i]))
            steps_of[i] += 1
        else:
            h_reqs.append(Request(i, *bufs[i], t_arrival=float(h_t[k] - h_t[0])))
    h_done = srv.run(h_reqs)
    torch.cuda.synchronize()
    hs = latency_stats(h_done)
    line = dict(metric=METRIC, value=st["charges"] / wall, unit=UNIT, n_gpus=1, steps=steps, warmup=warm,
                ms_per_step=wall * 1e3 / steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype={"fp64": "f64", "mixed": "f32+f64", "mixed_simt": "f32+f64"}[args.precision],
                data="synthetic (seeded +-1 electrolytes)",
                config=dict(workload=args.workload, replicas=len(reps), requests_per_step=cfg["per_step"],
                            arrival_rate_per_s=cfg["rate"], streams=cfg["nstreams"],
                            workspace_budget_gb=budget / 1e9,
                            l2="grids of 10 MB to 2 GB per request, requests interleaved; no flush"),
                latency_ms=dict(p50=st["p50_ms"], p99=st["p99_ms"]),
                half_load=dict(arrival_rate_per_s=half_rate, requests=hs.get("requests", 0),
                               latency_ms=dict(p50=hs.get("p50_ms"), p99=hs.get("p99_ms")),
                               charges_per_s=hs.get("charges_per_s")),
                service_ms=dict(p50=svc[len(svc) // 2], p99=svc[min(len(svc) - 1, int(0.99 * len(svc)))]),
                requests=st["requests"], failed=st.get("failed", 0), charges=st["charges"],
                request_kind="Brownian-dynamics step (solve + steric + update)" if cfg["bd"] else "solve",
                bd_retries=int(sum(r.retries or 0 for r in done)) if cfg["bd"] else None,
                admission=dict(counters, peak_workspace_gb=srv.peak_ws_bytes / 1e9,
                               resident_plans_gb=srv.plan_bytes() / 1e9, register_s=t_register),
                sequential_value=seq_rate, served_over_sequential=(st["charges"] / wall) / seq_rate,
                clocks=ck)
    print(json.dumps(line))
    srv.close()
    return 0


def main():
    args = parse()
    if args.workload in BATCH_WORKLOADS:
        return bench_batch(args)
    if args.workload in SERVE_WORKLOADS:
        return bench_serve(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_2101_07088_b300 import synth
    pos, q, p = synth.workload(args.workload)
    n = len(q)
    wl = synth.WORKLOADS[args.workload]
    config = dict(workload=args.workload, charges=n, box=[p["Lx"], p["Ly"], p["H"]],
                  grid=[p["nx"], p["ny"], p["nz"]], eps_wall_over_eps=[p["eps_b"], p["eps_t"]],
                  gw=p["gw"], r_cut=p["r_cut"], tol=p["tol"], precision=args.precision,
                  parallelism=f"replicas{world}", l2="512 MiB memset between timed steps")

    sample_name = CPU_SAMPLE.get(args.workload, args.workload)
    if args.impl == "reference":
        if rank != 0:
            return 0
        budget = max(30.0, args.cpu_budget_s)
        spos, sq, sp = synth.workload(sample_name)
        times, threads = oracle_rate(spos, sq, sp, budget, max(1, args.steps))
        mean = sum(times) / len(times)
        value = len(sq) / mean
        line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus,
                    steps=len(times), warmup=0, ms_per_step=mean * 1e3, higher_is_better=True,
                    scaling="weak", vs_baseline=None, dtype="f64", data="synthetic", config=config,
                    cpu_baseline=dict(value=value, unit=UNIT, cores=threads, kind="oracle",
                                      sample=f"{len(times)} oracle solves of {sample_name} "
                                             f"({len(sq)} charges, same slab/spacing/density as {args.workload}; "
                                             f"steps capped by a {budget:.0f} s budget, {args.steps} requested); "
                                             f"host {cpu_model()}, {os.cpu_count()} logical CPUs"),
                    e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
        print(json.dumps(line))
        return 0

    import numpy as np
    import torch
    from paper_2101_07088_b300 import build, dpslab, replicas
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    # each rank solves its own system (independent seed)
    if world > 1:
        pos, q = synth.electrolyte(n, p["Lx"], p["Ly"], 1.0, p["H"] - 1.0, replicas.replica_seed(wl["seed"], rank))
    prec = {"mixed": dpslab.MIXED, "mixed_simt": dpslab.MIXED_SIMT, "fp64": dpslab.FP64}[args.precision]
    plan = dpslab.Plan(dpslab.make_params(precision=prec, **p), n)
    d = plan.derived
    pos_t = torch.tensor(pos, dtype=torch.float64, device=dev)
    q_t = torch.tensor(q, dtype=torch.float64, device=dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    force = torch.empty((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    # launch shapes of the xy transforms by the library's autotuner (before
    # the warm-up, outside the timed region)
    default_knobs = plan.tuning()
    knobs = plan.autotune(pos_t, q_t, reps=3) if not args.no_autotune else default_knobs
    config["tuning"] = dict(knobs=knobs, default=default_knobs, autotuned=not args.no_autotune)

    for _ in range(max(3, args.warmup)):
        plan.solve(pos_t, q_t, phi, force)

    def timed(steps, profiled):
        """`steps` solves, each bracketed by CUDA events on the solve's stream
        with an L2 flush in between (outside the events); per-step ms and,
        when profiled, the summed stage times."""
        plan.profile(profiled)
        ms, stages = [], {}
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            energy[0], _ = plan.solve(pos_t, q_t, phi, force, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            if profiled:
                for k, v in plan.stage_times().items():
                    stages[k] = stages.get(k, 0.0) + v
        plan.profile(False)
        return ms, stages

    energy = [None]
    clocks = Clocks(local)
    clocks.start()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks.begin()
    t_wall = time.perf_counter()
    # the product path: plain solves (near field on the plan's second stream)
    step_ms, _ = timed(args.steps, False)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t_wall
    launches = plan.last_launch_count() * args.steps
    # stage times: a second timed set of the same solves with stage events
    # (the near field still on its second stream, timed there)
    prof_steps = max(5, min(args.steps, 20))
    prof_ms, stage_sum = timed(prof_steps, True)
    torch.cuda.synchronize(dev)
    clocks.end()
    clk = clocks.stop()
    mean_ms, value = replicas.job_rate(sum(step_ms) / len(step_ms), n, dist, dev)
    if dist:
        dist.barrier()
    srt = sorted(step_ms)
    p50 = srt[len(srt) // 2]
    p99 = srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)]

    # e2e: host buffers through dpslab_solve_host (H2D of pos, q; D2H of phi, force, U)
    pin_pos = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
    pin_q = torch.empty(n, dtype=torch.float64, pin_memory=True)
    pin_phi = torch.empty(n, dtype=torch.float64, pin_memory=True)
    pin_force = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
    pin_pos.copy_(torch.from_numpy(pos))
    pin_q.copy_(torch.from_numpy(q))
    hp, hq, hphi, hforce = pin_pos.numpy(), pin_q.numpy(), pin_phi.numpy(), pin_force.numpy()
    for _ in range(2):
        plan.solve_host(hp, hq, stream=stream, phi=hphi, force=hforce)
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.solve_host(hp, hq, stream=stream, phi=hphi, force=hforce)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_mean, e2e_value = replicas.job_rate(sum(e2e_ms) / len(e2e_ms), n, dist, dev)

    # accuracy of the timed path against the FP64 path on the same inputs, and
    # the FP64 path's own step time (outside the timed region)
    accuracy, fp64_ms = None, None
    if args.precision != "fp64":
        plan64 = dpslab.Plan(dpslab.make_params(precision=dpslab.FP64, **p), n)
        phi64 = torch.empty_like(phi)
        force64 = torch.empty_like(force)
        U64, _ = plan64.solve(pos_t, q_t, phi64, force64)
        t64 = []
        for _ in range(2):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan64.solve(pos_t, q_t, phi64, force64, stream=stream)
            e1.record(stream)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1))
        fp64_ms = min(t64)
        Um, _ = plan.solve(pos_t, q_t, phi, force)
        accuracy = dict(vs="FP64 GPU path on the same inputs (itself within 1e-14 of the FP64 oracle)",
                        force_rel_l2=float(torch.linalg.norm(force - force64) / torch.linalg.norm(force64)),
                        energy_rel=abs(Um - U64) / abs(U64),
                        potential_rel_max=float(torch.max(torch.abs(phi - phi64)) / torch.max(torch.abs(phi64))))
        plan64.close()

    # roofline of the dominant stage
    over = int(np.sum((pos[:, 2] <= 2 * d["HE"]) | (pos[:, 2] >= p["H"] - 2 * d["HE"])))
    fo, ff = node_fractions(dpslab.make_params(precision=prec, **p), d) if args.precision == "mixed" else (1.0, 1.0)
    work, fft_flops = stage_work(d, n, over, wbytes=4 if args.precision != "fp64" else 8, fo=fo, ff=ff)
    stage_ms = {k: v / prof_steps for k, v in stage_sum.items()}
    top = max(SINGLE_KERNEL_STAGES, key=lambda k: stage_ms.get(k, 0.0))
    pk = peaks()
    bound, amount = work[top]
    secs = stage_ms[top] * 1e-3
    if bound == "hbm":
        achieved = amount / secs / 1e9
        traffic = None
        if args.precision == "mixed" and top in NCU_TRAFFIC_C3Q:
            traffic = NCU_TRAFFIC_C3Q[top] * (d["ny"] * (d["nx"] // 2 + 1)) / NCU_TRAFFIC_COLUMNS
        roof = dict(bound="hbm", achieved=achieved, peak=pk["hbm_gbs"], unit="GB/s",
                    frac=achieved / pk["hbm_gbs"], traffic=traffic, algorithmic_bytes=amount, kernel=top,
                    peak_source=pk["source"] + " (MEASURED_PEAKS hbm_gbs)")
    else:
        achieved = amount / secs / 1e12
        fp64_peak = measure_fp64_tflops(dev)
        roof = dict(bound="alu", achieved=achieved, peak=fp64_peak, unit="TFLOP/s",
                    frac=achieved / fp64_peak, traffic=None, kernel=top,
                    peak_source="measured here: FP64 cuBLAS GEMM 8192^3, best of 5 (CUDA events)")
    roof["stage_ms"] = {k: round(v, 4) for k, v in stage_ms.items()}
    roof["stage_timing"] = (f"{prof_steps} profiled solves after the timed ones; the near field runs beside the "
                            f"far field, so the stages add up to more than a solve")
    roof["profiled_ms_per_step"] = sum(prof_ms) / len(prof_ms)

    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=mean_ms, p50_ms=p50, p99_ms=p99, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64" if args.precision == "fp64" else "f32+f64", data="synthetic (seeded +-1 electrolyte)",
                config=config,
                e2e=dict(value=e2e_value, unit=UNIT, ms_per_step=e2e_mean,
                         h2d_bytes_per_step=n * 4 * 8, d2h_bytes_per_step=n * 4 * 8 + 8 + 8 * 8 + 4),
                gpu_launches=launches, roofline=roof, clocks=clk, wall_s=wall,
                energy=energy[0], plan_device_bytes=plan.device_bytes)
    if accuracy is not None:
        line["accuracy"] = accuracy
        line["fp64_ms_per_step"] = fp64_ms
        line["fp64_value"] = n * world / (fp64_ms * 1e-3)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        spos, sq, sp = synth.workload(sample_name)
        times, threads = oracle_rate(spos, sq, sp, 40.0, 1)
        line["cpu_baseline"] = dict(value=len(sq) / times[0], unit=UNIT, cores=threads, kind="oracle",
                                    sample=f"1 oracle solve of {sample_name} ({len(sq)} charges, same slab, "
                                           f"spacing and density as {args.workload}; {times[0]:.1f} s); "
                                           f"host {cpu_model()}, {os.cpu_count()} logical CPUs")
    if rank == 0:
        print(json.dumps(line))
    plan.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
