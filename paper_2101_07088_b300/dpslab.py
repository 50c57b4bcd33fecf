"""Python binding of the C ABI in include/dpslab.h (argument marshalling only).

Every solve runs in the CUDA library libdpslab.so built from csrc/; this
module only converts arguments. Device buffers are PyTorch CUDA tensors
(float64, contiguous); streams are torch.cuda streams. If the library is
missing the import fails: there is no CPU path.
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdpslab.so")

OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "NOT_NEUTRAL", -3: "OUT_OF_SLAB", -4: "CUTOFF_TOO_LARGE",
    -5: "SPLIT_CONSTRAINT", -6: "CAPACITY", -7: "CUDA", -8: "NO_DEVICE", -9: "GRID", -10: "UNSUPPORTED",
    -11: "BD_REJECTED", -12: "TIMEOUT",
}
(ERR_INVALID_ARG, ERR_NOT_NEUTRAL, ERR_OUT_OF_SLAB, ERR_CUTOFF_TOO_LARGE, ERR_SPLIT_CONSTRAINT, ERR_CAPACITY,
 ERR_CUDA, ERR_NO_DEVICE, ERR_GRID, ERR_UNSUPPORTED, ERR_BD_REJECTED, ERR_TIMEOUT) = range(-1, -13, -1)
WAIT_LIMIT_DEFAULT = 1 << 26         # default polls of a bounded wait (dpslab_plan_set_wait_limit)
PENDING = 1                          # DPSLAB_PENDING
FP64, MIXED, MIXED_SIMT = 0, 1, 2   # DPSLAB_FP64, DPSLAB_MIXED, DPSLAB_MIXED_SIMT
NSTAGES = 12
NKNOBS = 7                           # DPSLAB_NKNOBS
BATCH_STREAMS, BATCH_WAVES = 0, 1    # DPSLAB_BATCH_STREAMS, DPSLAB_BATCH_WAVES


class DpslabError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dpslab error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("H", ctypes.c_double),
                ("eps", ctypes.c_double), ("eps_b", ctypes.c_double), ("eps_t", ctypes.c_double),
                ("gw", ctypes.c_double), ("tol", ctypes.c_double),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("xi", ctypes.c_double), ("r_cut", ctypes.c_double), ("n_sigma", ctypes.c_double),
                ("precision", ctypes.c_int), ("strict", ctypes.c_int)]


class Derived(ctypes.Structure):
    _fields_ = [("hx", ctypes.c_double), ("hy", ctypes.c_double), ("h", ctypes.c_double),
                ("xi", ctypes.c_double), ("gt", ctypes.c_double),
                ("n_sigma", ctypes.c_double), ("HE", ctypes.c_double),
                ("r_cut", ctypes.c_double), ("r_nf", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("Hbar", ctypes.c_double),
                ("kmax", ctypes.c_double),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("support_x", ctypes.c_int), ("support_y", ctypes.c_int), ("violations", ctypes.c_int)]


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2101_07088_b300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, D = ctypes.POINTER(Params), ctypes.POINTER(Derived)
        vp, dp, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
        sig = {
            "dpslab_derive": (ctypes.c_int, [P, D]),
            "dpslab_table": (ctypes.c_int, [P, ctypes.c_int, dp, ctypes.c_int]),
            "dpslab_plan_create": (ctypes.c_int, [P, i64, ctypes.POINTER(vp)]),
            "dpslab_plan_derived": (ctypes.c_int, [vp, D]),
            "dpslab_plan_device_bytes": (i64, [vp]),
            "dpslab_solve": (ctypes.c_int, [vp, i64, vp, vp, dp, vp, vp, vp]),
            "dpslab_solve_host": (ctypes.c_int, [vp, i64, vp, vp, dp, vp, vp, vp]),
            "dpslab_debug_fetch": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_size_t]),
            "dpslab_last_launch_count": (ctypes.c_int, [vp]),
            "dpslab_plan_set_wait_limit": (ctypes.c_int, [vp, i64]),
            "dpslab_plan_destroy": (ctypes.c_int, [vp]),
            "dpslab_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "dpslab_plan_footprint": (ctypes.c_int, [P, i64, ctypes.POINTER(i64)]),
            "dpslab_plan_create_unbound": (ctypes.c_int, [P, i64, ctypes.POINTER(vp)]),
            "dpslab_plan_set_wall_charge": (ctypes.c_int, [vp, vp, vp, vp]),
            "dpslab_bd_init_noise": (ctypes.c_int, [ctypes.c_uint64, i64, vp, vp]),
            "dpslab_bd_step_enqueue": (ctypes.c_int, [vp, ctypes.POINTER(BdParams), i64, vp, vp, vp, ctypes.c_uint64,
                                                      vp, vp]),
            "dpslab_bd_last_retries": (ctypes.c_int, [vp]),
            "dpslab_plan_autotune": (ctypes.c_int, [vp, i64, vp, vp, ctypes.c_int, vp]),
            "dpslab_plan_tuning": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
            "dpslab_plan_set_tuning": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
            "dpslab_plan_work_bytes": (i64, [vp]),
            "dpslab_plan_bind_work": (ctypes.c_int, [vp, vp, i64]),
            "dpslab_solve_enqueue": (ctypes.c_int, [vp, i64, vp, vp, vp, vp, vp]),
            "dpslab_solve_poll": (ctypes.c_int, [vp, dp]),
            "dpslab_batch_create": (ctypes.c_int, [P, ctypes.POINTER(i64), ctypes.c_int, ctypes.c_int,
                                                   ctypes.POINTER(vp)]),
            "dpslab_batch_solve": (ctypes.c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(vp), ctypes.POINTER(vp), dp,
                                                  ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                  ctypes.POINTER(ctypes.c_int), vp]),
            "dpslab_batch_device_bytes": (i64, [vp]),
            "dpslab_batch_last_launch_count": (ctypes.c_int, [vp]),
            "dpslab_batch_set_schedule": (ctypes.c_int, [vp, ctypes.c_int]),
            "dpslab_batch_schedule": (ctypes.c_int, [vp]),
            "dpslab_batch_autotune": (ctypes.c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                     ctypes.c_int, vp]),
            "dpslab_batch_destroy": (ctypes.c_int, [vp]),
            "dpslab_profile": (ctypes.c_int, [vp, ctypes.c_int]),
            "dpslab_stage_times": (ctypes.c_int, [vp, dp, ctypes.c_int]),
            "dpslab_stage_name": (ctypes.c_char_p, [ctypes.c_int]),
            "dpslab_near_field_static": (ctypes.c_int, [P, i64, vp, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _check(code):
    if code != OK:
        raise DpslabError(code, lib().dpslab_strerror(code).decode())


def make_params(Lx, Ly, H, gw, tol, nx, ny, nz=0, eps=1.0, eps_b=1.0, eps_t=1.0, xi=0.0,
                r_cut=0.0, n_sigma=0.0, precision=FP64, strict=0):
    return Params(float(Lx), float(Ly), float(H), float(eps), float(eps_b), float(eps_t), float(gw),
                  float(tol), int(nx), int(ny), int(nz), float(xi), float(r_cut), float(n_sigma),
                  int(precision), int(strict))


def _as_params(p):
    return p if isinstance(p, Params) else make_params(**p)


def derive(params):
    """dpslab_derive: the derived quantities as a dict (host only)."""
    d = Derived()
    _check(lib().dpslab_derive(ctypes.byref(_as_params(params)), ctypes.byref(d)))
    return {name: getattr(d, name) for name, _ in Derived._fields_}


def table(params, which):
    """dpslab_table: 0 nodes, 1 quadrature weights, 2 gauge weights."""
    p = _as_params(params)
    nz = derive(p)["nz"]
    out = np.zeros(nz)
    _check(lib().dpslab_table(ctypes.byref(p), int(which), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nz))
    return out


def near_field_static(params, pos, q, out, stream=None, check=True):
    """dpslab_near_field_static: near-field part only, no allocation by the
    library (for callers that cannot allocate device memory). pos [n, 3],
    q [n], out [n, 4]: float64 contiguous CUDA tensors. Returns the code."""
    import torch
    p = _as_params(params)
    st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = lib().dpslab_near_field_static(ctypes.byref(p), q.shape[0], pos.data_ptr(), q.data_ptr(),
                                        out.data_ptr(), st)
    if check:
        _check(rc)
    return rc


class BdParams(ctypes.Structure):
    """dpslab_bd_params (Brownian dynamics, Sec. 7.1)."""
    _fields_ = [("dt", ctypes.c_double), ("mu", ctypes.c_double), ("kT", ctypes.c_double),
                ("a", ctypes.c_double), ("U0", ctypes.c_double), ("r_m", ctypes.c_double),
                ("p", ctypes.c_int), ("max_retries", ctypes.c_int), ("max_disp", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


def bd_params(dt, mu, kT, a, U0, r_m, p, max_retries=8, max_disp=0.0, seed=0):
    return BdParams(float(dt), float(mu), float(kT), float(a), float(U0), float(r_m), int(p), int(max_retries),
                    float(max_disp), int(seed))


def bd_init_noise(seed, W, stream=None):
    """dpslab_bd_init_noise: W^0 into the CUDA float64 tensor W [n, 3]."""
    import torch
    st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    _check(lib().dpslab_bd_init_noise(int(seed), W.shape[0], W.data_ptr(), st))


def plan_bytes(params, max_n):
    """dpslab_plan_footprint: device bytes a plan for (params, max_n) takes."""
    p = _as_params(params)
    b = ctypes.c_int64(0)
    _check(lib().dpslab_plan_footprint(ctypes.byref(p), int(max_n), ctypes.byref(b)))
    return b.value


class Plan:
    """dpslab_plan_create / dpslab_solve / dpslab_plan_destroy. With
    own_work=False the plan is created unbound (dpslab_plan_create_unbound):
    bind a workspace with bind_work() before solving."""

    def __init__(self, params, max_n, own_work=True):
        self.params = _as_params(params)
        h = ctypes.c_void_p()
        create = lib().dpslab_plan_create if own_work else lib().dpslab_plan_create_unbound
        _check(create(ctypes.byref(self.params), int(max_n), ctypes.byref(h)))
        self._h = h
        self.max_n = int(max_n)
        d = Derived()
        _check(lib().dpslab_plan_derived(self._h, ctypes.byref(d)))
        self.derived = {name: getattr(d, name) for name, _ in Derived._fields_}
        self.device_bytes = lib().dpslab_plan_device_bytes(self._h)
        self.work_bytes = lib().dpslab_plan_work_bytes(self._h)
        self.work = None

    def bd_enqueue(self, bp, pos, q, W, step, force=None, stream=None):
        """dpslab_bd_step_enqueue: one Brownian-dynamics step on `stream`
        (pos and W updated in place when accepted); finish with poll()."""
        import torch
        st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
        _check(lib().dpslab_bd_step_enqueue(self._h, ctypes.byref(bp), q.shape[0], pos.data_ptr(), q.data_ptr(),
                                            W.data_ptr(), int(step),
                                            force.data_ptr() if force is not None else None, st))

    def autotune(self, pos, q, reps=5, stream=None):
        """dpslab_plan_autotune on device inputs; returns the chosen knobs."""
        import torch
        st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
        _check(lib().dpslab_plan_autotune(self._h, q.shape[0], pos.data_ptr(), q.data_ptr(), int(reps), st))
        return self.tuning()

    def tuning(self):
        """The NKNOBS launch-shape knobs (dpslab_plan_tuning)."""
        k = (ctypes.c_int * NKNOBS)()
        _check(lib().dpslab_plan_tuning(self._h, k, NKNOBS))
        return list(k)

    def set_tuning(self, knobs):
        """Apply 4 (FFT shapes only) or NKNOBS knobs (dpslab_plan_set_tuning)."""
        k = (ctypes.c_int * len(knobs))(*[int(v) for v in knobs])
        _check(lib().dpslab_plan_set_tuning(self._h, k, len(knobs)))

    def last_bd_retries(self):
        return lib().dpslab_bd_last_retries(self._h)

    def bd_step(self, bp, pos, q, W, step, force=None, stream=None, check=True):
        """One step, waited for: returns (code, retries used)."""
        self.bd_enqueue(bp, pos, q, W, step, force, stream)
        while True:
            code, _ = self.poll()
            if code != PENDING:
                break
        if check:
            _check(code)
        return code, lib().dpslab_bd_last_retries(self._h)

    def set_wall_charge(self, sigma_b=None, sigma_t=None, stream=None):
        """dpslab_plan_set_wall_charge: numpy arrays (ny, nx) of the wall
        charge densities at (i hx, j hy) ([j, i]), or None."""
        import numpy as np
        import torch
        keep = []

        def ptr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            d = self.derived
            if a.shape != (d["ny"], d["nx"]):
                raise ValueError(f"wall charge grid must be (ny, nx) = ({d['ny']}, {d['nx']})")
            keep.append(a)
            return a.ctypes.data

        st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
        _check(lib().dpslab_plan_set_wall_charge(self._h, ptr(sigma_b), ptr(sigma_t), st))
        self.device_bytes = lib().dpslab_plan_device_bytes(self._h)

    def bind_work(self, work):
        """dpslab_plan_bind_work: `work` a CUDA uint8 tensor of at least
        work_bytes bytes (kept referenced while bound), or None to unbind."""
        if work is None:
            _check(lib().dpslab_plan_bind_work(self._h, None, 0))
        else:
            _check(lib().dpslab_plan_bind_work(self._h, work.data_ptr(), work.numel() * work.element_size()))
        self.work = work

    def close(self):
        if getattr(self, "_h", None):
            lib().dpslab_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, pos, q, phi=None, force=None, energy=True, stream=None, check=True):
        """pos [n, 3], q [n]: float64 contiguous CUDA tensors. phi [n] and
        force [n, 3] are optional output tensors (None skips that output).
        Returns (U or None, return code)."""
        import torch
        for t in (pos, q):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("pos and q must be contiguous float64 CUDA tensors")
        n = q.shape[0]
        U = ctypes.c_double(math.nan)
        st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
        rc = lib().dpslab_solve(self._h, n, pos.data_ptr(), q.data_ptr(),
                                ctypes.byref(U) if energy else None,
                                phi.data_ptr() if phi is not None else None,
                                force.data_ptr() if force is not None else None, st)
        if check:
            _check(rc)
        return (U.value if energy else None), rc

    def enqueue(self, pos, q, phi=None, force=None, stream=None):
        """dpslab_solve_enqueue: start the solve on `stream` and return at
        once (poll() tells when it is done)."""
        import torch
        for t in (pos, q):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("pos and q must be contiguous float64 CUDA tensors")
        st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
        _check(lib().dpslab_solve_enqueue(self._h, q.shape[0], pos.data_ptr(), q.data_ptr(),
                                          phi.data_ptr() if phi is not None else None,
                                          force.data_ptr() if force is not None else None, st))

    def poll(self):
        """dpslab_solve_poll: (PENDING, None) while running, then (code, U)."""
        U = ctypes.c_double(math.nan)
        rc = lib().dpslab_solve_poll(self._h, ctypes.byref(U))
        return (rc, None) if rc == PENDING else (rc, U.value)

    def solve_host(self, pos, q, want_phi=True, want_force=True, stream=None, check=True, phi=None, force=None):
        """Host (numpy) buffers; copies happen inside the library call.
        phi [n] and force [n, 3] may be given as C-contiguous float64 arrays
        (pinned memory, e.g. a pinned torch tensor's .numpy(), makes the
        device-to-host copies asynchronous and fast); otherwise they are
        allocated. Returns (U, phi or None, force or None, return code)."""
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.float64)
        n = q.shape[0]

        def out(a, shape, want):
            if not want:
                return None
            if a is None:
                return np.empty(shape)
            if a.shape != shape or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or not a.flags["WRITEABLE"]:
                raise ValueError(f"output must be a writeable C-contiguous float64 array of shape {shape}")
            return a
        phi = out(phi, (n,), want_phi)
        force = out(force, (n, 3), want_force)
        U = ctypes.c_double(math.nan)
        st = None
        if stream is not None:
            st = stream.cuda_stream
        rc = lib().dpslab_solve_host(self._h, n, pos.ctypes.data, q.ctypes.data, ctypes.byref(U),
                                     phi.ctypes.data if phi is not None else None,
                                     force.ctypes.data if force is not None else None, st)
        if check:
            _check(rc)
        return U.value, phi, force, rc

    def debug_fetch(self, which, n):
        d = self.derived
        shapes = {0: (2, d["nz"], d["ny"], d["nx"]), 1: (d["nz"], d["ny"], d["nx"], 4),
                  2: (n, 4), 3: (n, 4), 4: (4,)}
        out = np.zeros(shapes[which])
        _check(lib().dpslab_debug_fetch(self._h, int(which), out.ctypes.data, out.nbytes))
        return out

    def last_launch_count(self):
        return lib().dpslab_last_launch_count(self._h)

    def set_wait_limit(self, polls=WAIT_LIMIT_DEFAULT):
        """dpslab_plan_set_wait_limit: polls of each bounded wait of the
        tensor-core z transforms before the solve reports ERR_TIMEOUT."""
        _check(lib().dpslab_plan_set_wait_limit(self._h, int(polls)))

    def profile(self, on=True, near_in_line=False):
        """Stage timing on (the near field stays on the second stream and is
        timed there) or off; near_in_line runs the near field in line."""
        _check(lib().dpslab_profile(self._h, (2 if near_in_line else 1) if on else 0))

    def stage_times(self):
        """{stage name: device ms} of the last solve (profiling on)."""
        ms = (ctypes.c_double * NSTAGES)()
        _check(lib().dpslab_stage_times(self._h, ms, NSTAGES))
        return {lib().dpslab_stage_name(i).decode(): ms[i] for i in range(NSTAGES)}


class Batch:
    """dpslab_batch_create / dpslab_batch_solve / dpslab_batch_destroy: many
    independent systems solved by one call (one CUDA graph, replayed while
    the buffers stay the same)."""

    def __init__(self, params_list, max_n_list, nstreams=8):
        self.count = len(params_list)
        self._params = (Params * self.count)(*[_as_params(p) for p in params_list])
        mx = (ctypes.c_int64 * self.count)(*[int(v) for v in max_n_list])
        h = ctypes.c_void_p()
        _check(lib().dpslab_batch_create(self._params, mx, self.count, int(nstreams), ctypes.byref(h)))
        self._h = h
        self.device_bytes = lib().dpslab_batch_device_bytes(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().dpslab_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, pos, q, phi=None, force=None, stream=None, check=True):
        """pos, q: lists of float64 contiguous CUDA tensors ([n_i, 3], [n_i]);
        phi, force: lists of output tensors (or None). Returns (U [count],
        status [count]) as numpy arrays."""
        import torch
        c = self.count
        vp = ctypes.c_void_p
        for t in list(pos) + list(q):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("pos and q must be contiguous float64 CUDA tensors")
        n = (ctypes.c_int64 * c)(*[int(t.shape[0]) for t in q])
        P = (vp * c)(*[t.data_ptr() for t in pos])
        Q = (vp * c)(*[t.data_ptr() for t in q])
        PH = (vp * c)(*[t.data_ptr() if t is not None else None for t in phi]) if phi is not None else None
        FO = (vp * c)(*[t.data_ptr() if t is not None else None for t in force]) if force is not None else None
        U = np.zeros(c)
        status = np.zeros(c, dtype=np.int32)
        st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
        rc = lib().dpslab_batch_solve(self._h, n, P, Q, U.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), PH, FO,
                                      status.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), st)
        if check:
            _check(rc)
        return U, status

    def last_launch_count(self):
        """Kernels launched by the last solve, over all systems."""
        return lib().dpslab_batch_last_launch_count(self._h)

    def set_schedule(self, schedule):
        """BATCH_STREAMS or BATCH_WAVES (dpslab_batch_set_schedule)."""
        _check(lib().dpslab_batch_set_schedule(self._h, int(schedule)))

    def schedule(self):
        return lib().dpslab_batch_schedule(self._h)

    def autotune(self, pos, q, reps=3, stream=None):
        """dpslab_batch_autotune on device inputs; returns the schedule kept."""
        import torch
        c = self.count
        vp = ctypes.c_void_p
        n = (ctypes.c_int64 * c)(*[int(t.shape[0]) for t in q])
        P = (vp * c)(*[t.data_ptr() for t in pos])
        Q = (vp * c)(*[t.data_ptr() for t in q])
        st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
        _check(lib().dpslab_batch_autotune(self._h, n, P, Q, int(reps), st))
        return self.schedule()
