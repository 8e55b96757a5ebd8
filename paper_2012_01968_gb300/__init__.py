"""Python binding of the GB300 negacyclic RNS NTT library (libntt_gb300.so).

The functions mirror the C ABI in include/ntt_gb300.h one to one and only
marshal arguments: every transform step runs in the library's CUDA kernels.
Device buffers may be given as torch CUDA tensors (uint64 or int64, contiguous)
or as raw integer addresses; streams as torch.cuda.Stream, a raw handle, or
None (torch's current stream when a tensor is passed, else the default
stream).  There is no CPU fallback: if the library is missing, importing the
functions raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libntt_gb300.so")
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "ntt_gb300.h")

NTT_OK = 0
NTT_ERR_INVALID_ARG = 1
NTT_ERR_BAD_PRIME = 2
NTT_ERR_MISALIGNED = 3
NTT_ERR_CUDA = 4
NTT_ERR_OOM = 5
NTT_ERR_BUSY = 6
NTT_ERR_TIMEOUT = 7
NTT_ERR_DEVICE = 8
NTT_ERR_LIMIT = 9

NTT_NOALLOC_MAX_LIMBS = 8192

NTT_TWIDDLE_AUTO = 0
NTT_TWIDDLE_TABLE = 1
NTT_TWIDDLE_OT = 2

NTT_KERNEL_AUTO = 0
NTT_KERNEL_FUSED = 1
NTT_KERNEL_PER_PASS = 2
NTT_KERNEL_RADIX2 = 3
NTT_KERNEL_HIGH_RADIX = 4
NTT_KERNEL_CLUSTER = 5

NTT_GEOMETRY_DEFAULT = 0
NTT_GEOMETRY_SMALL_ROW_TILE = 1
NTT_GEOMETRY_ALT_SPLIT = 2

NTT_PLAN_L2_TWIDDLES = 1

NTT_OP_FORWARD = 1
NTT_OP_INVERSE = 2

NTT_REQ_HOST = 1

_u32, _u64, _vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
_u64p = ctypes.POINTER(ctypes.c_uint64)


class PlanOpts(ctypes.Structure):
    _fields_ = [("twiddle_mode", _u32), ("ot_stages", _u32), ("kernel", _u32), ("geometry", _u32),
                ("flags", _u32), ("radix_log2", _u32), ("ctas_per_sm", _u32), ("reserved", _u32)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("opts", PlanOpts), ("forward_us", ctypes.c_double), ("inverse_us", ctypes.c_double),
                ("status", ctypes.c_int), ("reserved", _u32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("N", _u32), ("L", _u32), ("log2_N", _u32), ("passes", _u32),
                ("pass1_log2", _u32), ("twiddle_mode", _u32), ("ot_stages", _u32),
                ("device", _u32), ("kernel", _u32), ("device_bytes", _u64), ("geometry", _u32),
                ("row_tile_log2", _u32), ("radix_log2", _u32), ("ctas_per_sm", _u32)]


class Job(ctypes.Structure):
    _fields_ = [("plan", _vp), ("data", _vp), ("batch", _u32), ("levels", _u32), ("op", _u32),
                ("reserved", _u32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", _u64), ("arena_bytes", _u64), ("max_batch_jobs", _u32),
                ("slots", _u32), ("max_queue", _u32), ("reserved", _u32 * 3)]


class Request(ctypes.Structure):
    _fields_ = [("plan", _vp), ("data", _vp), ("host_out", _vp), ("batch", _u32), ("levels", _u32),
                ("op", _u32), ("flags", _u32)]


class RequestTimes(ctypes.Structure):
    _fields_ = [("submit_ns", ctypes.c_int64), ("start_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
                ("device_ns", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("batches", _u64), ("requests", _u64), ("max_launch_ns", ctypes.c_int64),
                ("max_loop_gap_ns", ctypes.c_int64), ("max_completion_gap_ns", ctypes.c_int64),
                ("max_device_ns", ctypes.c_int64), ("reserved", ctypes.c_int64 * 4)]


class NttError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib().ntt_status_string(status).decode()
        if status == NTT_ERR_CUDA:
            msg += " (" + _lib().ntt_last_cuda_error().decode() + ")"
        super().__init__(f"{where}: {msg}")


_lock = threading.Lock()
_L = None


def build(verbose: bool = False) -> str:
    from . import builder
    return builder.build(verbose=verbose)


def _lib():
    global _L
    if _L is not None:
        return _L
    with _lock:
        if _L is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run paper_2012_01968_gb300.build() or python -m paper_2012_01968_gb300.builder)")
            L = ctypes.CDLL(LIB_PATH)
            S = ctypes.c_int
            L.ntt_plan_create.restype = S
            L.ntt_plan_create.argtypes = [ctypes.POINTER(_vp), _u32, _u64p, _u32, ctypes.POINTER(PlanOpts)]
            L.ntt_plan_destroy.restype = None
            L.ntt_plan_destroy.argtypes = [_vp]
            L.ntt_plan_clone.restype = S
            L.ntt_plan_clone.argtypes = [ctypes.POINTER(_vp), _vp]
            L.ntt_plan_set_ctas_per_sm.restype = S
            L.ntt_plan_set_ctas_per_sm.argtypes = [_vp, _u32]
            for f in ("ntt_forward", "ntt_inverse"):
                getattr(L, f).restype = S
                getattr(L, f).argtypes = [_vp, _vp, _u32, _vp]
            for f in ("ntt_forward_levels", "ntt_inverse_levels"):
                getattr(L, f).restype = S
                getattr(L, f).argtypes = [_vp, _vp, _u32, _u32, _vp]
            L.ntt_mul_negacyclic.restype = S
            L.ntt_mul_negacyclic.argtypes = [_vp, _vp, _vp, _vp, _u32, _vp]
            L.ntt_mul_pointwise.restype = S
            L.ntt_mul_pointwise.argtypes = [_vp, _vp, _vp, _vp, _u32, _vp]
            L.ntt_execute.restype = S
            L.ntt_execute.argtypes = [_vp, _vp, _u32, _u32, _vp]
            for f in ("ntt_execute_host", "ntt_execute_host_async"):
                getattr(L, f).restype = S
                getattr(L, f).argtypes = [_vp, _vp, _vp, _u32, _u32, _vp]
            L.ntt_transform_noalloc.restype = S
            L.ntt_transform_noalloc.argtypes = [_vp, _vp, _u32, _u32, _u32, _vp]
            L.ntt_batch_create.restype = S
            L.ntt_batch_create.argtypes = [ctypes.POINTER(_vp)]
            L.ntt_batch_destroy.restype = None
            L.ntt_batch_destroy.argtypes = [_vp]
            L.ntt_batch_submit.restype = S
            L.ntt_batch_submit.argtypes = [_vp, ctypes.POINTER(Job), _u32, _vp]
            L.ntt_batch_device_status.restype = S
            L.ntt_batch_device_status.argtypes = [_vp, ctypes.POINTER(_u32)]
            L.ntt_server_create.restype = S
            L.ntt_server_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(ServerOpts)]
            L.ntt_server_destroy.restype = None
            L.ntt_server_destroy.argtypes = [_vp]
            L.ntt_server_submit.restype = S
            L.ntt_server_submit.argtypes = [_vp, ctypes.POINTER(Request), ctypes.POINTER(_u64)]
            L.ntt_server_wait.restype = S
            L.ntt_server_wait.argtypes = [_vp, _u64, _u64]
            L.ntt_server_request_times.restype = S
            L.ntt_server_request_times.argtypes = [_vp, _u64, ctypes.POINTER(RequestTimes)]
            L.ntt_server_release.restype = S
            L.ntt_server_release.argtypes = [_vp, _u64]
            L.ntt_server_stats_get.restype = S
            L.ntt_server_stats_get.argtypes = [_vp, ctypes.POINTER(ServerStats)]
            L.ntt_measure_butterfly_rate.restype = S
            L.ntt_measure_butterfly_rate.argtypes = [ctypes.POINTER(ctypes.c_double)]
            L.ntt_plan_query.restype = S
            L.ntt_plan_query.argtypes = [_vp, ctypes.POINTER(PlanInfo)]
            L.ntt_plan_device_status.restype = S
            L.ntt_plan_device_status.argtypes = [_vp, ctypes.POINTER(_u32)]
            L.ntt_plan_psi.restype = S
            L.ntt_plan_psi.argtypes = [_vp, _u32, _u64p]
            L.ntt_autotune.restype = S
            L.ntt_autotune.argtypes = [_u32, _u64p, _u32, _u32, _u32, ctypes.POINTER(PlanOpts),
                                       ctypes.POINTER(TuneEntry), _u32, ctypes.POINTER(_u32)]
            L.ntt_plan32_create.restype = S
            L.ntt_plan32_create.argtypes = [ctypes.POINTER(_vp), _u32, ctypes.POINTER(_u32), _u32, _u32, _u32]
            L.ntt_plan32_device_status.restype = S
            L.ntt_plan32_device_status.argtypes = [_vp, ctypes.POINTER(_u32)]
            L.ntt_plan32_destroy.restype = None
            L.ntt_plan32_destroy.argtypes = [_vp]
            for f in ("ntt_forward32", "ntt_inverse32"):
                getattr(L, f).restype = S
                getattr(L, f).argtypes = [_vp, _vp, _u32, _vp]
            L.ntt_plan32_psi.restype = S
            L.ntt_plan32_psi.argtypes = [_vp, _u32, ctypes.POINTER(_u32)]
            L.ntt_status_string.restype = ctypes.c_char_p
            L.ntt_status_string.argtypes = [S]
            L.ntt_last_cuda_error.restype = ctypes.c_char_p
            L.ntt_last_cuda_error.argtypes = []
            _L = L
    return _L


def lib():
    """The loaded ctypes library (raises if it was not built)."""
    return _lib()


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------
def _addr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return int(x.data_ptr())
    raise TypeError(f"cannot take a device address of {type(x)!r}")


def _stream(stream, like=None) -> int:
    if stream is None:
        if like is not None and hasattr(like, "data_ptr"):
            import torch
            return int(torch.cuda.current_stream(like.device).cuda_stream)
        return 0
    if isinstance(stream, int):
        return stream
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    raise TypeError(f"bad stream {type(stream)!r}")


def _check(st: int, where: str):
    if st != NTT_OK:
        raise NttError(st, where)


# --------------------------------------------------------------------------
# C ABI, same names
# --------------------------------------------------------------------------
def ntt_plan_create(N: int, primes, twiddle_mode: int = NTT_TWIDDLE_AUTO, ot_stages: int = 0,
                    kernel: int = NTT_KERNEL_AUTO, geometry: int = NTT_GEOMETRY_DEFAULT, flags: int = 0,
                    radix_log2: int = 0, ctas_per_sm: int = 0) -> int:
    """Create a plan; returns the opaque handle (an int).  Raises NttError."""
    primes = [int(p) for p in primes]
    arr = (_u64 * len(primes))(*primes)
    opts = PlanOpts(twiddle_mode, ot_stages, kernel, geometry, flags, radix_log2, ctas_per_sm)
    out = _vp()
    _check(_lib().ntt_plan_create(ctypes.byref(out), N, arr, len(primes), ctypes.byref(opts)),
           "ntt_plan_create")
    return int(out.value)


def ntt_plan_create_status(N: int, primes, twiddle_mode: int = 0, ot_stages: int = 0, reserved=None,
                           kernel: int = 0, geometry: int = 0, flags: int = 0, radix_log2: int = 0,
                           ctas_per_sm: int = 0):
    """Like ntt_plan_create but returns (status, handle) without raising."""
    primes = [int(p) for p in primes]
    arr = (_u64 * max(1, len(primes)))(*primes)
    opts = PlanOpts(twiddle_mode, ot_stages, kernel, geometry, flags, radix_log2, ctas_per_sm)
    if reserved:
        opts.reserved = int(reserved[0])
    out = _vp()
    st = _lib().ntt_plan_create(ctypes.byref(out), N, arr if primes else None, len(primes),
                                ctypes.byref(opts))
    return st, (int(out.value) if out.value else 0)


def ntt_plan_destroy(plan: int) -> None:
    _lib().ntt_plan_destroy(plan)


def ntt_forward(plan: int, data, batch: int, stream=None) -> None:
    _check(_lib().ntt_forward(plan, _addr(data), batch, _stream(stream, data)), "ntt_forward")


def ntt_inverse(plan: int, data, batch: int, stream=None) -> None:
    _check(_lib().ntt_inverse(plan, _addr(data), batch, _stream(stream, data)), "ntt_inverse")


def ntt_forward_levels(plan: int, data, batch: int, levels: int, stream=None) -> None:
    _check(_lib().ntt_forward_levels(plan, _addr(data), batch, levels, _stream(stream, data)),
           "ntt_forward_levels")


def ntt_inverse_levels(plan: int, data, batch: int, levels: int, stream=None) -> None:
    _check(_lib().ntt_inverse_levels(plan, _addr(data), batch, levels, _stream(stream, data)),
           "ntt_inverse_levels")


def ntt_mul_pointwise(plan: int, a, b, c, batch: int, stream=None) -> None:
    _check(_lib().ntt_mul_pointwise(plan, _addr(a), _addr(b), _addr(c), batch, _stream(stream, a)),
           "ntt_mul_pointwise")


def ntt_mul_negacyclic(plan: int, a, b, c, batch: int, stream=None) -> None:
    """c = a * b mod (X^N + 1) per limb; a factor that c does not alias is left
    holding its transform.  With c aliasing a or b (fused plans) the inverse's
    first pass applies the element-wise product."""
    _check(_lib().ntt_mul_negacyclic(plan, _addr(a), _addr(b), _addr(c), batch, _stream(stream, a)),
           "ntt_mul_negacyclic")


def ntt_execute(plan: int, data, batch: int, ops: int, stream=None) -> None:
    """Device data in place: forward, inverse, or both (one launch for fused plans)."""
    _check(_lib().ntt_execute(plan, _addr(data), batch, ops, _stream(stream, data)), "ntt_execute")


def _host_ptr(x) -> int:
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    return int(x)


def ntt_execute_host(plan: int, host_in, host_out, batch: int, ops: int, stream=None) -> None:
    """host_in / host_out: numpy uint64 arrays or CPU torch tensors (pinned for speed)."""
    _check(_lib().ntt_execute_host(plan, _host_ptr(host_in), _host_ptr(host_out), batch, ops, _stream(stream)),
           "ntt_execute_host")


def ntt_execute_host_async(plan: int, host_in, host_out, batch: int, ops: int, stream=None) -> None:
    """As ntt_execute_host without waiting: `stream` is ordered after the result
    lands in host_out; keep both buffers alive (and host_in unchanged) until then."""
    _check(_lib().ntt_execute_host_async(plan, _host_ptr(host_in), _host_ptr(host_out), batch, ops,
                                         _stream(stream)), "ntt_execute_host_async")


def ntt_transform_noalloc(plan: int, data, batch: int, levels: int, op: int, stream=None) -> None:
    """One forward or inverse transform that allocates nothing (fixed device
    work area shared by all such calls on a device; calls must not overlap)."""
    _check(_lib().ntt_transform_noalloc(plan, _addr(data), batch, levels, op, _stream(stream, data)),
           "ntt_transform_noalloc")


def ntt_batch_create() -> int:
    h = _vp()
    _check(_lib().ntt_batch_create(ctypes.byref(h)), "ntt_batch_create")
    return h.value


def ntt_batch_destroy(batch: int) -> None:
    _lib().ntt_batch_destroy(batch)


def make_jobs(jobs):
    """jobs: iterable of (plan handle, data, batch, levels, op) -> ctypes array of Job."""
    jobs = list(jobs)
    arr = (Job * len(jobs))()
    for i, (plan, data, batch, levels, op) in enumerate(jobs):
        arr[i] = Job(plan, _addr(data), batch, levels, op, 0)
    return arr


def ntt_batch_submit(batch: int, jobs, stream=None) -> None:
    """jobs: a ctypes Job array (make_jobs) or an iterable of (plan, data, batch, levels, op)."""
    like = None
    if not isinstance(jobs, ctypes.Array):
        jobs = list(jobs)
        like = next((j[1] for j in jobs if hasattr(j[1], "data_ptr")), None)
        jobs = make_jobs(jobs)
    _check(_lib().ntt_batch_submit(batch, jobs, len(jobs), _stream(stream, like)), "ntt_batch_submit")


def ntt_batch_device_status(batch: int) -> int:
    v = _u32()
    _check(_lib().ntt_batch_device_status(batch, ctypes.byref(v)), "ntt_batch_device_status")
    return v.value


def ntt_measure_butterfly_rate() -> float:
    """Butterflies per second (1e9) of a register-only loop of the transform's butterfly."""
    v = ctypes.c_double()
    _check(_lib().ntt_measure_butterfly_rate(ctypes.byref(v)), "ntt_measure_butterfly_rate")
    return v.value


def ntt_plan_query(plan: int) -> PlanInfo:
    info = PlanInfo()
    _check(_lib().ntt_plan_query(plan, ctypes.byref(info)), "ntt_plan_query")
    return info


def ntt_plan_device_status(plan: int) -> int:
    v = _u32()
    _check(_lib().ntt_plan_device_status(plan, ctypes.byref(v)), "ntt_plan_device_status")
    return int(v.value)


def ntt_plan_psi(plan: int, l: int) -> int:
    v = _u64()
    _check(_lib().ntt_plan_psi(plan, l, ctypes.byref(v)), "ntt_plan_psi")
    return int(v.value)


def ntt_autotune(N: int, primes, batch: int = 1, reps: int = 0, entries: bool = True):
    """Time every compiled configuration on the current device; returns
    (best PlanOpts, [TuneEntry, ...]).  With entries=False the cached choice is
    returned when there is one (and the list is empty)."""
    primes = [int(p) for p in primes]
    arr = (_u64 * max(1, len(primes)))(*primes)
    best = PlanOpts()
    cap = 64
    buf = (TuneEntry * cap)() if entries else None
    cnt = _u32()
    _check(_lib().ntt_autotune(N, arr, len(primes), batch, reps, ctypes.byref(best), buf, cap if entries else 0,
                               ctypes.byref(cnt)), "ntt_autotune")
    out = [buf[i] for i in range(min(cnt.value, cap))] if entries else []
    return best, out


def ntt_plan32_create_status(N: int, primes, kernel: int = NTT_KERNEL_AUTO, twiddle_mode: int = NTT_TWIDDLE_AUTO):
    """Create a 32-bit plan; returns (status, handle) without raising."""
    primes = [int(p) for p in primes]
    arr = (_u32 * max(1, len(primes)))(*primes)
    out = _vp()
    st = _lib().ntt_plan32_create(ctypes.byref(out), N, arr if primes else None, len(primes), kernel, twiddle_mode)
    return st, (int(out.value) if out.value else 0)


def ntt_plan32_create(N: int, primes, kernel: int = NTT_KERNEL_AUTO, twiddle_mode: int = NTT_TWIDDLE_AUTO) -> int:
    """Create a 32-bit plan (primes q < 2^28); returns the handle.  Raises NttError."""
    st, h = ntt_plan32_create_status(N, primes, kernel, twiddle_mode)
    _check(st, "ntt_plan32_create")
    return h


def ntt_plan32_destroy(plan: int) -> None:
    _lib().ntt_plan32_destroy(plan)


def ntt_forward32(plan: int, data, batch: int, stream=None) -> None:
    _check(_lib().ntt_forward32(plan, _addr(data), batch, _stream(stream, data)), "ntt_forward32")


def ntt_inverse32(plan: int, data, batch: int, stream=None) -> None:
    _check(_lib().ntt_inverse32(plan, _addr(data), batch, _stream(stream, data)), "ntt_inverse32")


def ntt_plan32_device_status(plan: int) -> int:
    v = _u32()
    _check(_lib().ntt_plan32_device_status(plan, ctypes.byref(v)), "ntt_plan32_device_status")
    return int(v.value)


def ntt_plan32_psi(plan: int, l: int) -> int:
    v = _u32()
    _check(_lib().ntt_plan32_psi(plan, l, ctypes.byref(v)), "ntt_plan32_psi")
    return int(v.value)


def ntt_status_string(status: int) -> str:
    return _lib().ntt_status_string(status).decode()


def ntt_last_cuda_error() -> str:
    return _lib().ntt_last_cuda_error().decode()


class Plan:
    """RAII wrapper over a plan handle."""

    def __init__(self, N: int, primes, twiddle_mode: int = NTT_TWIDDLE_AUTO, ot_stages: int = 0,
                 kernel: int = NTT_KERNEL_AUTO, geometry: int = NTT_GEOMETRY_DEFAULT, flags: int = 0,
                 radix_log2: int = 0, ctas_per_sm: int = 0):
        self.N = N
        self.primes = [int(p) for p in primes]
        self.L = len(self.primes)
        self.handle = ntt_plan_create(N, self.primes, twiddle_mode, ot_stages, kernel, geometry, flags, radix_log2,
                                      ctas_per_sm)

    @classmethod
    def from_opts(cls, N: int, primes, opts: PlanOpts, flags: int | None = None, ctas_per_sm: int | None = None):
        """A plan with the options an autotuner run returned (flags, ctas_per_sm: overrides)."""
        return cls(N, primes, opts.twiddle_mode, opts.ot_stages, opts.kernel, opts.geometry,
                   opts.flags if flags is None else flags, opts.radix_log2,
                   opts.ctas_per_sm if ctas_per_sm is None else ctas_per_sm)

    def clone(self) -> "Plan":
        """A plan sharing this one's device tables, with its own work area
        (ntt_plan_clone): for calls that overlap on another stream."""
        out = _vp()
        _check(_lib().ntt_plan_clone(ctypes.byref(out), self.handle), "ntt_plan_clone")
        c = object.__new__(type(self))
        c.N, c.primes, c.L, c.handle = self.N, list(self.primes), self.L, out.value
        return c

    def set_ctas_per_sm(self, ctas_per_sm: int) -> None:
        """Persistent CTAs per SM of this plan's fused launches (ntt_plan_set_ctas_per_sm)."""
        _check(_lib().ntt_plan_set_ctas_per_sm(self.handle, ctas_per_sm), "ntt_plan_set_ctas_per_sm")

    def forward(self, data, batch: int = 1, stream=None):
        ntt_forward(self.handle, data, batch, stream)

    def inverse(self, data, batch: int = 1, stream=None):
        ntt_inverse(self.handle, data, batch, stream)

    def execute(self, data, ops: int, batch: int = 1, stream=None):
        ntt_execute(self.handle, data, batch, ops, stream)

    def info(self) -> PlanInfo:
        return ntt_plan_query(self.handle)

    def device_status(self) -> int:
        return ntt_plan_device_status(self.handle)

    def close(self):
        if self.handle:
            ntt_plan_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan32:
    """RAII wrapper over a 32-bit plan handle (residues in int32/uint32 tensors)."""

    def __init__(self, N: int, primes, kernel: int = NTT_KERNEL_AUTO, twiddle_mode: int = NTT_TWIDDLE_AUTO):
        self.N = N
        self.primes = [int(p) for p in primes]
        self.L = len(self.primes)
        self.handle = ntt_plan32_create(N, self.primes, kernel, twiddle_mode)

    def device_status(self) -> int:
        return ntt_plan32_device_status(self.handle)

    def forward(self, data, batch: int = 1, stream=None):
        ntt_forward32(self.handle, data, batch, stream)

    def inverse(self, data, batch: int = 1, stream=None):
        ntt_inverse32(self.handle, data, batch, stream)

    def close(self):
        if self.handle:
            ntt_plan32_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def declared_symbols() -> list[str]:
    """Function names declared in include/ntt_gb300.h."""
    import re
    with open(HEADER) as f:
        txt = f.read()
    return sorted(set(re.findall(r"^(?:ntt_status|void|const char\*)\s+(ntt_\w+)\s*\(", txt, re.M)))


class Batch:
    """Owner of an ntt_batch handle (usable as a context manager)."""

    def __init__(self):
        self.handle = ntt_batch_create()

    def submit(self, jobs, stream=None):
        ntt_batch_submit(self.handle, jobs, stream)

    def device_status(self) -> int:
        return ntt_batch_device_status(self.handle)

    def close(self):
        if self.handle:
            ntt_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_addr(x) -> int:
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    return int(x)


class Server:
    """Owner of an ntt_server handle: submit requests, wait for them."""

    def __init__(self, hbm_budget_bytes: int, arena_bytes: int = 0, max_batch_jobs: int = 0, slots: int = 0,
                 max_queue: int = 0):
        o = ServerOpts(hbm_budget_bytes, arena_bytes, max_batch_jobs, slots, max_queue, (_u32 * 3)())
        h = _vp()
        _check(_lib().ntt_server_create(ctypes.byref(h), ctypes.byref(o)), "ntt_server_create")
        self.handle = h.value

    def submit_status(self, plan: int, data, batch: int, levels: int, op: int, host_out=None):
        """(status, ticket) without raising; host_out given => a host-buffer request."""
        host = host_out is not None
        r = Request(plan, _host_addr(data) if host else _addr(data), _host_addr(host_out) if host else None,
                    batch, levels, op, NTT_REQ_HOST if host else 0)
        t = _u64()
        st = _lib().ntt_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t))
        return st, t.value

    def submit(self, plan: int, data, batch: int, levels: int, op: int, host_out=None) -> int:
        st, t = self.submit_status(plan, data, batch, levels, op, host_out)
        _check(st, "ntt_server_submit")
        return t

    def wait_status(self, ticket: int, timeout_s: float = 60.0) -> int:
        return _lib().ntt_server_wait(self.handle, ticket, int(timeout_s * 1e9))

    def wait(self, ticket: int, timeout_s: float = 60.0) -> None:
        _check(self.wait_status(ticket, timeout_s), "ntt_server_wait")

    def times(self, ticket: int):
        """(submit_ns, start_ns, done_ns) on the steady clock, and the device
        time of the request's batch (device_ns)."""
        t = RequestTimes()
        _check(_lib().ntt_server_request_times(self.handle, ticket, ctypes.byref(t)), "ntt_server_request_times")
        return t.submit_ns, t.start_ns, t.done_ns, t.device_ns

    def release_status(self, ticket: int) -> int:
        return _lib().ntt_server_release(self.handle, ticket)

    def release(self, ticket: int) -> None:
        """Forget a finished request (its ticket and times)."""
        _check(self.release_status(ticket), "ntt_server_release")

    def stats(self) -> dict:
        """The scheduler's counters since creation (ntt_server_stats)."""
        st = ServerStats()
        _check(_lib().ntt_server_stats_get(self.handle, ctypes.byref(st)), "ntt_server_stats_get")
        return {k: int(getattr(st, k)) for k, _ in ServerStats._fields_ if k != "reserved"}

    def close(self):
        if self.handle:
            _lib().ntt_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
