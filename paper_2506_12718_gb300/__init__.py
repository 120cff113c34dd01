"""Permutation-avoiding FFT convolution on GB300 — Python binding of libpac.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libpac.so`` (built from ``csrc/`` for sm_103a).  The functions
below carry the C-ABI names of ``include/pac.h`` and raise ``PacError`` when a
call returns a non-zero status.  PyTorch is used by callers for device memory
and streams; ``Plan`` accepts torch tensors and passes their data pointers.

There is no fallback: if the library is missing or cannot be loaded, every
call raises.  Build it with ``python -m paper_2506_12718_gb300._build`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import enum
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpac.so")
_lib = None

C64, C128, C128_DF = 0, 1, 2
# dtype names: "c64" complex FP32, "c128" complex FP64, "c128df" complex FP64
# arrays computed in double-float arithmetic (PAC_C128_DF)
_DTYPE_CODES = {"c64": C64, "c128": C128, "c128df": C128_DF}


def _dtype_code(dtype) -> int:
    if isinstance(dtype, str):
        if dtype not in _DTYPE_CODES:
            raise ValueError(f"dtype must be one of {sorted(_DTYPE_CODES)}, not {dtype!r}")
        return _DTYPE_CODES[dtype]
    return int(dtype)


class Status(enum.IntEnum):
    OK = 0
    PENDING = 1
    ERR_ARG = -1
    ERR_SIZE = -2
    ERR_NO_SPECTRUM = -3
    ERR_NOMEM = -4
    ERR_CUDA = -5
    ERR_BUSY = -6
    ERR_TIMEOUT = -7
    ERR_NOT_FOUND = -8


Q_NDIM, Q_N_TOTAL, Q_ELEM_BYTES, Q_LAUNCHES_CONVOLVE, Q_LAUNCHES_PERMUTED, Q_LAUNCHES_FORWARD, \
    Q_DEVICE_BYTES, Q_HAS_SPECTRUM, Q_DEVICE_ERROR, Q_GROUPS, Q_PLANE, Q_GROUP_CAP, Q_NARROW = range(13)

# every entry point of include/pac.h: name -> (restype, argtypes)
_vp, _i64, _i32, _u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
_SIGS = {
    "pac_plan_create": (_i32, [_i32, ctypes.POINTER(_i64), _i32, _i32, ctypes.POINTER(_vp)]),
    "pac_plan_create_stages": (_i32, [_i32, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), _i32, ctypes.POINTER(_vp)]),
    "pac_plan_destroy": (_i32, [_vp]),
    "pac_filter_spectrum": (_i32, [_vp, _vp]),
    "pac_convolve": (_i32, [_vp, _vp, _vp, _vp]),
    "pac_convolve_host": (_i32, [_vp, _vp, _vp, _vp]),
    "pac_convolve_many": (_i32, [_i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp]),
    "pac_convolve_many_launches": (_i32, [_i32, ctypes.POINTER(_vp), ctypes.POINTER(_i32)]),
    "pac_queue_create": (_i32, [ctypes.c_size_t, _i32, ctypes.POINTER(_vp)]),
    "pac_submit": (_i32, [_vp, _vp, _vp, _vp, ctypes.POINTER(_u64)]),
    "pac_poll": (_i32, [_vp, _u64, ctypes.POINTER(ctypes.c_double)]),
    "pac_queue_drain": (_i32, [_vp, _i32]),
    "pac_queue_destroy": (_i32, [_vp]),
    "pac_last_error": (ctypes.c_char_p, []),
    "pac_plan_stages": (_i32, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "pac_plan_reverse_table": (_i32, [_vp, _i32, ctypes.POINTER(_i64)]),
    "pac_forward_unordered": (_i32, [_vp, _vp, _vp, _vp]),
    "pac_convolve_permuted": (_i32, [_vp, _vp, _vp, _vp]),
    "pac_fft": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "pac_convolve_permuted_noalloc": (_i32, [_vp, _vp, _vp, _vp]),
    "pac_plan_query": (_i32, [_vp, _i32, ctypes.POINTER(_i64)]),
    "pac_measure_fma_peak": (_i32, [_i32, ctypes.POINTER(ctypes.c_double)]),
    "pac_tune": (_i32, [_i32, ctypes.POINTER(_i64), _i32, _i32, _i32, ctypes.POINTER(ctypes.c_double)]),
    "pac_convolve_timed": (_i32, [_vp, _i32, _vp, _vp, _vp, _i32, ctypes.POINTER(ctypes.c_float),
                                  ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "pac_stage_list": (_i32, [_i64, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "pac_plan_groups": (_i32, [_i32, ctypes.POINTER(_i64), _i32, _i32, _i32, _i32, ctypes.POINTER(_i32),
                               ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "pac_reverse_table": (_i32, [_i32, ctypes.POINTER(_i32), ctypes.POINTER(_i64)]),
    "pac_test_barrier_timeout": (_i32, [_vp, _vp, _vp, _vp, _i32]),
    "pac_test_batch_timeout": (_i32, [_i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, _i32]),
    "pac_plan_twiddles": (_i32, [_i32, ctypes.POINTER(_i64), _i32, _i32, _i32, _i32, _i32, _i32, _vp,
                                 ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "pac_test_host_steps": (_i32, [_i32, ctypes.POINTER(_i64), _i32, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp,
                                   ctypes.POINTER(_i64), ctypes.POINTER(_i64), _vp, ctypes.POINTER(_i32)]),
    "pac_version": (ctypes.c_char_p, []),
    "pac_pfa_create": (_i32, [_i64, _i32, ctypes.POINTER(_vp)]),
    "pac_pfa_destroy": (_i32, [_vp]),
    "pac_pfa_filter_spectrum": (_i32, [_vp, _vp]),
    "pac_pfa_convolve": (_i32, [_vp, _vp, _vp, _vp]),
    "pac_pfa_shape": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64)]),
    "pac_pfa_query": (_i32, [_vp, _i32, ctypes.POINTER(_i64)]),
    "pac_pfa_plan": (_i32, [_vp, ctypes.POINTER(_vp)]),
}


class PacError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = int(status)
        try:
            name = Status(self.status).name
        except ValueError:
            name = str(self.status)
        super().__init__(f"{name}: {message}")


def load():
    """Load libpac.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpac.so not built at {LIB_PATH}; run python -m paper_2506_12718_gb300._build")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int) -> int:
    if rc < 0:
        raise PacError(rc, load().pac_last_error().decode(errors="replace"))
    return rc


def _ptr(t) -> int:
    """Device or host address of a torch tensor, numpy array or integer."""
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return int(t.data_ptr())
    if hasattr(t, "ctypes"):
        return int(t.ctypes.data)
    raise TypeError(f"cannot take the address of {type(t)}")


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ------------------------------------------------------------- C-ABI mirrors


def pac_version() -> str:
    return load().pac_version().decode()


def pac_last_error() -> str:
    return load().pac_last_error().decode(errors="replace")


def _mixed_flags(mixed) -> int:
    # None: the default rule (groups spanning bases where each has a compiled kernel)
    return 2 if mixed is None else (1 if mixed else 0)


def pac_plan_groups(dims, radix: int, dtype: int = 0, mixed=False, cap: int = 0) -> list:
    """Host only: the pass groups of a plan, forward order, as (axis, M, rounds).
    mixed: True / False allow / forbid groups spanning prime bases, None the default rule."""
    vals = [int(v) for v in dims]
    d = (ctypes.c_int64 * max(3, len(vals)))(*(vals + [1] * (3 - len(vals))))
    room = 64
    ax = (ctypes.c_int * room)()
    sz = (ctypes.c_int * room)()
    rr = (ctypes.c_int * (8 * room))()
    cnt = ctypes.c_int(room)
    _check(load().pac_plan_groups(len(vals), d, int(radix), int(dtype), _mixed_flags(mixed), int(cap), ax, sz, rr,
                                  ctypes.byref(cnt)))
    return [(ax[g], sz[g], [r for r in rr[8 * g:8 * g + 8] if r]) for g in range(cnt.value)]


def pac_plan_twiddles(dims, radix: int, dtype: int, group: int, which: int, mixed=False, cap: int = 0):
    """Host only: twiddle table `which` (0 round, 1 external low, 2 external high) of group `group`
    of the schedule pac_plan_groups gives, as uploaded by a plan; returns (values, L, T) with values a
    numpy complex64 / complex128 array (C128_DF: a float32 array of shape (n, 4), the pairs
    re.hi, re.lo, im.hi, im.lo)."""
    import numpy as np
    vals = [int(v) for v in dims]
    d = (ctypes.c_int64 * max(3, len(vals)))(*(vals + [1] * (3 - len(vals))))
    cnt, L, T = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    args = (len(vals), d, int(radix), int(dtype), _mixed_flags(mixed), int(cap), int(group), int(which))
    _check(load().pac_plan_twiddles(*args, None, ctypes.byref(cnt), ctypes.byref(L), ctypes.byref(T)))
    if int(dtype) == C128_DF:
        out = np.zeros((max(1, cnt.value), 4), np.float32)
    else:
        out = np.zeros(max(1, cnt.value), np.complex64 if int(dtype) == C64 else np.complex128)
    _check(load().pac_plan_twiddles(*args, out.ctypes.data, ctypes.byref(cnt), None, None))
    return out[: cnt.value], L.value, T.value


def pac_test_host_steps(dims, radix: int, dtype: int, cap: int = 0, flags: int = 0, h=None, x=None, y=None, spec=None,
                        scratch=None, tables=None, steps=None, room: int = 0):
    """Host-only test hook: the step records of a plan of this problem for the CPU emulation of the
    kernels (pointer arguments: host addresses as ints, or None).  Returns (table_bytes, spec_elems,
    number of steps)."""
    vals = [int(v) for v in dims]
    d = (ctypes.c_int64 * max(3, len(vals)))(*(vals + [1] * (3 - len(vals))))
    tb, se, ns = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int(int(room))
    _check(load().pac_test_host_steps(len(vals), d, int(radix), int(dtype), int(cap), int(flags), h, x, y, spec, scratch,
                                      tables, ctypes.byref(tb), ctypes.byref(se), steps, ctypes.byref(ns)))
    return tb.value, se.value, ns.value


def pac_stage_list(n: int, radix: int) -> list[int]:
    cnt = ctypes.c_int(64)
    arr = (ctypes.c_int * 64)()
    _check(load().pac_stage_list(int(n), int(radix), arr, ctypes.byref(cnt)))
    return list(arr[: cnt.value])


def pac_reverse_table(stages) -> list[int]:
    stages = list(stages)
    n = 1
    for s in stages:
        n *= s
    arr = (ctypes.c_int * max(1, len(stages)))(*stages)
    out = (ctypes.c_int64 * n)()
    _check(load().pac_reverse_table(len(stages), arr, out))
    return list(out)


def pac_plan_create(ndim: int, dims, radix: int, dtype: int) -> int:
    vals = [int(v) for v in dims]
    d = (ctypes.c_int64 * max(3, len(vals)))(*(vals + [1] * (3 - len(vals))))
    out = ctypes.c_void_p()
    _check(load().pac_plan_create(int(ndim), d, int(radix), int(dtype), ctypes.byref(out)))
    return out.value


def pac_plan_create_stages(dims, stages_per_axis, dtype: int) -> int:
    vals = [int(v) for v in dims]
    if len(stages_per_axis) != len(vals):
        raise ValueError("one stage list per axis")
    d = (ctypes.c_int64 * max(3, len(vals)))(*(vals + [1] * (3 - len(vals))))
    counts = (ctypes.c_int * max(1, len(vals)))(*[len(st) for st in stages_per_axis])
    flat = [int(r) for st in stages_per_axis for r in st]
    arr = (ctypes.c_int * max(1, len(flat)))(*flat)
    out = ctypes.c_void_p()
    _check(load().pac_plan_create_stages(len(vals), d, counts, arr, int(dtype), ctypes.byref(out)))
    return out.value


def pac_plan_destroy(plan: int) -> None:
    _check(load().pac_plan_destroy(plan))


def pac_filter_spectrum(plan: int, h_dev) -> None:
    _check(load().pac_filter_spectrum(plan, _ptr(h_dev)))


def pac_convolve(plan: int, x_dev, y_dev, stream=None) -> None:
    _check(load().pac_convolve(plan, _ptr(x_dev), _ptr(y_dev), _stream(stream)))


def pac_convolve_host(plan: int, x_host, y_host, stream=None) -> None:
    _check(load().pac_convolve_host(plan, _ptr(x_host), _ptr(y_host), _stream(stream)))


def pac_convolve_many(plans, xs, ys, stream=None) -> None:
    n = len(plans)
    P = (ctypes.c_void_p * n)(*plans)
    X = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    Y = (ctypes.c_void_p * n)(*[_ptr(y) for y in ys])
    _check(load().pac_convolve_many(n, P, X, Y, _stream(stream)))


def pac_test_batch_timeout(plans, xs, ys, wait_us: int, stream=None) -> None:
    """Test hook: the batch as one persistent launch whose dependency waits all run out."""
    n = len(plans)
    P = (ctypes.c_void_p * n)(*plans)
    X = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    Y = (ctypes.c_void_p * n)(*[_ptr(y) for y in ys])
    _check(load().pac_test_batch_timeout(n, P, X, Y, _stream(stream), int(wait_us)))


def pac_convolve_many_launches(plans) -> int:
    n = len(plans)
    P = (ctypes.c_void_p * max(1, n))(*plans)
    out = ctypes.c_int(0)
    _check(load().pac_convolve_many_launches(n, P, ctypes.byref(out)))
    return out.value


def pac_forward_unordered(plan: int, x_dev, xhat_dev, stream=None) -> None:
    _check(load().pac_forward_unordered(plan, _ptr(x_dev), _ptr(xhat_dev), _stream(stream)))


def pac_fft(plan: int, in_dev, out_dev, inverse: bool = False, stream=None) -> None:
    """Ordered DFT (DIF passes + index-reversal permutation) or its inverse (with 1/N)."""
    _check(load().pac_fft(plan, _ptr(in_dev), _ptr(out_dev), 1 if inverse else 0, _stream(stream)))


def pac_convolve_permuted(plan: int, x_dev, y_dev, stream=None) -> None:
    _check(load().pac_convolve_permuted(plan, _ptr(x_dev), _ptr(y_dev), _stream(stream)))


def pac_test_barrier_timeout(plan: int, x_dev, y_dev, spin_limit: int, stream=None) -> None:
    """Test hook: the convolution as one cooperative launch whose bounded barrier waits all run out."""
    _check(load().pac_test_barrier_timeout(plan, _ptr(x_dev), _ptr(y_dev), _stream(stream), int(spin_limit)))


def pac_convolve_permuted_noalloc(plan: int, x_dev, y_dev, stream=None) -> None:
    """Allocation-free permuted convolution (fixed 8 MiB static scratch; see include/pac.h)."""
    _check(load().pac_convolve_permuted_noalloc(plan, _ptr(x_dev), _ptr(y_dev), _stream(stream)))


def pac_plan_stages(plan: int, axis: int) -> list[int]:
    cnt = ctypes.c_int(64)
    arr = (ctypes.c_int * 64)()
    _check(load().pac_plan_stages(plan, int(axis), arr, ctypes.byref(cnt)))
    return list(arr[: cnt.value])


def pac_plan_reverse_table(plan: int, axis: int, n: int) -> list[int]:
    out = (ctypes.c_int64 * int(n))()
    _check(load().pac_plan_reverse_table(plan, int(axis), out))
    return list(out)


KERNEL_NAMES = {0: "dif_pass", 1: "fused_dif_mul_dit_pass", 2: "dit_pass", 3: "permute", 4: "pointwise",
                5: "conv_kernel", 6: "plane_pass"}


def pac_convolve_timed(plan: int, which: int, x_dev, y_dev, stream=None, max_launches: int = 64):
    """Returns [(kernel_name, ms), ...] for each launch of one convolution (synchronises)."""
    ms = (ctypes.c_float * max_launches)()
    ids = (ctypes.c_int * max_launches)()
    n = ctypes.c_int(0)
    _check(load().pac_convolve_timed(plan, int(which), _ptr(x_dev), _ptr(y_dev), _stream(stream), max_launches,
                                     ms, ids, ctypes.byref(n)))
    return [(KERNEL_NAMES.get(ids[i], str(ids[i])), float(ms[i])) for i in range(n.value)]


def pac_measure_fma_peak(dtype: str = "c128") -> float:
    """Measured peak FMA rate (GFLOP/s) of the device for FP32 ("c64") or FP64 ("c128")."""
    g = ctypes.c_double(0.0)
    _check(load().pac_measure_fma_peak(C64 if dtype == "c64" else C128, ctypes.byref(g)))
    return g.value


def pac_tune(dims, radix: int, dtype: str = "c64", reps: int = 5) -> float:
    """Autotune the pass schedule of this problem; returns the winner's time per convolution (us)."""
    vals = [int(v) for v in dims]
    d = (ctypes.c_int64 * max(3, len(vals)))(*(vals + [1] * (3 - len(vals))))
    us = ctypes.c_double(0.0)
    _check(load().pac_tune(len(vals), d, int(radix), _dtype_code(dtype), int(reps), ctypes.byref(us)))
    return us.value


def pac_pfa_create(n: int, dtype: int) -> int:
    out = ctypes.c_void_p()
    _check(load().pac_pfa_create(int(n), int(dtype), ctypes.byref(out)))
    return out.value


def pac_pfa_destroy(p: int) -> None:
    _check(load().pac_pfa_destroy(p))


def pac_pfa_filter_spectrum(p: int, h_dev) -> None:
    _check(load().pac_pfa_filter_spectrum(p, _ptr(h_dev)))


def pac_pfa_convolve(p: int, x_dev, y_dev, stream=None) -> None:
    _check(load().pac_pfa_convolve(p, _ptr(x_dev), _ptr(y_dev), _stream(stream)))


def pac_pfa_shape(p: int) -> tuple:
    t = ctypes.c_int()
    dims = (ctypes.c_int64 * 3)()
    _check(load().pac_pfa_shape(p, ctypes.byref(t), dims))
    return tuple(dims[3 - max(t.value, 1):])


def pac_pfa_query(p: int, key: int) -> int:
    v = ctypes.c_int64()
    _check(load().pac_pfa_query(p, int(key), ctypes.byref(v)))
    return v.value


def pac_pfa_plan(p: int) -> int:
    out = ctypes.c_void_p()
    _check(load().pac_pfa_plan(p, ctypes.byref(out)))
    return out.value


def pac_plan_query(plan: int, key: int) -> int:
    v = ctypes.c_int64()
    _check(load().pac_plan_query(plan, int(key), ctypes.byref(v)))
    return v.value


def pac_queue_create(hbm_budget_bytes: int, max_inflight: int) -> int:
    out = ctypes.c_void_p()
    _check(load().pac_queue_create(int(hbm_budget_bytes), int(max_inflight), ctypes.byref(out)))
    return out.value


def pac_submit(queue: int, plan: int, x_dev, y_dev) -> int:
    t = ctypes.c_uint64()
    _check(load().pac_submit(queue, plan, _ptr(x_dev), _ptr(y_dev), ctypes.byref(t)))
    return t.value


def pac_poll(queue: int, ticket: int):
    """Returns (status, latency_us); status is Status.OK or Status.PENDING, raises on failure."""
    lat = ctypes.c_double(0.0)
    rc = _check(load().pac_poll(queue, int(ticket), ctypes.byref(lat)))
    return Status(rc), lat.value


def pac_queue_drain(queue: int, timeout_ms: int = 60000) -> None:
    _check(load().pac_queue_drain(queue, int(timeout_ms)))


def pac_queue_destroy(queue: int) -> None:
    _check(load().pac_queue_destroy(queue))


# ------------------------------------------------------------ convenience


class Plan:
    """A convolution plan bound to torch tensors (complex64 for "c64",
    complex128 for "c128" and "c128df", on CUDA)."""

    def __init__(self, dims, radix: int, dtype: str = "c64", stages=None):
        """radix in {2,3,4,5,8}, or 0 for mixed radix (dims 2^a 3^b 5^c); or
        explicit per-axis DIF stage lists `stages` (radix is then ignored)."""
        self.dims = tuple(int(d) for d in dims)
        self.radix = int(radix) if stages is None else -1
        self.dtype = dtype
        code = _dtype_code(dtype)
        if stages is None:
            self.handle = pac_plan_create(len(self.dims), self.dims, self.radix, code)
        else:
            self.handle = pac_plan_create_stages(self.dims, [list(st) for st in stages], code)

    def _tensor_check(self, t, name):
        import torch
        want = torch.complex64 if self.dtype == "c64" else torch.complex128
        if t.dtype != want or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != self.dims:
            raise ValueError(f"{name}: need a contiguous CUDA {want} tensor of shape {self.dims}")

    def filter_spectrum(self, h) -> None:
        self._tensor_check(h, "h")
        pac_filter_spectrum(self.handle, h)

    def convolve(self, x, y=None, stream=None):
        import torch
        self._tensor_check(x, "x")
        if y is None:
            y = torch.empty_like(x)
        self._tensor_check(y, "y")
        pac_convolve(self.handle, x, y, stream)
        return y

    def convolve_permuted(self, x, y=None, stream=None):
        import torch
        self._tensor_check(x, "x")
        if y is None:
            y = torch.empty_like(x)
        pac_convolve_permuted(self.handle, x, y, stream)
        return y

    def forward_unordered(self, x, out=None, stream=None):
        import torch
        self._tensor_check(x, "x")
        if out is None:
            out = torch.empty_like(x)
        pac_forward_unordered(self.handle, x, out, stream)
        return out

    def stages(self, axis: int) -> list[int]:
        return pac_plan_stages(self.handle, axis)

    def reverse_table(self, axis: int) -> list[int]:
        return pac_plan_reverse_table(self.handle, axis, self.dims[axis])

    def query(self, key: int) -> int:
        return pac_plan_query(self.handle, key)

    def close(self) -> None:
        if self.handle:
            pac_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pfa:
    """Prime factor convolution of a 1-D length n = 2^a 3^b 5^c (Section 7.2),
    bound to torch tensors (complex64 / complex128, on CUDA)."""

    def __init__(self, n: int, dtype: str = "c64"):
        self.n = int(n)
        self.dtype = dtype
        self.handle = pac_pfa_create(self.n, C64 if dtype == "c64" else C128)

    @property
    def shape(self) -> tuple:
        """The tensor shape (n_t, ..., n_1) the convolution runs on."""
        return pac_pfa_shape(self.handle)

    def _tensor_check(self, t, name):
        import torch
        want = torch.complex64 if self.dtype == "c64" else torch.complex128
        if t.dtype != want or not t.is_cuda or not t.is_contiguous() or t.numel() != self.n:
            raise ValueError(f"{name}: need a contiguous CUDA {want} tensor of {self.n} elements")

    def filter_spectrum(self, h) -> None:
        self._tensor_check(h, "h")
        pac_pfa_filter_spectrum(self.handle, h)

    def convolve(self, x, y=None, stream=None):
        import torch
        self._tensor_check(x, "x")
        if y is None:
            y = torch.empty_like(x)
        self._tensor_check(y, "y")
        pac_pfa_convolve(self.handle, x, y, stream)
        return y

    def query(self, key: int) -> int:
        return pac_pfa_query(self.handle, key)

    def close(self) -> None:
        if self.handle:
            pac_pfa_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
