"""Python binding of ``libtsmm.so``: the GB300 pre-packed tall-and-skinny GEMM.

C = alpha * A * B + beta * C0  (Eq. 1 of AutoTSMM, arXiv 2208.08088), with B
packed once (PACKB of Algorithm 1) and reused by many executions (COMPUTE).

Two layers, both argument marshalling only -- every step of the computation
runs in the CUDA kernels of the shared library:

* ``tsmm_*`` functions with the C ABI's names and arguments (raw device
  pointers as ints, sizes, a stream handle), raising ``TsmmError`` on a
  non-OK status;
* ``pack_b`` / ``plan`` / ``execute`` conveniences taking torch CUDA tensors
  that hold column-major matrices (stride(0) == 1) and using the current
  torch stream.

The library must have been built first (``python paper_2208_08088_gb300/build.py``
or ``__graft_entry__.build()``); importing the binding without it raises
``ImportError`` -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

__all__ = [
    "TsmmError", "F32", "F64", "PREC_NATIVE", "PREC_BF16X3", "lib", "library_path",
    "tsmm_pack_b_ex", "tsmm_plan_ex",
    "tsmm_status_string", "tsmm_version", "tsmm_pack_b", "tsmm_packed_b_destroy",
    "tsmm_packed_b_info", "tsmm_packed_b_read", "tsmm_plan", "tsmm_plan_destroy", "tsmm_plan_info", "tsmm_execute",
    "tsmm_plan_check", "tsmm_plan_launches_per_execute", "tsmm_autotune",
    "tsmm_plan_cache_load", "tsmm_plan_cache_save", "tsmm_plan_cache_clear", "tsmm_plan_cache_size",
    "tsmm_execute_noalloc", "tsmm_last_cuda_error", "tsmm_diag_bounded_wait", "diag_bounded_wait",
    "tsmm_diag_fp_peak", "diag_fp_peak", "DIAG_FFMA", "DIAG_FFMA2", "DIAG_DFMA", "DIAG_DMMA",
    "autotune", "execute_grouped", "tsmm_execute_grouped", "GroupItem",
    "Server", "ServerConfig", "Request", "Completion", "tsmm_server_clock",
    "tsmm_server_create", "tsmm_server_submit", "tsmm_server_poll", "tsmm_server_drain",
    "tsmm_server_destroy", "tsmm_diag_server_inject_timeout",
    "PackedB", "Plan", "pack_b", "plan", "execute", "colmajor", "ld_of",
]

F32, F64 = 0, 1
PREC_NATIVE, PREC_BF16X3 = 0, 1
DIAG_FFMA, DIAG_FFMA2, DIAG_DFMA, DIAG_DMMA = 0, 1, 2, 3
STATUS = {
    0: "TSMM_OK", 1: "TSMM_ERR_INVALID_ARG", 2: "TSMM_ERR_UNSUPPORTED_SHAPE",
    3: "TSMM_ERR_MISMATCH", 4: "TSMM_ERR_MISALIGNED", 5: "TSMM_ERR_OUT_OF_MEMORY",
    6: "TSMM_ERR_CUDA", 7: "TSMM_ERR_TIMEOUT",
}

library_path = _build.LIB


class TsmmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class GroupItem(ctypes.Structure):
    """struct tsmm_group_item of include/tsmm.h."""
    _fields_ = [("plan", ctypes.c_void_p), ("alpha", ctypes.c_double), ("A_dev", ctypes.c_void_p),
                ("lda", ctypes.c_int64), ("pb", ctypes.c_void_p), ("beta", ctypes.c_double),
                ("C_dev", ctypes.c_void_p), ("ldc", ctypes.c_int64)]


class ServerConfig(ctypes.Structure):
    """struct tsmm_server_config."""
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("arena_bytes", ctypes.c_size_t),
                ("num_streams", ctypes.c_int), ("max_batch", ctypes.c_int), ("dtype", ctypes.c_int)]


class Request(ctypes.Structure):
    """struct tsmm_request."""
    _fields_ = [("id", ctypes.c_uint64), ("pb", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("A_dev", ctypes.c_void_p),
                ("lda", ctypes.c_int64), ("C_dev", ctypes.c_void_p), ("ldc", ctypes.c_int64),
                ("arrival_s", ctypes.c_double)]


class Completion(ctypes.Structure):
    """struct tsmm_completion."""
    _fields_ = [("id", ctypes.c_uint64), ("arrival_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("launch_s", ctypes.c_double), ("complete_s", ctypes.c_double), ("status", ctypes.c_int)]


def _load():
    if not os.path.exists(library_path):
        raise ImportError(
            f"{library_path} is missing: build the CUDA library first "
            "(python paper_2208_08088_gb300/build.py); there is no CPU fallback")
    L = ctypes.CDLL(library_path)
    i64, dbl, vp, ci = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
    sz = ctypes.c_size_t
    L.tsmm_status_string.restype = ctypes.c_char_p
    L.tsmm_status_string.argtypes = [ci]
    L.tsmm_version.restype = ci
    L.tsmm_version.argtypes = []
    L.tsmm_last_cuda_error.restype = ctypes.c_char_p
    L.tsmm_last_cuda_error.argtypes = []
    L.tsmm_pack_b.restype = ci
    L.tsmm_pack_b.argtypes = [ci, i64, i64, vp, i64, vp, ctypes.POINTER(vp)]
    L.tsmm_pack_b_ex.restype = ci
    L.tsmm_pack_b_ex.argtypes = [ci, ci, i64, i64, vp, i64, vp, ctypes.POINTER(vp)]
    L.tsmm_plan_ex.restype = ci
    L.tsmm_plan_ex.argtypes = [i64, i64, i64, ci, ci, ctypes.POINTER(vp)]
    L.tsmm_packed_b_destroy.restype = ci
    L.tsmm_packed_b_destroy.argtypes = [vp]
    L.tsmm_packed_b_info.restype = ci
    L.tsmm_packed_b_info.argtypes = [vp, ctypes.POINTER(ci)] + [ctypes.POINTER(i64)] * 5 + [
        ctypes.POINTER(vp), ctypes.POINTER(sz)]
    L.tsmm_packed_b_read.restype = ci
    L.tsmm_packed_b_read.argtypes = [vp, vp, sz]
    L.tsmm_plan.restype = ci
    L.tsmm_plan.argtypes = [i64, i64, i64, ci, ctypes.POINTER(vp)]
    L.tsmm_plan_destroy.restype = ci
    L.tsmm_plan_destroy.argtypes = [vp]
    L.tsmm_plan_info.restype = ci
    L.tsmm_plan_info.argtypes = [vp] + [ctypes.POINTER(ci)] * 4 + [ctypes.POINTER(sz)]
    L.tsmm_execute.restype = ci
    L.tsmm_execute.argtypes = [vp, dbl, vp, i64, vp, dbl, vp, i64, vp]
    L.tsmm_plan_check.restype = ci
    L.tsmm_plan_check.argtypes = [vp]
    L.tsmm_plan_launches_per_execute.restype = ci
    L.tsmm_plan_launches_per_execute.argtypes = [vp]
    L.tsmm_execute_grouped.restype = ci
    L.tsmm_execute_grouped.argtypes = [ctypes.POINTER(GroupItem), ci, vp]
    L.tsmm_server_create.restype = ci
    L.tsmm_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    L.tsmm_server_submit.restype = ci
    L.tsmm_server_submit.argtypes = [vp, ctypes.POINTER(Request), ci]
    L.tsmm_server_drain.restype = ci
    L.tsmm_server_drain.argtypes = [vp, dbl]
    L.tsmm_server_poll.restype = i64
    L.tsmm_server_poll.argtypes = [vp, ctypes.POINTER(Completion), i64]
    L.tsmm_server_destroy.restype = ci
    L.tsmm_server_destroy.argtypes = [vp]
    L.tsmm_diag_server_inject_timeout.restype = ci
    L.tsmm_diag_server_inject_timeout.argtypes = [vp, ci]
    L.tsmm_server_clock.restype = dbl
    L.tsmm_server_clock.argtypes = []
    L.tsmm_autotune.restype = ci
    L.tsmm_autotune.argtypes = [i64, i64, i64, ci, vp, i64, vp, vp, i64, vp, ci, ctypes.POINTER(vp)]
    for name in ("tsmm_plan_cache_load", "tsmm_plan_cache_save"):
        getattr(L, name).restype = ci
        getattr(L, name).argtypes = [ctypes.c_char_p]
    L.tsmm_plan_cache_clear.restype = ci
    L.tsmm_plan_cache_clear.argtypes = []
    L.tsmm_plan_cache_size.restype = i64
    L.tsmm_plan_cache_size.argtypes = []
    L.tsmm_diag_bounded_wait.restype = ci
    L.tsmm_diag_bounded_wait.argtypes = [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(dbl)]
    L.tsmm_diag_fp_peak.restype = ci
    L.tsmm_diag_fp_peak.argtypes = [ci, ctypes.c_uint32, ci, ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                    ctypes.POINTER(ctypes.c_uint64)]
    L.tsmm_execute_noalloc.restype = ci
    L.tsmm_execute_noalloc.argtypes = [ci, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, vp]
    return L


lib = _load()


def _check(status: int, where: str):
    if status != 0:
        detail = lib.tsmm_last_cuda_error().decode() if status in (5, 6) else ""
        raise TsmmError(status, where, detail)


# ------------------------------------------------------------------ C ABI names
def tsmm_status_string(status: int) -> str:
    return lib.tsmm_status_string(int(status)).decode()


def tsmm_version() -> int:
    return int(lib.tsmm_version())


def tsmm_pack_b(dtype: int, k: int, n: int, B_dev: int, ldb: int, stream: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(lib.tsmm_pack_b(dtype, k, n, B_dev or None, ldb, stream or None, ctypes.byref(out)),
           "tsmm_pack_b")
    return out.value


def tsmm_pack_b_ex(dtype: int, precision: int, k: int, n: int, B_dev: int, ldb: int,
                   stream: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(lib.tsmm_pack_b_ex(dtype, precision, k, n, B_dev or None, ldb, stream or None,
                              ctypes.byref(out)), "tsmm_pack_b_ex")
    return out.value


def tsmm_plan_ex(m: int, n: int, k: int, dtype: int, precision: int) -> int:
    out = ctypes.c_void_p()
    _check(lib.tsmm_plan_ex(m, n, k, dtype, precision, ctypes.byref(out)), "tsmm_plan_ex")
    return out.value


def tsmm_packed_b_destroy(pb: int) -> None:
    _check(lib.tsmm_packed_b_destroy(pb), "tsmm_packed_b_destroy")


def tsmm_packed_b_info(pb: int) -> dict:
    dt = ctypes.c_int()
    k, n, kp, w, nt = (ctypes.c_int64() for _ in range(5))
    data = ctypes.c_void_p()
    nbytes = ctypes.c_size_t()
    _check(lib.tsmm_packed_b_info(pb, ctypes.byref(dt), ctypes.byref(k), ctypes.byref(n),
                                  ctypes.byref(kp), ctypes.byref(w), ctypes.byref(nt),
                                  ctypes.byref(data), ctypes.byref(nbytes)), "tsmm_packed_b_info")
    return dict(dtype=dt.value, k=k.value, n=n.value, kp=kp.value, w=w.value, ntiles=nt.value,
                data=data.value or 0, bytes=nbytes.value)


def tsmm_packed_b_read(pb: int, host_dst: int, nbytes: int) -> None:
    _check(lib.tsmm_packed_b_read(pb, host_dst or None, nbytes), "tsmm_packed_b_read")


def tsmm_plan(m: int, n: int, k: int, dtype: int) -> int:
    out = ctypes.c_void_p()
    _check(lib.tsmm_plan(m, n, k, dtype, ctypes.byref(out)), "tsmm_plan")
    return out.value


def tsmm_plan_destroy(plan: int) -> None:
    _check(lib.tsmm_plan_destroy(plan), "tsmm_plan_destroy")


def tsmm_plan_info(plan: int) -> dict:
    regime, np_, bm, splits = (ctypes.c_int() for _ in range(4))
    ws = ctypes.c_size_t()
    _check(lib.tsmm_plan_info(plan, ctypes.byref(regime), ctypes.byref(np_), ctypes.byref(bm),
                              ctypes.byref(splits), ctypes.byref(ws)), "tsmm_plan_info")
    return dict(regime=regime.value, np=np_.value, bm=bm.value, splits=splits.value,
                workspace_bytes=ws.value)


def tsmm_execute(plan: int, alpha: float, A_dev: int, lda: int, pb: int, beta: float, C_dev: int,
                 ldc: int, stream: int = 0) -> None:
    _check(lib.tsmm_execute(plan, float(alpha), A_dev or None, lda, pb, float(beta), C_dev or None,
                            ldc, stream or None), "tsmm_execute")


def tsmm_plan_check(plan: int) -> None:
    _check(lib.tsmm_plan_check(plan), "tsmm_plan_check")


def tsmm_plan_launches_per_execute(plan: int) -> int:
    return int(lib.tsmm_plan_launches_per_execute(plan))


def tsmm_execute_grouped(items, stream: int = 0) -> None:
    """items: sequence of (plan, alpha, A_dev, lda, pb, beta, C_dev, ldc) tuples of raw handles."""
    arr = (GroupItem * max(1, len(items)))()
    for i, (pl, alpha, A, lda, pb, beta, C, ldc) in enumerate(items):
        arr[i] = GroupItem(pl, float(alpha), A or None, lda, pb, float(beta), C or None, ldc)
    _check(lib.tsmm_execute_grouped(arr, len(items), stream or None), "tsmm_execute_grouped")


def tsmm_autotune(m: int, n: int, k: int, dtype: int, A_dev: int, lda: int, pb: int, C_dev: int,
                  ldc: int, stream: int = 0, reps: int = 5) -> int:
    out = ctypes.c_void_p()
    _check(lib.tsmm_autotune(m, n, k, dtype, A_dev or None, lda, pb, C_dev or None, ldc,
                             stream or None, reps, ctypes.byref(out)), "tsmm_autotune")
    return out.value


def tsmm_execute_noalloc(dtype: int, m: int, n: int, k: int, alpha: float, A_dev: int, lda: int,
                         B_dev: int, ldb: int, beta: float, C_dev: int, ldc: int,
                         stream: int = 0) -> None:
    """Allocation-free C = alpha*A*B + beta*C0 for regime (i) shapes: B is
    packed into the library's built-in device scratch on every call."""
    _check(lib.tsmm_execute_noalloc(dtype, m, n, k, alpha, A_dev or None, lda, B_dev or None, ldb,
                                    beta, C_dev or None, ldc, stream or None),
           "tsmm_execute_noalloc")


def tsmm_last_cuda_error() -> str:
    """Text of the last CUDA error the library saw (empty if none)."""
    return lib.tsmm_last_cuda_error().decode()


def tsmm_plan_cache_load(path: str) -> None:
    _check(lib.tsmm_plan_cache_load(os.fsencode(path)), "tsmm_plan_cache_load")


def tsmm_plan_cache_save(path: str) -> None:
    _check(lib.tsmm_plan_cache_save(os.fsencode(path)), "tsmm_plan_cache_save")


def tsmm_plan_cache_clear() -> None:
    _check(lib.tsmm_plan_cache_clear(), "tsmm_plan_cache_clear")


def tsmm_plan_cache_size() -> int:
    return int(lib.tsmm_plan_cache_size())


# ------------------------------------------------------------------ torch layer
def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    if t == torch.float32:
        return F32
    if t == torch.float64:
        return F64
    raise TypeError(f"unsupported dtype {t}")


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def colmajor(rows: int, cols: int, dtype, device="cuda", ld: int | None = None, fill=None):
    """A rows x cols column-major tensor (stride(0) == 1, stride(1) == ld)."""
    torch = _torch()
    ld = max(1, rows) if ld is None else ld
    base = torch.empty((max(cols, 1), ld), dtype=dtype, device=device)
    if fill is not None:
        base.fill_(fill)
    return base.t()[:rows, :cols]


def ld_of(t) -> int:
    """Leading dimension of a column-major 2-D tensor."""
    if t.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    if t.shape[0] > 1 and t.stride(0) != 1:
        raise ValueError("tensor is not column-major (stride(0) != 1)")
    rows = max(1, int(t.shape[0]))
    if t.shape[1] > 1:
        return int(t.stride(1))
    # one column: its stride is free; keep it when it is a valid leading dimension
    return int(t.stride(1)) if t.stride(1) >= rows else rows


class PackedB:
    """Owner of a packed B handle (tsmm_pack_b / tsmm_packed_b_destroy)."""

    def __init__(self, handle: int, k: int, n: int, dtype: int):
        self.handle, self.k, self.n, self.dtype = handle, k, n, dtype

    def info(self) -> dict:
        return tsmm_packed_b_info(self.handle)

    def read(self):
        """The packed storage as a flat numpy array (synchronous copy)."""
        import numpy as np
        inf = self.info()
        out = np.empty(inf["bytes"] // (8 if self.dtype == F64 else 4),
                       dtype=np.float64 if self.dtype == F64 else np.float32)
        tsmm_packed_b_read(self.handle, out.ctypes.data, out.nbytes)
        return out

    def close(self):
        if self.handle:
            tsmm_packed_b_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owner of a plan handle (tsmm_plan / tsmm_plan_destroy)."""

    def __init__(self, handle: int, m: int, n: int, k: int, dtype: int):
        self.handle, self.m, self.n, self.k, self.dtype = handle, m, n, k, dtype

    def info(self) -> dict:
        return tsmm_plan_info(self.handle)

    def check(self):
        tsmm_plan_check(self.handle)

    def launches_per_execute(self) -> int:
        return tsmm_plan_launches_per_execute(self.handle)

    def close(self):
        if self.handle:
            tsmm_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_b(B, stream=None, precision: int = PREC_NATIVE) -> PackedB:
    """Pack a column-major k x n CUDA tensor (enqueued on the current stream)."""
    k, n = B.shape
    dt = _dtype_code(B.dtype)
    h = tsmm_pack_b_ex(dt, precision, k, n, B.data_ptr() if B.numel() else 0,
                       ld_of(B) if k else 1, _stream_handle(stream))
    pb = PackedB(h, k, n, dt)
    pb.precision = precision
    return pb


def plan(m: int, n: int, k: int, dtype, precision: int = PREC_NATIVE) -> Plan:
    dt = dtype if isinstance(dtype, int) else _dtype_code(dtype)
    p = Plan(tsmm_plan_ex(m, n, k, dt, precision), m, n, k, dt)
    p.precision = precision
    return p


def execute_grouped(problems, stream=None) -> None:
    """problems: sequence of (plan, alpha, A, pb, beta, C) with column-major CUDA
    tensors; all run with as few launches as the library can manage."""
    items = []
    for (p, alpha, A, pb, beta, C) in problems:
        lda = ld_of(A) if p.m > 0 and p.k > 0 else max(1, p.m)
        items.append((p.handle, alpha, A.data_ptr() if A.numel() else 0, lda, pb.handle, beta,
                      C.data_ptr() if C.numel() else 0, ld_of(C) if p.n > 0 else max(1, p.m)))
    tsmm_execute_grouped(items, _stream_handle(stream))


def tsmm_diag_bounded_wait(polls: int):
    """Same-named form of diag_bounded_wait: (status, cycles, seconds)."""
    return diag_bounded_wait(polls)


def diag_bounded_wait(polls: int):
    """Run the library's bounded mbarrier wait against a barrier that nothing
    completes (tsmm_diag_bounded_wait); returns (status, cycles, seconds) --
    status TIMEOUT (7) is the expected outcome."""
    cyc = ctypes.c_uint64(0)
    sec = ctypes.c_double(0.0)
    st = lib.tsmm_diag_bounded_wait(int(polls), ctypes.byref(cyc), ctypes.byref(sec))
    return int(st), int(cyc.value), float(sec.value)


def tsmm_diag_fp_peak(pipe: int, iters: int, blocks_per_sm: int = 4):
    """Same-named form of diag_fp_peak: (flops, ms, cycles)."""
    return diag_fp_peak(pipe, iters, blocks_per_sm)


def diag_fp_peak(pipe: int, iters: int, blocks_per_sm: int = 4):
    """Throughput of one arithmetic pipe (DIAG_FFMA, DIAG_FFMA2, DIAG_DFMA,
    DIAG_DMMA) on the current GPU (tsmm_diag_fp_peak): returns (flops, ms,
    cycles) of one timed launch; flops / ms is the rate, cycles / ms the SM
    clock it ran at."""
    fl = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    cyc = ctypes.c_uint64(0)
    _check(lib.tsmm_diag_fp_peak(int(pipe), int(iters), int(blocks_per_sm), ctypes.byref(fl),
                                 ctypes.byref(ms), ctypes.byref(cyc)), "tsmm_diag_fp_peak")
    return float(fl.value), float(ms.value), int(cyc.value)


def autotune(A, pb: PackedB, C, reps: int = 5, stream=None) -> Plan:
    """Time candidate plans on these operands (C is overwritten), remember the
    winner in the plan cache and return a plan that uses it."""
    m, k = A.shape
    n = C.shape[1]
    dt = _dtype_code(A.dtype)
    h = tsmm_autotune(m, n, k, dt, A.data_ptr(), ld_of(A), pb.handle, C.data_ptr(), ld_of(C),
                      _stream_handle(stream), reps)
    return Plan(h, m, n, k, dt)


def execute(p: Plan, alpha: float, A, pb: PackedB, beta: float, C, stream=None) -> None:
    """C = alpha * A @ B + beta * C in place (column-major CUDA tensors)."""
    if A.shape != (p.m, p.k) or C.shape != (p.m, p.n):
        raise ValueError(f"shape mismatch: plan {(p.m, p.n, p.k)}, A {tuple(A.shape)}, C {tuple(C.shape)}")
    lda = ld_of(A) if p.m > 0 and p.k > 0 else max(1, p.m)
    tsmm_execute(p.handle, alpha, A.data_ptr() if A.numel() else 0, lda, pb.handle, beta,
                 C.data_ptr() if C.numel() else 0, ld_of(C) if p.n > 0 else max(1, p.m),
                 _stream_handle(stream))


# ------------------------------------------------------------------ serving
def tsmm_server_clock() -> float:
    return float(lib.tsmm_server_clock())


def tsmm_server_create(cfg: "ServerConfig") -> int:
    """A tsmm_server_t handle (as an int) for the given ServerConfig."""
    out = ctypes.c_void_p()
    _check(lib.tsmm_server_create(ctypes.byref(cfg), ctypes.byref(out)), "tsmm_server_create")
    return out.value


def tsmm_server_submit(server: int, reqs, count: int) -> None:
    """Submit `count` entries of a ctypes array of Request."""
    _check(lib.tsmm_server_submit(server, reqs, count), "tsmm_server_submit")


def tsmm_server_poll(server: int, out, max_items: int) -> int:
    """Fill a ctypes array of Completion; returns how many were written."""
    return int(lib.tsmm_server_poll(server, out, max_items))


def tsmm_server_drain(server: int, timeout_s: float) -> None:
    _check(lib.tsmm_server_drain(server, timeout_s), "tsmm_server_drain")


def tsmm_server_destroy(server: int) -> None:
    _check(lib.tsmm_server_destroy(server), "tsmm_server_destroy")


def tsmm_diag_server_inject_timeout(server: int, units: int) -> None:
    """The next `units` launch units of the server finish as if a bounded wait
    in their kernels had run out (diagnostics of the serving failure path)."""
    _check(lib.tsmm_diag_server_inject_timeout(server, int(units)), "tsmm_diag_server_inject_timeout")


class Server:
    """Owner of a tsmm_server_t: continuous batching of TSMM requests against
    device-resident packed B matrices (see include/tsmm.h)."""

    def __init__(self, budget_bytes: int, dtype=F32, num_streams: int = 4, max_batch: int = 48,
                 arena_bytes: int = 0):
        dt = dtype if isinstance(dtype, int) else _dtype_code(dtype)
        cfg = ServerConfig(budget_bytes, arena_bytes, num_streams, max_batch, dt)
        out = ctypes.c_void_p()
        _check(lib.tsmm_server_create(ctypes.byref(cfg), ctypes.byref(out)), "tsmm_server_create")
        self.handle = out.value

    def submit(self, requests) -> None:
        """requests: sequence of (id, packed_b, m, alpha, A, beta, C, arrival_s) with
        column-major CUDA tensors A (m x k) and C (m x n)."""
        arr = (Request * max(1, len(requests)))()
        for i, (rid, pb, m, alpha, A, beta, C, t) in enumerate(requests):
            lda = ld_of(A) if m > 0 and A.shape[1] > 0 else max(1, m)
            ldc = ld_of(C) if m > 0 and C.shape[1] > 0 else max(1, m)
            arr[i] = Request(rid, pb.handle, m, float(alpha), float(beta),
                             A.data_ptr() if A.numel() else None, lda,
                             C.data_ptr() if C.numel() else None, ldc, float(t))
        _check(lib.tsmm_server_submit(self.handle, arr, len(requests)), "tsmm_server_submit")

    def submit_raw(self, arr, count: int) -> None:
        """Submit a prepared ctypes array of Request."""
        _check(lib.tsmm_server_submit(self.handle, arr, count), "tsmm_server_submit")

    def drain(self, timeout_s: float = 600.0) -> None:
        _check(lib.tsmm_server_drain(self.handle, timeout_s), "tsmm_server_drain")

    def poll(self, max_items: int = 1 << 16):
        """Completed requests as a list of dicts."""
        buf = (Completion * max_items)()
        n = int(lib.tsmm_server_poll(self.handle, buf, max_items))
        return [dict(id=c.id, arrival_s=c.arrival_s, admit_s=c.admit_s, launch_s=c.launch_s,
                     complete_s=c.complete_s, status=c.status) for c in buf[:n]]

    def inject_timeout(self, units: int = 1) -> None:
        """tsmm_diag_server_inject_timeout on this server."""
        tsmm_diag_server_inject_timeout(self.handle, units)

    def close(self):
        if self.handle:
            lib.tsmm_server_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
