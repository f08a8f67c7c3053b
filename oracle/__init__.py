"""CPU oracle for C = alpha*A*B + beta*C0 (Eq. 1 of AutoTSMM, arXiv 2208.08088).

THIS IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library under ``paper_2208_08088_gb300/`` and neither imports the other.

The arithmetic lives in ``tsmm_oracle.c`` (plain C, FP64 accumulation, the
compensated Dot2 dot product for FP64 operands); this module compiles it with
gcc and calls it through ctypes on numpy arrays.

Parity status: every function here is pinned by the CPU tests in
``tests/test_oracle_pins.py`` (exhaustive ternary brute force, exact integer
products, closed forms, transpose symmetry, leading-dimension padding, and
exact-rational checks of the FP64 compensated path).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsmm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
            "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            i64, dbl, vp = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            for name in ("oracle_tsmm_f32", "oracle_tsmm_f64"):
                fn = getattr(lib, name)
                fn.restype = ctypes.c_int
                fn.argtypes = [i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, vp, vp]
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_num_threads.argtypes = []
            _lib = lib
    return _lib


def num_threads() -> int:
    """Threads the oracle's parallel loop uses (OMP_NUM_THREADS or all cores)."""
    return int(_load().oracle_num_threads())


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def tsmm(alpha, A, B, beta, C0, *, m=None, n=None, k=None, lda=None, ldb=None, ldc=None,
         dtype=None):
    """Evaluate Eq. 1 on column-major host arrays.

    ``A``, ``B``, ``C0`` are either Fortran-ordered 2-D arrays (shapes m x k,
    k x n, m x n; leading dimensions taken from their strides) or flat 1-D
    buffers with explicit ``m, n, k, lda, ldb, ldc``.  ``C0`` may be None when
    ``beta == 0``; ``A``/``B`` may be None when ``alpha == 0`` or ``k == 0``.

    Returns ``(Cref, E)``: float64 Fortran-ordered m x n arrays with the exact-
    ish result and the componentwise acceptance bound.
    """
    def ld_of(x, rows):
        if x is None:
            return max(1, rows)
        if x.ndim == 2:
            if x.shape[0] > 1 and x.strides[0] != x.itemsize:
                raise ValueError("2-D arguments must be column-major (Fortran order)")
            return x.strides[1] // x.itemsize if x.shape[1] > 1 else max(1, x.shape[0])
        raise ValueError("1-D buffers need explicit leading dimensions")

    if dtype is None:
        for x in (A, B, C0):
            if x is not None:
                dtype = x.dtype
                break
    dtype = np.dtype(dtype)
    if dtype not in (np.dtype(np.float32), np.dtype(np.float64)):
        raise TypeError("oracle supports float32 and float64")
    if m is None:
        if A is not None and A.ndim == 2:
            m, k = A.shape
        elif C0 is not None and C0.ndim == 2:
            m = C0.shape[0]
    if n is None:
        if B is not None and B.ndim == 2:
            k2, n = B.shape
            if k is None:
                k = k2
        elif C0 is not None and C0.ndim == 2:
            n = C0.shape[1]
    if k is None:
        k = 0
    if lda is None:
        lda = ld_of(A, m) if A is not None else max(1, m)
    if ldb is None:
        ldb = ld_of(B, k) if B is not None else max(1, k)
    if ldc is None:
        ldc = ld_of(C0, m) if C0 is not None else max(1, m)
    for x in (A, B, C0):
        if x is not None and x.dtype != dtype:
            raise TypeError("mixed dtypes")
    Cref = np.zeros((m, n), dtype=np.float64, order="F")
    E = np.zeros((m, n), dtype=np.float64, order="F")
    lib = _load()
    fn = lib.oracle_tsmm_f32 if dtype == np.float32 else lib.oracle_tsmm_f64
    rc = fn(int(m), int(n), int(k), float(alpha), _ptr(A), int(lda), _ptr(B), int(ldb),
            float(beta), _ptr(C0), int(ldc), _ptr(Cref), _ptr(E))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (code {rc})")
    return Cref, E


def round_to(x: np.ndarray, dtype) -> np.ndarray:
    """Round the oracle's double result to the working precision (RN-even)."""
    return np.asarray(x, dtype=np.float64).astype(dtype)


def check(C, Cref, E, dtype):
    """Componentwise acceptance test |C - Cref| <= E.

    Where E == 0 (no accumulation took place: k == 0, or alpha*A*B vanishes and
    beta == 0) the result is a single correctly rounded operation, so C must
    equal Cref rounded to the working precision bit for bit.  NaN must match
    NaN, infinities must match exactly.  Returns (ok, max_ratio, n_bad) where
    max_ratio = max |C - Cref| / E over entries with E > 0.
    """
    C = np.asarray(C, dtype=np.float64)
    Cref = np.asarray(Cref, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    nan_c, nan_r = np.isnan(C), np.isnan(Cref)
    bad = nan_c != nan_r
    fin = ~(nan_c | nan_r)
    inf_mix = fin & (np.isinf(C) | np.isinf(Cref))
    bad |= inf_mix & (C != Cref)
    reg = fin & ~inf_mix
    diff = np.abs(C - Cref)
    exact = reg & (E == 0)
    bad |= exact & (C != round_to(Cref, dtype).astype(np.float64))
    pos = reg & (E > 0)
    bad |= pos & (diff > E)
    ratio = float(np.max(diff[pos] / E[pos])) if np.any(pos) else 0.0
    return (not bool(np.any(bad))), ratio, int(np.count_nonzero(bad))
