"""tsmm_execute_noalloc: the allocation-free entry point for callers that
cannot call cudaMalloc (code whose device memory is owned by a host framework,
latency-critical loops that cannot take cudaMalloc's implicit synchronisation).

Called through the C ABI (ctypes on libtsmm.so) on two calls in a row and
checked, like every parity test here, against the CPU oracle: within the
componentwise bound E = 4*k*u*(|alpha||A||B| + |beta||C0|) of the oracle's
result, and bit for bit equal to the oracle's result rounded to the working
precision on integer-valued inputs.  As a second check each result is also
compared with the allocating path tsmm_pack_b / tsmm_plan / tsmm_execute on the
same inputs (within E of it; identical bits on integer inputs).  This file is
collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2208_08088_gb300 as tsmm
import tsmm_inputs as ti

pytestmark = pytest.mark.gpu

_fn = tsmm.lib.tsmm_execute_noalloc
_fn.restype = ctypes.c_int
_fn.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]


def dev(X, ld=None, offset=0):
    rows, cols = X.shape
    ld = max(1, rows) if ld is None else ld
    base = torch.full((offset + ld * cols + 64,), float("nan"),
                      dtype=torch.float32 if X.dtype == np.float32 else torch.float64, device="cuda")
    v = torch.as_strided(base, (rows, cols), (1, ld), storage_offset=offset)
    v.copy_(torch.from_numpy(np.ascontiguousarray(X)))
    return v


def noalloc(dtype_code, A, B, C, alpha, beta, lda, ldb, ldc):
    m, k = A.shape
    n = B.shape[1]
    stream = torch.cuda.current_stream().cuda_stream
    return _fn(dtype_code, m, n, k, alpha, A.data_ptr(), lda, B.data_ptr(), ldb, beta,
               C.data_ptr(), ldc, stream or None)


CASES = [
    # (m, n, k, dist, lda_pad, a_offset): split-K with TMA; one slab per split
    (300, 16, 20000, "uniform", 0, 0),
    (2048, 16, 2048, "integer", 0, 0),
    (1000, 64, 777, "uniform", 0, 0),
    (301, 5, 3000, "uniform", 2, 1),      # unaligned A: the plain-load kernel
    (32768, 8, 4096, "uniform", 0, 0),    # many slabs: split limited by the scratch
    (700, 40, 3000, "uniform", 0, 0),     # width 48
]


@pytest.mark.parametrize("npdt", [np.float32, np.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("m,n,k,dist,lda_pad,a_off", CASES)
def test_noalloc_matches_allocating_path(npdt, m, n, k, dist, lda_pad, a_off):
    code = tsmm.F32 if npdt == np.float32 else tsmm.F64
    A = ti.matrix_np(m, k, ti.SEED_A, dist, npdt)
    B = ti.matrix_np(k, n, ti.SEED_B, dist, npdt)
    C0 = ti.matrix_np(m, n, ti.SEED_C0, dist, npdt)
    lda = m + lda_pad
    dA = dev(A, lda, a_off)
    dB = dev(B)
    alpha, beta = 1.5, 0.5

    # the oracle: Eq. 1 in plain C on the host, and its componentwise bound
    Cref, E = oracle.tsmm(alpha, A, B, beta, C0)

    # the allocating entry points, for the second check
    dC_lib = dev(C0)
    pl = tsmm.plan(m, n, k, dA.dtype)
    tsmm.execute(pl, alpha, dA, tsmm.pack_b(dB), beta, dC_lib)
    pl.check()
    C_lib = dC_lib.cpu().numpy()

    for call in range(2):  # two calls in a row share (and must re-clear) the scratch
        dC = dev(C0)
        st = noalloc(code, dA, dB, dC, alpha, beta, lda, k, m)
        assert st == 0, tsmm.tsmm_status_string(st)
        torch.cuda.synchronize()
        C = dC.cpu().numpy()
        ok, ratio, nbad = oracle.check(C, Cref, E, npdt)
        assert ok, f"call {call}: {nbad} entries outside the oracle's bound (max ratio {ratio:.3g})"
        if dist == "integer":
            np.testing.assert_array_equal(C, oracle.round_to(Cref, npdt))
        ok, _, nbad = oracle.check(C, C_lib, E, npdt)
        assert ok, f"call {call}: {nbad} entries differ from tsmm_execute by more than E"
        if dist == "integer":
            np.testing.assert_array_equal(C, C_lib)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    """Packed B of k = 2^20 rows x 64 columns (256 MiB) exceeds the 32 MiB
    scratch: rejected before any device work; n > 64 is not this kernel."""
    dummy = torch.zeros(1024, device="cuda")
    p = dummy.data_ptr()
    assert _fn(tsmm.F32, 128, 64, 1 << 20, 1.0, p, 128, p, 1 << 20, 0.0, p, 128, None) == 2
    assert _fn(tsmm.F32, 128, 65, 16, 1.0, p, 128, p, 16, 0.0, p, 128, None) == 2
    assert _fn(tsmm.F32, 128, 16, 16, 1.0, p, 127, p, 16, 0.0, p, 128, None) == 1  # lda < m


def test_noalloc_split_limited_by_scratch_integer_bitwise():
    """Packed B of 16 MiB leaves room for only a few 2 MiB partial-tile splits:
    the k split is reduced to fit, and the integer-valued result (every partial
    sum exact) must equal the oracle's bit for bit on sampled rows, twice, and
    the allocating path's everywhere."""
    m, n, k = 4096, 64, 65536
    dA = torch.empty((k, m), dtype=torch.float32, device="cuda")
    ti.fill_torch(dA, ti.SEED_A, "integer")
    dA = dA.t()
    dB = torch.empty((n, k), dtype=torch.float32, device="cuda")
    ti.fill_torch(dB, ti.SEED_B, "integer")
    dB = dB.t()
    C0 = torch.empty((n, m), dtype=torch.float32, device="cuda")
    ti.fill_torch(C0, ti.SEED_C0, "integer")
    C0 = C0.t()

    # oracle on 64 sampled rows (first and last included), inputs regenerated on the host
    rows = np.sort(np.random.default_rng(11).choice(m, size=64, replace=False))
    rows[0], rows[-1] = 0, m - 1
    A_r = np.asfortranarray(ti.rows_np(rows, m, k, ti.SEED_A, "integer", np.float32))
    B = ti.matrix_np(k, n, ti.SEED_B, "integer", np.float32)
    C0_r = np.asfortranarray(ti.rows_np(rows, m, n, ti.SEED_C0, "integer", np.float32))
    Cref, E = oracle.tsmm(1.5, A_r, B, 0.5, C0_r)
    want = oracle.round_to(Cref, np.float32)

    dC_lib = torch.empty((n, m), dtype=torch.float32, device="cuda").t()
    dC_lib.copy_(C0)
    pl = tsmm.plan(m, n, k, torch.float32)
    assert pl.info()["splits"] > 1
    tsmm.execute(pl, 1.5, dA, tsmm.pack_b(dB), 0.5, dC_lib)
    pl.check()
    sel = torch.as_tensor(rows, device="cuda")
    for _ in range(2):
        dC = torch.empty((n, m), dtype=torch.float32, device="cuda").t()
        dC.copy_(C0)
        st = noalloc(tsmm.F32, dA, dB, dC, 1.5, 0.5, m, k, m)
        assert st == 0, tsmm.tsmm_status_string(st)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dC[sel].cpu().numpy(), want)
        assert torch.equal(dC, dC_lib)
