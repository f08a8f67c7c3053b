"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element
by element, on seeded inputs at sizes that span several tiles and ragged tails.

Acceptance (Eq. 1 with the componentwise bound of the library's contract):
|C - C_ref| <= 4*k*u*(|alpha| |A||B| + |beta| |C0|), u = 2^-24 / 2^-53; and
bit-exact equality on integer-valued inputs whose partial sums are exactly
representable (entries in [-4, 4], dyadic alpha and beta)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2208_08088_gb300 as tsmm
import tsmm_inputs as ti
from gpu_util import assert_parity, run, to_device

pytestmark = pytest.mark.gpu

DT = [np.float32, np.float64]


def gen(m, n, k, dtype, dist="uniform", seeds=(ti.SEED_A, ti.SEED_B, ti.SEED_C0)):
    return (ti.matrix_np(m, k, seeds[0], dist, dtype), ti.matrix_np(k, n, seeds[1], dist, dtype),
            ti.matrix_np(m, n, seeds[2], dist, dtype))


# ------------------------------------------------------------- m = k = 2048, n = 16, alpha = 1.5, beta = 0.5
@pytest.mark.parametrize("dist", ["uniform", "integer"])
@pytest.mark.parametrize("dtype", DT)
def test_2048x2048x16_alpha_beta(dist, dtype):
    """m = k = 2048, n = 16, alpha = 1.5, beta = 0.5, B packed once."""
    A, B, C0 = gen(2048, 16, 2048, dtype, dist)
    C, pl, _ = run(A, B, C0, 1.5, 0.5)
    assert_parity(C, A, B, C0, 1.5, 0.5, exact=(dist == "integer"))


# ------------------------------------------------------------- regime (i) sweep
@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 9, 16, 17, 20, 24, 31, 32, 33, 40, 48, 63, 64])
def test_tall_all_n_ragged(dtype, n):
    """m, k not multiples of the tile sizes (256/128/64-row slabs, 32-column
    stages), every padded width (1, 2, 4, 8, 16, 24, 32, 48, 64)."""
    m, k = 1000, 777
    A, B, C0 = gen(m, n, k, dtype)
    C, pl, _ = run(A, B, C0, -1.25, 0.75)
    assert pl.info()["regime"] == 1
    assert_parity(C, A, B, C0, -1.25, 0.75)


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (1, 16, 1), (3, 7, 2), (5, 64, 33), (129, 16, 31),
                                   (128, 16, 32), (64, 64, 64), (257, 2, 4097)])
def test_tall_small_and_edges(dtype, m, n, k):
    A, B, C0 = gen(m, n, k, dtype)
    C, _, _ = run(A, B, C0, 1.0, 1.0)
    assert_parity(C, A, B, C0, 1.0, 1.0)


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n", [1, 16, 24, 32, 48, 64])
def test_tall_split_k_integer_exact(dtype, n):
    """Few m-slabs and long k force split-K (S > 1); integer inputs make the
    result independent of the summation order, so it must be bit-exact."""
    m, k = 300, 20000
    A, B, C0 = gen(m, n, k, dtype, "integer")
    C, pl, _ = run(A, B, C0, 1.5, 0.5)
    assert pl.info()["splits"] > 1
    assert_parity(C, A, B, C0, 1.5, 0.5, exact=True)


@pytest.mark.parametrize("dtype", DT)
def test_tall_split_k_uniform(dtype):
    m, n, k = 700, 16, 30000
    A, B, C0 = gen(m, n, k, dtype)
    C, pl, _ = run(A, B, C0, 1.0, -1.0)
    assert pl.info()["splits"] > 1
    assert_parity(C, A, B, C0, 1.0, -1.0)


@pytest.mark.parametrize("dtype", DT)
def test_deterministic_repeats(dtype):
    """Fixed-order split-K: repeated executions give identical bits."""
    A, B, C0 = gen(500, 16, 9000, dtype)
    outs, pl, _ = run(A, B, C0, 1.0, 0.5, repeats=3)
    assert pl.info()["splits"] > 1
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


# ------------------------------------------------------------- layouts / paths
@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n", [4, 16, 64])
def test_padded_leading_dimensions_tma_path(dtype, n):
    """lda, ldb, ldc larger than the matrix (16-byte multiples keep TMA); the
    padding holds NaN and must never be read or written."""
    m, k = 333, 515
    A, B, C0 = gen(m, n, k, dtype)
    C, _, _ = run(A, B, C0, 1.5, 0.5, lda=352, ldb=520, ldc=340)
    assert_parity(C, A, B, C0, 1.5, 0.5)


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n", [1, 16, 64])
def test_unaligned_A_takes_plain_load_path(dtype, n):
    """An odd lda (rows not 16-byte aligned) and an A pointer one element off
    a 16-byte boundary: the kernel without TMA must give the same result."""
    m, k = 301, 250
    A, B, C0 = gen(m, n, k, dtype)
    C1, _, _ = run(A, B, C0, 1.0, 1.0, lda=303)
    assert_parity(C1, A, B, C0, 1.0, 1.0)
    C2, _, _ = run(A, B, C0, 1.0, 1.0, a_offset=1)
    assert_parity(C2, A, B, C0, 1.0, 1.0)


@pytest.mark.parametrize("dtype", DT)
def test_unaligned_integer_matches_tma_bitwise(dtype):
    A, B, C0 = gen(640, 16, 3000, dtype, "integer")
    C_tma, _, _ = run(A, B, C0, 1.5, 0.5)
    C_gen, _, _ = run(A, B, C0, 1.5, 0.5, a_offset=1)
    assert np.array_equal(C_tma, C_gen)
    assert_parity(C_tma, A, B, C0, 1.5, 0.5, exact=True)


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n", [1, 5, 16, 24, 40, 64])
@pytest.mark.parametrize("m,k,lda_pad,a_off", [(1027, 333, 1, 0), (1026, 700, 2, 1), (2049, 3001, 3, 3),
                                               (257, 40, 0, 2), (513, 20000, 1, 1)])
def test_unaligned_A_every_offset_integer_exact(dtype, n, m, k, lda_pad, a_off):
    """A whose column stride or base is not 16-byte aligned streams through the
    cp.async kernel, which places each column at its own offset within 16
    bytes: every offset (a_off 0..3, lda = m + 1..3), a ragged last slab, k not a
    multiple of 32, and split-K (k = 20000).  Integer inputs: equal to the TMA
    path bit for bit and to the oracle."""
    A, B, C0 = gen(m, n, k, dtype, "integer")
    C_tma, _, _ = run(A, B, C0, 1.5, 0.5, lda=m + (4 - m % 4) % 4)
    C_un, _, _ = run(A, B, C0, 1.5, 0.5, lda=m + lda_pad, a_offset=a_off)
    np.testing.assert_array_equal(C_un, C_tma)
    assert_parity(C_un, A, B, C0, 1.5, 0.5, exact=True)


# ------------------------------------------------------------- special cases
@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n,k", [(16, 100), (200, 64)])
def test_alpha_zero_reads_neither_A_nor_B(dtype, n, k):
    m = 150
    A = np.full((m, k), np.nan, dtype=dtype, order="F")
    B = np.asfortranarray(np.full((k, n), np.inf, dtype=dtype))
    C0 = ti.matrix_np(m, n, 3, "uniform", dtype)
    C, _, _ = run(A, B, C0, 0.0, 1.5)
    np.testing.assert_array_equal(C, (C0.astype(np.float64) * 1.5).astype(dtype))


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n,k", [(16, 100), (200, 64)])
@pytest.mark.parametrize("m", [150, 152])  # 152: C meets the TMA rules
def test_beta_zero_overwrites_nan(dtype, n, k, m):
    A, B, _ = gen(m, n, k, dtype)
    C, _, _ = run(A, B, None, 2.0, 0.0)
    assert np.all(np.isfinite(C))
    assert_parity(C, A, B, None, 2.0, 0.0)


@pytest.mark.parametrize("dtype", DT)
def test_k_zero_is_beta_scale(dtype):
    m, n = 77, 9
    C0 = ti.matrix_np(m, n, 3, "uniform", dtype)
    A = np.zeros((m, 0), dtype=dtype, order="F")
    B = np.zeros((0, n), dtype=dtype, order="F")
    C, _, _ = run(A, B, C0, 1.0, 0.5)
    np.testing.assert_array_equal(C, (C0.astype(np.float64) * 0.5).astype(dtype))


@pytest.mark.parametrize("dtype", DT)
def test_empty_m_or_n_is_noop(dtype):
    for (m, n, k) in ((0, 16, 10), (10, 0, 10)):
        pl = tsmm.plan(m, n, k, gpu_dtype(dtype))
        dB = to_device(np.zeros((k, n), dtype=dtype, order="F"))
        pb = tsmm.pack_b(dB)
        dA = to_device(np.zeros((m, k), dtype=dtype, order="F"))
        dC = to_device(np.zeros((m, n), dtype=dtype, order="F"))
        tsmm.execute(pl, 1.0, dA, pb, 1.0, dC)
        pl.check()
        assert pl.launches_per_execute() == 0


def gpu_dtype(dtype):
    return torch.float32 if dtype == np.float32 else torch.float64


@pytest.mark.parametrize("dtype", DT)
def test_ieee_specials_propagate(dtype):
    m, n, k = 130, 4, 70
    A, B, C0 = gen(m, n, k, dtype)
    A = A.copy(order="F")
    A[5, 3] = np.inf
    A[77, 10] = np.nan
    C, _, _ = run(A, B, C0, 1.0, 1.0)
    assert_parity(C, A, B, C0, 1.0, 1.0)


# ------------------------------------------------------------- regime (ii)
@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("k", [1, 4, 7, 16, 17, 32, 37, 48, 64, 127, 128])
def test_rankk_ragged(dtype, k):
    m, n = 1000, 300
    A, B, C0 = gen(m, n, k, dtype)
    C, pl, _ = run(A, B, C0, 1.0, 1.0)
    assert pl.info()["regime"] == 2
    assert_parity(C, A, B, C0, 1.0, 1.0)


@pytest.mark.parametrize("dtype", DT)
def test_rankk_integer_exact_and_padded(dtype):
    m, n, k = 513, 257, 100
    A, B, C0 = gen(m, n, k, dtype, "integer")
    C, _, _ = run(A, B, C0, 1.5, 0.5, lda=520, ldb=104, ldc=516)
    assert_parity(C, A, B, C0, 1.5, 0.5, exact=True)
    C2, _, _ = run(A, B, C0, 1.5, 0.5, lda=515, ldc=514, a_offset=1, c_offset=1)
    assert np.array_equal(C, C2)


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("k", [4, 16, 32, 64, 128])
def test_rankk_unaligned_A_equals_aligned(dtype, k):
    """An A that a tensor map cannot describe (lda*s or the base not a multiple
    of 16 bytes) is copied into an aligned scratch buffer on the stream, so
    regime (ii) then runs the same kernels: bit for bit the aligned result, with
    C aligned (TMA epilogue) and not (plain epilogue)."""
    m, n = 1001, 700
    A, B, C0 = gen(m, n, k, dtype)
    pl = pb = None
    for ldc in (1004, 1001):  # C described by a tensor map, and not
        ref, pl, pb = run(A, B, C0, 1.25, 0.75, lda=1004, ldc=ldc, plan=pl, pb=pb)
        for lda, off in ((1001, 0), (1003, 2), (1004, 1)):
            C, _, _ = run(A, B, C0, 1.25, 0.75, lda=lda, ldc=ldc, a_offset=off, plan=pl, pb=pb)
            assert np.array_equal(C, ref), f"lda={lda} offset={off} ldc={ldc}"
        assert_parity(ref, A, B, C0, 1.25, 0.75)


# ------------------------------------------------------------- packing + ABI errors
@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("k,n", [(1, 1), (33, 5), (100, 64), (7, 65), (128, 300)])
def test_pack_roundtrip_bitwise(dtype, k, n):
    """Unpacking the packed storage with a reader written from the layout
    documented in include/tsmm.h reproduces B bit for bit, with +0 padding."""
    B = ti.matrix_np(k, n, 9, "uniform", dtype)
    pb = tsmm.pack_b(to_device(B, ld=k + 3))
    info = pb.info()
    flat = pb.read()
    kp, w, nt = info["kp"], info["w"], info["ntiles"]
    assert flat.size == kp * w * nt and kp >= k and w * nt >= n
    tiles = flat.reshape(nt, kp, w)
    full = np.concatenate([tiles[t] for t in range(nt)], axis=1)  # kp x (nt*w)
    assert np.ascontiguousarray(full[:k, :n]).tobytes() == np.ascontiguousarray(B).tobytes()
    pad = full.copy()
    pad[:k, :n] = 0
    assert np.all(pad == 0) and not np.any(np.signbit(pad))


def test_mismatch_and_misaligned_errors():
    B = to_device(ti.matrix_np(100, 16, 1, "uniform", np.float32))
    pb = tsmm.pack_b(B)
    A = to_device(ti.matrix_np(50, 101, 1, "uniform", np.float32))
    C = to_device(np.zeros((50, 16), dtype=np.float32, order="F"))
    with pytest.raises(tsmm.TsmmError) as e:
        tsmm.execute(tsmm.plan(50, 16, 101, torch.float32), 1.0, A, pb, 0.0, C)
    assert e.value.status == 3
    A64 = to_device(ti.matrix_np(50, 100, 1, "uniform", np.float64))
    with pytest.raises(tsmm.TsmmError) as e:
        tsmm.execute(tsmm.plan(50, 16, 100, torch.float64), 1.0, A64, pb, 0.0, C)
    assert e.value.status == 3
    pl = tsmm.plan(50, 16, 100, torch.float32)
    with pytest.raises(tsmm.TsmmError) as e:  # C pointer not 4-byte aligned
        tsmm.tsmm_execute(pl.handle, 1.0, A.data_ptr(), 50, pb.handle, 0.0, C.data_ptr() + 2, 50)
    assert e.value.status == 4
    with pytest.raises(tsmm.TsmmError) as e:  # lda < m
        tsmm.tsmm_execute(pl.handle, 1.0, A.data_ptr(), 49, pb.handle, 0.0, C.data_ptr(), 50)
    assert e.value.status == 1


def test_plan_reuse_across_A_pointers():
    """The plan caches its TMA descriptor per A pointer; a new A must be seen."""
    m, n, k = 400, 8, 600
    A1, B, C0 = gen(m, n, k, np.float32)
    A2 = ti.matrix_np(m, k, 77, "uniform", np.float32)
    pl = tsmm.plan(m, n, k, torch.float32)
    pb = tsmm.pack_b(to_device(B))
    for A in (A1, A2, A1):
        C, _, _ = run(A, B, C0, 1.0, 0.0, plan=pl, pb=pb)
        assert_parity(C, A, B, None, 1.0, 0.0)


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("k", [3, 16, 32, 33, 100])
@pytest.mark.parametrize("beta", [0.0, 1.0, -0.5])
@pytest.mark.parametrize("m", [2050, 2048])
def test_rankk_persistent_many_tiles(dtype, k, beta, m):
    """More tiles than resident blocks: every block walks several tiles, reusing
    its k-chunk ring and its C buffers (m = 2048: C meets the TMA rules, so C0
    and C move by tensor copies; m = 2050: plain loads and stores)."""
    n = 1000
    A, B, C0 = gen(m, n, k, dtype)
    C, pl, _ = run(A, B, C0 if beta != 0 else None, 1.0 if k != 33 else 0.75, beta)
    assert pl.info()["regime"] == 2
    assert_parity(C, A, B, C0 if beta != 0 else None, 1.0 if k != 33 else 0.75, beta)


@pytest.mark.parametrize("beta", [0.0, 1.0])
@pytest.mark.parametrize("k", [33, 64, 128])
@pytest.mark.parametrize("m,n", [(129, 65), (1000, 80), (1000, 96), (384, 97), (640, 70), (1000, 130),
                                 (2048, 1000)])
def test_rankk_tma_epilogue_edges_integer_exact(m, n, k, beta):
    """FP32 with k > 32 and C meeting the TMA rules (m = 129 does not: the plain
    epilogue) moves C0 and C as 128 x 64 tiles by tensor copies: ragged m and n
    whose last tile is a quarter to seven eighths beyond m or n, beta = 0 over a
    NaN-filled C, integer inputs (exact)."""
    A, B, C0 = gen(m, n, k, np.float32, "integer")
    C, pl, _ = run(A, B, C0 if beta != 0 else None, 1.5, beta)
    assert pl.info()["regime"] == 2
    assert pl.info()["bm"] == 128
    assert_parity(C, A, B, C0 if beta != 0 else None, 1.5, beta, exact=True)


@pytest.mark.parametrize("beta", [0.0, 1.0])
@pytest.mark.parametrize("k", [40, 100])
@pytest.mark.parametrize("m", [2048, 2050])
def test_rankk_wide_several_tiles_per_block(m, k, beta):
    """FP32 with k > 32 over 1216 or more 128 x 64 tiles (n = 4864), so that
    every one of the 2 x 152 persistent blocks walks four tiles or more through
    its k-chunk ring and its C buffer (m = 2048: tensor copies for C0 and C;
    m = 2050: plain loads and stores); k = 40 and 100 end in a partial chunk
    of 32.  Integer inputs (exact)."""
    n = 4864
    A, B, C0 = gen(m, n, k, np.float32, "integer")
    C, pl, _ = run(A, B, C0 if beta != 0 else None, 1.5, beta)
    assert pl.info()["regime"] == 2
    assert_parity(C, A, B, C0 if beta != 0 else None, 1.5, beta, exact=True)


@pytest.mark.parametrize("alpha", [1.0, -0.5])
@pytest.mark.parametrize("k", [64, 128])
@pytest.mark.parametrize("m", [1024, 1001])
def test_rankk_beta_one_subnormals_exact(m, k, alpha):
    """FP32, k > 32, beta = 1 (C = C0 + alpha*AB in one rounding: by a TMA
    reduce-add of alpha*acc when C meets the TMA rules, m = 1024, and by the
    plain epilogue's fma(1, C0, alpha*acc), m = 1001): subnormals are
    neither read nor written as zero.  In the first half of the rows A is zero
    and C keeps its subnormal C0; in the other half alpha*AB is alpha * 2^-126
    (alpha = -0.5: itself subnormal) and C0 = s - alpha * 2^-126 with s a
    subnormal, so C = s exactly."""
    n = 320
    rng = np.random.default_rng(11)
    A = np.zeros((m, k), np.float32, order="F")
    B = np.zeros((k, n), np.float32, order="F")
    half = m // 2
    A[half:, 3] = np.float32(2.0 ** -63)
    B[3, :] = np.float32(2.0 ** -63)
    tiny = 2.0 ** -149
    s = rng.integers(-(2 ** 20), 2 ** 20, size=(m, n)).astype(np.float64) * tiny
    C0 = s.copy()
    C0[half:] -= alpha * 2.0 ** -126
    C0 = np.asfortranarray(C0.astype(np.float32))
    assert np.array_equal(C0.astype(np.float64), np.where(np.arange(m)[:, None] < half, s,
                                                          s - alpha * 2.0 ** -126))  # exact
    C, pl, _ = run(A, B, C0, alpha, 1.0)
    assert pl.info()["regime"] == 2
    np.testing.assert_array_equal(C, s.astype(np.float32))
    assert_parity(C, A, B, C0, alpha, 1.0, exact=True)


@pytest.mark.parametrize("k", [16, 64])
@pytest.mark.parametrize("m", [1024, 1001])
def test_rankk_ieee_specials_propagate(m, k):
    """FP32 regime (ii) with beta = 1 (k = 64: the TMA reduce-add into C when C
    meets the TMA rules, m = 1024): infinities and NaNs in A and in C0 reach C as
    the oracle has them, including inf + (-inf) = NaN between the product and C0."""
    n = 300
    A, B, C0 = gen(m, n, k, np.float32)
    A, B, C0 = A.copy(order="F"), np.abs(B).astype(np.float32, order="F"), C0.copy(order="F")
    A[5, 3] = np.inf
    A[77, 10] = np.nan
    A[300, :] = 0.0
    A[300, 0] = np.inf        # row 300: +inf products (B >= 0, B[0] > 0 where checked)
    B[0, :] = np.maximum(B[0, :], np.float32(0.25))
    C0[300, 100] = -np.inf    # +inf + (-inf) = NaN
    C0[300, 101] = np.inf     # +inf + inf = inf
    C0[200, 17] = np.nan
    C0[400, 250] = -np.inf
    C, pl, _ = run(A, B, C0, 1.0, 1.0)
    assert pl.info()["regime"] == 2
    assert np.isnan(C[300, 100]) and C[300, 101] == np.inf and np.isnan(C[200, 17]) and C[400, 250] == -np.inf
    assert_parity(C, A, B, C0, 1.0, 1.0)


@pytest.mark.parametrize("k", [1, 8, 32])
def test_rankk_f64_alpha_beta_one_integer_exact(k):
    """FP64 with alpha = beta = 1 and k within one chunk starts its
    accumulators from C0 (another summation order of the same terms): exact on
    integers, over several tiles per block."""
    m, n = 2048, 1000
    A, B, C0 = gen(m, n, k, np.float64, "integer")
    C, pl, _ = run(A, B, C0, 1.0, 1.0)
    assert pl.info()["regime"] == 2
    assert_parity(C, A, B, C0, 1.0, 1.0, exact=True)


def test_2048x2048x16_integer_matches_golden_fixture():
    """GPU rows of the m = k = 2048, n = 16 integer workload equal the committed
    fixture (written by tests/golden/make_golden.py from the oracle) bit for bit."""
    import json
    import os
    fx = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                     "tsmm_2048x2048x16_integer_rows.json")))
    m, n, k = fx["m"], fx["n"], fx["k"]
    A, B, C0 = gen(m, n, k, np.float32, "integer")
    C, _, _ = run(A, B, C0, fx["alpha"], fx["beta"])
    np.testing.assert_array_equal(C[fx["rows"]], np.array(fx["C_rows"], dtype=np.float32))


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("m,n,k", [(4000, 64, 3000), (1000, 16, 20000), (3000, 200, 100)])
def test_row_slabs_match_whole_problem_integer(world, m, n, k):
    """The multi-GPU row split (bench.py --split rows) on one GPU: each slab of
    rows [lo, hi) from bench.row_slab gets its own plan and runs on views of the
    same A and C (lda = ldc = m, offset lo); together they must equal the whole
    problem's execute and the oracle bit for bit (integer inputs: every partial
    sum exact, whatever the slab's split of k)."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "bench", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    A, B, C0 = gen(m, n, k, np.float32, "integer")
    whole, pl, pb = run(A, B, C0, 1.5, 0.5)
    dA = to_device(A)
    dC = to_device(C0)
    bm = pl.info()["bm"]
    for r in range(world):
        lo, hi = bench.row_slab(m, r, world, bm)
        pl_r = tsmm.plan(hi - lo, n, k, torch.float32)
        tsmm.execute(pl_r, 1.5, dA[lo:hi], pb, 0.5, dC[lo:hi])
        pl_r.check()
    split = dC.cpu().numpy()
    np.testing.assert_array_equal(split, whole)
    assert_parity(split, A, B, C0, 1.5, 0.5, exact=True)
