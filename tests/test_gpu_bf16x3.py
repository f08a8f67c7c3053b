"""BF16x3 precision mode (tcgen05 tensor cores, FP32 accumulation in TMEM).

Integer-valued inputs in [-4, 4] are exact in BF16 (x_lo = 0) and every
partial sum is exact in FP32, so the tensor-core result must equal the oracle
bit for bit -- this pins the operand layouts, the k chunking and the split-K
finish exactly.  General inputs are checked against the mode's stated bound
(2^-13 + 4*k*2^-24) * (|alpha||A||B| + |beta||C0|)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2208_08088_gb300 as tsmm
import tsmm_inputs as ti
from gpu_util import to_device

pytestmark = pytest.mark.gpu
X3 = tsmm.PREC_BF16X3


def run_x3(A, B, C0, alpha, beta, lda=None, a_offset=0, repeats=1):
    m, k = A.shape
    n = B.shape[1]
    if lda is None:
        lda = (m + 3) // 4 * 4  # this mode needs lda*4 to be a multiple of 16
    dA = to_device(A, lda, a_offset)
    pb = tsmm.pack_b(to_device(B), precision=X3)
    pl = tsmm.plan(m, n, k, torch.float32, precision=X3)
    outs = []
    for _ in range(repeats):
        dC = to_device(C0 if C0 is not None else np.full((m, n), np.nan, np.float32, order="F"))
        tsmm.execute(pl, alpha, dA, pb, beta, dC)
        pl.check()
        outs.append(dC.cpu().numpy())
    return outs if repeats > 1 else outs[0], pl


def x3_bound(A, B, C0, alpha, beta):
    k = A.shape[1]
    G = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
    c = np.abs(C0.astype(np.float64)) if C0 is not None else 0.0
    return (2.0 ** -13 + 4 * k * 2.0 ** -24) * (abs(alpha) * G + abs(beta) * c)


@pytest.mark.parametrize("m,n,k", [(1000, 64, 777), (300, 16, 20000), (129, 17, 64), (2048, 32, 2048),
                                   (5, 3, 1), (640, 64, 4096), (257, 40, 130),
                                   # several work items per persistent block, with and without split-K
                                   (20000, 64, 4000), (40000, 32, 64)])
def test_bf16x3_integer_bit_exact(m, n, k):
    A = ti.matrix_np(m, k, 21, "integer", np.float32)
    B = ti.matrix_np(k, n, 22, "integer", np.float32)
    C0 = ti.matrix_np(m, n, 23, "integer", np.float32)
    C, pl = run_x3(A, B, C0, 1.5, 0.5)
    Cref, _ = oracle.tsmm(1.5, A, B, 0.5, C0)
    np.testing.assert_array_equal(C, oracle.round_to(Cref, np.float32))


@pytest.mark.parametrize("m,n,k,beta", [(1000, 64, 777, 1.0), (300, 16, 20000, 0.0), (2048, 32, 2048, -0.5),
                                        (4096, 64, 6000, 1.0), (77, 9, 100, 1.0)])
def test_bf16x3_uniform_within_mode_bound(m, n, k, beta):
    A = ti.matrix_np(m, k, 31, "uniform", np.float32)
    B = ti.matrix_np(k, n, 32, "uniform", np.float32)
    C0 = ti.matrix_np(m, n, 33, "uniform", np.float32)
    C, pl = run_x3(A, B, C0 if beta != 0 else None, 1.25, beta)
    Cref, _ = oracle.tsmm(1.25, A, B, beta, C0 if beta != 0 else None)
    E3 = x3_bound(A, B, C0 if beta != 0 else None, 1.25, beta)
    err = np.abs(C.astype(np.float64) - Cref)
    assert np.all(np.isfinite(C))
    assert np.all(err <= E3), f"max err/bound {np.max(err / E3):.3g}"


def test_bf16x3_deterministic_split_k():
    A = ti.matrix_np(700, 30000, 41, "uniform", np.float32)
    B = ti.matrix_np(30000, 64, 42, "uniform", np.float32)
    C0 = ti.matrix_np(700, 64, 43, "uniform", np.float32)
    outs, pl = run_x3(A, B, C0, 1.0, 1.0, repeats=3)
    assert pl.info()["splits"] > 1
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


def test_bf16x3_errors():
    B = to_device(ti.matrix_np(100, 16, 1, "uniform", np.float32))
    pb_native = tsmm.pack_b(B)
    pl_x3 = tsmm.plan(50, 16, 100, torch.float32, precision=X3)
    A = to_device(ti.matrix_np(50, 100, 1, "uniform", np.float32))
    C = to_device(np.zeros((50, 16), np.float32, order="F"))
    with pytest.raises(tsmm.TsmmError) as e:  # mode mismatch between plan and packed B
        tsmm.execute(pl_x3, 1.0, A, pb_native, 0.0, C)
    assert e.value.status == 3
    with pytest.raises(tsmm.TsmmError) as e:  # FP64 has no BF16x3 mode
        tsmm.plan(50, 16, 100, torch.float64, precision=X3)
    assert e.value.status == 1


@pytest.mark.parametrize("m,n,k,pad,offset", [(1000, 64, 777, 1, 0), (300, 16, 20000, 2, 1), (257, 40, 130, 3, 3),
                                              (2050, 32, 4000, 1, 2), (129, 17, 64, 0, 1), (5, 3, 1, 1, 1),
                                              # several work items per persistent block, with split-K
                                              (20000, 64, 4000, 3, 0), (40001, 32, 70, 2, 0)])
def test_bf16x3_unaligned_A_equals_aligned(m, n, k, pad, offset):
    """Regime (i) with an A that a tensor map cannot describe (lda*4 or the base
    not a multiple of 16 bytes): its columns are copied one by one into padded
    slots and read at their offsets, then split and multiplied exactly as the
    tensor-copy path does, so the result equals that path's on the same values
    bit for bit (and the mode bound holds against the oracle)."""
    A = ti.matrix_np(m, k, 51, "uniform", np.float32)
    B = ti.matrix_np(k, n, 52, "uniform", np.float32)
    C0 = ti.matrix_np(m, n, 53, "uniform", np.float32)
    ref, _ = run_x3(A, B, C0, 1.25, 0.5)  # lda rounded up to 4, base aligned: tensor copies
    C, _ = run_x3(A, B, C0, 1.25, 0.5, lda=m + pad, a_offset=offset)
    assert np.array_equal(C, ref)
    Cref, _ = oracle.tsmm(1.25, A, B, 0.5, C0)
    assert np.all(np.abs(C.astype(np.float64) - Cref) <= x3_bound(A, B, C0, 1.25, 0.5))


@pytest.mark.parametrize("m,n,k,pad,offset", [(1003, 64, 777, 1, 0), (258, 40, 130, 3, 2)])
def test_bf16x3_unaligned_A_integer_bit_exact(m, n, k, pad, offset):
    A = ti.matrix_np(m, k, 61, "integer", np.float32)
    B = ti.matrix_np(k, n, 62, "integer", np.float32)
    C0 = ti.matrix_np(m, n, 63, "integer", np.float32)
    C, _ = run_x3(A, B, C0, 1.5, 0.5, lda=m + pad, a_offset=offset)
    Cref, _ = oracle.tsmm(1.5, A, B, 0.5, C0)
    np.testing.assert_array_equal(C, oracle.round_to(Cref, np.float32))


def test_bf16x3_pack_layout_roundtrip():
    """hi + lo of every packed element reproduces B to BF16x2 accuracy, and the
    hi/lo tiles sit where the layout documented in tsmm.h puts them."""
    k, n = 130, 40
    B = ti.matrix_np(k, n, 51, "uniform", np.float32)
    pb = tsmm.pack_b(to_device(B), precision=X3)
    info = pb.info()
    kp, w = info["kp"], info["w"]
    assert kp == 192 and w == 64 and info["bytes"] == kp * w * 4
    raw = np.empty(info["bytes"] // 2, dtype=np.uint16)
    tsmm.tsmm_packed_b_read(pb.handle, raw.ctypes.data, raw.nbytes)

    def bf16(u):
        return (u.astype(np.uint32) << 16).view(np.float32)

    rec = np.zeros((kp, w), dtype=np.float64)
    for c in range(kp // 64):
        base = c * 2 * w * 64
        for j in range(w):
            for kk in range(64):
                off = ((j // 8) * 1024 + (kk // 8) * 128 + (j % 8) * 16 + (kk % 8) * 2) // 2
                rec[c * 64 + kk, j] = float(bf16(raw[base + off : base + off + 1])[0]) + \
                    float(bf16(raw[base + w * 64 + off : base + w * 64 + off + 1])[0])
    err = np.abs(rec[:k, :n] - B.astype(np.float64))
    assert np.all(err <= 2.0 ** -16 * np.abs(B))
    assert np.all(rec[k:, :] == 0) and np.all(rec[:, n:] == 0)


def test_bf16x3_full_size_sampled():
    """m = k = 32768, n = 64 (the FP32 sweep's FMA-bound point) in this mode."""
    m = k = 32768
    n = 64
    dA = torch.empty((k, m), dtype=torch.float32, device="cuda")
    ti.fill_torch(dA, ti.SEED_A, "uniform")
    dA = dA.t()
    dB = torch.empty((n, k), dtype=torch.float32, device="cuda")
    ti.fill_torch(dB, ti.SEED_B, "uniform")
    dB = dB.t()
    pl = tsmm.plan(m, n, k, torch.float32, precision=X3)
    pb = tsmm.pack_b(dB, precision=X3)
    dC = torch.zeros((n, m), dtype=torch.float32, device="cuda").t()
    tsmm.execute(pl, 1.0, dA, pb, 0.0, dC)
    pl.check()
    rows = np.sort(np.random.default_rng(3).choice(m, 32, replace=False))
    A_r = np.asfortranarray(ti.rows_np(rows, m, k, ti.SEED_A, "uniform", np.float32))
    B = ti.matrix_np(k, n, ti.SEED_B, "uniform", np.float32)
    Cref, _ = oracle.tsmm(1.0, A_r, B, 0.0, None)
    C = dC[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    E3 = x3_bound(A_r, B, None, 1.0, 0.0)
    err = np.abs(C.astype(np.float64) - Cref)
    assert np.all(err <= E3), f"max err/bound {np.max(err / E3):.3g}"


@pytest.mark.parametrize("m,n,k,beta", [(1000, 300, 64, 1.0), (2050, 1000, 128, 1.0), (515, 129, 33, 0.0),
                                        (4096, 2048, 100, -0.5), (300, 5000, 16, 1.0),
                                        # beta = 0: plain stores (ldc*4 not a multiple of 16)
                                        (2050, 1000, 128, 0.0),
                                        # beta = 0 with TMA stores; C starts as NaN
                                        (1024, 1000, 100, 0.0),
                                        # items of 6 n-tiles, the last chunk ragged
                                        (8192, 8000, 72, 1.0)])
def test_bf16x3_rankk_integer_bit_exact(m, n, k, beta):
    """Regime (ii) in the tensor-core mode: integer inputs are exact."""
    A = ti.matrix_np(m, k, 61, "integer", np.float32)
    B = ti.matrix_np(k, n, 62, "integer", np.float32)
    C0 = ti.matrix_np(m, n, 63, "integer", np.float32)
    C, pl = run_x3(A, B, C0 if beta else None, 1.5, beta)
    assert pl.info()["regime"] == 2
    Cref, _ = oracle.tsmm(1.5, A, B, beta, C0 if beta else None)
    np.testing.assert_array_equal(C, oracle.round_to(Cref, np.float32))


@pytest.mark.parametrize("m,n,k,pad,offset,beta,ldc_pad", [(1000, 700, 128, 1, 0, 0.5, 0), (257, 300, 40, 3, 2, 0.0, 0),
                                                             (2050, 130, 96, 2, 1, 1.0, 1), (131, 129, 64, 0, 3, 0.5, 0),
                                                             (4099, 1000, 17, 1, 1, 0.5, 3)])
def test_bf16x3_rankk_unaligned_A_equals_aligned(m, n, k, pad, offset, beta, ldc_pad):
    """Regime (ii) in the tensor-core mode with an A that a tensor map cannot
    describe: the item's A tile is copied column by column into padded slots
    and split as the tensor-copy path does, so the result equals that path's on
    the same values bit for bit, and integer inputs are exact."""
    for dist, seeds in (("uniform", (71, 72, 73)), ("integer", (74, 75, 76))):
        A = ti.matrix_np(m, k, seeds[0], dist, np.float32)
        B = ti.matrix_np(k, n, seeds[1], dist, np.float32)
        C0 = ti.matrix_np(m, n, seeds[2], dist, np.float32)
        pb = tsmm.pack_b(to_device(B), precision=X3)
        pl = tsmm.plan(m, n, k, torch.float32, precision=X3)
        assert pl.info()["regime"] == 2
        outs = []
        for lda, off in (((m + 3) // 4 * 4, 0), (m + pad, offset)):
            dC = to_device(C0, m + ldc_pad)
            tsmm.execute(pl, 1.25, to_device(A, lda, off), pb, beta, dC)
            pl.check()
            outs.append(dC.cpu().numpy())
        assert np.array_equal(outs[1], outs[0])
        Cref, _ = oracle.tsmm(1.25, A, B, beta, C0 if beta else None)
        if dist == "integer":
            np.testing.assert_array_equal(outs[1], oracle.round_to(Cref, np.float32))
        else:
            E3 = x3_bound(A, B, C0 if beta else None, 1.25, beta)
            assert np.all(np.abs(outs[1].astype(np.float64) - Cref) <= E3)


@pytest.mark.parametrize("beta", [1.5, 0.0])
@pytest.mark.parametrize("ldc_pad,c_offset", [(0, 0), (4, 0), (1, 0), (0, 1), (12, 3)])
def test_bf16x3_rankk_c_layouts(ldc_pad, c_offset, beta):
    """C0 loads and C stores go through TMA when C's base and column stride
    are 16-byte aligned, else through 4-byte cp.async and plain stores; both
    give the exact result, and padding rows of C stay untouched."""
    m, n, k = 1028, 700, 96
    A = ti.matrix_np(m, k, 64, "integer", np.float32)
    B = ti.matrix_np(k, n, 65, "integer", np.float32)
    C0 = ti.matrix_np(m, n, 66, "integer", np.float32)
    dA = to_device(A, m)
    pb = tsmm.pack_b(to_device(B), precision=X3)
    pl = tsmm.plan(m, n, k, torch.float32, precision=X3)
    ldc = m + ldc_pad
    dC = to_device(C0, ldc, c_offset)
    tsmm.execute(pl, -2.0, dA, pb, beta, dC)
    pl.check()
    Cref, _ = oracle.tsmm(-2.0, A, B, beta, C0 if beta else None)
    np.testing.assert_array_equal(dC.cpu().numpy(), oracle.round_to(Cref, np.float32))
    if ldc_pad:
        full = torch.as_strided(dC, (ldc, n), (1, ldc)).cpu().numpy()
        assert np.all(np.isnan(full[m:, :]))


@pytest.mark.parametrize("m,n,k", [(2000, 1500, 128), (1000, 700, 64)])
def test_bf16x3_rankk_uniform_within_mode_bound(m, n, k):
    A = ti.matrix_np(m, k, 71, "uniform", np.float32)
    B = ti.matrix_np(k, n, 72, "uniform", np.float32)
    C0 = ti.matrix_np(m, n, 73, "uniform", np.float32)
    C, _ = run_x3(A, B, C0, 1.0, 1.0)
    Cref, _ = oracle.tsmm(1.0, A, B, 1.0, C0)
    E3 = x3_bound(A, B, C0, 1.0, 1.0)
    err = np.abs(C.astype(np.float64) - Cref)
    assert np.all(err <= E3), f"max err/bound {np.max(err / E3):.3g}"


def test_bf16x3_rankk_full_size_sampled():
    """m = n = 16384, k = 128 (the precision workload's rank-k shape)."""
    m = n = 16384
    k = 128
    dA = torch.empty((k, m), dtype=torch.float32, device="cuda")
    ti.fill_torch(dA, ti.SEED_A, "uniform")
    dA = dA.t()
    dB = torch.empty((n, k), dtype=torch.float32, device="cuda")
    ti.fill_torch(dB, ti.SEED_B, "uniform")
    dB = dB.t()
    dC = torch.empty((n, m), dtype=torch.float32, device="cuda")
    ti.fill_torch(dC, ti.SEED_C0, "uniform")
    dC = dC.t()
    pl = tsmm.plan(m, n, k, torch.float32, precision=X3)
    tsmm.execute(pl, 1.0, dA, tsmm.pack_b(dB, precision=X3), 1.0, dC)
    pl.check()
    rows = np.sort(np.random.default_rng(9).choice(m, 16, replace=False))
    A_r = np.asfortranarray(ti.rows_np(rows, m, k, ti.SEED_A, "uniform", np.float32))
    B = ti.matrix_np(k, n, ti.SEED_B, "uniform", np.float32)
    C0_r = np.asfortranarray(ti.rows_np(rows, m, n, ti.SEED_C0, "uniform", np.float32))
    Cref, _ = oracle.tsmm(1.0, A_r, B, 1.0, C0_r)
    C = dC[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    E3 = x3_bound(A_r, B, C0_r, 1.0, 1.0)
    err = np.abs(C.astype(np.float64) - Cref)
    assert np.all(err <= E3), f"max err/bound {np.max(err / E3):.3g}"
