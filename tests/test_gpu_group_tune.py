"""Grouped execution, autotuning + plan cache, and CUDA-graph capture, all
checked against the single-problem path (bitwise: same plan, same arithmetic)
and against the oracle bound."""
import numpy as np
import pytest
import torch

import oracle
import paper_2208_08088_gb300 as tsmm
import tsmm_inputs as ti
from gpu_util import assert_parity, to_device

pytestmark = pytest.mark.gpu

T = {np.float32: torch.float32, np.float64: torch.float64}


def problem(m, n, k, dtype, seed, dist="uniform", a_offset=0):
    A = ti.matrix_np(m, k, seed, dist, dtype)
    B = ti.matrix_np(k, n, seed + 1, dist, dtype)
    C0 = ti.matrix_np(m, n, seed + 2, dist, dtype)
    return A, B, C0, to_device(A, offset=a_offset), to_device(B)


MIX = [  # (m, n, k, alpha, beta, a_offset)
    (1000, 16, 777, 1.5, 0.5, 0), (4096, 1, 3000, 1.0, 0.0, 0), (300, 64, 5000, -1.0, 1.0, 0),
    (129, 3, 64, 2.0, -0.5, 0), (2048, 16, 2048, 1.5, 0.5, 0), (700, 17, 9000, 1.0, 1.0, 0),
    (512, 200, 40, 1.0, 1.0, 0),      # regime (ii): own launch
    (333, 8, 100, 0.0, 1.5, 0),       # alpha = 0: scale launch
    (301, 5, 250, 1.0, 1.0, 1),       # unaligned A: plain-load launch
    (64, 64, 64, 1.0, 0.0, 0),
    (900, 40, 1500, 1.0, 1.0, 0),     # width 48
    (650, 24, 333, 1.5, 0.5, 0),      # width 24, with n = 17 above
]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_grouped_equals_single_launches(dtype):
    probs = []
    for i, (m, n, k, alpha, beta, off) in enumerate(MIX):
        A, B, C0, dA, dB = problem(m, n, k, dtype, 100 + 10 * i, a_offset=off)
        probs.append((m, n, k, alpha, beta, A, B, C0, dA, tsmm.pack_b(dB)))
    # one launch per problem
    singles = []
    for (m, n, k, alpha, beta, A, B, C0, dA, pb) in probs:
        dC = to_device(C0)
        pl = tsmm.plan(m, n, k, T[dtype])
        tsmm.execute(pl, alpha, dA, pb, beta, dC)
        pl.check()
        singles.append(dC.cpu().numpy())
    # grouped
    plans, outs, items = [], [], []
    for (m, n, k, alpha, beta, A, B, C0, dA, pb) in probs:
        pl = tsmm.plan(m, n, k, T[dtype])
        dC = to_device(C0)
        plans.append(pl)
        outs.append(dC)
        items.append((pl, alpha, dA, pb, beta, dC))
    tsmm.execute_grouped(items)
    for pl in plans:
        pl.check()
    for i, (m, n, k, alpha, beta, A, B, C0, dA, pb) in enumerate(probs):
        C = outs[i].cpu().numpy()
        assert np.array_equal(C, singles[i]), f"problem {i} differs from its single launch"
        assert_parity(C, A, B, C0 if beta != 0 else None, alpha, beta)


UNALIGNED_MIX = [  # (m, n, k, a_offset, lda_pad): A not describable by a tensor map
    (1027, 1, 333, 0, 1), (2050, 5, 3001, 1, 0), (777, 16, 20000, 3, 2), (4099, 24, 1500, 2, 1),
    (515, 33, 700, 1, 3), (1030, 48, 2222, 0, 2), (2047, 64, 5000, 3, 0), (129, 8, 40, 2, 1),
]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_grouped_unaligned_mix_equals_single_launches(dtype):
    """Problems whose A has a column stride or base that is not 16-byte aligned
    run in the grouped kernel's element/bulk-copy form: bit for bit the single
    launches (same plan, same arithmetic) and exact against the oracle on
    integer inputs, over every padded width, every offset within 16 bytes,
    split-K and ragged slabs."""
    probs = []
    for i, (m, n, k, off, pad) in enumerate(UNALIGNED_MIX):
        A = ti.matrix_np(m, k, 300 + 10 * i, "integer", dtype)
        B = ti.matrix_np(k, n, 301 + 10 * i, "integer", dtype)
        C0 = ti.matrix_np(m, n, 302 + 10 * i, "integer", dtype)
        dA = to_device(A, ld=m + pad, offset=off)
        probs.append((m, n, k, A, B, C0, dA, tsmm.pack_b(to_device(B))))
    singles = []
    for (m, n, k, A, B, C0, dA, pb) in probs:
        dC = to_device(C0)
        pl = tsmm.plan(m, n, k, T[dtype])
        tsmm.execute(pl, 1.5, dA, pb, 0.5, dC)
        pl.check()
        singles.append(dC.cpu().numpy())
    plans, outs, items = [], [], []
    for (m, n, k, A, B, C0, dA, pb) in probs:
        pl = tsmm.plan(m, n, k, T[dtype])
        dC = to_device(C0)
        plans.append(pl)
        outs.append(dC)
        items.append((pl, 1.5, dA, pb, 0.5, dC))
    tsmm.execute_grouped(items)
    for pl in plans:
        pl.check()
    for i, (m, n, k, A, B, C0, dA, pb) in enumerate(probs):
        C = outs[i].cpu().numpy()
        assert np.array_equal(C, singles[i]), f"problem {i} differs from its single launch"
        assert_parity(C, A, B, C0, 1.5, 0.5, exact=True)


def test_grouped_many_problems_span_several_launches():
    """60 problems of one class exceed the 48-per-launch limit."""
    dtype = np.float32
    items, refs = [], []
    for i in range(60):
        m, n, k = 100 + 37 * i, 8, 200 + 13 * i
        A, B, C0, dA, dB = problem(m, n, k, dtype, 1000 + i, "integer")
        pl = tsmm.plan(m, n, k, torch.float32)
        dC = to_device(C0)
        items.append((pl, 1.5, dA, tsmm.pack_b(dB), 0.5, dC))
        refs.append((A, B, C0))
    tsmm.execute_grouped(items)
    for (pl, _, _, _, _, dC), (A, B, C0) in zip(items, refs):
        pl.check()
        assert_parity(dC.cpu().numpy(), A, B, C0, 1.5, 0.5, exact=True)


def test_grouped_rejects_shared_plan():
    A, B, C0, dA, dB = problem(200, 4, 100, np.float32, 7)
    pl = tsmm.plan(200, 4, 100, torch.float32)
    pb = tsmm.pack_b(dB)
    with pytest.raises(tsmm.TsmmError) as e:
        tsmm.execute_grouped([(pl, 1.0, dA, pb, 0.0, to_device(C0)),
                              (pl, 1.0, dA, pb, 0.0, to_device(C0))])
    assert e.value.status == 1


def test_autotune_records_and_reuses_plan(tmp_path):
    m, n, k = 2048, 16, 32768
    A, B, C0, dA, dB = problem(m, n, k, np.float32, 55, "integer")
    pb = tsmm.pack_b(dB)
    tsmm.tsmm_plan_cache_clear()
    dC = to_device(np.zeros((m, n), dtype=np.float32, order="F"))
    tuned = tsmm.autotune(dA, pb, dC, reps=3)
    splits = tuned.info()["splits"]
    assert tsmm.tsmm_plan_cache_size() == 2  # the exact entry and its m bucket
    # tsmm_plan now returns the tuned choice for this shape, and for another m
    # of the same quarter octave (2048 <= m < 2435)
    assert tsmm.plan(m, n, k, torch.float32).info()["splits"] == splits
    assert tsmm.plan(2300, n, k, torch.float32).info()["splits"] == splits
    # the tuned plan is correct (integer inputs: bit-exact)
    dC = to_device(C0)
    tsmm.execute(tuned, 1.5, dA, pb, 0.5, dC)
    tuned.check()
    assert_parity(dC.cpu().numpy(), A, B, C0, 1.5, 0.5, exact=True)
    # the cache file round-trips the entry
    path = tmp_path / "plans.txt"
    tsmm.tsmm_plan_cache_save(str(path))
    tsmm.tsmm_plan_cache_clear()
    tsmm.tsmm_plan_cache_load(str(path))
    assert tsmm.plan(m, n, k, torch.float32).info()["splits"] == splits
    tsmm.tsmm_plan_cache_clear()


def test_cuda_graph_replay_matches_eager():
    """tsmm_execute launches can be captured in a CUDA graph (no allocation or
    synchronisation inside) and replayed."""
    shapes = [(2048, 16, 2048), (1000, 64, 3000), (4000, 300, 32)]
    ops = []
    for i, (m, n, k) in enumerate(shapes):
        A, B, C0, dA, dB = problem(m, n, k, np.float32, 300 + 10 * i)
        pl = tsmm.plan(m, n, k, torch.float32)
        pb = tsmm.pack_b(dB)
        dC = to_device(np.zeros((m, n), dtype=np.float32, order="F"))
        ops.append((pl, dA, pb, dC, A, B))
    # regime (ii) with an A that a tensor map cannot describe: its scratch copy is
    # allocated and freed on the stream (memory nodes of the graph)
    m, n, k = 3001, 200, 40
    A, B, C0, _, dB = problem(m, n, k, np.float32, 340)
    ops.append((tsmm.plan(m, n, k, torch.float32), to_device(A, ld=m), tsmm.pack_b(dB),
                to_device(np.zeros((m, n), dtype=np.float32, order="F")), A, B))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for (pl, dA, pb, dC, A, B) in ops:  # warm-up outside capture
            tsmm.execute(pl, 1.0, dA, pb, 0.0, dC)
    torch.cuda.synchronize()
    eager = [dC.cpu().numpy().copy() for (_, _, _, dC, _, _) in ops]
    for (_, _, _, dC, _, _) in ops:
        dC.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for (pl, dA, pb, dC, A, B) in ops:
            tsmm.execute(pl, 1.0, dA, pb, 0.0, dC, stream=s)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for (pl, dA, pb, dC, A, B), ref in zip(ops, eager):
        pl.check()
        assert np.array_equal(dC.cpu().numpy(), ref)
        assert_parity(ref, A, B, None, 1.0, 0.0)
