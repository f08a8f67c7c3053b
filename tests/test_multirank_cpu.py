"""The bench's multi-GPU paths on CPU, as world_size-2 gloo ranks: independent
replicas report all ranks' flops over the slowest rank's time, and the row
split partitions one problem's m rows into slabs (B replicated, no exchange on
the data path) whose gathered results equal a single-rank run."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    # rank r "took" 100*(r+1) ms for 10 steps of 1e9 flops each
    ms, value = bench.aggregate_over_ranks(100.0 * (rank + 1), 1e9, 10, world)
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 200.0                      # max over ranks
        assert value == pytest.approx(2 * 1e9 * 10 / 0.2 / 1e9)  # both ranks' work / slowest time


def _load_bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return bench


def test_row_slabs_partition_m():
    """bench.row_slab: contiguous, disjoint slabs covering [0, m), boundaries on
    the plan's row granule, the last rank taking the rest (empty slabs allowed)."""
    bench = _load_bench()
    for m, world, g in [(32768, 2, 128), (32768, 8, 256), (1000, 2, 64), (1000, 3, 64), (100, 4, 64),
                        (1, 2, 64), (0, 2, 64), (16384, 5, 128)]:
        slabs = [bench.row_slab(m, r, world, g) for r in range(world)]
        assert slabs[0][0] == 0 and slabs[-1][1] == m
        for (lo, hi), (lo2, _) in zip(slabs, slabs[1:]):
            assert hi == lo2 and lo <= hi
        assert all(lo % g == 0 for lo, _ in slabs)


def _split_rank(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench = _load_bench()
    import oracle
    import tsmm_inputs as ti

    m, n, k, granule = 1000, 13, 300, 64
    lo, hi = bench.row_slab(m, rank, world, granule)
    rows = np.arange(lo, hi)
    A_r = np.asfortranarray(ti.rows_np(rows, m, k, ti.SEED_A, "integer", np.float32))
    B = ti.matrix_np(k, n, ti.SEED_B, "integer", np.float32)
    C0_r = np.asfortranarray(ti.rows_np(rows, m, n, ti.SEED_C0, "integer", np.float32))
    C_r, _ = oracle.tsmm(1.5, A_r, B, 0.5, C0_r, m=hi - lo, n=n, k=k, dtype=np.float32)
    got = [None] * world
    dist.all_gather_object(got, (lo, hi, oracle.round_to(C_r, np.float32)))
    ok = True
    if rank == 0:
        C = np.full((m, n), np.nan, dtype=np.float32)
        for (a, b, part) in got:
            C[a:b] = part
        A = ti.matrix_np(m, k, ti.SEED_A, "integer", np.float32)
        C0 = ti.matrix_np(m, n, ti.SEED_C0, "integer", np.float32)
        ref, _ = oracle.tsmm(1.5, A, B, 0.5, C0)
        ok = bool(np.array_equal(C, oracle.round_to(ref, np.float32)))
    q.put((rank, lo, hi, ok))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_row_split_matches_single_rank():
    """The bench's --split rows path on CPU: two gloo ranks take the row slabs of
    one problem (B replicated), each computes its rows with the oracle, and the
    gathered C equals a single-rank oracle run of the whole problem bit for bit
    (integer inputs: every partial sum exact)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + os.getpid() % 1000
    procs = [ctx.Process(target=_split_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(lo, hi) for (_, lo, hi, _) in out] == [(0, 448), (448, 1000)]
    assert all(ok for (*_, ok) in out)
