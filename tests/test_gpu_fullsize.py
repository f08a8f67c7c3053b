"""Parity at the full workload sizes, in the launch configuration the bench
times (the same planner output for the same shape): inputs are generated on
the device by the shared seeded generator, and sampled rows of C are checked
against the oracle fed with the same rows regenerated on the host.

Workloads: m = k = 32768 with n in {1,2,4,8,16,32,64}, FP32 and FP64, beta in
{0, 1} (the memory-bound sweep), and m = n = 16384 with k in {4..128}, beta = 1
(the rank-k shape whose cost is the output)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2208_08088_gb300 as tsmm
import tsmm_inputs as ti

pytestmark = pytest.mark.gpu

N_SAMPLE = 48


def device_matrix(rows, cols, seed, dist, dtype):
    t = torch.empty((cols, rows), dtype=dtype, device="cuda")  # storage = column-major rows x cols
    ti.fill_torch(t, seed, dist)
    return t.t()


def sample_rows(m, seed=0):
    rng = np.random.default_rng(seed)
    rows = rng.choice(m, size=N_SAMPLE, replace=False)
    rows[:2] = [0, m - 1]
    return np.sort(rows)


def check_rows(C_dev, rows, m, n, k, alpha, beta, dist, npdt, exact=False):
    A_r = np.asfortranarray(ti.rows_np(rows, m, k, ti.SEED_A, dist, npdt))
    B = ti.matrix_np(k, n, ti.SEED_B, dist, npdt)
    C0_r = np.asfortranarray(ti.rows_np(rows, m, n, ti.SEED_C0, dist, npdt)) if beta != 0 else None
    Cref, E = oracle.tsmm(alpha, A_r, B, beta, C0_r, m=len(rows), n=n, k=k, dtype=npdt)
    C = C_dev[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    ok, ratio, nbad = oracle.check(C, Cref, E, npdt)
    assert ok, f"{nbad} sampled entries outside the bound (max ratio {ratio:.3g})"
    if exact:
        np.testing.assert_array_equal(C, oracle.round_to(Cref, npdt))
    return ratio


@pytest.fixture(scope="module", params=[torch.float32, torch.float64], ids=["f32", "f64"])
def tall_A(request):
    dtype = request.param
    A = device_matrix(32768, 32768, ti.SEED_A, "uniform", dtype)
    yield dtype, A
    del A
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64])
def test_tall_sweep_32768(tall_A, n):
    dtype, A = tall_A
    npdt = np.float32 if dtype == torch.float32 else np.float64
    m = k = 32768
    B = device_matrix(k, n, ti.SEED_B, "uniform", dtype)
    pb = tsmm.pack_b(B)
    pl = tsmm.plan(m, n, k, dtype)
    rows = sample_rows(m, n)
    for beta in (0.0, 1.0):
        C = device_matrix(m, n, ti.SEED_C0, "uniform", dtype)
        tsmm.execute(pl, 1.0, A, pb, beta, C)
        pl.check()
        check_rows(C, rows, m, n, k, 1.0, beta, "uniform", npdt)


def test_tall_32768_integer_bit_exact():
    """|sum| <= 16 * 32768 = 2^19: exactly representable, so bit-exact."""
    m = k = 32768
    n = 16
    A = device_matrix(m, k, ti.SEED_A, "integer", torch.float32)
    B = device_matrix(k, n, ti.SEED_B, "integer", torch.float32)
    C = device_matrix(m, n, ti.SEED_C0, "integer", torch.float32)
    pl = tsmm.plan(m, n, k, torch.float32)
    tsmm.execute(pl, 1.5, A, tsmm.pack_b(B), 0.5, C)
    pl.check()
    check_rows(C, sample_rows(m, 99), m, n, k, 1.5, 0.5, "integer", np.float32, exact=True)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("k", [4, 8, 16, 32, 64, 128])
def test_rankk_16384(dtype, k):
    npdt = np.float32 if dtype == torch.float32 else np.float64
    m = n = 16384
    A = device_matrix(m, k, ti.SEED_A, "uniform", dtype)
    B = device_matrix(k, n, ti.SEED_B, "uniform", dtype)
    C = device_matrix(m, n, ti.SEED_C0, "uniform", dtype)
    pl = tsmm.plan(m, n, k, dtype)
    assert pl.info()["regime"] == 2
    tsmm.execute(pl, 1.0, A, tsmm.pack_b(B), 1.0, C)
    pl.check()
    check_rows(C, sample_rows(m, k), m, n, k, 1.0, 1.0, "uniform", npdt)
