"""The shared seeded input generator: determinism, ranges, exact
representability, and agreement of its numpy and torch implementations."""
import numpy as np
import pytest
import torch

import tsmm_inputs as ti


def test_mul32_matches_bigint():
    rng = np.random.default_rng(0)
    xs = rng.integers(0, 2 ** 32, size=2000, dtype=np.int64)
    for c in (0x7FEB352D, 0x846CA68B, 0xFFFFFFFF, 1, 0):
        got = ti._mul32(xs, c)
        want = np.array([(int(x) * c) % 2 ** 32 for x in xs], dtype=np.int64)
        np.testing.assert_array_equal(got, want)


def test_hash32_reference_steps():
    """The mixer written out with Python big integers, step by step."""
    def h(x):
        x ^= x >> 16
        x = (x * 0x7FEB352D) % 2 ** 32
        x ^= x >> 15
        x = (x * 0x846CA68B) % 2 ** 32
        x ^= x >> 16
        return x
    for x in [0, 1, 2, 12345, 2 ** 31, 2 ** 32 - 1, 0xDEADBEEF]:
        assert ti._hash32_int(x) == h(x)
    assert h(0) == 0


@pytest.mark.parametrize("dist,lo,hi", [("uniform", -1.0, 1.0), ("integer", -4, 4), ("ternary", -1, 1)])
def test_ranges_and_exactness(dist, lo, hi):
    v = ti.values_np(np.arange(200000), 7, dist)
    assert v.min() >= lo and v.max() <= hi
    np.testing.assert_array_equal(v.astype(np.float32).astype(np.float64), v)
    if dist == "uniform":
        assert v.max() < 1.0
        assert abs(v.mean()) < 0.01 and abs(v.var() - 1 / 3) < 0.01
        np.testing.assert_array_equal(np.round(v * 2 ** 23), v * 2 ** 23)
    else:
        np.testing.assert_array_equal(np.round(v), v)
        assert set(np.unique(v).tolist()) == set(range(int(lo), int(hi) + 1))


def test_seeds_and_streams_differ_and_repeat():
    a = ti.values_np(np.arange(1000), 1)
    assert np.array_equal(a, ti.values_np(np.arange(1000), 1))
    assert not np.array_equal(a, ti.values_np(np.arange(1000), 2))
    assert not np.array_equal(a, ti.values_np(np.arange(1000), 1, stream=1))


def test_large_indices_use_high_bits():
    i = np.array([5, 5 + 2 ** 32], dtype=np.int64)
    v = ti.values_np(i, 3)
    assert v[0] != v[1]


def test_matrix_layout_and_rows():
    M = ti.matrix_np(7, 5, 9, "uniform", np.float32)
    assert M.flags.f_contiguous and M.shape == (7, 5)
    flat = ti.values_np(np.arange(35), 9).astype(np.float32)
    np.testing.assert_array_equal(M.ravel(order="F"), flat)
    R = ti.rows_np([0, 3, 6], 7, 5, 9, "uniform", np.float32)
    np.testing.assert_array_equal(R, M[[0, 3, 6], :])


@pytest.mark.parametrize("dist", ["uniform", "integer"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_torch_fill_matches_numpy(dist, dtype):
    t = torch.empty(5, 13, dtype=dtype)  # viewed as flat column-major storage
    ti.fill_torch(t, 4, dist, chunk=17)
    want = ti.values_np(np.arange(65), 4, dist)
    np.testing.assert_array_equal(t.view(-1).double().numpy(), want)


def test_normal_scaled_shape_and_scale():
    Z = ti.normal_scaled_np(400, 300, 5)
    assert Z.shape == (400, 300) and np.all(np.isfinite(Z))
    rs = np.abs(Z).max(axis=1)
    assert rs.max() / rs.min() > 1e3  # rows span several decades


def test_normal_scaled_torch_matches_numpy():
    t = torch.empty(6, 9, dtype=torch.float64)  # 9 x 6 column-major matrix
    ti.normal_scaled_torch(t, 3, chunk=7)
    Z = ti.normal_scaled_np(9, 6, 3, np.float64)
    np.testing.assert_allclose(t.t().numpy(), Z, rtol=1e-13, atol=0)
