"""Pins for the CPU oracle (Eq. 1, C = alpha*A*B + beta*C0), all on the CPU.

Each test fixes the oracle against something other than itself: exhaustive
brute force in exact rational arithmetic, exact integer products, closed forms
(identity / permutation / rank-1 / all-ones operands, the alpha = 0, beta = 0
and k = 0 special cases), the transpose identity (A B)^T = B^T A^T, invariance
under leading-dimension padding, IEEE special-value propagation, and the
accuracy of the FP64 compensated dot product on ill-conditioned sums checked
against exact rationals.  A dropped term, a wrong sign, a swapped index or a
transposed operand in the oracle fails at least one of them.
"""
import itertools
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import oracle
import tsmm_inputs as ti

DTYPES = [np.float32, np.float64]
U = {np.float32: 2.0 ** -24, np.float64: 2.0 ** -53}
SCALARS = [0.0, 1.0, -1.0, 1.5, 0.5]


def F(x):
    return np.asfortranarray(x)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("m,n,k", list(itertools.product([1, 2], repeat=3)))
def test_exhaustive_ternary(dtype, m, n, k):
    """Every A in {-1,0,1}^(m x k) against every B in {-1,0,1}^(k x n), all
    alpha, beta in {0, +-1, 1.5, 0.5}; expected values from exact rational
    arithmetic written out element by element."""
    a_all = [np.array(v, dtype=dtype).reshape(k, m).T for v in
             itertools.product([-1, 0, 1], repeat=m * k)]
    A = F(np.vstack(a_all))  # all A's stacked: shared B, independent rows
    M = A.shape[0]
    C0 = F(np.array([[((i * 7 + j * 5) % 3) - 1 for j in range(n)] for i in range(M)],
                    dtype=dtype))
    for bv in itertools.product([-1, 0, 1], repeat=k * n):
        B = F(np.array(bv, dtype=dtype).reshape(n, k).T)
        for alpha, beta in itertools.product(SCALARS, SCALARS):
            Cref, E = oracle.tsmm(alpha, A, B, beta, C0)
            for i in range(M):
                for j in range(n):
                    s = sum(Fraction(int(A[i, p])) * Fraction(int(B[p, j])) for p in range(k))
                    want = Fraction(alpha) * s + Fraction(beta) * Fraction(int(C0[i, j]))
                    assert Fraction(Cref[i, j]) == want
                    g = sum(abs(int(A[i, p])) * abs(int(B[p, j])) for p in range(k))
                    e_want = 4 * k * U[dtype] * (abs(alpha) * g + abs(beta) * abs(int(C0[i, j])))
                    assert E[i, j] == e_want


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("m,n,k", [(17, 9, 33), (1, 1, 1), (16, 4, 7), (5, 13, 2), (33, 1, 65)])
def test_random_integer_exact(dtype, m, n, k):
    """Integer entries in [-4, 4]: every partial sum is exactly representable,
    so the oracle must equal exact int64 arithmetic (alpha=1.5, beta=0.5 are
    dyadic, so 2*C is an integer)."""
    A = ti.matrix_np(m, k, 11, "integer", dtype)
    B = ti.matrix_np(k, n, 12, "integer", dtype)
    C0 = ti.matrix_np(m, n, 13, "integer", dtype)
    Cref, _ = oracle.tsmm(1.5, A, B, 0.5, C0)
    Ai, Bi, Ci = A.astype(np.int64), B.astype(np.int64), C0.astype(np.int64)
    twice = 3 * (Ai @ Bi) + Ci
    np.testing.assert_array_equal(Cref * 2, twice.astype(np.float64))


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("dtype", DTYPES)
def test_identity_B(dtype):
    m, k = 37, 19
    A = ti.matrix_np(m, k, 21, "uniform", dtype)
    C0 = ti.matrix_np(m, k, 22, "uniform", dtype)
    B = F(np.eye(k, dtype=dtype))
    Cref, E = oracle.tsmm(1.0, A, B, 1.0, C0)
    # alpha = 1, one nonzero product per entry: C = A + C0 up to one rounding in double
    np.testing.assert_array_equal(Cref, A.astype(np.float64) + C0.astype(np.float64))


@pytest.mark.parametrize("dtype", DTYPES)
def test_permutation_B(dtype):
    m, k, n = 23, 11, 6
    rng = np.random.default_rng(5)
    perm = rng.permutation(k)[:n]
    A = ti.matrix_np(m, k, 31, "uniform", dtype)
    B = np.zeros((k, n), dtype=dtype)
    for j in range(n):
        B[perm[j], j] = 1
    B = F(B)
    Cref, _ = oracle.tsmm(-1.0, A, B, 0.0, None)
    np.testing.assert_array_equal(Cref, -A[:, perm].astype(np.float64))


@pytest.mark.parametrize("dtype", DTYPES)
def test_rank1_A(dtype):
    """A = u v^T with integer u, v: C = alpha * u (v^T B) + beta*C0 exactly."""
    m, k, n = 29, 41, 7
    u = ti.values_np(np.arange(m), 41, "integer")
    v = ti.values_np(np.arange(k), 42, "integer")
    A = F(np.outer(u, v).astype(dtype))
    B = ti.matrix_np(k, n, 43, "integer", dtype)
    C0 = ti.matrix_np(m, n, 44, "integer", dtype)
    Cref, _ = oracle.tsmm(0.5, A, B, -1.0, C0)
    vB = [sum(int(v[p]) * int(B[p, j]) for p in range(k)) for j in range(n)]
    want = np.array([[0.5 * int(u[i]) * vB[j] - float(C0[i, j]) for j in range(n)]
                     for i in range(m)])
    np.testing.assert_array_equal(Cref, want)


@pytest.mark.parametrize("dtype", DTYPES)
def test_all_ones_and_bound(dtype):
    """All-ones A and B: C = alpha*k + beta*C0, E = 4ku(|alpha| k + |beta||C0|)."""
    m, k, n = 13, 50, 3
    A = F(np.ones((m, k), dtype=dtype))
    B = F(np.ones((k, n), dtype=dtype))
    C0 = F(np.full((m, n), 2.0, dtype=dtype))
    Cref, E = oracle.tsmm(1.5, A, B, -0.5, C0)
    assert np.all(Cref == 1.5 * k - 1.0)
    assert np.all(E == 4 * k * U[dtype] * (1.5 * k + 0.5 * 2.0))


@pytest.mark.parametrize("dtype", DTYPES)
def test_alpha_zero_does_not_read_A_B(dtype):
    m, k, n = 9, 5, 4
    A = F(np.full((m, k), np.nan, dtype=dtype))
    B = F(np.full((k, n), np.inf, dtype=dtype))
    C0 = ti.matrix_np(m, n, 51, "uniform", dtype)
    Cref, E = oracle.tsmm(0.0, A, B, 1.5, C0)
    np.testing.assert_array_equal(Cref, 1.5 * C0.astype(np.float64))
    Cref2, _ = oracle.tsmm(0.0, None, None, 1.5, C0, m=m, n=n, k=k, lda=m, ldb=k)
    np.testing.assert_array_equal(Cref2, Cref)


@pytest.mark.parametrize("dtype", DTYPES)
def test_beta_zero_does_not_read_C0(dtype):
    m, k, n = 9, 5, 4
    A = ti.matrix_np(m, k, 61, "integer", dtype)
    B = ti.matrix_np(k, n, 62, "integer", dtype)
    C0 = F(np.full((m, n), np.nan, dtype=dtype))
    Cref, _ = oracle.tsmm(2.0, A, B, 0.0, C0)
    want = 2.0 * (A.astype(np.int64) @ B.astype(np.int64))
    np.testing.assert_array_equal(Cref, want.astype(np.float64))
    Cref2, E2 = oracle.tsmm(2.0, A, B, 0.0, None)
    np.testing.assert_array_equal(Cref2, Cref)


@pytest.mark.parametrize("dtype", DTYPES)
def test_k_zero(dtype):
    m, n = 6, 5
    C0 = ti.matrix_np(m, n, 71, "uniform", dtype)
    Cref, E = oracle.tsmm(3.0, None, None, 0.5, C0, m=m, n=n, k=0)
    np.testing.assert_array_equal(Cref, 0.5 * C0.astype(np.float64))
    assert np.all(E == 0)


def test_empty_and_bad_args():
    Cref, E = oracle.tsmm(1.0, None, None, 0.0, None, m=0, n=5, k=3, dtype=np.float32)
    assert Cref.shape == (0, 5)
    with pytest.raises(ValueError):
        oracle.tsmm(1.0, None, None, 0.0, None, m=-1, n=5, k=3, dtype=np.float32)
    A = ti.matrix_np(4, 3, 1, "uniform", np.float32)
    B = ti.matrix_np(3, 2, 2, "uniform", np.float32)
    with pytest.raises(ValueError):  # lda < m
        oracle.tsmm(1.0, A.ravel(order="F"), B, 0.0, None, m=4, n=2, k=3, lda=3, ldb=3)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("dtype", DTYPES)
def test_transpose_identity(dtype):
    """(alpha A B + beta C0)^T == alpha B^T A^T + beta C0^T bit for bit: every
    entry is the same products summed in the same order p = 0..k-1."""
    m, k, n = 31, 27, 12
    A = ti.matrix_np(m, k, 81, "uniform", dtype)
    B = ti.matrix_np(k, n, 82, "uniform", dtype)
    C0 = ti.matrix_np(m, n, 83, "uniform", dtype)
    Cref, E = oracle.tsmm(1.5, A, B, 0.5, C0)
    CrefT, ET = oracle.tsmm(1.5, F(B.T), F(A.T), 0.5, F(C0.T))
    np.testing.assert_array_equal(Cref, CrefT.T)
    np.testing.assert_array_equal(E, ET.T)


@pytest.mark.parametrize("dtype", DTYPES)
def test_leading_dimension_padding(dtype):
    """Padding rows (filled with NaN) beyond m / k must never be read."""
    m, k, n = 21, 14, 5
    A = ti.matrix_np(m, k, 91, "uniform", dtype)
    B = ti.matrix_np(k, n, 92, "uniform", dtype)
    C0 = ti.matrix_np(m, n, 93, "uniform", dtype)
    Cref, E = oracle.tsmm(-1.5, A, B, 0.5, C0)

    def pad(X, extra):
        P = np.full((X.shape[0] + extra, X.shape[1]), np.nan, dtype=dtype, order="F")
        P[: X.shape[0], :] = X
        return P[: X.shape[0], :]

    Cp, Ep = oracle.tsmm(-1.5, pad(A, 3), pad(B, 7), 0.5, pad(C0, 1))
    np.testing.assert_array_equal(Cp, Cref)
    np.testing.assert_array_equal(Ep, E)


@pytest.mark.parametrize("dtype", DTYPES)
def test_linearity_and_k_split(dtype):
    """Exact on integers: A(B1 + B2) = A B1 + A B2 and splitting the k range."""
    m, k, n = 19, 23, 6
    A = ti.matrix_np(m, k, 101, "integer", dtype)
    B1 = ti.matrix_np(k, n, 102, "integer", dtype)
    B2 = ti.matrix_np(k, n, 103, "integer", dtype)
    C12, _ = oracle.tsmm(1.0, A, F(B1 + B2), 0.0, None)
    C1, _ = oracle.tsmm(1.0, A, B1, 0.0, None)
    C2, _ = oracle.tsmm(1.0, A, B2, 0.0, None)
    np.testing.assert_array_equal(C12, C1 + C2)
    k1 = 9
    Ca, _ = oracle.tsmm(1.0, F(A[:, :k1]), F(B1[:k1]), 0.0, None)
    Cb, _ = oracle.tsmm(1.0, F(A[:, k1:]), F(B1[k1:]), 0.0, None)
    np.testing.assert_array_equal(C1, Ca + Cb)


@pytest.mark.parametrize("dtype", DTYPES)
def test_ieee_special_values(dtype):
    """Inf * nonzero -> +-Inf, Inf * 0 -> NaN, NaN propagates (IEEE 754)."""
    A = F(np.array([[np.inf, 1.0], [1.0, 1.0], [np.nan, 0.0]], dtype=dtype))
    B = F(np.array([[1.0, 0.0, -2.0], [1.0, 1.0, 1.0]], dtype=dtype))
    Cref, _ = oracle.tsmm(1.0, A, B, 0.0, None)
    assert Cref[0, 0] == np.inf and np.isnan(Cref[0, 1]) and Cref[0, 2] == -np.inf
    np.testing.assert_array_equal(Cref[1], [2.0, 1.0, -1.0])
    assert np.all(np.isnan(Cref[2]))


def test_subnormals_are_ordinary_values():
    """FP32 subnormals (below 2^-126) are kept, not flushed: with a zero
    product C = C0 exactly; a product of 2^-126 plus a C0 of -0.75 * 2^-126
    gives the subnormal 2^-128; products 2^-138 + 2^-149 sum to a subnormal
    exactly (values fixed by hand)."""
    t = np.float32
    A = F(np.array([[0.0, 0.0], [2.0 ** -63, 0.0], [2.0 ** -75, 2.0 ** -75]], dtype=t))
    B = F(np.array([[2.0 ** -63, 1.0], [2.0 ** -74, 1.0]], dtype=t))
    C0 = F(np.array([[3 * 2.0 ** -149, -(2.0 ** -140)], [-0.75 * 2.0 ** -126, 0.0], [0.0, 0.0]], dtype=t))
    Cref, _ = oracle.tsmm(1.0, A, B, 1.0, C0)
    C = oracle.round_to(Cref, t)
    assert C[0, 0] == 3 * 2.0 ** -149 and C[0, 1] == -(2.0 ** -140)  # A = 0: C0 kept
    assert C[1, 0] == 2.0 ** -128                                     # 2^-126 - 0.75 * 2^-126
    assert C[2, 0] == 2.0 ** -138 + 2.0 ** -149                       # 2049 * 2^-149


# ---------------------------------------------------------------- accuracy
def _exact(A, B, alpha, beta, C0):
    m, k = A.shape
    n = B.shape[1]
    out = np.empty((m, n), dtype=object)
    for i in range(m):
        for j in range(n):
            s = sum(Fraction(float(A[i, p])) * Fraction(float(B[p, j])) for p in range(k))
            c = Fraction(float(C0[i, j])) if C0 is not None else Fraction(0)
            out[i, j] = Fraction(alpha) * s + Fraction(beta) * c
    return out


def test_f32_accuracy_vs_exact():
    """FP32 operands: the double-accumulated oracle is within k*2^-52*sum|ab|
    (plus two final roundings) of the exact rational result."""
    m, k, n = 7, 60, 3
    A = ti.matrix_np(m, k, 111, "uniform", np.float32)
    B = ti.matrix_np(k, n, 112, "uniform", np.float32)
    C0 = ti.matrix_np(m, n, 113, "uniform", np.float32)
    Cref, E = oracle.tsmm(1.5, A, B, 0.5, C0)
    X = _exact(A, B, 1.5, 0.5, C0)
    for i in range(m):
        for j in range(n):
            g = sum(abs(float(A[i, p]) * float(B[p, j])) for p in range(k))
            tol = (k + 3) * 2.0 ** -52 * (1.5 * g + 0.5 * abs(float(C0[i, j])))
            assert abs(Fraction(Cref[i, j]) - X[i, j]) <= Fraction(tol)
            # and the oracle's own error is a tiny fraction of the bound E
            assert float(abs(Fraction(Cref[i, j]) - X[i, j])) <= 1e-6 * E[i, j]


def _ill_conditioned_pairs(k, seed, rng_exp=60):
    """Dot products with heavy cancellation: random terms of widely spread
    magnitude followed by terms that cancel their running sum."""
    rng = np.random.default_rng(seed)
    half = k // 2
    x = np.empty(k)
    y = np.empty(k)
    e = rng.integers(0, rng_exp, size=half)
    x[:half] = rng.uniform(-1, 1, size=half) * 2.0 ** e
    y[:half] = rng.uniform(-1, 1, size=half) * 2.0 ** rng.integers(0, rng_exp, size=half)
    acc = Fraction(0)
    for p in range(half):
        acc += Fraction(x[p]) * Fraction(y[p])
    for p in range(half, k):
        # pick x[p]*y[p] ~= -acc (rounded), so the exact sum keeps cancelling
        target = -float(acc) * rng.uniform(0.5, 1.0) if p < k - 1 else -float(acc)
        y[p] = rng.uniform(1, 2)
        x[p] = target / y[p]
        acc += Fraction(x[p]) * Fraction(y[p])
    return x, y


@pytest.mark.parametrize("k", [2, 5, 16, 40])
def test_f64_dot2_ill_conditioned(k):
    """FP64: the compensated (Dot2) oracle meets the Ogita-Rump-Oishi bound
    |res - x.y| <= u|x.y| + gamma_k^2 sum|x_i y_i| on sums with cancellation
    where plain FP64 summation loses every significant digit."""
    m = 6
    # row i of A and the single column of B_i form one ill-conditioned pair
    xs, ys = [], []
    for i in range(m):
        x, y = _ill_conditioned_pairs(k, 1000 + i)
        xs.append(x)
        ys.append(y)
    A = F(np.array(xs))
    u = 2.0 ** -53
    gam = k * u / (1 - k * u)
    for j in range(m):
        B = F(np.array(ys[j]).reshape(k, 1))
        Cref, _ = oracle.tsmm(1.0, A, B, 0.0, None)
        x, y = xs[j], ys[j]
        exact = sum(Fraction(x[p]) * Fraction(y[p]) for p in range(k))
        absdot = sum(abs(Fraction(x[p]) * Fraction(y[p])) for p in range(k))
        err = abs(Fraction(Cref[j, 0]) - exact)
        assert err <= Fraction(u) * abs(exact) + Fraction(gam * gam) * absdot


def test_f64_final_combination_is_compensated():
    """alpha*S + beta*C0 with catastrophic cancellation between the two terms."""
    A = F(np.array([[2.0 ** 53, 1.0]]))
    B = F(np.array([[1.0], [1.0]]))
    C0 = F(np.array([[2.0 ** 53]]))
    Cref, _ = oracle.tsmm(1.0, A, B, -1.0, C0)
    assert Cref[0, 0] == 1.0
    # plain double evaluation would give 0 here
    assert (2.0 ** 53 + 1.0) - 2.0 ** 53 == 0.0


def test_thread_count_independent():
    """Row blocking makes every sum's order fixed: 1 thread == all threads."""
    code = (
        "import numpy as np, oracle, tsmm_inputs as ti;"
        "A=ti.matrix_np(1500,70,1,'uniform',np.float32);"
        "B=ti.matrix_np(70,5,2,'uniform',np.float32);"
        "C,E=oracle.tsmm(1.5,A,B,0.0,None);"
        "import sys; sys.stdout.buffer.write(C.tobytes())"
    )
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for nt in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=nt, PYTHONPATH=root)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, cwd=root,
                                   capture_output=True, check=True).stdout)
    assert outs[0] == outs[1] and len(outs[0]) == 1500 * 5 * 8


# ---------------------------------------------------------------- acceptance check
def test_check_semantics():
    Cref = np.array([[1.0, 2.0, np.nan, np.inf, 0.1]])
    E = np.array([[0.5, 0.0, 0.0, 0.0, 0.0]])
    C = np.array([[1.4, 2.0, np.nan, np.inf, np.float32(0.1)]])
    ok, ratio, nbad = oracle.check(C, Cref, E, np.float32)
    assert ok and abs(ratio - 0.8) < 1e-12
    ok, _, nbad = oracle.check(np.array([[1.6, 2.0, np.nan, np.inf, 0.1]]), Cref, E, np.float32)
    assert not ok and nbad == 2  # 1.6 out of bound; 0.1 (double) != fl32(0.1)


def test_golden_fixture_reproduces():
    """The committed fixture equals what its generator script computes now
    (exact integers: any change in the oracle's arithmetic would show)."""
    import json
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = os.path.join(root, "tests", "golden", "make_golden.py")
    spec = importlib.util.spec_from_file_location("make_golden", path)
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    stored = json.load(open(os.path.join(root, "tests", "golden", "tsmm_2048x2048x16_integer_rows.json")))
    assert mg.integer_2048x2048x16() == stored
    # and the stored values are integers / 2 (alpha = 1.5, beta = 0.5 on integers)
    assert all(float(2 * x).is_integer() for row in stored["C_rows"] for x in row)
