"""Helpers for the GPU parity tests: device placement of column-major host
matrices (with padded leading dimensions and element offsets), one call of the
library through its C ABI, and the comparison against the CPU oracle."""
import numpy as np
import torch

import oracle
import paper_2208_08088_gb300 as tsmm

NP2T = {np.float32: torch.float32, np.float64: torch.float64}


def to_device(X, ld=None, offset=0, pad_value=float("nan")):
    """Copy a host column-major matrix into a CUDA tensor with leading
    dimension `ld` starting `offset` elements into its allocation; unused
    storage holds `pad_value` (NaN by default, so stray reads show up)."""
    X = np.asarray(X)
    rows, cols = X.shape
    ld = max(1, rows) if ld is None else ld
    n_el = offset + ld * max(cols - 1, 0) + rows + 64
    base = torch.full((n_el,), pad_value, dtype=NP2T[X.dtype.type], device="cuda")
    view = torch.as_strided(base, (rows, cols), (1, ld), storage_offset=offset)
    if X.size:
        view.copy_(torch.from_numpy(np.ascontiguousarray(X)))
    return view


def run(A, B, C0, alpha, beta, *, lda=None, ldc=None, ldb=None, a_offset=0, c_offset=0,
        repeats=1, plan=None, pb=None):
    """C = alpha*A*B + beta*C0 through tsmm_pack_b / tsmm_plan / tsmm_execute."""
    m, k = A.shape
    n = B.shape[1]
    dA = to_device(A, lda, a_offset)
    dB = to_device(B, ldb)
    outs = []
    pb = pb or tsmm.pack_b(dB)
    pl = plan or tsmm.plan(m, n, k, NP2T[A.dtype.type])
    for _ in range(repeats):
        dC = to_device(C0 if C0 is not None else np.full((m, n), np.nan, dtype=A.dtype), ldc,
                       c_offset)
        tsmm.execute(pl, alpha, dA, pb, beta, dC)
        pl.check()
        outs.append(dC.cpu().numpy())
    return (outs if repeats > 1 else outs[0]), pl, pb


def assert_parity(C, A, B, C0, alpha, beta, exact=False):
    dtype = A.dtype.type
    Cref, E = oracle.tsmm(alpha, A, B, beta, C0 if beta != 0 else None,
                          m=A.shape[0], n=B.shape[1], k=A.shape[1], dtype=A.dtype)
    ok, ratio, nbad = oracle.check(C, Cref, E, dtype)
    assert ok, f"{nbad} entries outside the bound (max ratio {ratio:.3g})"
    if exact:
        np.testing.assert_array_equal(C, oracle.round_to(Cref, dtype))
    return ratio
