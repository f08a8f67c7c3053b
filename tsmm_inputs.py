"""Seeded, counter-based synthetic inputs shared by the oracle side and the GPU side.

This module holds no arithmetic of the TSMM method itself: it only turns
(seed, stream, element index) into matrix entries, so that the CPU oracle and
the CUDA path can be fed bit-identical inputs without either importing the
other.

Generator definition
--------------------
Every value is a pure function of ``(seed, stream, i)`` where ``i`` is the
element's linear index in a column-major array with a tight leading dimension
(``i = row + col * rows``).  The 32-bit mixer is Chris Wellons' "lowbias32"
integer hash (published in "Prospecting for Hash Functions", 2018)::

    x ^= x >> 16;  x *= 0x7feb352d;  x ^= x >> 15;  x *= 0x846ca68b;  x ^= x >> 16

(all mod 2**32).  A value is

    key  = H(seed_lo ^ H(stream ^ 0x9e3779b9) ^ H(seed_hi ^ 0x85ebca6b))
    h(i) = H(H(i_lo ^ key) ^ i_hi ^ 0x27d4eb2f)

with ``i_lo``/``i_hi`` the low/high 32 bits of ``i``.  The multiplications
are carried out in int64 on 16-bit limbs so no intermediate exceeds 2**49:
the result is the same on numpy, torch-CPU and torch-CUDA and never relies
on signed overflow.

Distributions (all exactly representable in FP32 and FP64):

* ``uniform``  : ``(h >> 8) * 2**-23 - 1``      -> 2**24 values in [-1, 1)
* ``integer``  : ``(h % 9) - 4``                -> integers in [-4, 4]
* ``ternary``  : ``(h % 3) - 1``                -> {-1, 0, 1}
* ``normal_scaled``: N(0,1) by Box-Muller from two uniform streams, times
  ``10**U`` with ``U`` uniform in [-3, 3] drawn once per row (the
  precision-mode workload's "scaled per row" inputs).
"""
from __future__ import annotations

import math

import numpy as np

_M32 = 0xFFFFFFFF

# Seeds of the standard workloads: one per operand.
SEED_A, SEED_B, SEED_C0 = 1, 2, 3


def _mul32(x, c: int):
    """(x * c) mod 2**32 for 0 <= x < 2**32, done on 16-bit limbs of c."""
    lo = c & 0xFFFF
    hi = c >> 16
    return (x * lo + (((x * hi) & 0xFFFF) << 16)) & _M32


def _hash32(x):
    x = x ^ (x >> 16)
    x = _mul32(x, 0x7FEB352D)
    x = x ^ (x >> 15)
    x = _mul32(x, 0x846CA68B)
    x = x ^ (x >> 16)
    return x


def _hash32_int(x: int) -> int:
    return int(_hash32(x & _M32))


def stream_key(seed: int, stream: int = 0) -> int:
    """32-bit key of one (seed, stream) pair."""
    s_lo = seed & _M32
    s_hi = (seed >> 32) & _M32
    return _hash32_int(s_lo ^ _hash32_int(stream ^ 0x9E3779B9) ^ _hash32_int(s_hi ^ 0x85EBCA6B))


def _bits(idx, key: int):
    """32 random bits for each int64 index in ``idx`` (numpy or torch)."""
    i_lo = idx & _M32
    i_hi = idx >> 32
    return _hash32(_hash32(i_lo ^ key) ^ i_hi ^ 0x27D4EB2F)


def _to_values(h, dist: str):
    if dist == "uniform":
        return (h >> 8) * (2.0 ** -23) - 1.0
    if dist == "integer":
        return (h % 9) - 4
    if dist == "ternary":
        return (h % 3) - 1
    raise ValueError(f"unknown distribution {dist!r}")


def bits_np(idx: np.ndarray, seed: int, stream: int = 0) -> np.ndarray:
    """Raw 32-bit hash values (as int64) for int64 indices, numpy."""
    idx = np.asarray(idx, dtype=np.int64)
    return _bits(idx, stream_key(seed, stream))


def values_np(idx: np.ndarray, seed: int, dist: str = "uniform", stream: int = 0,
              dtype=np.float64) -> np.ndarray:
    """Generator values at the given linear indices, numpy (host)."""
    h = bits_np(idx, seed, stream)
    return _to_values(h, dist).astype(dtype)


def matrix_np(rows: int, cols: int, seed: int, dist: str = "uniform", dtype=np.float32,
              stream: int = 0) -> np.ndarray:
    """A rows x cols column-major matrix (returned as a Fortran-ordered array)."""
    n = rows * cols
    idx = np.arange(n, dtype=np.int64)
    v = values_np(idx, seed, dist, stream, dtype=np.float64).astype(dtype)
    return np.asfortranarray(v.reshape(cols, rows).T)


def rows_np(row_idx, rows: int, cols: int, seed: int, dist: str = "uniform", dtype=np.float32,
            stream: int = 0) -> np.ndarray:
    """Selected rows (all columns) of the rows x cols matrix, shape (len(row_idx), cols)."""
    r = np.asarray(row_idx, dtype=np.int64)[:, None]
    c = np.arange(cols, dtype=np.int64)[None, :]
    idx = r + c * rows
    return values_np(idx, seed, dist, stream).astype(dtype)


def fill_torch(t, seed: int, dist: str = "uniform", stream: int = 0, chunk: int = 1 << 25):
    """Fill a contiguous torch tensor, viewed as the flat column-major storage of a
    matrix with tight leading dimension, with generator values.  Runs on the
    tensor's own device (torch elementwise ops only), in chunks."""
    import torch

    flat = t.view(-1)
    key = stream_key(seed, stream)
    n = flat.numel()
    for start in range(0, n, chunk):
        stop = min(n, start + chunk)
        idx = torch.arange(start, stop, dtype=torch.int64, device=t.device)
        h = _bits(idx, key)
        if dist == "uniform":
            v = (h >> 8).to(torch.float64) * (2.0 ** -23) - 1.0
        elif dist == "integer":
            v = (h % 9 - 4).to(torch.float64)
        elif dist == "ternary":
            v = (h % 3 - 1).to(torch.float64)
        else:
            raise ValueError(f"unknown distribution {dist!r}")
        flat[start:stop] = v.to(flat.dtype)
        del idx, h, v
    return t


def normal_scaled_np(rows: int, cols: int, seed: int, dtype=np.float32) -> np.ndarray:
    """N(0,1) entries (Box-Muller on two uniform streams) scaled by 10**U, U ~ U[-3,3]
    drawn once per row; column-major rows x cols."""
    n = rows * cols
    idx = np.arange(n, dtype=np.int64)
    u1 = ((bits_np(idx, seed, 11) >> 8).astype(np.float64) + 1.0) * 2.0 ** -24  # (0, 1]
    u2 = (bits_np(idx, seed, 12) >> 8).astype(np.float64) * 2.0 ** -24           # [0, 1)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    ridx = np.arange(rows, dtype=np.int64)
    e = (bits_np(ridx, seed, 13) >> 8).astype(np.float64) * 2.0 ** -24 * 6.0 - 3.0
    z = z.reshape(cols, rows).T * (10.0 ** e)[:, None]
    return np.asfortranarray(z.astype(dtype))


def normal_scaled_torch(t, seed: int, chunk: int = 1 << 24):
    """Device counterpart of normal_scaled_np: fill the contiguous storage of a
    rows x cols column-major matrix viewed as t.t() (t has shape cols x rows)
    with N(0,1) * 10**U[-3,3] (U drawn once per row) using torch float64 math
    on t's device.  Transcendentals may differ from numpy's in the last bits,
    so consumers that need the exact values read them back from the tensor."""
    import torch

    cols, rows = t.shape
    flat = t.view(-1)
    k1, k2, k3 = stream_key(seed, 11), stream_key(seed, 12), stream_key(seed, 13)
    ridx = torch.arange(rows, dtype=torch.int64, device=t.device)
    e = (_bits(ridx, k3) >> 8).to(torch.float64) * 2.0 ** -24 * 6.0 - 3.0
    scale = torch.pow(torch.tensor(10.0, dtype=torch.float64, device=t.device), e)
    n = flat.numel()
    for start in range(0, n, chunk):
        stop = min(n, start + chunk)
        idx = torch.arange(start, stop, dtype=torch.int64, device=t.device)
        u1 = ((_bits(idx, k1) >> 8).to(torch.float64) + 1.0) * 2.0 ** -24
        u2 = (_bits(idx, k2) >> 8).to(torch.float64) * 2.0 ** -24
        z = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
        flat[start:stop] = (z * scale[idx % rows]).to(flat.dtype)
    return t
