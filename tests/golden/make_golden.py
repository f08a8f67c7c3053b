"""Writes the golden fixtures of this directory.  Calls only the CPU oracle
(oracle/) and the shared seeded input generator; never the CUDA library.

    python tests/golden/make_golden.py

tsmm_2048x2048x16_integer_rows.json: the m = k = 2048, n = 16 workload (alpha = 1.5,
beta = 0.5) with integer-valued inputs in [-4, 4] (seeds A = 1, B = 2, C0 = 3):
every partial sum is an integer below 2^15, so C is exact in FP32 and the
stored rows are the unique correct result for any summation order.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import tsmm_inputs as ti  # noqa: E402

ROWS = [0, 1, 2, 127, 128, 1000, 1023, 1024, 2046, 2047]


def integer_2048x2048x16():
    m = k = 2048
    n = 16
    A = np.asfortranarray(ti.rows_np(ROWS, m, k, ti.SEED_A, "integer", np.float32))
    B = ti.matrix_np(k, n, ti.SEED_B, "integer", np.float32)
    C0 = np.asfortranarray(ti.rows_np(ROWS, m, n, ti.SEED_C0, "integer", np.float32))
    Cref, E = oracle.tsmm(1.5, A, B, 0.5, C0)
    return {"workload": "m=k=2048, n=16, alpha=1.5, beta=0.5, integer inputs in [-4,4], "
                        "seeds A=1 B=2 C0=3 (tsmm_inputs)",
            "m": m, "n": n, "k": k, "alpha": 1.5, "beta": 0.5, "rows": ROWS,
            "C_rows": [[float(x) for x in row] for row in Cref]}


def main():
    with open(os.path.join(HERE, "tsmm_2048x2048x16_integer_rows.json"), "w") as f:
        json.dump(integer_2048x2048x16(), f, indent=1)


if __name__ == "__main__":
    main()
