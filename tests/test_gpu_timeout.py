"""The timeout path of the library's bounded waits, run on a GPU without a
fault or a hang: tsmm_diag_bounded_wait polls an mbarrier that nothing
completes with the same wait every kernel uses, the kernel records
TSMM_ERR_TIMEOUT in its status word and returns, and the context stays usable
for the next TSMM."""
import numpy as np
import pytest
import torch

import oracle
import paper_2208_08088_gb300 as tsmm
import tsmm_inputs as ti
from gpu_util import run

pytestmark = pytest.mark.gpu
TIMEOUT = 7


def test_bounded_wait_runs_out_and_reports():
    st, cycles, seconds = tsmm.diag_bounded_wait(1 << 12)
    assert st == TIMEOUT
    assert cycles > 0 and seconds > 0
    st2, cycles2, _ = tsmm.diag_bounded_wait(1 << 14)
    assert st2 == TIMEOUT
    # the wait is a loop of polls: four times the polls take longer
    assert cycles2 > 2 * cycles
    print(f"\nbounded wait: {seconds / (1 << 12) * 1e9:.1f} ns per failed poll")


def test_bounded_wait_ends_on_the_clock():
    """With the library's own poll cap (2^24 polls, about a minute of polling)
    the wait ends on its one-second clock bound instead."""
    st, cycles, seconds = tsmm.diag_bounded_wait(1 << 24)
    assert st == TIMEOUT
    assert 0.5 < seconds < 3.0, seconds


def test_context_usable_after_timeout():
    assert tsmm.diag_bounded_wait(1 << 12)[0] == TIMEOUT
    m, n, k = 1000, 16, 700
    A = ti.matrix_np(m, k, 31, "integer", np.float32)
    B = ti.matrix_np(k, n, 32, "integer", np.float32)
    C0 = ti.matrix_np(m, n, 33, "integer", np.float32)
    C, pl, _ = run(A, B, C0, 1.5, 0.5)
    Cref, _ = oracle.tsmm(1.5, A, B, 0.5, C0)
    np.testing.assert_array_equal(C, oracle.round_to(Cref, np.float32))
    torch.cuda.synchronize()


def test_zero_polls_rejected():
    assert tsmm.diag_bounded_wait(0)[0] == 1  # INVALID_ARG
