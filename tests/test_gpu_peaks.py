"""The arithmetic-pipe probe (tsmm_diag_fp_peak) that supplies the roofline
denominators of the FMA-bound shapes and decides between FP64 fma and FP64
mma for the FP64 kernels (the GPU counterpart of the paper's install-time
selection of inner kernels, Section IV.B, taken by measurement).

Each pipe runs on every SM through the same harness; the test checks that the
figures are physically possible (the FP32 pipes cannot exceed 128 fmas per
clock per SM, i.e. 256 flop) and prints them, FP64 fma next to FP64 mma."""
import pytest
import torch

import paper_2208_08088_gb300 as tsmm

pytestmark = pytest.mark.gpu


def _rate(pipe, target_ms=30.0):
    fl, ms, cyc = tsmm.diag_fp_peak(pipe, 64, 4)
    iters = max(64, int(64 * target_ms / max(ms, 1e-3)))
    fl, ms, cyc = tsmm.diag_fp_peak(pipe, iters, 4)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return {"tflops": fl / (ms * 1e-3) / 1e12, "mhz": cyc / (ms * 1e3), "flop_per_clk_sm": fl / cyc / sms,
            "ms": ms}


def test_fp_pipe_rates_are_physical_and_fp64_choice_is_printed():
    torch.cuda.set_device(0)
    r = {name: _rate(pipe) for name, pipe in (("ffma", tsmm.DIAG_FFMA), ("ffma2", tsmm.DIAG_FFMA2),
                                              ("dfma", tsmm.DIAG_DFMA), ("dmma", tsmm.DIAG_DMMA))}
    for name, x in r.items():
        print(f"{name}: {x['tflops']:.3f} TFLOP/s at {x['mhz']:.0f} MHz, {x['flop_per_clk_sm']:.2f} flop/clk/SM")
        assert x["ms"] > 1.0 and x["tflops"] > 0
    for name in ("ffma", "ffma2"):
        assert r[name]["flop_per_clk_sm"] <= 256 * 1.02
    # the packed FP32x2 fma is what the FP32 kernels use; it must reach the
    # FP32 pipe (FFMA2 issues at half rate, leaving room for loop overhead)
    assert r["ffma2"]["flop_per_clk_sm"] >= r["ffma"]["flop_per_clk_sm"] * 0.99
    faster = "dfma" if r["dfma"]["tflops"] >= r["dmma"]["tflops"] else "dmma"
    print(f"FP64: {faster} is faster ({r['dfma']['tflops']:.3f} vs {r['dmma']['tflops']:.3f} TFLOP/s, fma vs mma)")


def test_fp_peak_rejects_bad_arguments():
    with pytest.raises(tsmm.TsmmError):
        tsmm.diag_fp_peak(9, 100)
    with pytest.raises(tsmm.TsmmError):
        tsmm.diag_fp_peak(tsmm.DIAG_FFMA, 100, blocks_per_sm=0)
