"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/tsmm.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import pytest

import paper_2208_08088_gb300 as tsmm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "tsmm.h")).read()
    return sorted(set(re.findall(r"TSMM_API[^;(]*?\b(tsmm_\w+)\s*\(", text)))


def test_header_declares_entry_points():
    syms = declared_symbols()
    for name in ("tsmm_pack_b", "tsmm_plan", "tsmm_execute", "tsmm_plan_destroy",
                 "tsmm_packed_b_destroy", "tsmm_status_string"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(tsmm.library_path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_exports_nothing_else():
    """Hidden visibility: only the extern "C" entry points are exported."""
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", tsmm.library_path],
                         capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported == set(declared_symbols())


def test_status_strings_and_version():
    for code, name in tsmm.STATUS.items():
        assert tsmm.tsmm_status_string(code) == name
    assert tsmm.tsmm_status_string(99) == "TSMM_ERR_UNKNOWN"
    assert tsmm.tsmm_version() >= 100


def test_argument_errors_before_device_work():
    L = tsmm.lib
    out = ctypes.c_void_p()
    # plan: negative size, bad dtype, NULL out, unsupported shape
    assert L.tsmm_plan(-1, 4, 4, 0, ctypes.byref(out)) == 1
    assert L.tsmm_plan(4, 4, 4, 7, ctypes.byref(out)) == 1
    assert L.tsmm_plan(4, 4, 4, 0, None) == 1
    assert L.tsmm_plan(1000, 65, 129, 0, ctypes.byref(out)) == 2
    # pack: NULL out, ldb < k, NULL B with nonzero size, misaligned B, unsupported
    assert L.tsmm_pack_b(0, 8, 4, None, 8, None, None) == 1
    assert L.tsmm_pack_b(0, 8, 4, 256, 7, None, ctypes.byref(out)) == 1
    assert L.tsmm_pack_b(0, 8, 4, None, 8, None, ctypes.byref(out)) == 1
    assert L.tsmm_pack_b(0, 8, 4, 258, 8, None, ctypes.byref(out)) == 4
    assert L.tsmm_pack_b(1, 8, 4, 260, 8, None, ctypes.byref(out)) == 4
    assert L.tsmm_pack_b(0, 129, 65, 256, 129, None, ctypes.byref(out)) == 2
    assert out.value is None  # never written on failure
    # execute / destroy / info with NULL handles
    assert L.tsmm_execute(None, 1.0, None, 1, None, 0.0, None, 1, None) == 1
    assert L.tsmm_plan_destroy(None) == 0
    assert L.tsmm_packed_b_destroy(None) == 0
    assert L.tsmm_plan_info(None, None, None, None, None, None) == 1
    assert L.tsmm_plan_check(None) == 1
    assert L.tsmm_plan_launches_per_execute(None) == 0


def test_python_raises_tsmm_error():
    with pytest.raises(tsmm.TsmmError) as ei:
        tsmm.tsmm_plan(10, 100, 1000, tsmm.F32)
    assert ei.value.status == 2


def test_plan_cache_file_roundtrip(tmp_path):
    """The plan cache's text format: load merges, save writes every entry,
    malformed files are rejected without touching the cache (host only)."""
    tsmm.tsmm_plan_cache_clear()
    assert tsmm.tsmm_plan_cache_size() == 0
    src = tmp_path / "cache.txt"
    src.write_text("# comment\nf32 32768 16 32768 152 19\nf64 4096 8 4096 152 3\nf32q 60 16 32768 152 7\n\n")
    tsmm.tsmm_plan_cache_load(str(src))
    assert tsmm.tsmm_plan_cache_size() == 3
    dst = tmp_path / "out.txt"
    tsmm.tsmm_plan_cache_save(str(dst))
    lines = [l for l in dst.read_text().splitlines() if not l.startswith("#")]
    assert sorted(lines) == sorted(["f32 32768 16 32768 152 19", "f64 4096 8 4096 152 3",
                                    "f32q 60 16 32768 152 7"])
    bad = tmp_path / "bad.txt"
    bad.write_text("f16 1 2 3 4 5\n")
    with pytest.raises(tsmm.TsmmError):
        tsmm.tsmm_plan_cache_load(str(bad))
    with pytest.raises(tsmm.TsmmError):
        tsmm.tsmm_plan_cache_load(str(tmp_path / "missing.txt"))
    assert tsmm.tsmm_plan_cache_size() == 3
    tsmm.tsmm_plan_cache_clear()
    assert tsmm.tsmm_plan_cache_size() == 0


def test_last_cuda_error_string():
    assert isinstance(tsmm.lib.tsmm_last_cuda_error().decode(), str)


def test_binding_has_every_entry_point_under_its_c_name():
    """The Python binding is the C ABI under the same names (marshalling only)."""
    missing = [s for s in declared_symbols() if not callable(getattr(tsmm, s, None))]
    assert not missing, missing


def test_noalloc_argument_errors_before_device_work():
    with pytest.raises(tsmm.TsmmError) as e:
        tsmm.tsmm_execute_noalloc(tsmm.F32, -1, 4, 4, 1.0, 0, 1, 0, 4, 0.0, 0, 1)
    assert e.value.status == 1
    with pytest.raises(tsmm.TsmmError) as e:
        tsmm.tsmm_execute_noalloc(tsmm.F32, 100, 65, 8, 1.0, 0, 100, 0, 8, 0.0, 0, 100)
    assert e.value.status == 2
    with pytest.raises(tsmm.TsmmError) as e:
        tsmm.tsmm_execute_noalloc(tsmm.F32, 100, 8, 8, 1.0, 0, 99, 0, 8, 0.0, 0, 100)
    assert e.value.status == 1
    # m = 0 or n = 0: nothing to do, no device touched
    tsmm.tsmm_execute_noalloc(tsmm.F32, 0, 8, 8, 1.0, 0, 1, 0, 8, 0.0, 0, 1)


def test_fp_peak_argument_errors_before_device_work():
    L = tsmm.lib
    assert L.tsmm_diag_fp_peak(4, 10, 4, None, None, None) == 1   # no such pipe
    assert L.tsmm_diag_fp_peak(-1, 10, 4, None, None, None) == 1
    assert L.tsmm_diag_fp_peak(0, 0, 4, None, None, None) == 1    # iters == 0
    assert L.tsmm_diag_fp_peak(0, 10, 0, None, None, None) == 1   # blocks per SM outside 1..8
    assert L.tsmm_diag_fp_peak(0, 10, 9, None, None, None) == 1
    with pytest.raises(tsmm.TsmmError) as e:
        tsmm.diag_fp_peak(tsmm.DIAG_DMMA, 0)
    assert e.value.status == 1
