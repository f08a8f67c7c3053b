"""bench.py's reference arm runs on the host alone (the CPU oracle on a bounded
sample of the workload) and prints the contract's JSON line: the same metric,
unit and direction as the GPU arm, marked impl = reference, with a cpu_baseline
describing the run and an e2e record that moves no bytes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    env = dict(os.environ, RANK="0")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600, check=True).stdout
    line = json.loads(out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"].startswith("TSMM GFLOP/s") and line["unit"] == "GFLOP/s"
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1")
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert res.returncode == 0 and res.stdout.strip() == ""


def test_workloads_and_roofline_arithmetic():
    """The default step is the FP32 sweep m = k = 32768, n in {1, 2, 4, 8, 16, 32,
    64}, beta in {0, 1}; the rank-k workload is m = n = 16384, k in {4..128},
    beta = 1; flops are 2mnk (Eq. 7) and algorithmic bytes read A and B once,
    write C once and read C0 only when beta != 0."""
    sys.path.insert(0, ROOT)
    import bench

    saved = sys.argv
    try:
        sys.argv = ["bench.py"]
        pts = bench.workload_points(bench.parse())
        sys.argv = ["bench.py", "--workload", "rankk"]
        rk = bench.workload_points(bench.parse())
    finally:
        sys.argv = saved
    assert len(pts) == 14 and bench.SWEEP_N == [1, 2, 4, 8, 16, 32, 64]
    assert {(m, k) for (m, _, k, _) in pts} == {(32768, 32768)}
    assert {b for (*_, b) in pts} == {0.0, 1.0}
    assert [(m, n, k, b) for (m, n, k, b) in rk] == [(16384, 16384, k, 1.0) for k in (4, 8, 16, 32, 64, 128)]
    assert bench.flops(3, 5, 7) == 210.0
    assert bench.alg_bytes(10, 2, 3, 0.0, 4) == 4 * (30 + 6 + 20)
    assert bench.alg_bytes(10, 2, 3, 0.5, 8) == 8 * (30 + 6 + 40)
    # the derived FP32 peak: 152 SMs x 128 lanes x 2 flop x 2070 MHz
    assert abs(bench.SMS * bench.FP32_LANES_PER_SM * 2 * bench.SM_MAX_MHZ * 1e6 / 1e12 - 80.55) < 0.01


def test_serving_stall_metric():
    """longest_stall_ms: the longest interval with a request outstanding and no
    completion.  A 100-ms pause that holds the requests arriving in it shows as
    the pause; an idle gap with nothing outstanding does not count; a request
    outstanding from time 0 counts from its arrival."""
    sys.path.insert(0, ROOT)
    import bench

    comps = []
    for i in range(100):
        a = i * 0.001
        c = 0.15 + 0.0001 * i if 0.05 <= a < 0.15 else a + 0.0005
        comps.append({"arrival_s": a, "complete_s": c})
    assert abs(bench.longest_stall_ms(comps) - 105.0) < 1e-6
    idle = [{"arrival_s": 0.0, "complete_s": 0.001}, {"arrival_s": 0.5, "complete_s": 0.501}]
    assert abs(bench.longest_stall_ms(idle) - 1.0) < 1e-6
    held = [{"arrival_s": 0.0, "complete_s": 0.001}, {"arrival_s": 0.0, "complete_s": 0.2}]
    assert abs(bench.longest_stall_ms(held) - 199.0) < 1e-6
    assert bench.longest_stall_ms(held[:1]) == 0.0


def test_kernel_source_hash_follows_code_not_comments():
    """The traffic records are tied to a kernel family's code: comments and
    whitespace do not change code_text, a changed token does."""
    sys.path.insert(0, ROOT)
    import bench

    a = "int x = 1; // one\n/* block\n comment */ int y = x +  2;\n"
    b = "int x = 1;   // other words\nint y = x + 2; /* c */\n"
    c = "int x = 1;\nint y = x + 3;\n"
    assert bench.code_text(a) == bench.code_text(b) == "int x = 1; int y = x + 2;"
    assert bench.code_text(c) != bench.code_text(a)
    assert len(bench.kernel_source_hash("tall")) == 16
