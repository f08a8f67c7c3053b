"""Benchmark of the pre-packed tall-and-skinny GEMM on GB300.

Workload (default, FP32): the memory-bound sweep  m = k = 32768,
n in {1,2,4,8,16,32,64}, beta in {0,1}, alpha = 1, A and C0 uniform[-1,1] from
the shared seeded generator, B packed once per n (packing untimed, as in the
paper's evaluation, Section V).  One step = one tsmm_execute per (n, beta)
point, 14 launches over a resident 4 GiB A (larger than L2, so no flush is
needed between calls).  `--dtype f64` runs the same sweep in FP64.
`--workload rankk` runs m = n = 16384, k in {4,...,128}, beta = 1;
`--workload grouped` times tsmm_execute_grouped against back-to-back single
launches on mixes of uneven problems.

Metric: GFLOP/s by Eq. 7 (2*m*n*k / t) aggregated over the step, with the
roofline of the dominant kernel against peaks measured in the same run (the
library's FP pipe throughput probe for FMA-bound kernels, the measured copy
bandwidth for HBM-bound ones).  The default line also carries the rest of the
metric: the FP64 sweep, the rank-k shapes in FP32 and FP64, and a serving
session (p50/p90/p99 latency, capacity, aggregate GFLOP/s).  The CPU oracle on
the host cores is timed on a bounded sample of the same workload as a
baseline, with all cores and with one.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype f32|f64]
                  [--workload tall|rankk|precision|serving|grouped] [--impl ours|reference]
                  [--split replicas|rows]

Under torchrun (N > 1) every rank runs the full workload on its own GPU
(independent problems, weak scaling; `--split replicas`, the default), or the
ranks split each problem's m rows into slabs with B replicated (`--split rows`,
strong scaling: the multi-thread optimizer's split of Section IV.A.2, with no
exchange between ranks).  No collective touches the data; rank 0 prints the
JSON line with value = all ranks' flops / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TSMM GFLOP/s & % HBM/FP roofline vs plain kernel; serving p50/p99 latency"
UNIT = "GFLOP/s"
SMS = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (non-tensor) nominal rate

SWEEP_N = [1, 2, 4, 8, 16, 32, 64]
SWEEP_BETA = [0.0, 1.0]
RANKK_K = [4, 8, 16, 32, 64, 128]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    p.add_argument("--workload", choices=["tall", "rankk", "precision", "serving", "grouped"], default="tall")
    p.add_argument("--requests", type=int, default=10000, help="serving: number of requests")
    p.add_argument("--load", type=float, default=0.8, help="serving: arrival rate / measured capacity")
    p.add_argument("--streams", type=int, default=4, help="serving: the server's CUDA streams")
    p.add_argument("--precision", choices=["native", "bf16x3"], default="native",
                   help="arithmetic of the tall sweep: IEEE FMA (default) or the BF16x3 tensor-core mode")
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--size", type=int, default=None,
                   help="profiling/small runs: m = k (tall) or m = n (rankk) instead of the workload's")
    p.add_argument("--only", type=int, default=None,
                   help="profiling/small runs: keep only this n (tall) or k (rankk)")
    p.add_argument("--beta", type=float, default=None, help="profiling/small runs: one beta only")
    p.add_argument("--lda-pad", type=int, default=0,
                   help="store A with lda = m + PAD (PAD not a multiple of 16/element size: the path "
                        "for an A that a tensor map cannot describe)")
    p.add_argument("--split", choices=["replicas", "rows"], default="replicas",
                   help="N > 1: independent replicas (weak scaling) or one problem's rows split over ranks")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the FP64 sweep, rank-k and serving keys of the default line")
    return p.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload_points(args):
    """(m, n, k, beta) per launch of one step."""
    betas = SWEEP_BETA if args.beta is None else [args.beta]
    if args.workload == "tall":
        s = args.size or 32768
        ns = SWEEP_N if args.only is None else [args.only]
        return [(s, n, s, b) for n in ns for b in betas]
    s = args.size or 16384
    ks = RANKK_K if args.only is None else [args.only]
    return [(s, s, k, 1.0 if args.beta is None else args.beta) for k in ks]


def workload_name(args):
    pad = f", A stored with lda = m + {args.lda_pad}" if getattr(args, "lda_pad", 0) else ""
    if args.size or args.only or args.beta is not None:
        return "reduced case for profiling: " + ", ".join(
            f"m={m} n={n} k={k} beta={b}" for (m, n, k, b) in workload_points(args)) + pad
    if args.workload == "tall":
        mode = "" if args.precision == "native" else " in the BF16x3 tensor-core mode"
        return (f"memory-bound sweep {args.dtype.upper()} m=k=32768, n in {SWEEP_N}, "
                f"beta in {{0,1}}, alpha=1, B pre-packed and reused{mode}{pad}")
    return f"rank-k {args.dtype.upper()} m=n=16384, k in {RANKK_K}, beta=1, B pre-packed"


def alg_bytes(m, n, k, beta, es):
    """Algorithmic bytes: A and B read once, C written once, C0 read if beta != 0."""
    return es * (m * k + k * n + m * n * (1 + (1 if beta != 0 else 0)))


def flops(m, n, k):
    return 2.0 * m * n * k


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        # median under load: samples within 30% of the top observed clock
        top = max(sm) if sm else 0
        loaded = [x for x in sm if x >= 0.3 * top] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(rows), "reasons": reasons}


# --------------------------------------------------------------------- oracle leg
def oracle_sample_rows(cores, m):
    """Rows of the CPU oracle's bounded sample: the oracle splits rows into
    blocks of 512 over its threads, so 512 per thread keeps every thread busy."""
    return int(min(m, 512 * max(1, cores)))


def oracle_time_sample(args, A_rows, m_s, repeats=1):
    """Time the oracle, as it stands, on the first m_s rows of every point of
    the workload (A_rows[(m, k)]: those rows of A, column-major on the host).
    Returns (GFLOP/s, flops, seconds) of the best of `repeats` passes."""
    import oracle
    import tsmm_inputs as ti

    npdt = np.float32 if args.dtype == "f32" else np.float64
    pts = workload_points(args)
    Bs = {(n, k): ti.matrix_np(k, n, ti.SEED_B, "uniform", npdt) for (_, n, k, _) in pts}
    C0s = {(m, n): np.asfortranarray(ti.rows_np(np.arange(m_s), m, n, ti.SEED_C0, "uniform", npdt))
           for (m, n, _, _) in pts}
    best = None
    for _ in range(repeats):
        t0 = time.perf_counter()
        fl = 0.0
        for (m, n, k, beta) in pts:
            oracle.tsmm(1.0, A_rows[(m, k)], Bs[(n, k)], beta, C0s[(m, n)] if beta != 0 else None)
            fl += flops(m_s, n, k)
        t = time.perf_counter() - t0
        if best is None or t < best[2]:
            best = (fl / t / 1e9, fl, t)
    return best


def oracle_one_core(args, m_s=256):
    """The oracle on one core (OMP_NUM_THREADS=1 in a child process that touches
    no GPU): GFLOP/s on the first m_s rows of every point of the workload."""
    code = ("import json, sys; sys.path.insert(0, {root!r}); sys.argv = {argv!r}; import bench, numpy as np, "
            "tsmm_inputs as ti; a = bench.parse(); "
            "dt = np.float32 if a.dtype == 'f32' else np.float64; "
            "A = {{(m, k): np.asfortranarray(ti.rows_np(np.arange({ms}), m, k, ti.SEED_A, 'uniform', dt)) "
            "for (m, k) in {{(p[0], p[2]) for p in bench.workload_points(a)}}}}; "
            "r = bench.oracle_time_sample(a, A, {ms}); import oracle; "
            "print(json.dumps({{'value': round(r[0], 3), 'threads': oracle.num_threads(), "
            "'gflop': round(r[1] / 1e9, 2), 'seconds': round(r[2], 2)}}))").format(
                root=ROOT, argv=["bench.py", "--dtype", args.dtype, "--workload", args.workload]
                + (["--size", str(args.size)] if args.size else []) + (["--only", str(args.only)] if args.only else [])
                + (["--beta", str(args.beta)] if args.beta is not None else []), ms=m_s)
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=300, check=True).stdout
        d = json.loads(out.strip().splitlines()[-1])
        return {"value": d["value"], "unit": UNIT, "cores": d["threads"], "kind": "oracle",
                "sample": f"first {m_s} rows of each point of the workload "
                          f"({d['gflop']} GFLOP in {d['seconds']} s), OMP_NUM_THREADS=1"}
    except Exception as e:  # the baseline is reported, not required
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": str(e)[:200]}


def oracle_sample(args, A_dev):
    """The CPU-baseline leg of our arm: the oracle on the machine's host cores on the
    first 512 x threads rows of every point (rows copied from the resident
    device A, made by the same seeded generator), plus the same on one core."""
    import oracle

    pts = workload_points(args)
    cores = oracle.num_threads()
    m_s = oracle_sample_rows(cores, pts[0][0])

    def rows_of(m, k):
        a = A_dev[(m, k)][:m_s]  # column-major m_s x k view
        return np.asfortranarray(a.t().contiguous().cpu().numpy().T)

    A_rows = {mk: rows_of(*mk) for mk in {(m, k) for (m, _, k, _) in pts}}
    gfs, fl, t = oracle_time_sample(args, A_rows, m_s)
    return {"value": round(gfs, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {m_s} rows (512 per thread) of each of the {len(pts)} points of the workload "
                      f"({fl / 1e9:.1f} GFLOP in {t:.1f} s)",
            "one_core": oracle_one_core(args)}


# --------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0  # rank 0 alone runs the CPU oracle
    import oracle
    import tsmm_inputs as ti

    oracle.build()
    npdt = np.float32 if args.dtype == "f32" else np.float64
    pts = workload_points(args)
    cores = oracle.num_threads()
    # one step = the first 512 x threads rows of every point (every thread has row blocks)
    m_s = oracle_sample_rows(cores, pts[0][0])
    A_rows = {(m, k): np.asfortranarray(ti.rows_np(np.arange(m_s), m, k, ti.SEED_A, "uniform", npdt))
              for (m, k) in {(m, k) for (m, _, k, _) in pts}}
    for _ in range(args.warmup):
        oracle_time_sample(args, A_rows, m_s)
    t0 = time.perf_counter()
    fl = 0.0
    for _ in range(args.steps):
        fl += oracle_time_sample(args, A_rows, m_s)[1]
    t = time.perf_counter() - t0
    value = fl / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": workload_name(args), "sample_rows": m_s},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {m_s} rows (512 per thread) of every point of the workload per step",
                         "one_core": oracle_one_core(args)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------- our arm
KERNEL_SOURCES = {  # the files that define each kernel family's device code
    "tall": ["tsmm_tall.cuh", "tsmm_device.cuh"],
    "rankk": ["tsmm_rankk.cu", "tsmm_device.cuh"],
}


def code_text(source):
    """C++/CUDA source without its comments and with whitespace collapsed: what
    the hash of a kernel family follows (its code, not its documentation)."""
    import re

    source = re.sub(r"/\*.*?\*/", " ", source, flags=re.S)
    source = re.sub(r"//[^\n]*", " ", source)
    return " ".join(source.split())


def kernel_source_hash(family):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2208_08088_gb300", "csrc")
    for name in KERNEL_SOURCES[family]:
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(name.encode())
            h.update(code_text(f.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key, family):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    from the committed ncu record, if it was taken on the current sources of
    this kernel family; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    ent = d.get(kernel_key)
    if not ent or ent.get("source_hash") != kernel_source_hash(family):
        return None
    return ent.get("dram_bytes_per_launch")


def aggregate_over_ranks(elapsed_ms, step_flops, steps, world):
    """Whole-job throughput of `world` replicas: every rank's flops divided by
    the slowest rank's time (max over ranks; no collective touches the data).
    Works with any torch.distributed backend (gloo on CPU in the tests)."""
    import torch
    import torch.distributed as dist

    if world > 1:
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    value = world * step_flops * steps / (elapsed_ms * 1e-3) / 1e9
    return elapsed_ms, value


def row_slab(m, rank, world, granule):
    """Rows [lo, hi) of an m-row problem that rank `rank` of `world` computes when
    one TSMM is split along m, the multi-thread optimizer's split (Section
    IV.A.2): contiguous blocks of rows, B replicated, n never split, no exchange
    between ranks.  Boundaries sit at m*r/world rounded down to a multiple of
    `granule` (the plan's rows per thread block, so no block straddles two
    ranks); the last rank takes the rest.  Slabs may be empty when m is small."""
    def edge(r):
        return m if r >= world else (m * r // world) // granule * granule
    return edge(rank), edge(rank + 1)


def measure_fp_peaks(tsmm):
    """Arithmetic-pipe peaks of this GPU, measured now by the library's probe
    (tsmm_diag_fp_peak): FP32 fma, packed FP32x2 fma, FP64 fma and FP64 mma,
    each as the best of two ~60 ms launches on every SM.  cycles/ms gives the SM
    clock each ran at.  Nothing here changes a GPU setting."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = {}
    for name, pipe in (("ffma", tsmm.DIAG_FFMA), ("ffma2", tsmm.DIAG_FFMA2), ("dfma", tsmm.DIAG_DFMA),
                       ("dmma", tsmm.DIAG_DMMA)):
        fl, ms, cyc = tsmm.diag_fp_peak(pipe, 64, 4)
        iters = max(64, int(64 * 60.0 / max(ms, 1e-3)))
        best = None
        for _ in range(2):
            fl, ms, cyc = tsmm.diag_fp_peak(pipe, iters, 4)
            tf = fl / (ms * 1e-3) / 1e12
            if best is None or tf > best["tflops"]:
                best = {"tflops": round(tf, 3), "ms": round(ms, 2), "sm_mhz": round(cyc / (ms * 1e3), 1),
                        "flop_per_clk_per_sm": round(fl / max(cyc, 1) / sms, 2)}
        out[name] = best
    f32 = max(("ffma", "ffma2"), key=lambda k: out[k]["tflops"])
    f64 = max(("dfma", "dmma"), key=lambda k: out[k]["tflops"])
    out["fp32"] = {"tflops": out[f32]["tflops"], "from": f32}
    out["fp64"] = {"tflops": out[f64]["tflops"], "from": f64}
    out["derived_fp32_tflops"] = round(SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12, 2)
    out["nominal_fp64_tflops"] = FP64_NOMINAL_TFLOPS
    return out


def time_points(tsmm, torch, pts, tdt, steps, warmup, precision=0, world=1, rank=0, split="replicas",
                sampler=None, lda_pad=0):
    """Resident inputs for every point (one A per distinct (m, k), B packed once
    per (n, k), C0 per point), `warmup` untimed steps, then `steps` timed steps
    with CUDA events around each launch on the launching stream.  With split =
    rows each rank computes only its row slab of every problem (same plans'
    shapes restricted to the slab).  Returns (points, elapsed_ms, launches,
    state) where state holds the resident tensors for the e2e leg."""
    import tsmm_inputs as ti

    stream = torch.cuda.current_stream()

    def dmat(rows, cols, seed, pad=0):
        t = torch.empty((cols, rows + pad), dtype=tdt, device="cuda")
        ti.fill_torch(t, seed, "uniform")
        return t.t()[:rows]

    A, packed, plans, C, pack_ms, slab = {}, {}, {}, {}, {}, {}
    for (m, n, k, beta) in pts:
        if (m, k) not in A:
            A[(m, k)] = dmat(m, k, ti.SEED_A, lda_pad)
    for (m, n, k, beta) in pts:
        if (n, k) not in packed:
            Bsrc = dmat(k, n, ti.SEED_B)
            tsmm.pack_b(Bsrc, precision=precision)  # first call: kernel attributes, module load
            p0 = torch.cuda.Event(enable_timing=True)
            p1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            p0.record(stream)
            packed[(n, k)] = tsmm.pack_b(Bsrc, precision=precision)
            p1.record(stream)
            torch.cuda.synchronize()
            pack_ms[f"n={n},k={k}"] = round(p0.elapsed_time(p1), 4)
        if (m, n) not in C:
            C[(m, n)] = dmat(m, n, ti.SEED_C0)  # C0; beta != 0 updates it in place
        if (m, n, k) not in plans:
            bm = tsmm.plan(m, n, k, tdt, precision=precision).info()["bm"]
            lo, hi = row_slab(m, rank, world, bm) if split == "rows" else (0, m)
            slab[(m, n, k)] = (lo, hi)
            plans[(m, n, k)] = tsmm.plan(hi - lo, n, k, tdt, precision=precision)
    torch.cuda.synchronize()

    def one(pt):
        m, n, k, beta = pt
        lo, hi = slab[(m, n, k)]
        tsmm.execute(plans[(m, n, k)], 1.0, A[(m, k)][lo:hi], packed[(n, k)], beta, C[(m, n)][lo:hi])

    for _ in range(warmup):
        for pt in pts:
            one(pt)
    torch.cuda.synchronize()
    for pl in plans.values():
        pl.check()
    ev = {pt: [] for pt in pts}
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if sampler is not None:
        sampler.start()
        time.sleep(0.3)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        for pt in pts:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one(pt)
            e1.record(stream)
            ev[pt].append((e0, e1))
    stop.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler is not None else None
    elapsed_ms = start.elapsed_time(stop)
    for pl in plans.values():
        pl.check()
    points = []
    for pt in pts:
        m, n, k, beta = pt
        durs = [a.elapsed_time(b) for (a, b) in ev[pt]]
        lo, hi = slab[(m, n, k)]
        points.append({"m": m, "n": n, "k": k, "beta": beta, "rows": [lo, hi],
                       "avg_ms": sum(durs) / len(durs), "total_ms": sum(durs)})
    # regime (ii) in the native precision first copies, with a kernel of its own,
    # an A that a tensor map cannot describe (column stride not a multiple of 16 bytes)
    es = torch.empty((), dtype=tdt).element_size()

    def per_execute(m, pl):
        copy = precision == 0 and pl.info()["regime"] == 2 and ((m + lda_pad) * es) % 16 != 0
        return pl.launches_per_execute() + (1 if copy else 0)

    launches = steps * sum(per_execute(m, plans[(m, n, k)]) for (m, n, k, _) in pts)
    state = {"A": A, "packed": packed, "plans": plans, "C": C, "slab": slab, "pack_ms": pack_ms,
             "clocks": clocks}
    return points, elapsed_ms, launches, state


def rate_points(points, es, hbm_peak, fp_peak_tf):
    """Per point: GFLOP/s (Eq. 7), algorithmic GB/s, the roof that binds (the
    slower of HBM and the FP pipe at their peaks) and the fraction of it."""
    out = []
    for p in points:
        m, n, k, beta = p["m"], p["n"], p["k"], p["beta"]
        rows = p["rows"][1] - p["rows"][0]
        ms = p["avg_ms"]
        gb = alg_bytes(rows, n, k, beta, es) / 1e9
        gbs = gb / (ms * 1e-3)
        tf = flops(rows, n, k) / (ms * 1e-3) / 1e12
        bound = "hbm" if gb / hbm_peak >= flops(rows, n, k) / (fp_peak_tf * 1e12) else "alu"
        frac = (gbs / hbm_peak) if bound == "hbm" else (tf / fp_peak_tf)
        q = {"m": m, "n": n, "k": k, "beta": beta, "avg_ms": round(ms, 4), "gflops": round(tf * 1e3, 1),
             "alg_gbs": round(gbs, 1), "bound": bound, "frac": round(frac, 4)}
        if rows != m:
            q["rows"] = p["rows"]
        out.append(q)
    return out


def run_ours(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2208_08088_gb300 as tsmm

    tdt = torch.float32 if args.dtype == "f32" else torch.float64
    es = 4 if args.dtype == "f32" else 8
    pts = workload_points(args)
    prec = tsmm.PREC_BF16X3 if args.precision == "bf16x3" else tsmm.PREC_NATIVE

    # peaks of this GPU, measured before the timed region (roofline denominators)
    peaks = measure_fp_peaks(tsmm)
    hbm_peak, hbm_src = load_peaks()
    if args.precision == "bf16x3":
        # three BF16 tensor-core products per FP32 product: the measured dense
        # BF16 peak / 3 (MEASURED_PEAKS.json bf16_tflops)
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                fp_peak_tf = float(json.load(f)["bf16_tflops"]) / 3.0
        except Exception:
            fp_peak_tf = 1900.0 / 3.0
        fp_src = "measured dense BF16 peak (MEASURED_PEAKS.json bf16_tflops) / 3 products"
    else:
        key = "fp32" if args.dtype == "f32" else "fp64"
        fp_peak_tf = peaks[key]["tflops"]
        fp_src = (f"measured now: tsmm_diag_fp_peak {peaks[key]['from']} at "
                  f"{peaks[peaks[key]['from']]['sm_mhz']} MHz (context: "
                  + (f"derived {peaks['derived_fp32_tflops']} TFLOP/s = 152 SMs x 128 lanes x 2 x 2070 MHz)"
                     if args.dtype == "f32" else f"nominal GB300 FP64 {FP64_NOMINAL_TFLOPS} TFLOP/s)"))

    sampler = ClockSampler(local)
    points, elapsed_ms, launches, st = time_points(tsmm, torch, pts, tdt, args.steps, args.warmup, prec, world,
                                                   rank, args.split, sampler, args.lda_pad)
    clocks = st["clocks"]
    step_flops = sum(flops(p["rows"][1] - p["rows"][0], p["n"], p["k"]) for p in points)
    if args.split == "rows":
        # every rank's slab flops summed, over the slowest rank's time: the whole problem
        total = torch.tensor([step_flops], dtype=torch.float64, device="cuda")
        if world > 1:
            torch.distributed.all_reduce(total)
        elapsed_ms, _ = aggregate_over_ranks(elapsed_ms, 0.0, args.steps, world)
        value = float(total.item()) * args.steps / (elapsed_ms * 1e-3) / 1e9
    else:
        elapsed_ms, value = aggregate_over_ranks(elapsed_ms, step_flops, args.steps, world)

    rated = rate_points(points, es, hbm_peak, fp_peak_tf)
    dom_i = max(range(len(points)), key=lambda i: points[i]["total_ms"])
    dom = rated[dom_i]
    m, n, k, beta = dom["m"], dom["n"], dom["k"], dom["beta"]
    kernel_key = f"{args.workload}_{args.dtype}_n{n}_k{k}"
    if dom["bound"] == "hbm":
        roof = {"bound": "hbm", "achieved": dom["alg_gbs"], "peak": hbm_peak, "unit": "GB/s",
                "frac": round(dom["alg_gbs"] / hbm_peak, 4),
                "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        ach = dom["gflops"] / 1e3
        roof = {"bound": "alu", "achieved": round(ach, 2), "peak": round(fp_peak_tf, 2),
                "unit": "TFLOP/s", "frac": round(ach / fp_peak_tf, 4), "peak_source": fp_src}
    roof["traffic"] = recorded_traffic(kernel_key, args.workload) if args.split != "rows" or world == 1 else None
    roof["kernel"] = f"{'tall' if args.workload == 'tall' else 'rankk'} {args.dtype} m={m} n={n} k={k} beta={beta}"
    roof["alg_bytes_per_launch"] = alg_bytes(m, n, k, beta, es)

    # ---------------- end to end: host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e and args.split == "replicas" and not args.lda_pad:
        e2e = run_e2e(args, tsmm, torch, tdt, es, pts, st["A"], st["packed"], st["plans"], world)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample(args, st["A"])
    pack_ms = st["pack_ms"]
    del st
    torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(elapsed_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "strong" if args.split == "rows" else "weak", "vs_baseline": None, "dtype": args.dtype,
        "data": "synthetic",
        "config": {"workload": workload_name(args), "launches_per_step": len(pts),
                   "alpha": 1.0, "l2": "no flush: each launch streams a >= 1 GiB operand, "
                                         "larger than the 129 MB L2",
                   "parallelism": (f"rows of each problem split over {world} ranks (B replicated, no exchange)"
                                   if args.split == "rows" else
                                   f"replicas x{world} (independent problems per GPU)")},
        "clocks": clocks, "gpu_launches": launches, "e2e": e2e, "roofline": roof,
        "points": rated, "pack_ms": pack_ms,
        "peaks": peaks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if (rank == 0 and world == 1 and not args.no_extras and args.workload == "tall" and args.dtype == "f32"
            and args.precision == "native" and not (args.size or args.only or args.beta is not None)
            and not args.lda_pad):
        line.update(run_extras(args, tsmm, torch, peaks, hbm_peak))
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_extras(args, tsmm, torch, peaks, hbm_peak):
    """The rest of the metric, in the default line: the FP64 sweep (m = k =
    32768, the same 14 points), the rank-k shapes m = n = 16384, k in
    {4..128}, beta = 1 in FP32 and FP64, and a serving session.  Each sweep runs
    a few warm-up and timed steps; fractions are against the peaks measured in
    this run."""
    extras = {}
    ns = argparse.Namespace(**vars(args))
    for key, dtype, workload, steps, warmup in (("f64_sweep", "f64", "tall", 3, 2),
                                                ("rankk_f32", "f32", "rankk", 10, 3),
                                                ("rankk_f64", "f64", "rankk", 3, 2)):
        ns.dtype, ns.workload = dtype, workload
        tdt = torch.float32 if dtype == "f32" else torch.float64
        es = 4 if dtype == "f32" else 8
        pts = workload_points(ns)
        points, elapsed_ms, _, st = time_points(tsmm, torch, pts, tdt, steps, warmup)
        del st
        torch.cuda.empty_cache()
        fp = peaks["fp32" if dtype == "f32" else "fp64"]["tflops"]
        rated = rate_points(points, es, hbm_peak, fp)
        fl = sum(flops(p["m"], p["n"], p["k"]) for p in points)
        extras[key] = {"workload": workload_name(ns), "steps": steps, "warmup": warmup,
                       "ms_per_step": round(elapsed_ms / steps, 3),
                       "gflops": round(fl * steps / (elapsed_ms * 1e-3) / 1e9, 1),
                       "fp_peak_tflops": fp, "points": rated}
    extras["serving"] = serving_session(args, tsmm, torch, args.requests, args.load, args.streams)
    return extras


def run_e2e(args, tsmm, torch, tdt, es, pts, A, packed, plans, world):
    """Same metric through the public API with HOST buffers: each step copies
    A (once, shared by every point) and the C0 of each beta != 0 point from
    pinned host memory, executes, and reads every C back.  The inputs stream
    through two sets of device buffers on a copy stream, so step s+1's inputs
    cross the host link while step s computes (a streaming caller's pipeline);
    each result is read back on a third stream as soon as its launch is done,
    so the kernels never wait for a read-back.  The timed region runs from
    before the first copy to after the last read-back.  CUDA events on each
    stream give every step's upload, kernels and read-back tail: the record
    carries their medians, and the uploads that took far longer than the
    median (the host link stalling), so the end-to-end time can be read
    against max(upload, kernels)."""
    stream = torch.cuda.current_stream()
    copy_stream = torch.cuda.Stream()
    rb_stream = torch.cuda.Stream()
    hostA = {key: torch.empty_strided(a.shape, a.stride(), dtype=tdt, pin_memory=True)
             for key, a in A.items()}
    for key, h in hostA.items():
        h.copy_(A[key])
    # per point: C0 (read by beta != 0 points) and the result, both pinned
    hostC0, hostC = {}, {}
    for pt in pts:
        m, n = pt[0], pt[1]
        hostC0[pt] = torch.empty_strided((m, n), (1, m), dtype=tdt, pin_memory=True)
        hostC0[pt].fill_(0.5)
        hostC[pt] = torch.empty_strided((m, n), (1, m), dtype=tdt, pin_memory=True)
    devA = [{key: torch.empty_strided(h.shape, h.stride(), dtype=tdt, device="cuda")
             for key, h in hostA.items()} for _ in range(2)]
    devC = [{pt: torch.empty_strided((pt[0], pt[1]), (1, pt[0]), dtype=tdt, device="cuda") for pt in pts}
            for _ in range(2)]
    h2d = d2h = 0
    for key, h in hostA.items():
        h2d += h.numel() * es
    for (m, n, k, beta) in pts:
        if beta != 0:
            h2d += m * n * es
        d2h += m * n * es
    steps = max(3, args.steps)
    a_ready = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    launched = {(b, pt): torch.cuda.Event() for b in range(2) for pt in pts}

    def T():
        return torch.cuda.Event(enable_timing=True)

    def copy_in(s, ev):
        b = s % 2
        with torch.cuda.stream(copy_stream):
            if s >= 2:
                copy_stream.wait_event(done[b])  # step s-2 is done with these buffers
            if ev:
                ev["u0"][s].record(copy_stream)
            for pt in pts:
                if pt[3] != 0:
                    devC[b][pt].copy_(hostC0[pt], non_blocking=True)
            for key in hostA:
                devA[b][key].copy_(hostA[key], non_blocking=True)
            if ev:
                ev["u1"][s].record(copy_stream)
            a_ready[b].record(copy_stream)

    def compute(s, ev):
        b = s % 2
        stream.wait_event(a_ready[b])
        if ev:
            ev["c0"][s].record(stream)
        for pt in pts:
            m, n, k, beta = pt
            tsmm.execute(plans[(m, n, k)], 1.0, devA[b][(m, k)], packed[(n, k)], beta, devC[b][pt])
            launched[(b, pt)].record(stream)
            rb_stream.wait_event(launched[(b, pt)])
            with torch.cuda.stream(rb_stream):
                hostC[pt].copy_(devC[b][pt], non_blocking=True)
        if ev:
            ev["c1"][s].record(stream)
            ev["r1"][s].record(rb_stream)
        done[b].record(rb_stream)

    def run(nsteps, ev=None):
        copy_stream.wait_stream(stream)
        copy_in(0, ev)
        for s in range(nsteps):
            if s + 1 < nsteps:
                copy_in(s + 1, ev)
            compute(s, ev)
        stream.wait_stream(rb_stream)

    run(2)  # warm-up
    torch.cuda.synchronize()
    # the host link's own rate at this moment (uploads of A, nothing else running;
    # the best of three, as a one-off copy can catch an unrelated stall)
    key0 = next(iter(hostA))
    a = T()
    b = T()
    best_ms = None
    for _ in range(3):
        a.record(stream)
        devA[0][key0].copy_(hostA[key0], non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b)
        best_ms = t if best_ms is None else min(best_ms, t)
    link_gbs = hostA[key0].numel() * es / (best_ms * 1e-3) / 1e9
    ev = {name: [T() for _ in range(steps)] for name in ("u0", "u1", "c0", "c1", "r1")}
    if world > 1:
        torch.distributed.barrier()
    a.record(stream)
    run(steps, ev)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    up = [ev["u0"][s].elapsed_time(ev["u1"][s]) for s in range(steps)]
    kern = [ev["c0"][s].elapsed_time(ev["c1"][s]) for s in range(steps)]
    tail = [ev["c1"][s].elapsed_time(ev["r1"][s]) for s in range(steps)]
    up_med = statistics.median(up)
    stalls = [[s, round(x, 2)] for s, x in enumerate(up) if x > 1.5 * up_med]
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    fl = sum(flops(m, n, k) for (m, n, k, _) in pts)
    del hostA, devA, devC
    return {"value": round(world * fl * steps / (ms * 1e-3) / 1e9, 1), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "ms_per_step": round(ms / steps, 3), "host_to_device_gbs": round(link_gbs, 1),
            "breakdown": {"upload_ms_median": round(up_med, 3), "upload_ms_max": round(max(up), 3),
                          "kernels_ms_median": round(statistics.median(kern), 3),
                          "readback_tail_ms_median": round(statistics.median(tail), 3),
                          "floor_ms": round(max(h2d / (link_gbs * 1e9) * 1e3, statistics.median(kern)), 3),
                          "stalled_uploads": stalls},
            "pipeline": "inputs double-buffered on a copy stream (step s+1's upload overlaps step s), "
                        "read-backs on their own stream"}


def run_precision(args):
    """Precision-mode workload: m = k = 32768 with n = 64, and m = n = 16384 with
    k in {64, 128}; A and B entries N(0,1) * 10**U[-3,3] per row, alpha = 1,
    beta = 0.  Each shape is computed in FP32 (IEEE FMA), in the BF16x3
    tensor-core mode and in FP64 (FMA) on the same inputs; the JSON line gives
    each launch's time and its error on 32 sampled rows against the exactly
    rounded result: the inputs are FP32 values, so every product is exact in
    FP64, and math.fsum returns the correctly rounded sum of the k products."""
    import math

    import torch

    import paper_2208_08088_gb300 as tsmm
    import tsmm_inputs as ti

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    shapes = [(32768, 64, 32768), (16384, 16384, 64), (16384, 16384, 128)]
    if args.size:
        shapes = [(args.size, args.only or 64, args.size)]
    out = []
    for (m, n, k) in shapes:
        A32 = torch.empty((k, m), dtype=torch.float32, device="cuda")
        ti.normal_scaled_torch(A32, ti.SEED_A)
        A32 = A32.t()
        B32 = torch.empty((n, k), dtype=torch.float32, device="cuda")
        ti.normal_scaled_torch(B32, ti.SEED_B)
        B32 = B32.t()
        rows = np.sort(np.random.default_rng(7).choice(m, 32, replace=False))
        A_rows = np.asfortranarray(A32[torch.as_tensor(rows, device="cuda")].cpu().numpy().astype(np.float64))
        B_host = np.asfortranarray(B32.cpu().numpy().astype(np.float64))
        Cref = np.empty((len(rows), n))
        for ri in range(len(rows)):
            P = A_rows[ri][:, None] * B_host  # k x n exact products
            Cref[ri] = [math.fsum(P[:, j]) for j in range(n)]
        G = np.abs(A_rows) @ np.abs(B_host)
        for name, dt, prec in (("fp32_fma", torch.float32, tsmm.PREC_NATIVE),
                               ("bf16x3_tcgen05", torch.float32, tsmm.PREC_BF16X3),
                               ("fp64_fma", torch.float64, tsmm.PREC_NATIVE)):
            A = A32 if dt == torch.float32 else A32.t().double().t()
            B = B32 if dt == torch.float32 else B32.t().double().t()
            pb = tsmm.pack_b(B, precision=prec)
            pl = tsmm.plan(m, n, k, dt, precision=prec)
            C = torch.zeros((n, m), dtype=dt, device="cuda").t()
            reps = args.steps if dt == torch.float32 else max(1, min(args.steps, 2))
            for _ in range(args.warmup):
                tsmm.execute(pl, 1.0, A, pb, 0.0, C)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                tsmm.execute(pl, 1.0, A, pb, 0.0, C)
            e1.record()
            torch.cuda.synchronize()
            pl.check()
            ms = e0.elapsed_time(e1) / reps
            Cs = C[torch.as_tensor(rows, device="cuda")].cpu().numpy().astype(np.float64)
            err = np.abs(Cs - Cref)
            rel = err / np.maximum(np.abs(Cref), 1e-300)
            out.append({"m": m, "n": n, "k": k, "mode": name, "avg_ms": round(ms, 4),
                        "gflops": round(flops(m, n, k) / (ms * 1e-3) / 1e9, 1),
                        "max_abs_err_over_sum_abs": float(np.max(err / G)),
                        "max_rel_err": float(np.max(rel)), "median_rel_err": float(np.median(rel))})
            del A, B, C, pb, pl
            torch.cuda.empty_cache()
        del A32, B32
    x3 = [r for r in out if r["mode"] == "bf16x3_tcgen05"]
    tot_ms = sum(r["avg_ms"] for r in x3)
    tot_fl = sum(flops(r["m"], r["n"], r["k"]) for r in x3)
    line = {"metric": METRIC, "value": round(tot_fl / (tot_ms * 1e-3) / 1e9, 1), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot_ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (bf16x3 tensor-core mode)", "data": "synthetic",
            "config": {"workload": "precision mode: m=k=32768 n=64, and m=n=16384 k in {64,128}; "
                                   "A and B entries N(0,1)*10^U[-3,3] per row, alpha=1, beta=0; "
                                   "value = BF16x3 GFLOP/s over the three shapes",
                       "error_reference": "exactly rounded sums of the exact FP64 products "
                                          "(math.fsum) on 32 sampled rows"},
            "modes": out}
    print(json.dumps(line))
    return 0


def longest_stall_ms(comps):
    """Longest interval with a request outstanding (arrived, not complete)
    and no completion: a pause of the server or the GPU, not queueing.
    Between consecutive completions a < b, the requests completing at b
    or later that arrived before b are outstanding from their arrival on;
    the earliest of those arrivals (a suffix minimum in completion order)
    starts the interval, clipped at a."""
    order = sorted(comps, key=lambda c: c["complete_s"])
    done = np.array([c["complete_s"] for c in order])
    arr = np.array([c["arrival_s"] for c in order])
    first = np.minimum.accumulate(arr[::-1])[::-1]  # earliest arrival among completions i..end
    best = 0.0
    for i in range(1, len(order)):
        if first[i] < done[i]:
            best = max(best, done[i] - max(done[i - 1], first[i]))
    return round(float(best) * 1e3, 2)


# arrival rates of the serving load sweep, as fractions of the measured capacity
SERVING_LOADS = (0.5, 0.7, 0.9, 0.95)


def serving_session(args, tsmm, torch, N, load, num_streams):
    """Serving workload: 32 device-resident packed B (k log-uniform in
    [64, 8192], n log-uniform in [1, 64], drawn once from a seed); requests pick a
    B uniformly and m log-uniform in [1024, 262144]; FP32, alpha = 1, every third
    request with beta = 1 (reads its C0), the others beta = 0.  The server admits
    under a 40 GB budget and batches continuously (grouped launches, one block per work item, on
    `num_streams` lanes).  Capacity is measured with every request arriving at
    once; then Poisson arrivals at `load` x capacity give the p50 / p90 / p99
    arrival-to-completion latency and the aggregate GFLOP/s, and the same
    arrival sequence rescaled to each rate of SERVING_LOADS gives the latency
    sweep (`load_sweep`).

    A requests read windows of one resident, read-only pool (moving 10,000 A
    matrices over the host link would measure the link); the budget charges each
    request its full A, so admission is conservative against the bytes the pool
    physically pins.  C windows are disjoint slices of a 48 GB ring."""
    import tsmm_inputs as ti

    rng = np.random.default_rng(2208)
    NB = 32
    ks = np.round(np.exp(rng.uniform(np.log(64), np.log(8192), NB))).astype(np.int64)
    ns = np.round(np.exp(rng.uniform(np.log(1), np.log(64), NB))).astype(np.int64)
    packed = []
    for i in range(NB):
        B = torch.empty((int(ns[i]), int(ks[i])), dtype=torch.float32, device="cuda")
        ti.fill_torch(B, 100 + i, "uniform")
        packed.append(tsmm.pack_b(B.t()))
    b_idx = rng.integers(NB, size=N)
    ms = np.round(np.exp(rng.uniform(np.log(1024), np.log(262144), N))).astype(np.int64)
    betas = np.where(np.arange(N) % 3 == 2, 1.0, 0.0)
    mk = ms * ks[b_idx]
    mn = ms * ns[b_idx]
    fl = 2.0 * ms * ns[b_idx] * ks[b_idx]
    a_pool = torch.empty(int(mk.max()) + 1024, dtype=torch.float32, device="cuda")
    ti.fill_torch(a_pool, ti.SEED_A, "uniform")
    c_elems = (48 << 30) // 4
    c_pool = torch.zeros(c_elems, dtype=torch.float32, device="cuda")
    a_off = (rng.integers(0, (a_pool.numel() - mk) // 4 + 1) * 4).astype(np.int64)
    c_off = np.zeros(N, dtype=np.int64)
    pos = 0
    for i in range(N):
        if pos + mn[i] > c_elems:
            pos = 0
        c_off[i] = pos
        pos += (int(mn[i]) + 63) // 64 * 64
    a_base, c_base = a_pool.data_ptr(), c_pool.data_ptr()

    def requests(arrivals):
        arr = (tsmm.Request * N)()
        for i in range(N):
            m = int(ms[i])
            arr[i] = tsmm.Request(i, packed[b_idx[i]].handle, m, 1.0, float(betas[i]), a_base + 4 * int(a_off[i]),
                                  m, c_base + 4 * int(c_off[i]), m, float(arrivals[i]))
        return arr

    # autotuned plans: one tsmm_autotune per (packed B, quarter octave of m) present
    # in the stream, on the first request of each; the plan cache's bucket
    # entries hand the tuned split counts to every request of that bucket
    import math
    t_tune = time.time()
    seen = set()
    for i in range(N):
        key = (int(b_idx[i]), int(math.floor(4.0 * math.log2(int(ms[i])) + 1e-9)))
        if key in seen:
            continue
        seen.add(key)
        m, k, n = int(ms[i]), int(ks[b_idx[i]]), int(ns[b_idx[i]])
        A_i = a_pool[int(a_off[i]):int(a_off[i]) + m * k].view(k, m).t()
        C_i = c_pool[int(c_off[i]):int(c_off[i]) + m * n].view(n, m).t()
        tsmm.autotune(A_i, packed[b_idx[i]], C_i, reps=2)
    torch.cuda.synchronize()
    tune_s = time.time() - t_tune

    budget = 40 << 30
    srv = tsmm.Server(budget_bytes=budget, num_streams=num_streams, max_batch=48, arena_bytes=1 << 30)

    def session(arrivals):
        arr = requests(arrivals)
        srv.submit_raw(arr, N)
        srv.drain(3600.0)
        comps = srv.poll(N + 16)
        assert len(comps) == N and all(c["status"] == 0 for c in comps), "serving errors"
        return comps

    # warm-up (module load, kernel attributes), then capacity with all requests at once
    session(np.full(N, tsmm.tsmm_server_clock()))
    t0 = tsmm.tsmm_server_clock() + 0.01
    comps = session(np.full(N, t0))
    makespan = max(c["complete_s"] for c in comps) - t0
    capacity = N / makespan
    cap_gflops = fl.sum() / makespan / 1e9
    # open loop: Poisson arrivals at load x capacity (one seeded draw of unit
    # gaps, scaled to each rate), then the same at each load of the sweep
    unit_gaps = rng.exponential(1.0, N)

    def open_loop(ld):
        t0 = tsmm.tsmm_server_clock() + 0.05
        comps = session(t0 + np.cumsum(unit_gaps / (ld * capacity)))
        lat = np.array([c["complete_s"] - c["arrival_s"] for c in comps])
        span = max(c["complete_s"] for c in comps) - min(c["arrival_s"] for c in comps)
        return comps, lat, span

    lam = load * capacity
    comps, lat, span = open_loop(load)
    qwait = np.array([c["admit_s"] - c["arrival_s"] for c in comps])
    lwait = np.array([c["launch_s"] - c["arrival_s"] for c in comps])
    stall_main = longest_stall_ms(comps)
    sweep = []
    for ld in SERVING_LOADS:
        cs, lt, sp = open_loop(ld)
        sweep.append({"load": ld, "arrival_rate_per_s": round(ld * capacity, 1),
                      "gflops": round(fl.sum() / sp / 1e9, 1),
                      "p50_ms": round(float(np.percentile(lt, 50)) * 1e3, 3),
                      "p90_ms": round(float(np.percentile(lt, 90)) * 1e3, 3),
                      "p99_ms": round(float(np.percentile(lt, 99)) * 1e3, 3),
                      "longest_stall_ms": longest_stall_ms(cs)})
    srv.close()
    del a_pool, c_pool, packed
    torch.cuda.empty_cache()
    return {"workload": f"{N} FP32 TSMM requests, Poisson arrivals at {load:.2f} x measured capacity, "
                        "m log-uniform [1024, 262144], 32 resident packed B with k log-uniform [64, 8192], "
                        "n log-uniform [1, 64], beta = 1 for every third request; 40 GB admission budget; "
                        f"grouped launches (one block per work item) on {num_streams} lanes",
            "gflops": round(fl.sum() / span / 1e9, 1), "span_ms": round(span * 1e3, 2),
            "total_gflop": round(fl.sum() / 1e9, 1),
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)) * 1e3, 3),
                           "p90": round(float(np.percentile(lat, 90)) * 1e3, 3),
                           "p99": round(float(np.percentile(lat, 99)) * 1e3, 3),
                           "mean": round(float(lat.mean()) * 1e3, 3),
                           "queue_wait_p99": round(float(np.percentile(qwait, 99)) * 1e3, 3),
                           "launch_wait_p50": round(float(np.percentile(lwait, 50)) * 1e3, 3),
                           "launch_wait_p99": round(float(np.percentile(lwait, 99)) * 1e3, 3),
                           "longest_stall_ms": stall_main},
            "capacity": {"requests_per_s": round(capacity, 1), "gflops": round(cap_gflops, 1),
                         "makespan_ms": round(makespan * 1e3, 2)},
            "arrival_rate_per_s": round(lam, 1),
            "load_sweep": sweep,
            "plans": f"autotuned: {len(seen)} shapes (one per packed B and quarter octave of m), "
                     f"{tune_s:.1f} s, before the sessions",
            "a_storage": "windows of one read-only resident pool, each charged in full to the budget"}


def run_serving(args):
    """The serving workload alone (see serving_session), as its own JSON line."""
    import torch

    import paper_2208_08088_gb300 as tsmm

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    r = serving_session(args, tsmm, torch, args.requests, args.load, args.streams)
    line = {"metric": METRIC, "value": r["gflops"], "unit": UNIT, "n_gpus": 1,
            "steps": 1, "warmup": 1, "ms_per_step": r["span_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving: " + r["workload"], "total_gflop": r["total_gflop"],
                       "plans": r["plans"], "a_storage": r["a_storage"]},
            "latency_ms": r["latency_ms"], "capacity": r["capacity"],
            "arrival_rate_per_s": r["arrival_rate_per_s"], "load_sweep": r["load_sweep"]}
    print(json.dumps(line))
    return 0


# (n, problems, largest m) of each grouped mix
GROUPED_MIXES = [(1, 40, 65536), (6, 40, 65536), (16, 40, 65536), (40, 40, 65536), (64, 20, 262144),
                 (16, 40, 8192)]


def run_grouped(args):
    """Grouped execution against back-to-back single launches, as its own JSON
    line.  Each mix: FP32 problems with the same n, m log-uniform in [1024,
    largest m] (odd), k log-uniform in [64, 8192], beta = 0, drawn from a
    seed; once with lda = m (A not describable by a tensor map) and once with lda
    rounded up to a multiple of 4.  Both forms run on one stream; the median of
    7 timed repetitions (CUDA events) after one untimed; every mix's inputs are
    larger than L2."""
    import torch

    import paper_2208_08088_gb300 as tsmm
    import tsmm_inputs as ti

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()

    def timed(fn, reps=7):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    rng = np.random.default_rng(2208)
    mixes, total_fl, total_ms = [], 0.0, 0.0
    for mi, (n, count, mmax) in enumerate(GROUPED_MIXES):
        for aligned in (False, True):
            items, plans, keep = [], [], []
            fl = byts = 0.0
            for i in range(count):
                m = int(np.exp(rng.uniform(np.log(1024), np.log(mmax)))) | 1
                k = int(np.exp(rng.uniform(np.log(64), np.log(8192))))
                ld = (m + 3) // 4 * 4 if aligned else m
                buf = torch.empty(ld * k, dtype=torch.float32, device="cuda")
                ti.fill_torch(buf, ti.SEED_A + 1000 * mi + i, "uniform")
                A = buf.as_strided((m, k), (1, ld))
                B = torch.empty((n, k), dtype=torch.float32, device="cuda")
                ti.fill_torch(B, ti.SEED_B + 1000 * mi + i, "uniform")
                pb = tsmm.pack_b(B.t())
                C = torch.zeros((n, m), dtype=torch.float32, device="cuda").t()
                pl = tsmm.plan(m, n, k, torch.float32)
                plans.append(pl)
                keep.append(buf)
                items.append((pl, 1.0, A, pb, 0.0, C))
                fl += 2.0 * m * n * k
                byts += 4.0 * (m * k + k * n + m * n)
            t_grouped = timed(lambda: tsmm.execute_grouped(items))

            def singles():
                for it in items:
                    tsmm.execute(*it)

            t_single = timed(singles)
            for pl in plans:
                pl.check()
            total_fl += fl
            total_ms += t_grouped
            mixes.append({"n": n, "problems": count, "m_max": mmax, "lda": "m rounded up to 4" if aligned else "m",
                          "gflop": round(fl / 1e9, 2), "grouped_ms": round(t_grouped, 3),
                          "single_launches_ms": round(t_single, 3),
                          "grouped_GBs": round(byts / t_grouped / 1e6, 1),
                          "single_launches_GBs": round(byts / t_single / 1e6, 1),
                          "speedup": round(t_single / t_grouped, 2)})
            del items, plans, keep
            torch.cuda.empty_cache()
    line = {"metric": METRIC, "value": total_fl / total_ms / 1e6, "unit": UNIT, "n_gpus": 1,
            "steps": 7, "warmup": 1, "ms_per_step": total_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "grouped execution vs back-to-back single launches: FP32 mixes of 20-40 "
                                   "problems, m log-uniform [1024, m_max], k log-uniform [64, 8192], beta = 0, "
                                   "lda = m and lda rounded up to 4; inputs larger than L2",
                       "mixes": len(mixes)},
            "mixes": mixes}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.workload == "serving" and args.impl != "reference":
        return run_serving(args)
    if args.workload == "grouped" and args.impl != "reference":
        return run_grouped(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "precision":
        return run_precision(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
