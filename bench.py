"""Benchmark of the pre-packed tall-and-skinny GEMM on GB300.

Workload (default, FP32): the memory-bound sweep  m = k = 32768,
n in {1,2,4,8,16,32,64}, beta in {0,1}, alpha = 1, A and C0 uniform[-1,1] from
the shared seeded generator, B packed once per n (packing untimed, as in the
paper's evaluation, Section V).  One step = one tsmm_execute per (n, beta)
point, 14 launches over a resident 4 GiB A (larger than L2, so no flush is
needed between calls).  `--dtype f64` runs the same sweep in FP64.
`--workload rankk` runs m = n = 16384, k in {4,...,128}, beta = 1.

Metric: GFLOP/s by Eq. 7 (2*m*n*k / t) aggregated over the step, with the
roofline of the dominant kernel; the CPU oracle on the host cores is timed on
a bounded sample of the same workload as a baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype f32|f64]
                  [--workload tall|rankk] [--impl ours|reference]

Under torchrun (N > 1) every rank runs the full workload on its own GPU
(independent problems, weak scaling, no collective on the data path); rank 0
prints the JSON line with value = all ranks' flops / max-over-ranks time.
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
    p.add_argument("--workload", choices=["tall", "rankk", "precision", "serving"], default="tall")
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
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
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
    if args.size or args.only or args.beta is not None:
        return "reduced case for profiling: " + ", ".join(
            f"m={m} n={n} k={k} beta={b}" for (m, n, k, b) in workload_points(args))
    if args.workload == "tall":
        mode = "" if args.precision == "native" else " in the BF16x3 tensor-core mode"
        return (f"memory-bound sweep {args.dtype.upper()} m=k=32768, n in {SWEEP_N}, "
                f"beta in {{0,1}}, alpha=1, B pre-packed and reused{mode}")
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
def oracle_sample(args, A_dev, budget_s=10.0):
    """Time the CPU oracle, as it stands, on a bounded sample of the workload:
    the first m_s rows of every point (same n, k, beta), with m_s sized from a
    short calibration run so the sample takes about `budget_s` seconds.  The
    rows of A are copied from the resident device A (same seeded generator)."""
    import torch

    import oracle
    import tsmm_inputs as ti

    npdt = np.float32 if args.dtype == "f32" else np.float64
    pts = workload_points(args)
    cores = oracle.num_threads()

    def rows_of(m, k, m_s):
        a = A_dev[(m, k)][:m_s]  # column-major m_s x k view
        return np.asfortranarray(a.t().contiguous().cpu().numpy().T)

    m0, n0, k0, _ = max(pts, key=lambda p: p[1] * p[2])
    m_cal = min(m0, 512 * max(1, min(cores, 16)))
    Acal = rows_of(m0, k0, m_cal)
    Bcal = ti.matrix_np(k0, n0, ti.SEED_B, "uniform", npdt)
    t0 = time.perf_counter()
    oracle.tsmm(1.0, Acal, Bcal, 0.0, None)
    rate = flops(m_cal, n0, k0) / max(time.perf_counter() - t0, 1e-4)
    per_row = sum(flops(1, n, k) for (_, n, k, _) in pts)
    m_s = int(budget_s * rate / per_row) // 256 * 256
    m_s = max(256, min(m0, 8192, m_s))
    sample = {}
    for (m, n, k, beta) in pts:
        if (m, k) not in sample:
            sample[(m, k)] = rows_of(m, k, m_s)
    Bs = {(n, k): ti.matrix_np(k, n, ti.SEED_B, "uniform", npdt) for (_, n, k, _) in pts}
    C0s = {(m, n): np.asfortranarray(ti.rows_np(np.arange(m_s), m, n, ti.SEED_C0, "uniform", npdt))
           for (m, n, _, _) in pts}
    t0 = time.perf_counter()
    fl = 0.0
    for (m, n, k, beta) in pts:
        oracle.tsmm(1.0, sample[(m, k)], Bs[(n, k)], beta, C0s[(m, n)] if beta != 0 else None)
        fl += flops(m_s, n, k)
    t = time.perf_counter() - t0
    del torch
    return {"value": round(fl / t / 1e9, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {m_s} rows of each of the {len(pts)} points of the workload "
                      f"({fl / 1e9:.1f} GFLOP in {t:.1f} s)"}


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
    kmax = max(k for (_, _, k, _) in pts)
    # one step = the first m_s rows of every point; m_s sized for ~4 s per step
    m_s = 256 * max(1, min(cores, 16)) // (2 if args.dtype == "f64" else 1)
    m_s = min(m_s, pts[0][0])
    A = ti.matrix_np(m_s, kmax, ti.SEED_A, "uniform", npdt)
    Bs = {(n, k): ti.matrix_np(k, n, ti.SEED_B, "uniform", npdt) for (_, n, k, _) in pts}
    C0s = {n: ti.matrix_np(m_s, n, ti.SEED_C0, "uniform", npdt) for (_, n, _, _) in pts}

    def step():
        fl = 0.0
        for (m, n, k, beta) in pts:
            Ak = A if k == kmax else np.asfortranarray(A[:, :k])
            oracle.tsmm(1.0, Ak, Bs[(n, k)], beta, C0s[n] if beta != 0 else None)
            fl += flops(m_s, n, k)
        return fl

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    fl = 0.0
    for _ in range(args.steps):
        fl += step()
    t = time.perf_counter() - t0
    value = fl / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": workload_name(args), "sample_rows": m_s},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {m_s} rows of every point of the workload per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------- our arm
KERNEL_SOURCES = {  # the files that define each kernel family's device code
    "tall": ["tsmm_tall.cuh", "tsmm_device.cuh"],
    "rankk": ["tsmm_rankk.cu", "tsmm_device.cuh"],
}


def kernel_source_hash(family):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2208_08088_gb300", "csrc")
    for name in KERNEL_SOURCES[family]:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
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
    import tsmm_inputs as ti

    tdt = torch.float32 if args.dtype == "f32" else torch.float64
    es = 4 if args.dtype == "f32" else 8
    pts = workload_points(args)
    stream = torch.cuda.current_stream()

    def dmat(rows, cols, seed):
        t = torch.empty((cols, rows), dtype=tdt, device="cuda")
        ti.fill_torch(t, seed, "uniform")
        return t.t()

    # resident inputs: one A per distinct k, one packed B + plan + C0 per point
    A = {}
    for (m, n, k, beta) in pts:
        if (m, k) not in A:
            A[(m, k)] = dmat(m, k, ti.SEED_A)
    packed, plans, C = {}, {}, {}
    pack_ms = {}  # tsmm_pack_b time per B (once per B, outside the timed steps)
    prec = tsmm.PREC_BF16X3 if args.precision == "bf16x3" else tsmm.PREC_NATIVE
    for (m, n, k, beta) in pts:
        if (n, k) not in packed:
            Bsrc = dmat(k, n, ti.SEED_B)
            tsmm.pack_b(Bsrc, precision=prec)  # first call: kernel attributes, module load
            p0 = torch.cuda.Event(enable_timing=True)
            p1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            p0.record(stream)
            packed[(n, k)] = tsmm.pack_b(Bsrc, precision=prec)
            p1.record(stream)
            torch.cuda.synchronize()
            pack_ms[f"n={n},k={k}"] = round(p0.elapsed_time(p1), 4)
            plans[(m, n, k)] = tsmm.plan(m, n, k, tdt, precision=prec)
            C[(m, n)] = dmat(m, n, ti.SEED_C0)  # C0; beta = 1 updates it in place
    torch.cuda.synchronize()

    def one(pt):
        m, n, k, beta = pt
        tsmm.execute(plans[(m, n, k)], 1.0, A[(m, k)], packed[(n, k)], beta, C[(m, n)])

    # warm-up
    for _ in range(args.warmup):
        for pt in pts:
            one(pt)
    torch.cuda.synchronize()
    for pl in plans.values():
        pl.check()

    ev = {pt: [] for pt in pts}
    sampler = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
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
    clocks = sampler.stop()
    elapsed_ms = start.elapsed_time(stop)
    for pl in plans.values():
        pl.check()
    step_flops = sum(flops(m, n, k) for (m, n, k, _) in pts)
    elapsed_ms, value = aggregate_over_ranks(elapsed_ms, step_flops, args.steps, world)
    launches = args.steps * sum(plans[(m, n, k)].launches_per_execute() for (m, n, k, _) in pts)

    hbm_peak, hbm_src = load_peaks()
    fp32_peak_tf = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    fp_peak_tf = fp32_peak_tf if args.dtype == "f32" else FP64_NOMINAL_TFLOPS
    if args.precision == "bf16x3":
        # three BF16 tensor-core products per FP32 product: the measured dense
        # BF16 peak / 3 (MEASURED_PEAKS.json bf16_tflops)
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                fp_peak_tf = float(json.load(f)["bf16_tflops"]) / 3.0
        except Exception:
            fp_peak_tf = 1900.0 / 3.0

    points = []
    for pt in pts:
        m, n, k, beta = pt
        durs = [a.elapsed_time(b) for (a, b) in ev[pt]]
        avg_ms = sum(durs) / len(durs)
        gb = alg_bytes(m, n, k, beta, es) / 1e9
        gbs = gb / (avg_ms * 1e-3)
        tf = flops(m, n, k) / (avg_ms * 1e-3) / 1e12
        # which roof binds: time at the HBM roof vs time at the FP roof
        t_hbm = gb / hbm_peak
        t_fp = flops(m, n, k) / (fp_peak_tf * 1e12)
        bound = "hbm" if t_hbm >= t_fp else "alu"
        frac = (gbs / hbm_peak) if bound == "hbm" else (tf / fp_peak_tf)
        points.append({"m": m, "n": n, "k": k, "beta": beta, "avg_ms": round(avg_ms, 4),
                       "gflops": round(tf * 1e3, 1), "alg_gbs": round(gbs, 1),
                       "bound": bound, "frac": round(frac, 4), "total_ms": sum(durs)})
    dom = max(points, key=lambda p: p["total_ms"])
    m, n, k, beta = dom["m"], dom["n"], dom["k"], dom["beta"]
    kernel_key = f"{args.workload}_{args.dtype}_n{n}_k{k}"
    if dom["bound"] == "hbm":
        roof = {"bound": "hbm", "achieved": dom["alg_gbs"], "peak": hbm_peak, "unit": "GB/s",
                "frac": round(dom["alg_gbs"] / hbm_peak, 4),
                "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        ach = dom["gflops"] / 1e3
        roof = {"bound": "alu", "achieved": round(ach, 2), "peak": round(fp_peak_tf, 2),
                "unit": "TFLOP/s", "frac": round(ach / fp_peak_tf, 4),
                "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"
                                if args.dtype == "f32" else "nominal GB300 FP64 rate 1.25 TFLOP/s")}
    traffic = recorded_traffic(kernel_key, args.workload)
    roof["traffic"] = traffic
    roof["kernel"] = f"{'tall' if args.workload == 'tall' else 'rankk'} {args.dtype} m={m} n={n} k={k} beta={beta}"
    roof["alg_bytes_per_launch"] = alg_bytes(m, n, k, beta, es)
    for p in points:
        del p["total_ms"]

    # ---------------- end to end: host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, tsmm, torch, tdt, es, pts, A, packed, plans, world)

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(elapsed_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": workload_name(args), "launches_per_step": len(pts),
                   "alpha": 1.0, "l2": "no flush: each launch streams a >= 1 GiB operand, "
                                         "larger than the 129 MB L2",
                   "parallelism": f"replicas x{world} (independent problems per GPU)"},
        "clocks": clocks, "gpu_launches": launches, "e2e": e2e, "roofline": roof,
        "points": points, "pack_ms": pack_ms,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = oracle_sample(args, A)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_e2e(args, tsmm, torch, tdt, es, pts, A, packed, plans, world):
    """Same metric through the public API with HOST buffers: each step copies
    A (once, shared by every point) and the C0 of each beta != 0 point from
    pinned host memory, executes, and reads every C back.  The inputs stream
    through two sets of device buffers on a copy stream, so step s+1's inputs
    cross the host link while step s computes (a streaming caller's pipeline);
    the read-backs run on the compute stream, whose copies use the other
    direction of the link.  The timed region runs from before the first copy
    to after the last read-back."""
    stream = torch.cuda.current_stream()
    copy_stream = torch.cuda.Stream()
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
    steps = max(3, args.steps // 2)
    a_ready = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]

    def copy_in(s):
        b = s % 2
        with torch.cuda.stream(copy_stream):
            if s >= 2:
                copy_stream.wait_event(done[b])  # step s-2 is done with these buffers
            for pt in pts:
                if pt[3] != 0:
                    devC[b][pt].copy_(hostC0[pt], non_blocking=True)
            for key in hostA:
                devA[b][key].copy_(hostA[key], non_blocking=True)
            a_ready[b].record(copy_stream)

    def compute(s):
        b = s % 2
        stream.wait_event(a_ready[b])
        for pt in pts:
            m, n, k, beta = pt
            tsmm.execute(plans[(m, n, k)], 1.0, devA[b][(m, k)], packed[(n, k)], beta, devC[b][pt])
            hostC[pt].copy_(devC[b][pt], non_blocking=True)
        done[b].record(stream)

    def run(nsteps):
        copy_stream.wait_stream(stream)
        copy_in(0)
        for s in range(nsteps):
            if s + 1 < nsteps:
                copy_in(s + 1)
            compute(s)

    run(2)  # warm-up
    torch.cuda.synchronize()
    # the host link's own rate at this moment (uploads of A, nothing else running;
    # the best of three, as a one-off copy can catch an unrelated stall)
    key0 = next(iter(hostA))
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    best_ms = None
    for _ in range(3):
        a.record(stream)
        devA[0][key0].copy_(hostA[key0], non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b)
        best_ms = t if best_ms is None else min(best_ms, t)
    link_gbs = hostA[key0].numel() * es / (best_ms * 1e-3) / 1e9
    if world > 1:
        torch.distributed.barrier()
    a.record(stream)
    run(steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    fl = sum(flops(m, n, k) for (m, n, k, _) in pts)
    del hostA, devA, devC
    return {"value": round(world * fl * steps / (ms * 1e-3) / 1e9, 1), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "ms_per_step": round(ms / steps, 3), "host_to_device_gbs": round(link_gbs, 1),
            "pipeline": "inputs double-buffered on a copy stream: step s+1's upload overlaps step s"}


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


def run_serving(args):
    """Serving workload: 32 device-resident packed B (k log-uniform in
    [64, 8192], n log-uniform in [1, 64], drawn once from a seed); requests pick a
    B uniformly and m log-uniform in [1024, 262144]; FP32, alpha = 1, beta = 0.
    The server admits under a 40 GB budget and batches continuously (grouped
    persistent launches on 4 streams).  Capacity is measured with every request
    arriving at once; then Poisson arrivals at `--load` x capacity give the
    p50 / p99 arrival-to-completion latency and the aggregate GFLOP/s."""
    import torch

    import paper_2208_08088_gb300 as tsmm
    import tsmm_inputs as ti

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rng = np.random.default_rng(2208)
    NB = 32
    ks = np.round(np.exp(rng.uniform(np.log(64), np.log(8192), NB))).astype(np.int64)
    ns = np.round(np.exp(rng.uniform(np.log(1), np.log(64), NB))).astype(np.int64)
    packed = []
    for i in range(NB):
        B = torch.empty((int(ns[i]), int(ks[i])), dtype=torch.float32, device="cuda")
        ti.fill_torch(B, 100 + i, "uniform")
        packed.append(tsmm.pack_b(B.t()))
    N = args.requests
    b_idx = rng.integers(NB, size=N)
    ms = np.round(np.exp(rng.uniform(np.log(1024), np.log(262144), N))).astype(np.int64)
    mk = ms * ks[b_idx]
    mn = ms * ns[b_idx]
    fl = 2.0 * ms * ns[b_idx] * ks[b_idx]
    # A: windows into one resident pool (synthetic inputs already on the device);
    # C: disjoint windows of a pool larger than the budget, reused in a ring
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
            arr[i] = tsmm.Request(i, packed[b_idx[i]].handle, m, 1.0, 0.0, a_base + 4 * int(a_off[i]), m,
                                  c_base + 4 * int(c_off[i]), m, float(arrivals[i]))
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
    srv = tsmm.Server(budget_bytes=budget, num_streams=args.streams, max_batch=48, arena_bytes=1 << 30)

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
    # open loop: Poisson arrivals at load x capacity
    lam = args.load * capacity
    gaps = rng.exponential(1.0 / lam, N)
    t0 = tsmm.tsmm_server_clock() + 0.05
    arrivals = t0 + np.cumsum(gaps)
    comps = session(arrivals)
    lat = np.array([c["complete_s"] - c["arrival_s"] for c in comps])
    qwait = np.array([c["admit_s"] - c["arrival_s"] for c in comps])
    lwait = np.array([c["launch_s"] - c["arrival_s"] for c in comps])
    span = max(c["complete_s"] for c in comps) - min(c["arrival_s"] for c in comps)
    srv.close()
    line = {"metric": METRIC, "value": round(fl.sum() / span / 1e9, 1), "unit": UNIT, "n_gpus": 1,
            "steps": 1, "warmup": 1, "ms_per_step": round(span * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving: {N} FP32 TSMM requests, Poisson arrivals at "
                                   f"{args.load:.2f} x measured capacity, m log-uniform [1024, 262144], "
                                   "32 resident packed B with k log-uniform [64, 8192], n log-uniform "
                                   f"[1, 64]; 40 GB admission budget; grouped persistent launches on {args.streams} streams",
                       "total_gflop": round(fl.sum() / 1e9, 1),
                       "plans": f"autotuned: {len(seen)} shapes (one per packed B and quarter octave of m), "
                                f"{tune_s:.1f} s, before the sessions"},
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)) * 1e3, 3),
                           "p90": round(float(np.percentile(lat, 90)) * 1e3, 3),
                           "p99": round(float(np.percentile(lat, 99)) * 1e3, 3),
                           "mean": round(float(lat.mean()) * 1e3, 3),
                           "queue_wait_p99": round(float(np.percentile(qwait, 99)) * 1e3, 3),
                           "launch_wait_p50": round(float(np.percentile(lwait, 50)) * 1e3, 3),
                           "launch_wait_p99": round(float(np.percentile(lwait, 99)) * 1e3, 3)},
            "capacity": {"requests_per_s": round(capacity, 1), "gflops": round(cap_gflops, 1),
                         "makespan_ms": round(makespan * 1e3, 2)},
            "arrival_rate_per_s": round(lam, 1)}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.workload == "serving" and args.impl != "reference":
        return run_serving(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "precision":
        return run_precision(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
