#!/usr/bin/env python
"""Benchmark of the H² × dense-block product (H2MM) and the block-CG solve.

Workload: n = 65536 points uniform on the unit sphere (seed 0), kernel
exp(-|x-y|/0.5) + 1e-2·I, leaf size 64, eta = 2, tensor Chebyshev order q = 4
(k = 64), m = 32 N(0,1) right-hand sides per GPU.

A timed step is one product Y += A·X (all phases: forward transformation,
transfer passes, coupling, nearfield, backward transformation) through the C
ABI on device-resident blocks, in the compute precision of the mixed solve
(FP32).  value = algorithmic H2MM GFLOP/s summed over ranks (weak scaling: each
rank owns its own 32 columns; columns never communicate).  The line also
carries the FP64 product rate, the block-CG time to a 1e-8 relative residual
for the mixed-precision and the FP64 solve, the roofline of the dominant
kernel (coupling), the end-to-end rate through the C ABI on pinned host
buffers, and the FP64 CPU oracle timed on this host as a baseline.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from workloads import CONFIGS, gaussian_rhs, sphere_points  # noqa: E402

WORKLOAD = "precision_n65536"
METRIC = "H2MM GFLOP/s (n=65536, q=4, m=32 per GPU; block-CG time to 1e-8 mixed vs FP64 reported alongside)"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
SM_COUNT = 152
FP32_FMA_PER_CLK_SM = 128
FP64_NOMINAL_TFLOPS = 1.25
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of the FP32 coupling kernel
# on precision_n65536 (k_tc_gemm<4,1>: the coupling with the transfer items above the upward
# cut), with the SHA-256 (first 16 hex digits) of the kernel's sources and of the work-list
# builder when the counters were taken.  The line reports the bytes only while the sources
# still hash to that value; after a change they are stale and `traffic` is null.
TC_F32_COUPLING_DRAM = {
    "kernel": "k_tc_gemm<4,1>",
    "bytes": 666707456,  # 654.177 MB read + 12.531 MB written
    "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
               "--clock-control none --kernel-name-base demangled -k regex:k_tc_gemm<(int)[41], (int)1> -c 2 "
               "python bench.py --steps 2 --warmup 1 --no-solve --no-cpu-baseline --no-batch --no-complex "
               "(the first of the two launches)",
    "sources": ("paper_2509_17257_gb300/csrc/h2_tc.cu", "paper_2509_17257_gb300/csrc/h2_async.cuh",
                "paper_2509_17257_gb300/csrc/h2_build.cu"),
    "source_sha16": "36c0f17dbfb27324",
}


def _sources_sha16(paths) -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the CPU baseline."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def workload_counts_from_info(info) -> dict:
    return {key: int(info[key]) for key in ("n_clusters", "n_adm", "n_near", "nnz_near", "depth")}


def bench_config(workload: str, cfg: dict, counts: dict, ws: int) -> dict:
    """The `config` dict of the bench line; both arms build it from the workload and the
    tree counts only, so the two lines name the same configuration."""
    k = cfg["q"] ** 3
    f32_bytes = 4 * (cfg["n"] * k + counts["n_clusters"] * k * k + counts["n_adm"] * k * k + counts["nnz_near"])
    return {"workload": workload, "n": cfg["n"], "q": cfg["q"], "k": k, "m_per_gpu": cfg["m"], "leaf": cfg["leaf"],
            "eta": cfg["eta"], "kernel": "exp(-r/0.5)+1e-2*I", "parallelism": f"column shards x{ws}",
            "l2": f"inputs larger than L2 (matrix data {f32_bytes / 1e9:.2f} GB FP32, "
                  f"{2 * f32_bytes / 1e9:.2f} GB FP64)",
            **counts}


def product_bytes(n, k, m, nc, n_adm, nnz_near, elt, elt_x=8, elt_acc=4):
    """Algorithmic bytes of one product: every matrix once (V twice: forward and backward),
    X read and Y read and written once, and the coefficient blocks x̂ and ŷ each written and
    read once."""
    return (elt * (2 * n * k + (nc - 1) * k * k + n_adm * k * k + nnz_near) + elt_x * 3 * n * m
            + 4 * nc * k * m * elt_acc)


def phase_bytes(n, k, m, nc, n_leaves, n_adm, nnz_near, elt, n_above=0):
    """Algorithmic bytes of each phase of the tensor-core FP32/BF16 product, as timed by
    h2_timing (coefficients, gathered X and leaf results in FP32; the caller's X, Y in FP64).
    n_above: clusters above the upward cut computed in the coupling launch (hybrid)."""
    a = 4  # coefficient / gathered-block element size
    return {
        "gather": 8 * n * m + a * n * m,
        "leaf_fwd": (elt * (n * k + (nc - 1 - 2 * n_above) * k * k) + a * n * m
                     + a * (nc - n_above) * k * m),  # upward pass fused in
        "coupling": elt * (n_adm + 2 * n_above) * k * k + 2 * a * nc * k * m + a * n_above * k * m,
        "down": elt * (nc - 1) * k * k + 2 * a * nc * k * m,
        "leaf_bwd_near": (elt * (n * k + nnz_near) + a * n_leaves * k * m + 2 * a * n * m
                          + a * n * m + 8 * n * m + 2 * 8 * n * m),  # leaf kernel, then the scatter into Y
    }


def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
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
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_rhs(n: int, m: int, seed: int, rank: int) -> np.ndarray:
    """Rank `rank`'s m right-hand sides: its own column shard of the job's block
    (weak scaling; the columns of a block product never interact)."""
    return gaussian_rhs(n, m, seed + 1000 * rank)


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The slowest rank's value, on every rank (x itself without a process group)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gflops(flops_per_rank_step: float, seconds_per_step: float, world_size: int) -> float:
    """Whole-job rate: the flops of every rank's step over the slowest rank's step time."""
    return flops_per_rank_step * world_size / seconds_per_step / 1e9


def _cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_flops(cfg, c) -> float:
    k = cfg["q"] ** 3
    return cfg["m"] * (4.0 * c["n"] * k + 4.0 * (c["n_clusters"] - 1) * k * k + 2.0 * c["n_adm"] * k * k
                       + 2.0 * c["nnz_near"] + 2.0 * c["n"])


def oracle_products(cfg, steps: int, warmup: int):
    """Time the FP64 CPU oracle's product on the workload (build untimed).
    Returns (flops per product, list of seconds, build seconds, oracle matrix)."""
    from oracle import h2_oracle as O

    pts = sphere_points(cfg["n"], cfg["point_seed"])
    t0 = time.perf_counter()
    H = O.H2Matrix(pts, q=cfg["q"], leaf_size=cfg["leaf"], eta=cfg["eta"], sigma=cfg["sigma"],
                   length=cfg["length"])
    build_s = time.perf_counter() - t0
    X = gaussian_rhs(cfg["n"], cfg["m"], cfg["rhs_seed"])
    for _ in range(warmup):
        O.h2mm(H, 1.0, X)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        O.h2mm(H, 1.0, X)
        times.append(time.perf_counter() - t0)
    return _oracle_flops(cfg, H.counts()), times, build_s, H


_SINGLE_THREAD_SNIPPET = """
import json, statistics, sys, time
sys.path.insert(0, {root!r})
from oracle import h2_oracle as O
from workloads import CONFIGS, gaussian_rhs, sphere_points
cfg = CONFIGS["fp64_n4096"]
H = O.H2Matrix(sphere_points(cfg["n"], cfg["point_seed"]), q=cfg["q"], leaf_size=cfg["leaf"], eta=cfg["eta"],
               sigma=cfg["sigma"], length=cfg["length"])
X = gaussian_rhs(cfg["n"], cfg["m"], cfg["rhs_seed"])
O.h2mm(H, 1.0, X)
ts = []
for _ in range(5):
    t0 = time.perf_counter(); O.h2mm(H, 1.0, X); ts.append(time.perf_counter() - t0)
print(json.dumps({{"median_s": statistics.median(ts), "counts": H.counts()}}))
"""


def cpu_baseline_extras(H2, cfg2, fp64_iterations):
    """The oracle's block CG and single-thread figures beside the product rate:
    the block CG to 1e-8 on the n = 4096 workload (full solve), the per-iteration
    cost on the bench workload (3 iterations, extrapolated to the iteration count of
    the GPU FP64 column-wise solve when one ran), and the n = 4096 product on one
    thread (a child process with every BLAS / OpenMP pool at one thread)."""
    from oracle import h2_oracle as O

    out = {}
    c1 = CONFIGS["fp64_n4096"]
    H1 = O.H2Matrix(sphere_points(c1["n"], c1["point_seed"]), q=c1["q"], leaf_size=c1["leaf"], eta=c1["eta"],
                    sigma=c1["sigma"], length=c1["length"])
    B1 = gaussian_rhs(c1["n"], c1["m"], c1["rhs_seed"] + 7)
    t0 = time.perf_counter()
    r1 = O.block_cg(lambda Z: O.h2mm(H1, 1.0, Z), B1, tol=1e-8, max_iter=5000)
    out["block_cg_fp64_n4096"] = {"seconds": round(time.perf_counter() - t0, 3), "iterations": int(r1.iterations),
                                  "status": r1.status, "m": c1["m"], "kind": "measured"}
    B2 = gaussian_rhs(cfg2["n"], cfg2["m"], cfg2["rhs_seed"] + 7)
    t0 = time.perf_counter()
    r2 = O.block_cg(lambda Z: O.h2mm(H2, 1.0, Z), B2, tol=1e-8, max_iter=3)
    per_it = (time.perf_counter() - t0) / max(int(r2.iterations), 1)
    row = {"seconds_per_iteration": round(per_it, 4), "iterations_timed": int(r2.iterations), "m": cfg2["m"]}
    if fp64_iterations:
        row.update(iterations=int(fp64_iterations), seconds=round(per_it * fp64_iterations, 1),
                   kind="extrapolated: oracle seconds per iteration x the GPU FP64 column-wise solve's "
                        "iteration count")
    out[f"block_cg_fp64_n{cfg2['n']}"] = row
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", _SINGLE_THREAD_SNIPPET.format(root=ROOT)], env=env,
                           capture_output=True, text=True, timeout=600)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        f1 = _oracle_flops(c1, d["counts"])
        out["single_thread_n4096"] = {"value": round(f1 / d["median_s"] / 1e9, 3), "unit": "GFLOP/s",
                                      "cores": 1, "sample": "median of 5 FP64 oracle products at n=4096, q=3, m=8"}
    except Exception as e:  # reported, not fatal: the main baseline stands
        out["single_thread_n4096"] = {"error": str(e)[:200]}
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    workload = args.workload
    cfg = CONFIGS[workload]
    flops, times, build_s, H = oracle_products(cfg, args.steps, args.warmup)
    t = statistics.median(times)
    v = flops / t / 1e9
    cores = _cpu_cores()
    c = H.counts()
    sample = (f"median of {args.steps} FP64 oracle products at n={cfg['n']}, q={cfg['q']}, m={cfg['m']} after "
              f"{args.warmup} warm-up; oracle build {build_s:.1f} s untimed; CPU {_cpu_model()}")
    line = {
        "metric": _metric(workload, cfg), "value": round(v, 3), "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": bench_config(workload, cfg, {key: int(c[key]) for key in
                                               ("n_clusters", "n_adm", "n_near", "nnz_near", "depth")}, args.gpus),
        "cpu_baseline": {"value": round(v, 3), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu_model": _cpu_model()},
        "e2e": {"value": round(v, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _metric(workload, cfg):
    if workload == WORKLOAD:
        return METRIC
    return (f"H2MM GFLOP/s (n={cfg['n']}, q={cfg['q']}, m={cfg['m']} per GPU; block-CG time to 1e-8 mixed vs FP64 "
            f"reported alongside)")


def run_ours(args):
    import torch

    import paper_2509_17257_gb300 as P

    ws, rank, local = _dist()
    if ws != args.gpus:
        args.gpus = ws
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    workload = args.workload
    cfg = CONFIGS[workload]
    n, m = cfg["n"], cfg["m"]
    peaks, peak_kind = _peaks()
    metric = _metric(workload, cfg)

    pts = sphere_points(n, cfg["point_seed"])
    t0 = time.perf_counter()
    G = P.H2Matrix(pts, q=cfg["q"], leaf_size=cfg["leaf"], eta=cfg["eta"], length=cfg["length"],
                   sigma=cfg["sigma"], precisions=("f32", "bf16"))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    info = G.info
    k = info["k"]
    X = torch.from_numpy(rank_rhs(n, m, cfg["rhs_seed"], rank)).to(dev)
    Y = torch.zeros_like(X)
    flops_step = G.flops(m)
    stream = torch.cuda.current_stream()

    def timed(dtype, steps, warmup, timing=False):
        for _ in range(warmup):
            G.matmul(X, Y, dtype=dtype)
        if timing:
            P.h2_timing_query(G.handle, reset=True)
            P.h2_timing_enable(G.handle, True)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            G.matmul(X, Y, dtype=dtype)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ms = e0.elapsed_time(e1) / steps
        phases = None
        if timing:
            P.h2_timing_enable(G.handle, False)
            phases, calls = P.h2_timing_query(G.handle, reset=True)
            phases = {kk: v / max(calls, 1) for kk, v in phases.items()}
        ms = max_over_ranks(ms, dist, dev)
        return ms, phases

    dtype = args.dtype
    clocks = ClockSampler(local)
    clocks.start()
    ms, phases = timed(dtype, args.steps, args.warmup, timing=True)
    clk = clocks.stop()
    value = job_gflops(flops_step, ms * 1e-3, ws)

    # FP64 product rate (fewer steps: it is ~50x slower)
    k64 = max(3, min(args.steps, 10))
    ms64, phases64 = timed("f64", k64, 3, timing=True)
    value64 = job_gflops(flops_step, ms64 * 1e-3, ws)

    # BF16 tensor-core product rate
    msbf, phasesbf = timed("bf16", args.steps, 3, timing=True)
    valuebf = job_gflops(flops_step, msbf * 1e-3, ws)

    # FP32 product with the matrix-free coupling (S_b evaluated from the nodes in the kernel)
    mf = None
    if dtype == "f32" and info["launches_tc"] > 0:
        kmf = max(3, min(args.steps, 10))
        msmf, phasesmf = timed("f32mf", kmf, 3, timing=True)
        mf = {"value": round(job_gflops(flops_step, msmf * 1e-3, ws), 3), "unit": "GFLOP/s",
              "ms_per_step": round(msmf, 4), "coupling_kernel_ms": round(phasesmf["coupling_kernel"], 4),
              "kernel_evaluations_per_step": int(info["n_adm"] * info["k"] * info["k"]),
              "s_bytes_not_read": int(info["n_adm"] * info["k"] * info["k"] * 4)}

    # the complex product (K = C): the same points and tree with the Helmholtz kernel
    # exp(i kappa r) / (4 pi sqrt(r^2 + delta^2)), m complex columns, FP64 and FP32 on
    # the CUDA cores; the coupling kernel against the ALU peak of its precision
    cx = None
    if not args.no_complex and workload == WORKLOAD:
        cx = complex_products(P, torch, dev, pts, cfg, rank, dist, clk, peaks)

    # roofline of the dominant kernel: the coupling phase (one launch per product)
    elt = 8 if dtype == "f64" else 4
    n_adm, nc = info["n_adm"], info["n_clusters"]
    coup_bytes = elt * (n_adm * k * k + 2 * nc * k * m)
    coup_flops = 2.0 * n_adm * k * k * m
    # the FP32 tensor-core product's coupling launch also computes the clusters above the
    # upward cut (hybrid): two Eᵀ per cluster read, its x̂ written, 2·2k²m flops
    hybrid = dtype == "f32" and info["launches_tc"] > 0 and info["hybrid"] == 1
    n_above = int(info["n_above_cut"]) if hybrid else 0
    coup_bytes += elt * (2 * n_above * k * k + n_above * k * m)
    coup_flops += 4.0 * n_above * k * k * m
    # the coupling kernel's own launch (events around it alone; the phase also packs x̂)
    coup_ms = phases.get("coupling_kernel") or phases["coupling"]
    clock_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    hbm_peak = peaks["hbm_gbs"]
    tensor_path = dtype in ("f32", "bf16") and info["launches_tc"] > 0
    if dtype == "f64":
        alu_peak_tf = FP64_NOMINAL_TFLOPS
        alu_note = "FP64 nominal 1.25 TFLOP/s (recipe table)"
    else:
        alu_peak_tf = SM_COUNT * FP32_FMA_PER_CLK_SM * 2 * clock_mhz * 1e6 / 1e12
        alu_note = f"FP32 FFMA: 152 SM x 128 FMA/clk x 2 x {clock_mhz:.0f} MHz (median SM clock under load)"
    t_hbm = coup_bytes / (hbm_peak * 1e9)
    t_alu = coup_flops / (alu_peak_tf * 1e12)
    if tensor_path:
        t_alu = 0.0  # tensor-core MMAs: 2x TF32 (or 1x BF16) work at <= 1.1 PFLOP/s is far below the HBM time
    if t_alu >= t_hbm:
        achieved = coup_flops / (coup_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(alu_peak_tf, 2),
                "unit": "TFLOP/s", "frac": round(achieved / alu_peak_tf, 4), "traffic": None,
                "kernel": "k_coupling", "peak_source": alu_note}
    else:
        achieved = coup_bytes / (coup_ms * 1e-3) / 1e9
        # DRAM bytes (read + write) of one launch of the FP32 tensor-core coupling kernel on this
        # workload from an earlier ncu capture, reported only while the kernel's sources are the
        # ones it was taken on
        cap = TC_F32_COUPLING_DRAM
        sha_now = _sources_sha16(cap["sources"])
        fresh = sha_now == cap["source_sha16"]
        kname = "k_tc_gemm<4,1>" if hybrid else ("k_tc_gemm<0,1>" if tensor_path else "k_coupling")
        applies = tensor_path and dtype == "f32" and args.workload == WORKLOAD and cap["kernel"] == kname
        measured = cap["bytes"] if (applies and fresh) else None
        what = (f" (coupling + {n_above} transfer items above the upward cut, split TF32)" if hybrid
                else (" (coupling, split TF32)" if tensor_path else ""))
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4), "traffic": measured, "kernel": kname + what,
                "peak_source": f"{peak_kind} hbm_gbs"}
        if applies:
            roof["traffic_source"] = {"capture": cap["capture"], "bytes": cap["bytes"],
                                      "kernel_source_sha16_at_capture": cap["source_sha16"],
                                      "kernel_source_sha16_now": sha_now,
                                      "state": "current" if fresh else "stale: kernel changed since the capture"}
    roof["algorithmic_bytes_per_launch"] = int(coup_bytes)
    roof["algorithmic_flops_per_launch"] = coup_flops
    roof["ms_per_launch"] = round(coup_ms, 4)

    # the whole product against its own HBM roofline, and each timed phase against its bytes
    n_leaves = int(info["n_leaves"])
    pbytes = product_bytes(n, k, m, nc, n_adm, info["nnz_near"], elt)
    roof_product = {"algorithmic_bytes": int(pbytes), "ms": round(ms, 4),
                    "achieved_GBps": round(pbytes / (ms * 1e-3) / 1e9, 1), "peak": hbm_peak,
                    "frac": round(pbytes / (ms * 1e-3) / 1e9 / hbm_peak, 4),
                    "formula": "elt*(2nk + (N_c-1)k^2 + N_adm k^2 + nnz_near) + 8*3nm + 4*N_c*k*m*4"}
    per_phase = None
    if tensor_path:
        per_phase = {}
        for ph, b in phase_bytes(n, k, m, nc, n_leaves, n_adm, info["nnz_near"], elt, n_above).items():
            t = phases.get(ph)
            if t and t > 0:
                per_phase[ph] = {"ms": round(t, 4), "algorithmic_bytes": int(b),
                                 "frac_hbm": round(b / (t * 1e-3) / 1e9 / hbm_peak, 4)}

    # end to end through the C ABI on pinned host buffers
    Xh = X.cpu().pin_memory()
    Yh = torch.zeros(n, m, dtype=torch.float64).pin_memory()
    for _ in range(2):
        G.matmul(Xh, Yh, dtype=dtype)
    ke = max(3, min(args.steps, 10))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        G.matmul(Xh, Yh, dtype=dtype)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / ke, dist, dev)
    e2e = {"value": round(job_gflops(flops_step, e2e_s, ws), 3), "unit": "GFLOP/s",
           "h2d_bytes_per_step": 2 * n * m * 8, "d2h_bytes_per_step": n * m * 8,
           "ms_per_step": round(e2e_s * 1e3, 3)}

    # block CG to a 1e-8 relative residual: mixed (FP32 inner, FP64 refinement) vs FP64
    solve = None
    if not args.no_solve:
        solve = {}
        B = torch.from_numpy(rank_rhs(n, m, cfg["rhs_seed"] + 7, rank)).to(dev)
        # name, product precision, refine (2 = reliable updates, 1 = restarted refinement), inner tol,
        # variant, preconditioner
        runs = (("mixed_f32", "f32", 2, 0.1, "columnwise", None),
                ("mixed_f32_restarted", "f32", 1, 1e-4, "columnwise", None),
                ("fp64", "f64", 0, 0.0, "columnwise", None),
                ("mixed_f32_gram", "f32", 2, 0.1, "gram", None),
                ("fp64_gram", "f64", 0, 0.0, "gram", None),
                ("mixed_f32_pcg", "f32", 2, 0.1, "columnwise", "block_jacobi"),
                ("fp64_pcg", "f64", 0, 0.0, "columnwise", "block_jacobi"),
                ("mixed_f32_gram_pcg", "f32", 2, 0.1, "gram", "block_jacobi"),
                ("fp64_gram_pcg", "f64", 0, 0.0, "gram", "block_jacobi"))
        big = workload != WORKLOAD
        for name, inner, refine, itol, variant, pc in runs:
            if variant == "gram" and m > 64:
                continue
            if big and name in ("mixed_f32_restarted",):
                continue
            # on the larger workloads the FP64 solves (~1 h) are run for a capped number of
            # iterations and reported per iteration
            cap = args.fp64_iter_cap if (big and inner == "f64") else args.solve_max_iter
            Xs = torch.zeros_like(B)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = G.block_cg(B, Xs, tol=1e-8, max_iter=cap, dtype=inner, refine=refine,
                           inner_tol=itol, check_every=4, variant=variant, precond=pc)
            torch.cuda.synchronize()
            secs = max_over_ranks(time.perf_counter() - t0, dist, dev)
            solve[name] = {"seconds": round(secs, 3), "status": r.status_name,
                           "iterations": int(r.iterations), "outer_steps": int(r.outer_steps),
                           "h2mm_calls": int(r.h2mm_calls),
                           "max_true_rel_residual": float(np.max(r.rel_residual))}
            if big:
                # on the larger workloads every solve reports its cost per iteration; the
                # FP64 ones are capped, and as specified (q = 4, sigma = 1e-2) the matrix is
                # not definite there, so no solve can reach the tolerance
                if inner == "f64":
                    solve[name]["status"] = "capped" if r.status_name != "ok" else "ok"
                solve[name]["seconds_per_iteration"] = round(secs / max(int(r.iterations), 1), 5)
        if solve["fp64"]["status"] == "ok" and solve["mixed_f32"]["status"] == "ok":
            solve["speedup_mixed_vs_fp64"] = round(solve["fp64"]["seconds"] / solve["mixed_f32"]["seconds"], 3)
        # the fastest mixed solve against the paper's FP64 block CG and against the fastest FP64 solve
        mixed = {k: v["seconds"] for k, v in solve.items() if k.startswith("mixed") and v["status"] == "ok"}
        fp64 = {k: v["seconds"] for k, v in solve.items() if k.startswith("fp64") and v["status"] == "ok"}
        if mixed and fp64 and "fp64" in fp64:
            best_m, best_f = min(mixed, key=mixed.get), min(fp64, key=fp64.get)
            solve["fastest_mixed"] = best_m
            solve["fastest_fp64"] = best_f
            solve["speedup_fastest_mixed_vs_fp64"] = round(solve["fp64"]["seconds"] / mixed[best_m], 3)
            solve["speedup_fastest_mixed_vs_fastest_fp64"] = round(fp64[best_f] / mixed[best_m], 3)

    # the batch workload: 64 independent systems (ellipsoids, n log-uniform in [2048, 32768],
    # m in 1..64, q in {3, 4}); one FP32 product of all of them per step, in two multi-system
    # launches (upward + coupling, downward + leaf) between the systems' gathers and scatters
    batch = None
    if not args.no_batch and workload == WORKLOAD:
        batch = batch_products(P, torch, dev, steps=max(5, min(args.steps, 20)), dist=dist)

    cpu = None
    # the oracle holds every block in host memory: timed on the default workload only
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and workload == WORKLOAD:
        c_flops, c_times, c_build, H2o = oracle_products(cfg, steps=5, warmup=0)
        ct = statistics.median(c_times)
        cpu = {"value": round(c_flops / ct / 1e9, 3), "unit": "GFLOP/s", "cores": _cpu_cores(), "kind": "oracle",
               "cpu_model": _cpu_model(),
               "sample": f"median of 5 FP64 oracle products at n={n}, q={cfg['q']}, m={m}; oracle build "
                         f"{c_build:.1f} s untimed"}
        fp64_it = None
        if solve and solve.get("fp64", {}).get("status") == "ok":
            fp64_it = solve["fp64"]["iterations"]
        cpu.update(cpu_baseline_extras(H2o, cfg, fp64_it))
        del H2o

    line = {
        "metric": metric, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": bench_config(workload, cfg, workload_counts_from_info(info), ws),
        "build_s": round(build_s, 2),
        "gflop_per_step": round(flops_step / 1e9, 4),
        "h2mm_f64": {"value": round(value64, 3), "unit": "GFLOP/s", "ms_per_step": round(ms64, 4)},
        "phases_ms": {kk: round(v, 4) for kk, v in phases.items()},
        "phases_ms_f64": {kk: round(v, 4) for kk, v in phases64.items()},
        "h2mm_bf16": {"value": round(valuebf, 3), "unit": "GFLOP/s", "ms_per_step": round(msbf, 4),
                      "coupling_GBps": round(n_adm * info["k"] * info["k"] * 2 / (phasesbf["coupling"] * 1e-3) / 1e9, 1),
                      "phases_ms": {kk: round(v, 4) for kk, v in phasesbf.items()}},
        "h2mm_f32_matrix_free": mf,
        "h2mm_complex": cx,
        "batch": batch,
        "roofline": roof,
        "roofline_product": roof_product,
        "phases_roofline": per_phase,
        "e2e": e2e,
        "solve": solve,
        "cpu_baseline": cpu,
        "clocks": clk,
        "gpu_launches": int(info["launches_tc"] if tensor_path else info["launches"]) * args.steps,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    G.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


KAPPA, DELTA = 1.0, 0.05  # the Helmholtz kernel's wave number (the paper's) and regularisation length


def complex_products(P, torch, dev, pts, cfg, rank, dist, clk, peaks) -> dict:
    n, m = cfg["n"], cfg["m"]
    G = P.H2Matrix(pts, q=cfg["q"], leaf_size=cfg["leaf"], eta=cfg["eta"], sigma=cfg["sigma"],
                   precisions=("f32",), kernel="helmholtz", kappa=KAPPA, delta=DELTA)
    info = G.info
    X = torch.from_numpy(rank_rhs(n, m, cfg["rhs_seed"], rank) + 1j * rank_rhs(n, m, cfg["rhs_seed"] + 1, rank)).to(dev)
    Y = torch.zeros_like(X)
    flops = G.flops(m)
    coup_flops = 8.0 * info["n_adm"] * info["k"] ** 2 * m
    clock_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    out = {"kernel": f"exp(i*{KAPPA}*r)/(4*pi*sqrt(r^2+{DELTA}^2)), sigma={cfg['sigma']}", "m_complex": m,
           "gflop_per_step": round(flops / 1e9, 4)}
    stream = torch.cuda.current_stream()
    for dt, steps in (("f64", 5), ("f32", 10)):
        for _ in range(3):
            G.matmul_complex(X, Y, dtype=dt)
        P.h2_timing_query(G.handle, reset=True)
        P.h2_timing_enable(G.handle, True)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            G.matmul_complex(X, Y, dtype=dt)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, dist, dev)
        P.h2_timing_enable(G.handle, False)
        ph, calls = P.h2_timing_query(G.handle, reset=True)
        cms = ph["coupling_kernel"] / max(calls, 1)
        if dt == "f32" and info["launches_tc"] > 0:
            # split-TF32 tensor cores: S_re and S_im streamed once, x̂ read and ŷ written once
            cbytes = 4 * (2 * info["n_adm"] * info["k"] ** 2 + 2 * info["n_clusters"] * info["k"] * 2 * m)
            ach = cbytes / (cms * 1e-3) / 1e9
            ck = {"ms": round(cms, 4), "bound": "hbm", "achieved_GBps": round(ach, 1), "peak_GBps": peaks["hbm_gbs"],
                  "frac": round(ach / peaks["hbm_gbs"], 4), "algorithmic_bytes": int(cbytes),
                  "kernel": "k_tc_gemm<0,1> (complex: S_re and S_im terms, split TF32)"}
        else:
            peak = FP64_NOMINAL_TFLOPS if dt == "f64" else SM_COUNT * FP32_FMA_PER_CLK_SM * 2 * clock_mhz * 1e6 / 1e12
            ach = coup_flops / (cms * 1e-3) / 1e12
            ck = {"ms": round(cms, 4), "bound": "alu", "achieved_TFLOPs": round(ach, 3), "peak_TFLOPs": round(peak, 2),
                  "frac": round(ach / peak, 4), "kernel": "k_coupling_c"}
        out[dt] = {"value": round(flops / (ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s", "ms_per_step": round(ms, 4),
                   "steps": steps, "coupling_kernel": ck}
    G.close()
    return out


def batch_products(P, torch, dev, steps: int, dist=None) -> dict:
    """Time the batched FP32 product of the 64-system batch workload (CUDA events)."""
    from workloads import batch_specs, ellipsoid_points
    specs = batch_specs(64, 3, 2048, 32768)
    mats = [P.H2Matrix(ellipsoid_points(sp["n"], sp["axes"], sp["point_seed"]), q=sp["q"], leaf_size=64, eta=2.0,
                       sigma=1e-2, precisions=("f32",)) for sp in specs]
    Xs = [torch.from_numpy(gaussian_rhs(sp["n"], sp["m"], sp["rhs_seed"])).to(dev) for sp in specs]
    Ys = [torch.zeros_like(x) for x in Xs]
    flops = sum(mm.flops(sp["m"]) for mm, sp in zip(mats, specs))
    Bt = P.H2Batch(mats)
    for _ in range(3):
        Bt.matmul(Xs, Ys, dtype="f32")
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    e0.record(st)
    for _ in range(steps):
        Bt.matmul(Xs, Ys, dtype="f32")
    e1.record(st)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, dist, dev)
    out = {"systems": len(specs), "total_n": sum(sp["n"] for sp in specs),
           "total_columns": sum(sp["m"] for sp in specs), "gflop_per_product": round(flops / 1e9, 3),
           "ms_per_product": round(ms, 4), "value": round(flops / (ms * 1e-3) / 1e9, 1), "unit": "GFLOP/s",
           "steps": steps, "launch": "two multi-system tensor-core launches per product (upward pass + coupling, "
                                     "downward pass + leaf phase) plus per-system gathers and scatters, one CUDA graph"}
    Bt.close()
    for mm in mats:
        mm.close()
    return out


def run_mvm_vs_mm(args):
    """The MVM-vs-MM experiment of Sec. 4 on one GPU: m products with one
    column each against one product with m columns, same matrix (the
    precision workload), for m in {10, 50, 100, 200}, FP64 and FP32.  Prints
    one JSON line; not a bench line."""
    import torch
    import paper_2509_17257_gb300 as P
    cfg = CONFIGS[WORKLOAD]
    n = cfg["n"]
    G = P.H2Matrix(sphere_points(n, cfg["point_seed"]), q=cfg["q"], leaf_size=cfg["leaf"], eta=cfg["eta"],
                   sigma=cfg["sigma"], precisions=("f32",))
    out = {"experiment": "mvm_vs_mm", "workload": WORKLOAD, "n": n, "q": cfg["q"], "rows": []}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def clock(fn, reps):
        fn()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(reps):
            fn()
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    for dtype in ("f64", "f32"):
        for m in (10, 50, 100, 200):
            X = torch.from_numpy(gaussian_rhs(n, m, 5)).cuda()
            Y = torch.zeros_like(X)
            cols = [X[:, j:j + 1].contiguous() for j in range(m)]
            ycols = [Y[:, j:j + 1].contiguous() for j in range(m)]

            def mm():
                G.matmul(X, Y, dtype=dtype)

            def mvm():
                for j in range(m):
                    G.matmul(cols[j], ycols[j], dtype=dtype)

            reps = 3 if dtype == "f64" else 5
            t_mm = clock(mm, reps)
            t_mvm = clock(mvm, 1 if dtype == "f64" else 2)
            out["rows"].append({"dtype": dtype, "m": m, "ms_mm": round(t_mm, 3), "ms_m_mvm": round(t_mvm, 3),
                                "speedup": round(t_mvm / t_mm, 2),
                                "mm_gflops": round(G.flops(m) / (t_mm * 1e-3) / 1e9, 1)})
    print(json.dumps(out), flush=True)
    G.close()
    return 0


def run_batch(args):
    """The batch workload on one GPU: 64 ellipsoid systems, n log-uniform in
    [2048, 32768], m in {1..64}, q in {3, 4}.  Times the FP32 product of all
    systems as one CUDA-graph launch against a loop of per-system products,
    after the autotuner picked each matrix's FP32 path, and the batched mixed
    solve (Gram variant).  Prints one JSON line; not a bench line."""
    import torch
    import paper_2509_17257_gb300 as P
    from workloads import batch_specs, ellipsoid_points
    specs = batch_specs(64, 3, 2048, 32768)
    mats = [P.H2Matrix(ellipsoid_points(sp["n"], sp["axes"], sp["point_seed"]), q=sp["q"], leaf_size=64, eta=2.0,
                       sigma=1e-2, precisions=("f32",)) for sp in specs]
    tuned = [P.h2_autotune(mm.handle, sp["m"]) for mm, sp in zip(mats, specs)]
    Xs = [torch.from_numpy(gaussian_rhs(sp["n"], sp["m"], sp["rhs_seed"])).cuda() for sp in specs]
    Ys = [torch.zeros_like(x) for x in Xs]
    flops = sum(mm.flops(sp["m"]) for mm, sp in zip(mats, specs))
    Bt = P.H2Batch(mats)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def clock(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(reps):
            fn()
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    def loop():
        for mm, x, y in zip(mats, Xs, Ys):
            mm.matmul(x, y, dtype="f32")

    t_loop = clock(loop, 10)
    t_graph = clock(lambda: Bt.matmul(Xs, Ys, dtype="f32"), 10)
    Bs = [torch.from_numpy(gaussian_rhs(sp["n"], sp["m"], sp["rhs_seed"] + 7)).cuda() for sp in specs]
    Xb = [torch.zeros_like(b) for b in Bs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = Bt.block_cg(Bs, Xb, tol=1e-8, max_iter=3000, dtype="f32", inner_tol=0.1, check_every=4, variant="gram")
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    out = {"experiment": "batch", "systems": len(specs), "total_n": sum(sp["n"] for sp in specs),
           "total_columns": sum(sp["m"] for sp in specs), "gflop_per_batched_product": round(flops / 1e9, 3),
           "ms_loop": round(t_loop, 3), "ms_graph": round(t_graph, 3),
           "gflops_graph": round(flops / (t_graph * 1e-3) / 1e9, 1), "graph_speedup": round(t_loop / t_graph, 2),
           "tensor_core_systems": sum(1 for a, b in tuned if 0 <= a <= b),
           "solve_seconds": round(t_solve, 3),
           "solve_status": {str(k): v for k, v in
                            __import__("collections").Counter(r.status_name for r in res).items()},
           "solve_max_iterations": max(r.iterations for r in res),
           "max_true_rel_residual_ok": max(float(r.rel_residual.max()) for r in res if r.status == 0)}
    print(json.dumps(out), flush=True)
    Bt.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--dtype", choices=["f32", "f64", "bf16"], default="f32")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-system batched product in the bench line")
    ap.add_argument("--no-complex", action="store_true", help="skip the complex (Helmholtz kernel) product")
    ap.add_argument("--solve-max-iter", type=int, default=8000)
    ap.add_argument("--workload", choices=sorted(CONFIGS), default=WORKLOAD,
                    help="workload of the bench line (default: the precision workload, n = 65536)")
    ap.add_argument("--fp64-iter-cap", type=int, default=60,
                    help="iteration cap of the FP64 solves on workloads other than the default")
    ap.add_argument("--batch", action="store_true", help="run the batch workload (64 systems) experiment")
    ap.add_argument("--mvm-vs-mm", action="store_true",
                    help="run the MVM-vs-MM experiment (m single-column products vs one m-column product)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.mvm_vs_mm:
        return run_mvm_vs_mm(args)
    if args.batch:
        return run_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
