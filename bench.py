"""Benchmark: fermion-drift evaluations per second on an 8^3 x 4 lattice.

One step = one drift evaluation of every replica of the batch: cl_factor
(multifrontal LU of D(m;mu)), cl_selinv_blocks (selected inversion + block
extraction) and cl_fermion_drift, links already resident in HBM.  The e2e
figure repeats the step through the same C ABI with the links copied from
pinned host memory and the drift copied back every step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64_emu|fp64|mixed]
                    [--batch B] [--impl ours|reference]

Precisions: fp64 = FP64 fronts on the FP64 MMA pipe; fp64_emu (default) = FP64
fronts whose GEMMs run as exact 7-digit BF16 products on the tensor cores
(held to the same FP64 parity bar in the tests); mixed = FP32 fronts.  The
JSON line also carries a quick comparison of the three on the same links
("precisions": rate and drift error against the native FP64 result).

Multi-GPU: replicas only (independent lattices per rank, no data-path
collective); value = evaluations of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fermion-drift evals/sec on 8^3x4 (FP64 vs mixed, stated drift error); front TFLOP/s vs peak"
NS, NT, M, MU = 8, 4, 0.05, 0.25
# DRAM bytes per digit-GEMM launch (dram__bytes_read + dram__bytes_write,
# averaged over the 269 GEMM launches of one 8^3x4 evaluation with
# 30-unknown panels, ncu, cold cache; profiles/gemm_emu_tcgen05_8x4.md);
# valid for the kernels it was taken on, keyed by (precision, batch, panel)
NCU_TRAFFIC = {("fp64_emu", 1, 30): 63.67e6}


def measured_bf16_tflops():
    """Sustained dense BF16 TFLOP/s of the GB300s (MEASURED_PEAKS.json
    beside this file), else the recipe's fallback; returns (value, note)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["bf16_tflops_sustained"])
        return v, "bf16_tflops_sustained %.0f TFLOP/s of measured (MEASURED_PEAKS.json)" % v
    except (OSError, KeyError, ValueError):
        return 1700.0, "1700 TFLOP/s BF16 sustained, of fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", choices=["fp64", "fp64_emu", "mixed"], default="fp64_emu")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 / emulated / mixed comparison")
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--panel", type=int, default=0, help="pivot-panel width (0: autotune)")
    return ap.parse_args()


def replica_seed(rank: int, bsz: int) -> int:
    """Seed of replica 0 of this rank: ranks hold disjoint replica streams."""
    from paper_1707_08874_gb300 import inputs
    return inputs.BASE_SEED + rank * bsz


def max_over_ranks(values, dist, device):
    """Element-wise max of per-rank timings (the slowest rank sets the rate)."""
    import torch
    if dist is None:
        return list(values)
    t = torch.tensor(list(values), device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample of one 8^3 x 4 evaluation)
# ---------------------------------------------------------------------------
def oracle_sample(lu_steps=2560, ncols=2048):
    """Time a bounded sample of the oracle's dense evaluation and scale it to
    one full evaluation by exact operation counts: the dense D, the first
    `lu_steps` of the N-step right-looking LU (step k costs (N-k)^2 updates)
    and `ncols` of the N column solves (each column costs the same)."""
    import oracle
    from paper_1707_08874_gb300 import inputs
    U = inputs.random_links(NS, NT, seed=inputs.BASE_SEED)
    N = 3 * NS ** 3 * NT
    t0 = time.perf_counter()
    D = oracle.dirac_dense(NS, NT, U, M, MU)
    t1 = time.perf_counter()
    LU, piv, _ = oracle.lu_steps(D, lu_steps)
    t2 = time.perf_counter()
    # the column solves run on the partly factored matrix (pivots beyond the
    # sample left in place): the same operations as on the finished factors
    piv[lu_steps:] = np.arange(lu_steps, N, dtype=np.int32)
    t3 = time.perf_counter()
    oracle.solve_unit_columns(LU, piv, np.arange(ncols))
    t4 = time.perf_counter()
    k = np.arange(N, dtype=np.float64)
    lu_scale = ((N - k) ** 2).sum() / ((N - k[:lu_steps]) ** 2).sum()
    t_eval = (t1 - t0) + (t2 - t1) * lu_scale + (t4 - t3) * (N / ncols)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample = ("8^3x4 oracle: dense D + first %d of %d LU steps (scaled by sum (N-k)^2) + %d of %d "
              "column solves (scaled linearly); measured %.1f s" % (lu_steps, N, ncols, N, t4 - t0))
    return 1.0 / t_eval, cores, sample, t_eval


def lapack_sample():
    """The paper's dense comparison (Sec. 3: the full inverse by LAPACK) on the
    host cores: dense D of the workload (oracle) and torch.linalg.inv in
    complex128, timed once; the drift itself is negligible beside it."""
    import torch
    import oracle
    from paper_1707_08874_gb300 import inputs
    U = inputs.random_links(NS, NT, seed=inputs.BASE_SEED)
    t0 = time.perf_counter()
    D = torch.from_numpy(oracle.dirac_dense(NS, NT, U, M, MU))
    t1 = time.perf_counter()
    torch.linalg.inv(D)
    t2 = time.perf_counter()
    sample = ("8^3x4 dense D (%.1f s) + torch.linalg.inv complex128 N=%d (%.1f s), one evaluation"
              % (t1 - t0, D.shape[0], t2 - t1))
    return 1.0 / (t2 - t0), torch.get_num_threads(), sample


def run_reference(args, rank, world):
    if rank != 0:
        return
    # each step: the dense D, the first 384 of the 6144 LU steps and 192 column
    # solves (~4 s on 16 cores), scaled to one evaluation by operation counts;
    # short samples overstate the rate (later LU steps parallelise worse)
    for _ in range(args.warmup):
        oracle_sample(lu_steps=384, ncols=192)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, cores, sample, t_eval = oracle_sample(lu_steps=384, ncols=192)
        vals.append(t_eval)
    wall = time.perf_counter() - t0
    t_eval = statistics.median(vals)
    value = 1.0 / t_eval
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_eval, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "8^3x4 lattice, m=0.05, mu=0.25, batch 1, dense CPU oracle",
                       "lattice": "8^3x4", "batch": 1, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": sample.split("; measured")[0] + "; %d samples in %.1f s" % (
                                 args.steps, wall)},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            os.makedirs(os.path.join(ROOT, "gpurun_out"), exist_ok=True)
            self.path = os.path.join(ROOT, "gpurun_out", "clocks_bench_%d.csv" % os.getpid())
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def compare_precisions(B, torch, links, bsz, steps=3):
    """Quick timing of the three front precisions on the same links, and the
    drift error of each against the native FP64 GPU result (replica 0)."""
    out, ref = {}, None
    names = [("fp64", B.CL_FP64), ("fp64_emu", B.CL_FP64_EMU), ("mixed", B.CL_MIXED_FP32)]
    for name, prec in names:
        plan = B.Plan.analyze(NS, NT, bsz, prec)
        o = plan.alloc_outputs()
        for _ in range(2):
            plan.drift_eval(links, M, MU, 1.0, None, o["Gfwd"], o["Gbwd"], o["Kf"])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.drift_eval(links, M, MU, 1.0, None, o["Gfwd"], o["Gbwd"], o["Kf"])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        K = o["Kf"][0].cpu().numpy()
        if ref is None:
            ref = K
        err = float(np.abs(K - ref).max() / np.abs(ref).max())
        out[name] = {"evals_per_s": bsz / (ms / 1e3), "ms_per_step": ms, "drift_rel_err_vs_fp64": err,
                     "launch": "direct"}
        plan.close()
    return out


def run_ours(args, rank, world, local):
    import torch
    from paper_1707_08874_gb300 import binding as B
    from paper_1707_08874_gb300 import inputs

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = {"fp64": B.CL_FP64, "fp64_emu": B.CL_FP64_EMU, "mixed": B.CL_MIXED_FP32}[args.precision]
    bsz = args.batch
    from paper_1707_08874_gb300 import autotune
    panel = args.panel or autotune.tune_panel(NS, NT, bsz, prec, use_cache=False)
    plan = B.Plan.analyze_ex(NS, NT, bsz, prec, panel)
    info = plan.info
    U = inputs.random_links(NS, NT, seed=replica_seed(rank, bsz), batch=bsz)
    links_host = torch.from_numpy(U).pin_memory()
    links = links_host.to("cuda", non_blocking=True)
    out = plan.alloc_outputs()
    kf_host = torch.empty(out["Kf"].shape, dtype=torch.complex128).pin_memory()
    stream = torch.cuda.current_stream()

    def step_direct():
        plan.drift_eval(links, M, MU, 1.0, None, out["Gfwd"], out["Gbwd"], out["Kf"], stream)

    for _ in range(max(3, args.warmup)):
        step_direct()
    torch.cuda.synchronize()
    # the evaluation's fixed schedule captured once into a CUDA graph (the
    # library's group API) and replayed: one launch per evaluation
    graph = B.Group([plan])
    graph.capture([links], M, MU, 1.0, [out["Gfwd"]], [out["Gbwd"]], [out["Kf"]])

    def step():
        graph.launch(stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    st, _ = plan.get_status()
    if st != B.CL_OK:
        raise RuntimeError("drift evaluation reported %s" % B.error_string(st))
    peak_unit = {B.CL_FP64: 0, B.CL_FP64_EMU: 3, B.CL_MIXED_FP32: 2}[prec]
    peak_gflops = B.measure_peak(peak_unit)
    peak_note = None
    if prec == B.CL_FP64_EMU:
        # the digit GEMM runs on tcgen05: its ceiling is the dense BF16 rate
        # (sustained: the kernel is timed inside a long step) over the 28
        # digit products of one FP64-equivalent product
        bf16, peak_note = measured_bf16_tflops()
        peak_gflops = bf16 * 1e3 / 28.0

    clocks = Clocks(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # per-kernel CUDA events over a pass of the same steps launched directly
    # (events between launches; this pass is not the headline number)
    plan.profile_enable(True)
    for _ in range(args.steps):
        step_direct()
    torch.cuda.synchronize()
    prof = plan.profile_read()
    plan.profile_enable(False)
    st, _ = plan.get_status()
    if st != B.CL_OK:
        raise RuntimeError("drift evaluation reported %s" % B.error_string(st))

    # end to end through the same ABI: H2D links, evaluation, D2H drift
    h2d = links_host.numel() * 16
    d2h = kf_host.numel() * 16
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        links.copy_(links_host, non_blocking=True)
        step()
        kf_host.copy_(out["Kf"], non_blocking=True)
    t1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = t0.elapsed_time(t1) / args.steps

    ms, e2e_ms = max_over_ranks([ms, e2e_ms], dist, "cuda")
    if rank != 0:
        return
    value = world * bsz / (ms / 1e3)
    g = prof.get("gemm", {})
    gemm_ms = g.get("total_ms", 0.0) / max(1, g.get("launches", 1))
    gemm_flops = g.get("flops", 0.0) / max(1, g.get("launches", 1))
    achieved = gemm_flops / (gemm_ms / 1e3) / 1e12 if gemm_ms > 0 else 0.0
    peak = peak_gflops / 1e3  # FP64-equivalent for the emulated path (BF16 peak / 28, above)
    total_prof_ms = sum(v["total_ms"] for v in prof.values())
    flops_eval = info["factor_flops"] + info["selinv_flops"]
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {B.CL_FP64: "f64", B.CL_FP64_EMU: "f64 (exact bf16 digit products, fp32 accumulate)",
                  B.CL_MIXED_FP32: "f32"}[prec], "data": "synthetic",
        "config": {"workload": "8^3x4 lattice, m=0.05, mu=0.25, links exp(i c.lambda), c ~ N(0,0.5)+iN(0,0.1)",
                   "lattice": "8^3x4", "batch": bsz, "precision": args.precision, "panel": panel,
                   "parallelism": "replicas" if world > 1 else "single",
                   "launch": "CUDA graph of one evaluation, replayed (cl_group_capture / cl_group_launch)",
                   "l2": "working set > L2 (front pool %.0f MB per replica)" % (info["front_bytes"] / bsz / 1e6)},
        "e2e": {"value": world * bsz / (e2e_ms / 1e3), "unit": "evals/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": info["launches_per_eval"] * args.steps,
        "roofline": {"bound": "alu" if prec == B.CL_MIXED_FP32 else "tensor", "kernel": "gemm",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None,
                     "peak_source": {B.CL_FP64: "FP64 MMA (mma.sync m8n8k4) throughput measured live on this GPU",
                                     B.CL_FP64_EMU: "%s / 28 digit products (FP64-equivalent ceiling of the "
                                                    "tcgen05 digit GEMM)" % peak_note,
                                     B.CL_MIXED_FP32: "FP32 FMA throughput measured live on this GPU"}[prec],
                     "traffic": NCU_TRAFFIC.get((args.precision, bsz, panel)),
                     "gemm_share_of_kernel_time": g.get("total_ms", 0.0) / total_prof_ms if total_prof_ms else None},
        "front_tflops": flops_eval * bsz / (ms / 1e3) / 1e12,
        "flops_per_eval": flops_eval,
        "kernel_ms_per_step": {k: v["total_ms"] / args.steps for k, v in prof.items()},
        "clocks": ck,
    }
    if not args.no_compare:
        line["precisions"] = compare_precisions(B, torch, links, bsz)
    if not args.no_cpu_baseline:
        v, cores, sample, _ = oracle_sample()
        line["cpu_baseline"] = {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample}
        lv, lcores, lsample = lapack_sample()
        line["cpu_lapack"] = {"value": lv, "unit": "evals/s", "cores": lcores, "kind": "dense LAPACK inverse",
                              "sample": lsample}
    print(json.dumps(line), flush=True)
    graph.close()
    plan.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
