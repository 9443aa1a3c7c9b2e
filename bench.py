"""Benchmark: fermion-drift evaluations per second on an 8^3 x 4 lattice.

One step = one drift evaluation of every replica of the batch: cl_factor
(multifrontal LU of D(m;mu)), cl_selinv_blocks (selected inversion + block
extraction) and cl_fermion_drift, links already resident in HBM.  The e2e
figure repeats the step through the same C ABI with the links copied from
pinned host memory and the drift copied back every step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64_emu|fp64|mixed|fp32]
                    [--batch B] [--impl ours|reference]

Precisions: fp64_emu (default) = the FP64 path, FP64 fronts whose GEMMs run as
8-digit BF16 products on the tcgen05 tensor cores (held to 1e-10 against the
oracle in the tests); fp64 = the same fronts with plain FP64 products on the
FP64 MMA pipe; mixed = split-BF16x3 Schur products with FP64 pivot blocks;
fp32 = all-FP32 fronts.  The JSON line also carries a comparison of the four on
the same links ("precisions": rate and drift error against the CPU oracle).

The CPU baseline and the reference arm time complete evaluations of the CPU
oracle (dense D, LU with partial pivoting, every column of D^{-1}, the
selected blocks and the drift), with no extrapolation.

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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fermion-drift evals/sec on 8^3x4 (FP64 vs mixed, stated drift error); front TFLOP/s vs peak"
NS, NT, M, MU = 8, 4, 0.05, 0.25
# DRAM bytes (dram__bytes_read + dram__bytes_write, ncu, caches flushed
# before each launch) of all digit-GEMM and split launches of one evaluation,
# the unit of `achieved` (538 launches at 8^3x4, batch 1, 30-unknown panels);
# keyed by (precision, batch, panel) and valid only for the kernel build it
# was taken on (profiles/gemm_dram_fp64_emu_8x4.md)
NCU_TRAFFIC = {("fp64_emu", 1, 30): 17.652e9}
# BF16 products per FP64-equivalent product of the digit GEMMs: digit pairs
# p + q <= ND - 1 of ND digits per operand (8 digits: 36)
DIGIT_PRODUCTS = {"fp64_emu": 36, "mixed": 6}


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
    ap.add_argument("--precision", choices=["fp64", "fp64_emu", "mixed", "fp32"], default="fp64_emu")
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
# CPU oracle timing: complete evaluations, no extrapolation
# ---------------------------------------------------------------------------
def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def oracle_eval():
    """One complete 8^3 x 4 evaluation of the CPU oracle, timed whole: dense D,
    LU with partial pivoting, all N column solves of D^{-1}, the selected
    blocks and the drift (OpenMP over the host cores).  Returns (seconds,
    oracle result)."""
    import oracle
    from paper_1707_08874_gb300 import inputs
    U = inputs.random_links(NS, NT, seed=inputs.BASE_SEED)
    t0 = time.perf_counter()
    ref = oracle.drift_eval(NS, NT, U, M, MU)
    return time.perf_counter() - t0, ref


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


# the reference arm times at most this many complete oracle evaluations (each
# ~33 s on the 16 Grace cores of a GPU machine) after at most one warm-up
# evaluation, so that a run of the default 20 steps ends within a few minutes
REF_MAX_STEPS = 4


def run_reference(args, rank, world):
    if rank != 0:
        return
    for _ in range(min(args.warmup, 1)):
        oracle_eval()
    steps = max(1, min(args.steps, REF_MAX_STEPS))
    vals = []
    t0 = time.perf_counter()
    for _ in range(steps):
        vals.append(oracle_eval()[0])
    wall = time.perf_counter() - t0
    t_eval = statistics.median(vals)
    value = 1.0 / t_eval
    sample = ("complete 8^3x4 evaluations of the CPU oracle (dense D, LU, all %d columns of D^-1, selected "
              "blocks, drift), no extrapolation: %d timed (median %.1f s, %.1f s in all) of the %d requested "
              "steps, after %d warm-up" % (3 * NS ** 3 * NT, steps, t_eval, wall, args.steps, min(args.warmup, 1)))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": steps, "steps_requested": args.steps, "warmup": min(args.warmup, 1),
            "ms_per_step": 1e3 * t_eval, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "8^3x4 lattice, m=0.05, mu=0.25, batch 1, dense CPU oracle",
                       "lattice": "8^3x4", "batch": 1, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": host_cores(), "kind": "oracle",
                             "sample": sample},
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
            fd, self.path = tempfile.mkstemp(prefix="clocks_bench_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
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
        lines = open(self.path).read().splitlines()
        os.unlink(self.path)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
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
PRECISIONS = ("fp64_emu", "fp64", "mixed", "fp32")


def prec_code(B, name):
    return {"fp64": B.CL_FP64, "fp64_emu": B.CL_FP64_EMU, "mixed": B.CL_MIXED_BF16X3,
            "fp32": B.CL_MIXED_FP32}[name]


def compare_precisions(B, torch, links, bsz, ref, steps=3):
    """Timing of the four front precisions on the same links (directly
    launched, `steps` evaluations after two warm-ups) and, when the oracle's
    result `ref` is given, the normwise errors of replica 0 against it: the G
    blocks (max_b |dG_b|_F / max_b |G_b|_F) and the drift (max |dK| / max |K|)."""
    out = {}
    for name in PRECISIONS:
        plan = B.Plan.analyze(NS, NT, bsz, prec_code(B, name))
        o = plan.alloc_outputs()
        for _ in range(2):
            plan.drift_eval(links, M, MU, 1.0, o["Gdiag"], o["Gfwd"], o["Gbwd"], o["Kf"])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.drift_eval(links, M, MU, 1.0, o["Gdiag"], o["Gfwd"], o["Gbwd"], o["Kf"])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        rec = {"evals_per_s": bsz / (ms / 1e3), "ms_per_step": ms, "launch": "direct"}
        if ref is not None:
            def blockwise(a, b):
                da = np.sqrt((np.abs(a - b) ** 2).sum((-1, -2)))
                return float(da.max() / np.sqrt((np.abs(b) ** 2).sum((-1, -2))).max())
            got = {k: o[k][0].cpu().numpy() for k in ("Gdiag", "Gfwd", "Gbwd", "Kf")}
            rec["g_rel_err_vs_oracle"] = max(blockwise(got[k], ref[k]) for k in ("Gdiag", "Gfwd", "Gbwd"))
            rec["drift_rel_err_vs_oracle"] = float(np.abs(got["Kf"] - ref["Kf"]).max() / np.abs(ref["Kf"]).max())
        out[name] = rec
        plan.close()
    return out


def compare_stochastic(B, torch, links, bsz, kf_exact, counts=(1, 16), steps=3):
    """The paper's comparison path (Sec. 3, Eq. 7): the drift from n Z4 noise
    vectors (factorisation, n row-vector solves with its factors, estimated
    blocks, drift) on the same links; rate and max |K_est - K| / max |K|
    against the exact selected-inversion drift of replica 0."""
    out = {}
    V = NS ** 3 * NT
    rng = np.random.default_rng(11)
    plan = B.Plan.analyze(NS, NT, bsz, B.CL_FP64_EMU)
    o = plan.alloc_outputs()
    K0 = kf_exact[0].cpu().numpy()
    for n in counts:
        eta = torch.from_numpy(rng.choice(np.array([1.0, 1j, -1.0, -1j]), size=(n, bsz * V, 3))).to("cuda")
        w = torch.empty_like(eta)
        work = plan.stochastic_drift(links, M, MU, 1.0, eta, w, None, o["Gfwd"], o["Gbwd"], o["Kf"])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.stochastic_drift(links, M, MU, 1.0, eta, w, None, o["Gfwd"], o["Gbwd"], o["Kf"])
        e1.record()
        torch.cuda.synchronize()
        del work
        ms = e0.elapsed_time(e1) / steps
        K = o["Kf"][0].cpu().numpy()
        out["noise_%d" % n] = {"evals_per_s": bsz / (ms / 1e3), "ms_per_step": ms,
                               "drift_rel_err_vs_exact": float(np.abs(K - K0).max() / np.abs(K0).max())}
    st, _ = plan.get_status()
    plan.close()
    if st != B.CL_OK:
        raise RuntimeError("stochastic drift reported %s" % B.error_string(st))
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
    prec = prec_code(B, args.precision)
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
    # ceiling of the front arithmetic: the digit GEMMs run on tcgen05, so their
    # FP64-equivalent ceiling is the dense BF16 rate (sustained: they are
    # timed inside a long step) over the BF16 products of one FP64-equivalent
    # product; the other precisions' pipes are measured live on this GPU
    if args.precision in DIGIT_PRODUCTS:
        bf16, bf16_note = measured_bf16_tflops()
        peak = bf16 / DIGIT_PRODUCTS[args.precision]
        peak_source = "%s / %d digit products (FP64-equivalent ceiling of the tcgen05 digit GEMM)" % (
            bf16_note, DIGIT_PRODUCTS[args.precision])
    else:
        peak = B.measure_peak(0 if prec == B.CL_FP64 else 2) / 1e3
        peak_source = ("FP64 MMA (mma.sync m8n8k4)" if prec == B.CL_FP64 else "FP32 FMA") + \
            " throughput measured live on this GPU by cl_measure_peak"

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
    growth = plan.pivot_growth()

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
    total_prof_ms = sum(v["total_ms"] for v in prof.values())
    flops_eval = info["factor_flops"] + info["selinv_flops"]
    # roofline of the front arithmetic from the timed (graph-replayed) step:
    # the algorithmic flops of one evaluation (cl_plan_info: 8 flops per
    # complex multiply-add of the factorisation and selected inversion) x batch
    # over ms_per_step; the GEMMs' own rate from per-launch CUDA events of a
    # profiled pass is given beside it
    achieved = flops_eval * bsz / (ms / 1e3) / 1e12
    gemm_only = g.get("flops", 0.0) / (g["total_ms"] / 1e3) / 1e12 if g.get("total_ms") else None
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp64_emu": "f64 (8-digit bf16 products, fp32 accumulate)",
                  "mixed": "f64 pivot blocks, split-bf16x3 Schur products", "fp32": "f32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": "8^3x4 lattice, m=0.05, mu=0.25, links exp(i c.lambda), c ~ N(0,0.5)+iN(0,0.1)",
                   "lattice": "8^3x4", "batch": bsz, "precision": args.precision, "panel": panel,
                   "parallelism": "replicas" if world > 1 else "single",
                   "launch": "CUDA graph of one evaluation, replayed (cl_group_capture / cl_group_launch)",
                   "l2": "working set > L2 (front pool %.0f MB per replica)" % (info["front_bytes"] / bsz / 1e6)},
        "e2e": {"value": world * bsz / (e2e_ms / 1e3), "unit": "evals/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": info["launches_per_eval"] * args.steps,
        # largest max|entry| / min|pivot| of the pivot blocks of the timed links
        # (cl_plan_pivot_growth): 11-62 over twenty 8^3x4 configurations with
        # pivots chosen among two panels' rows (~1e3 on the ill-conditioned
        # ones when pivots were restricted to a panel)
        "pivot_growth": growth,
        "roofline": {"bound": "tensor" if prec != B.CL_MIXED_FP32 else "alu",
                     "kernel": "front GEMMs (factorisation + selected inversion); achieved = flops_per_eval x "
                               "batch / ms_per_step of the timed step",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": peak_source,
                     "traffic": NCU_TRAFFIC.get((args.precision, bsz, panel)),
                     "traffic_unit": "bytes per evaluation (all digit-GEMM and split launches)",
                     "gemm_algorithmic_bytes": g.get("bytes", 0.0) / args.steps if g else None,
                     "gemm_only_tflops": gemm_only,
                     "gemm_share_of_kernel_time": g.get("total_ms", 0.0) / total_prof_ms if total_prof_ms else None},
        "flops_per_eval": flops_eval,
        "kernel_ms_per_step": {k: v["total_ms"] / args.steps for k, v in prof.items()},
        "clocks": ck,
    }
    ref = None
    if not args.no_cpu_baseline:
        t_eval, ref = oracle_eval()
        line["cpu_baseline"] = {"value": 1.0 / t_eval, "unit": "evals/s", "cores": host_cores(), "kind": "oracle",
                                "sample": "one complete 8^3x4 evaluation of the CPU oracle (dense D, LU, all %d "
                                          "columns of D^-1, selected blocks, drift), %.1f s, no extrapolation"
                                          % (3 * NS ** 3 * NT, t_eval)}
        lv, lcores, lsample = lapack_sample()
        line["cpu_lapack"] = {"value": lv, "unit": "evals/s", "cores": lcores, "kind": "dense LAPACK inverse",
                              "sample": lsample}
    if not args.no_compare:
        line["precisions"] = compare_precisions(B, torch, links, bsz, ref)
        line["stochastic_estimator"] = compare_stochastic(B, torch, links, bsz, out["Kf"])
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
