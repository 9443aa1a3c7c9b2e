"""Batched and ragged drift evaluations in one captured CUDA graph.

    python -m paper_1707_08874_gb300.run_batched [--precision fp64_emu|fp64|mixed|fp32]
        [--shapes 8x4:64]  or  [--shapes 4x4:16,6x4:16,8x6:8]  [--steps 5] [--tune]
        [--mode merged|streams]

Each --shapes entry is NsxNt:count (count replicas of that lattice).
--mode merged (default): one ragged plan (cl_analyze_ragged) whose schedule
runs every step of every level as one launch over the fronts of all lattices
of all shapes; --mode streams: one plan per shape, each on its own stream
(cl_group_*).  Either way the whole evaluation is captured once into a CUDA
graph and the timed loop replays it.  Prints one JSON line: evaluations per
second over all lattices, the FP64-equivalent front rate, and per shape the
drift error of replica 0 against a single-shape plan of the FP64 path
(CL_FP64_EMU, held to 1e-10 against the CPU oracle in the tests).
"""
from __future__ import annotations

import argparse
import json
import os


def parse_shapes(text):
    out = []
    for tok in text.split(","):
        dims, cnt = tok.split(":")
        ns, nt = dims.split("x")
        out.append((int(ns), int(nt), int(cnt)))
    return out


# BF16 products per FP64-class product of the digit GEMMs: 8 digits per
# operand (36 products) on the FP64 path, 3 (6 products) for the mixed form's
# Schur products; the other front precisions do not run on the BF16 pipe
DIGIT_PRODUCTS = {"fp64_emu": 36, "mixed": 6}


def roofline(precision, achieved_tflops):
    """Achieved front rate against the digit GEMM's ceiling: the measured
    sustained BF16 rate (MEASURED_PEAKS.json beside the package, else 1700
    TFLOP/s) over the BF16 products per FP64-class product."""
    if precision not in DIGIT_PRODUCTS:
        return None
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            bf16, src = float(json.load(f)["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        bf16, src = 1700.0, "fallback"
    peak = bf16 / DIGIT_PRODUCTS[precision]
    return {"bound": "tensor", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved_tflops / peak,
            "peak_source": "bf16 sustained %.0f TFLOP/s (%s) / %d products" % (bf16, src, DIGIT_PRODUCTS[precision])}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--shapes", default="8x4:64")
    ap.add_argument("--precision", choices=["fp64", "fp64_emu", "mixed", "fp32"], default="fp64_emu")
    ap.add_argument("--mode", choices=["merged", "streams"], default="merged")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--tune", action="store_true", help="autotune the panel width")
    ap.add_argument("--panel", type=int, default=0)
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--warm", type=int, default=2, help="graph launches before the timed ones")
    args = ap.parse_args(argv)

    import numpy as np
    import torch

    from . import autotune
    from . import binding as B
    from . import inputs

    prec = {"fp64": B.CL_FP64, "fp64_emu": B.CL_FP64_EMU, "mixed": B.CL_MIXED_BF16X3,
            "fp32": B.CL_MIXED_FP32}[args.precision]
    shapes = parse_shapes(args.shapes)
    U = [inputs.random_links(ns, nt, seed=inputs.BASE_SEED + 1000 * i, batch=cnt) for i, (ns, nt, cnt) in
         enumerate(shapes)]
    if args.mode == "merged":
        panel = args.panel or (autotune.tune_panel_ragged(shapes, prec) if args.tune else 0)
        plan = B.Plan.analyze_ragged(shapes, prec, panel)
        plans = [plan]
        links = [torch.from_numpy(np.concatenate([u.reshape((-1, 4, 3, 3)) for u in U])[None].copy()).to("cuda")]
        panels = [plan.info["panel"]]
    else:
        plans, links, panels = [], [], []
        for i, (ns, nt, cnt) in enumerate(shapes):
            if args.tune:
                plan, panel = autotune.tuned_plan(ns, nt, cnt, prec)
            else:
                plan = B.Plan.analyze_ex(ns, nt, cnt, prec, args.panel)
                panel = plan.info["panel"]
            plans.append(plan)
            panels.append(panel)
            links.append(torch.from_numpy(U[i]).to("cuda"))
    outs = [p.alloc_outputs() for p in plans]
    group = B.Group(plans)
    gf = [o["Gfwd"] for o in outs]
    gb = [o["Gbwd"] for o in outs]
    kf = [o["Kf"] for o in outs]
    group.drift_eval(links, 0.05, 0.25, 1.0, gf, gb, kf)   # warm-up, uncaptured
    group.capture(links, 0.05, 0.25, 1.0, gf, gb, kf)
    for _ in range(args.warm):
        group.launch()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        group.launch()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    for p in plans:
        st, _ = p.get_status()
        if st != B.CL_OK:
            raise RuntimeError(B.error_string(st))
    total = sum(c for _, _, c in shapes)
    flops = sum((p.info["factor_flops"] + p.info["selinv_flops"]) * p.info["batch"] for p in plans)
    rec = {"precision": args.precision, "mode": args.mode, "shapes": args.shapes, "replicas": total,
           "ms_per_step": ms, "evals_per_s": total / (ms / 1e3), "front_tflops": flops / (ms / 1e3) / 1e12,
           "panels": panels, "launches_per_step": sum(p.info["launches_per_eval"] for p in plans),
           "device_gb": sum(p.info["device_bytes"] for p in plans) / 1e9,
           "workspace_gb": sum(p.info["workspace_bytes"] for p in plans) / 1e9,
           "roofline": roofline(args.precision, flops / (ms / 1e3) / 1e12), "per_shape": []}
    site0 = 0
    for i, (ns, nt, cnt) in enumerate(shapes):
        V = ns ** 3 * nt
        entry = {"lattice": "%dx%d" % (ns, nt), "replicas": cnt}
        if args.mode == "merged":
            K = outs[0]["Kf"][0, site0:site0 + V].cpu().numpy()
        else:
            K = outs[i]["Kf"][0].cpu().numpy()
            entry["max_front"] = plans[i].info["max_front"]
        if not args.no_check:
            ref = B.Plan.analyze(ns, nt, 1, B.CL_FP64_EMU)
            r = ref.alloc_outputs()
            ref.drift_eval(torch.from_numpy(U[i][:1].copy()).to("cuda"), 0.05, 0.25, 1.0, None, r["Gfwd"],
                           r["Gbwd"], r["Kf"])
            torch.cuda.synchronize()
            want = r["Kf"][0].cpu().numpy()
            entry["drift_rel_err_vs_single_plan"] = float(np.abs(K - want).max() / np.abs(want).max())
            ref.close()
        rec["per_shape"].append(entry)
        site0 += cnt * V
    print(json.dumps(rec), flush=True)
    group.close()
    for p in plans:
        p.close()


if __name__ == "__main__":
    main()
