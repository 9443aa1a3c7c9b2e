"""Batched and ragged drift evaluations in one captured CUDA graph.

    python -m paper_1707_08874_gb300.run_batched [--precision fp64_emu|fp64|mixed]
        [--shapes 8x4:64]  or  [--shapes 4x4:16,6x4:16,8x6:8]  [--steps 5] [--tune]

Each --shapes entry is NsxNt:count (count replicas of that lattice).  All
shapes are evaluated side by side (one plan per shape on its own stream) and
the whole schedule is captured once into a CUDA graph; the timed loop replays
it.  Prints one JSON line: evaluations per second over all replicas, per
shape, and the drift error of replica 0 of every shape against the native
FP64 GPU path on the same links.
"""
from __future__ import annotations

import argparse
import json


def parse_shapes(text):
    out = []
    for tok in text.split(","):
        dims, cnt = tok.split(":")
        ns, nt = dims.split("x")
        out.append((int(ns), int(nt), int(cnt)))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--shapes", default="8x4:64")
    ap.add_argument("--precision", choices=["fp64", "fp64_emu", "mixed"], default="fp64_emu")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--tune", action="store_true", help="autotune the panel width per shape")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--warm", type=int, default=2, help="graph launches before the timed ones")
    args = ap.parse_args(argv)

    import numpy as np
    import torch

    from . import autotune
    from . import binding as B
    from . import inputs

    prec = {"fp64": B.CL_FP64, "fp64_emu": B.CL_FP64_EMU, "mixed": B.CL_MIXED_FP32}[args.precision]
    shapes = parse_shapes(args.shapes)
    plans, links, outs, panels = [], [], [], []
    for i, (ns, nt, cnt) in enumerate(shapes):
        if args.tune:
            plan, panel = autotune.tuned_plan(ns, nt, cnt, prec)
        else:
            plan = B.Plan.analyze(ns, nt, cnt, prec)
            panel = plan.info["panel"]
        plans.append(plan)
        panels.append(panel)
        links.append(torch.from_numpy(inputs.random_links(ns, nt, seed=inputs.BASE_SEED + 1000 * i,
                                                          batch=cnt)).to("cuda"))
        outs.append(plan.alloc_outputs())
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
    flops = sum((p.info["factor_flops"] + p.info["selinv_flops"]) * c for p, (_, _, c) in zip(plans, shapes))
    rec = {"precision": args.precision, "shapes": args.shapes, "replicas": total, "ms_per_step": ms,
           "evals_per_s": total / (ms / 1e3), "front_tflops": flops / (ms / 1e3) / 1e12, "panels": panels,
           "device_gb": sum(p.info["device_bytes"] for p in plans) / 1e9,
           "workspace_gb": sum(p.info["workspace_bytes"] for p in plans) / 1e9, "per_shape": []}
    for (ns, nt, cnt), p, o, l in zip(shapes, plans, outs, links):
        entry = {"lattice": "%dx%d" % (ns, nt), "replicas": cnt, "max_front": p.info["max_front"]}
        if not args.no_check and prec != B.CL_FP64:
            ref = B.Plan.analyze(ns, nt, 1, B.CL_FP64)
            r = ref.alloc_outputs()
            ref.drift_eval(l[:1].contiguous(), 0.05, 0.25, 1.0, None, r["Gfwd"], r["Gbwd"], r["Kf"])
            torch.cuda.synchronize()
            a = o["Kf"][0].cpu().numpy()
            b = r["Kf"][0].cpu().numpy()
            entry["drift_rel_err_vs_fp64"] = float(np.abs(a - b).max() / np.abs(b).max())
            ref.close()
        rec["per_shape"].append(entry)
    print(json.dumps(rec), flush=True)
    group.close()
    for p in plans:
        p.close()


if __name__ == "__main__":
    main()
