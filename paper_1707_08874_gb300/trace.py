"""Timeline of one profiled drift evaluation (cl_profile_trace).

    python -m paper_1707_08874_gb300.trace [--Ns 8] [--Nt 4] [--precision fp64_emu]
        [--panel 0] [--reps 20] [--out trace.json]

Runs a few unprofiled evaluations, then --reps evaluations with per-launch
events (cl_profile_enable), sampling the SM clock meanwhile, and prints per
tree level the medians over the repetitions of the span of the
factorisation's launches and of the busy time of each of its two streams (0:
panel chain, 1: bulk updates), the median duration of each kernel family on
the root front (and of a panel inverse per pivot column), and the span of the
selected inversion.  Profiled launches carry event records between them and
launch without programmatic overlap, so the timeline attributes time; the
headline rate comes from bench.py.  --out writes the last repetition's raw
records and the factorisation's op table as JSON.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile


def summarise(trace):
    """Per-level spans and stream busy times of the factorisation, root-front
    kernel medians, and the selected-inversion span, from profile records."""
    levels = {}
    for t in trace:
        if t["phase"] != 0:
            continue
        d = levels.setdefault(t["level"], dict(t0=float("inf"), t1=0.0, busy=[0.0, 0.0], launches=[0, 0]))
        d["t0"] = min(d["t0"], t["t0_us"])
        d["t1"] = max(d["t1"], t["t1_us"])
        d["busy"][t["stream"]] += t["t1_us"] - t["t0_us"]
        d["launches"][t["stream"]] += 1
    out = {"levels": {h: dict(span_us=d["t1"] - d["t0"], chain_busy_us=d["busy"][0], bulk_busy_us=d["busy"][1],
                              chain_launches=d["launches"][0], bulk_launches=d["launches"][1])
                      for h, d in sorted(levels.items())}}
    top = max((h for h in levels if h >= 0), default=None)
    fam = {}
    for t in trace:
        if t["phase"] == 0 and t["level"] == top:
            fam.setdefault("%s/stream%d" % (t["name"], t["stream"]), []).append(t["t1_us"] - t["t0_us"])
    out["root_median_us"] = {k: dict(launches=len(v), median=statistics.median(v)) for k, v in sorted(fam.items())}
    sel = [t for t in trace if t["phase"] == 1]
    if sel:
        out["selinv_span_us"] = max(t["t1_us"] for t in sel) - min(t["t0_us"] for t in sel)
    out["total_us"] = max(t["t1_us"] for t in trace) if trace else 0.0
    return out


def merge(summaries):
    """Medians over repetitions of the per-level and root-family figures."""
    med = statistics.median
    out = {"levels": {}, "root_median_us": {}, "reps": len(summaries)}
    for h in summaries[0]["levels"]:
        out["levels"][h] = {k: med(s["levels"][h][k] for s in summaries) for k in summaries[0]["levels"][h]}
    for k in summaries[0]["root_median_us"]:
        out["root_median_us"][k] = dict(launches=summaries[0]["root_median_us"][k]["launches"],
                                        median=med(s["root_median_us"][k]["median"] for s in summaries))
    for k in ("selinv_span_us", "total_us"):
        if k in summaries[0]:
            out[k] = med(s[k] for s in summaries)
    return out


class SmClock:
    """SM clock samples of one GPU (nvidia-smi, every 50 ms) while running."""

    def __enter__(self):
        self.samples = []
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_trace_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
            self.proc = subprocess.Popen(["nvidia-smi", "-i", dev, "--query-gpu=clocks.sm,clocks.max.sm",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is None:
            return False
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        for line in open(self.path).read().splitlines():
            f = [x.strip() for x in line.split(",")]
            try:
                self.samples.append((float(f[0]), float(f[1])))
            except (ValueError, IndexError):
                pass
        os.unlink(self.path)
        return False

    def summary(self):
        if not self.samples:
            return None
        return dict(sm_mhz=statistics.median(a for a, _ in self.samples),
                    sm_max_mhz=max(b for _, b in self.samples), samples=len(self.samples))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--Ns", type=int, default=8)
    ap.add_argument("--Nt", type=int, default=4)
    ap.add_argument("--precision", choices=["fp64", "fp64_emu", "mixed", "fp32"], default="fp64_emu")
    ap.add_argument("--panel", type=int, default=0)
    ap.add_argument("--seed", type=int, default=1707)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    import torch
    from . import binding as B, inputs
    prec = {"fp64": B.CL_FP64, "fp64_emu": B.CL_FP64_EMU, "mixed": B.CL_MIXED_BF16X3,
            "fp32": B.CL_MIXED_FP32}[args.precision]
    plan = B.Plan.analyze_ex(args.Ns, args.Nt, 1, prec, args.panel)
    U = torch.from_numpy(inputs.random_links(args.Ns, args.Nt, seed=args.seed)[None].copy()).cuda()
    o = plan.alloc_outputs()
    for _ in range(3):
        plan.drift_eval(U, 0.05, 0.25, 1.0, o["Gdiag"], o["Gfwd"], o["Gbwd"], o["Kf"])
    torch.cuda.synchronize()
    sums = []
    with SmClock() as clk:
        for _ in range(max(1, args.reps)):
            plan.profile_enable(True)  # clears the previous repetition's records
            plan.drift_eval(U, 0.05, 0.25, 1.0, o["Gdiag"], o["Gfwd"], o["Gbwd"], o["Kf"])
            torch.cuda.synchronize()
            trace = plan.profile_trace()
            sums.append(summarise(trace))
    plan.profile_enable(False)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(dict(trace=trace, factor_ops=plan.export_tables()["factor_ops"].tolist()), f)
    s = merge(sums)
    s["clocks"] = clk.summary()
    s["panel"] = plan.info["panel"]
    print("medians over %d profiled evaluations; SM clock %s" % (s["reps"], s["clocks"]))
    for h, d in s["levels"].items():
        print("level %2d: span %8.1f us  chain busy %8.1f us (%d launches)  bulk busy %8.1f us (%d)"
              % (h, d["span_us"], d["chain_busy_us"], d["chain_launches"], d["bulk_busy_us"], d["bulk_launches"]))
    for k, v in s["root_median_us"].items():
        print("root %-24s %4d launches, median %7.1f us" % (k, v["launches"], v["median"]))
    pin = s["root_median_us"].get("panel_inverse/stream0")
    if pin and s["panel"]:
        print("root panel inverse per pivot column %.2f us" % (pin["median"] / s["panel"]))
    if "selinv_span_us" in s:
        print("selected inversion span %.1f us" % s["selinv_span_us"])
    print("total %.1f us" % s["total_us"])
    print(json.dumps(dict(summary=s)))
    plan.close()


if __name__ == "__main__":
    main()
