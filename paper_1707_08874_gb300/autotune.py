"""Autotuner of the front schedule: picks the pivoting-panel width per lattice
shape, batch and precision by timing complete drift evaluations on the
device (narrow panels shorten the serial chain of FP64 panel inverses; wide
panels make fewer, larger GEMM launches).  Results are cached in a JSON file
keyed by GPU name, shape, batch and precision.

    plan, panel = autotune.tuned_plan(8, 4, batch=1, precision=B.CL_FP64_EMU)
"""
from __future__ import annotations

import json
import os

from . import binding as B
from . import inputs

CANDIDATES = (12, 24, 30, 48)


def cache_path() -> str:
    return os.environ.get("CLSELINV_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "clselinv", "panel_tuning.json"))


def _key(Ns, Nt, batch, precision):
    import torch
    return "%s|%dx%d|b%d|p%d" % (torch.cuda.get_device_name(), Ns, Nt, batch, precision)


def time_panel(Ns, Nt, batch, precision, panel, links, steps=2) -> float:
    """ms per drift evaluation of a plan with the given panel width."""
    import torch
    plan = B.Plan.analyze_ex(Ns, Nt, batch, precision, panel)
    o = plan.alloc_outputs()
    plan.drift_eval(links, 0.05, 0.25, 1.0, None, o["Gfwd"], o["Gbwd"], o["Kf"])
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan.drift_eval(links, 0.05, 0.25, 1.0, None, o["Gfwd"], o["Gbwd"], o["Kf"])
    e1.record()
    torch.cuda.synchronize()
    st, _ = plan.get_status()
    plan.close()
    if st != B.CL_OK:
        return float("inf")
    return e0.elapsed_time(e1) / steps


def tune_panel(Ns, Nt, batch=1, precision=B.CL_FP64_EMU, candidates=CANDIDATES, use_cache=True) -> int:
    import torch
    path = cache_path()
    key = _key(Ns, Nt, batch, precision)
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return int(cache[key]["panel"])
    links = torch.from_numpy(inputs.random_links(Ns, Nt, seed=inputs.BASE_SEED, batch=batch)).to("cuda")
    times = {p: time_panel(Ns, Nt, batch, precision, p, links) for p in candidates}
    best = min(times, key=times.get)
    if use_cache:
        cache[key] = {"panel": best, "ms": {str(k): v for k, v in times.items()}}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            json.dump(cache, open(path, "w"), indent=1)
        except OSError:
            pass
    return best


def tune_panel_ragged(shapes, precision=B.CL_FP64_EMU, candidates=CANDIDATES, steps=2) -> int:
    """Panel width of a ragged plan (one width for all its shapes), timed on
    the plan itself (not cached: the shape mix is the caller's)."""
    import numpy as np
    import torch
    links = torch.from_numpy(np.concatenate(
        [inputs.random_links(ns, nt, seed=inputs.BASE_SEED + i, batch=c).reshape((-1, 4, 3, 3))
         for i, (ns, nt, c) in enumerate(shapes)])[None].copy()).to("cuda")
    times = {}
    for panel in candidates:
        plan = B.Plan.analyze_ragged(shapes, precision, panel)
        o = plan.alloc_outputs()
        plan.drift_eval(links, 0.05, 0.25, 1.0, None, o["Gfwd"], o["Gbwd"], o["Kf"])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.drift_eval(links, 0.05, 0.25, 1.0, None, o["Gfwd"], o["Gbwd"], o["Kf"])
        e1.record()
        torch.cuda.synchronize()
        st, _ = plan.get_status()
        plan.close()
        times[panel] = e0.elapsed_time(e1) / steps if st == B.CL_OK else float("inf")
    return min(times, key=times.get)


def tuned_plan(Ns, Nt, batch=1, precision=B.CL_FP64_EMU, **kw):
    panel = tune_panel(Ns, Nt, batch, precision, **kw)
    return B.Plan.analyze_ex(Ns, Nt, batch, precision, panel), panel
