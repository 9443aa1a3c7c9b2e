"""Ragged groups of plans (several lattice shapes with their own replica
batches, evaluated side by side), CUDA-graph capture and replay of the whole
fixed schedule, and the panel-width autotuner."""
import numpy as np
import pytest

import oracle
from paper_1707_08874_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M, MU = 0.05, 0.25
SHAPES = [(4, 4, 2), (6, 4, 1), (4, 6, 2)]


def _B():
    from paper_1707_08874_gb300 import binding as B
    return B


def _setup(prec, seed0):
    B = _B()
    plans, links, outs = [], [], []
    for i, (ns, nt, b) in enumerate(SHAPES):
        plans.append(B.Plan.analyze(ns, nt, b, prec))
        links.append(torch.from_numpy(inputs.random_links(ns, nt, seed=seed0 + 10 * i, batch=b)).to("cuda"))
        outs.append(plans[-1].alloc_outputs())
    return plans, links, outs


@pytest.mark.parametrize("prec_name", ["fp64", "fp64_emu"])
def test_group_matches_plans_and_graph_replay(prec_name):
    B = _B()
    prec = B.CL_FP64 if prec_name == "fp64" else B.CL_FP64_EMU
    plans, links, outs = _setup(prec, 300)
    # reference: each plan on its own
    ref = []
    for p, l, o in zip(plans, links, outs):
        p.drift_eval(l, M, MU, 1.0, None, o["Gfwd"], o["Gbwd"], o["Kf"])
        torch.cuda.synchronize()
        ref.append(o["Kf"].cpu().numpy())
    g = B.Group(plans)
    outs2 = [p.alloc_outputs() for p in plans]
    g.drift_eval(links, M, MU, 1.0, [o["Gfwd"] for o in outs2], [o["Gbwd"] for o in outs2],
                 [o["Kf"] for o in outs2])
    torch.cuda.synchronize()
    for r, o in zip(ref, outs2):
        assert np.array_equal(r, o["Kf"].cpu().numpy())
    # capture once, then replay on new link values written into the same buffers
    outs3 = [p.alloc_outputs() for p in plans]
    g.capture(links, M, MU, 1.0, [o["Gfwd"] for o in outs3], [o["Gbwd"] for o in outs3],
              [o["Kf"] for o in outs3])
    for i, (ns, nt, b) in enumerate(SHAPES):
        links[i].copy_(torch.from_numpy(inputs.random_links(ns, nt, seed=900 + i, batch=b)))
    g.launch()
    torch.cuda.synchronize()
    for p, l, o3 in zip(plans, links, outs3):
        o = p.alloc_outputs()
        p.drift_eval(l, M, MU, 1.0, None, o["Gfwd"], o["Gbwd"], o["Kf"])
        torch.cuda.synchronize()
        assert np.array_equal(o["Kf"].cpu().numpy(), o3["Kf"].cpu().numpy())
        assert p.get_status()[0] == B.CL_OK
    # replica 0 of the 6^3x4 shape against the oracle
    U = links[1][0].cpu().numpy()
    want = oracle.drift_eval(6, 4, U, M, MU)["Kf"]
    got = outs3[1]["Kf"][0].cpu().numpy()
    assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()
    g.close()
    for p in plans:
        p.close()


def test_autotuner_picks_a_candidate(tmp_path, monkeypatch):
    B = _B()
    from paper_1707_08874_gb300 import autotune
    monkeypatch.setenv("CLSELINV_TUNE_CACHE", str(tmp_path / "tune.json"))
    panel = autotune.tune_panel(4, 4, 1, B.CL_FP64_EMU)
    assert panel in autotune.CANDIDATES
    assert (tmp_path / "tune.json").exists()
    plan, p2 = autotune.tuned_plan(4, 4, 1, B.CL_FP64_EMU)  # served from the cache
    assert p2 == panel and plan.info["panel"] == panel
    U = inputs.random_links(4, 4, seed=5)
    o = plan.alloc_outputs()
    plan.drift_eval(torch.from_numpy(U[None].copy()).to("cuda"), M, MU, 1.0, o["Gdiag"], o["Gfwd"], o["Gbwd"],
                    o["Kf"])
    torch.cuda.synchronize()
    want = oracle.drift_eval(4, 4, U, M, MU)["Kf"]
    assert np.abs(o["Kf"][0].cpu().numpy() - want).max() < 1e-10 * np.abs(want).max()
    plan.close()
