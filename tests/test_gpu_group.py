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


@pytest.mark.parametrize("prec_name", ["fp64_emu", "mixed"])
def test_ragged_plan_merged_schedule(prec_name):
    """cl_analyze_ragged: lattices of three shapes in one plan whose schedule
    runs every step of a level as one launch over all their fronts.  Each
    lattice's blocks and drift are bitwise those of its own single-shape plan
    (the same per-tile arithmetic), match the oracle at 1e-10 in the FP64
    path, and a captured graph of the ragged evaluation replays them."""
    B = _B()
    prec = B.CL_FP64_EMU if prec_name == "fp64_emu" else B.CL_MIXED_BF16X3
    plan = B.Plan.analyze_ragged(SHAPES, prec)
    assert plan.info["n_shapes"] == 3 and plan.info["batch"] == sum(c for _, _, c in SHAPES)
    Us, singles = [], []
    for i, (ns, nt, b) in enumerate(SHAPES):
        U = inputs.random_links(ns, nt, seed=500 + 10 * i, batch=b)
        Us.append(U)
        p = B.Plan.analyze(ns, nt, b, prec)
        o = p.alloc_outputs()
        p.drift_eval(torch.from_numpy(U).to("cuda"), M, MU, 1.0, o["Gdiag"], o["Gfwd"], o["Gbwd"], o["Kf"])
        torch.cuda.synchronize()
        assert p.get_status()[0] == B.CL_OK
        singles.append({k: v.cpu().numpy().reshape((-1,) + v.shape[2:]) for k, v in o.items()})
        p.close()
    links = torch.from_numpy(np.concatenate([U.reshape((-1, 4, 3, 3)) for U in Us])[None].copy()).to("cuda")
    out = plan.alloc_outputs()
    plan.drift_eval(links, M, MU, 1.0, out["Gdiag"], out["Gfwd"], out["Gbwd"], out["Kf"])
    torch.cuda.synchronize()
    assert plan.get_status()[0] == B.CL_OK
    got = {k: v[0].cpu().numpy() for k, v in out.items()}
    s0 = 0
    for i, (ns, nt, b) in enumerate(SHAPES):
        n = b * ns ** 3 * nt
        for k in ("Gdiag", "Gfwd", "Gbwd", "Kf"):
            assert np.array_equal(got[k][s0:s0 + n], singles[i][k]), (i, k)
        if prec_name == "fp64_emu":
            V = ns ** 3 * nt
            for r in range(b):
                ref = oracle.drift_eval(ns, nt, Us[i][r], M, MU)
                K = got["Kf"][s0 + r * V:s0 + (r + 1) * V]
                assert np.abs(K - ref["Kf"]).max() < 1e-10 * np.abs(ref["Kf"]).max()
        s0 += n
    # the whole ragged evaluation captured once as a graph and replayed
    g = B.Group([plan])
    out2 = plan.alloc_outputs()
    g.capture([links], M, MU, 1.0, [out2["Gfwd"]], [out2["Gbwd"]], [out2["Kf"]])
    g.launch()
    torch.cuda.synchronize()
    assert np.array_equal(out2["Kf"][0].cpu().numpy(), got["Kf"])
    g.close()
    # Langevin calls need a single-shape plan
    with pytest.raises(B.CLError):
        plan.gauge_drift(links, 5.0, torch.zeros((1, plan.info["V"], 4, 8), dtype=torch.complex128, device="cuda"))
    plan.close()
