"""Per-launch profiling: the aggregated records (cl_profile_read) and the
timeline (cl_profile_trace) of one evaluation through the C ABI."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _binding():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_08874_gb300 import binding as B
    return B


def test_profile_trace_matches_schedule():
    import torch
    from paper_1707_08874_gb300 import inputs
    B = _binding()
    plan = B.Plan.analyze(6, 4, 1, B.CL_FP64_EMU)
    U = torch.from_numpy(inputs.random_links(6, 4, seed=3)[None].copy()).cuda()
    o = plan.alloc_outputs()
    plan.drift_eval(U, 0.05, 0.25, 1.0, o["Gdiag"], o["Gfwd"], o["Gbwd"], o["Kf"])
    torch.cuda.synchronize()
    plan.profile_enable(True)
    plan.drift_eval(U, 0.05, 0.25, 1.0, o["Gdiag"], o["Gfwd"], o["Gbwd"], o["Kf"])
    torch.cuda.synchronize()
    agg = plan.profile_read()
    tr = plan.profile_trace()
    plan.profile_enable(False)
    # one record per profiled launch, the same count as the aggregate
    assert len(tr) == sum(v["launches"] for v in agg.values())
    for name, v in agg.items():
        recs = [t for t in tr if t["name"] == name]
        assert len(recs) == v["launches"]
        tot = sum(t["t1_us"] - t["t0_us"] for t in recs) * 1e-3
        assert tot == pytest.approx(v["total_ms"], rel=1e-3, abs=1e-3)
    tabs = plan.export_tables()
    n_factor, n_selinv = tabs["factor_ops"].shape[0], tabs["selinv_ops"].shape[0]
    for t in tr:
        assert t["t1_us"] >= t["t0_us"] >= 0.0
        assert t["phase"] in (-1, 0, 1)
        if t["phase"] == 0:
            assert 0 <= t["op"] < n_factor and t["stream"] in (0, 1)
        elif t["phase"] == 1:
            assert 0 <= t["op"] < n_selinv and t["stream"] == 0
    # the two-stream factorisation puts its bulk updates on stream 1
    assert any(t["stream"] == 1 for t in tr if t["phase"] == 0)
    assert tr[0]["t0_us"] == 0.0
    # the factorisation precedes the selected inversion on the caller's stream
    f_end = max(t["t1_us"] for t in tr if t["phase"] == 0)
    s_start = min(t["t0_us"] for t in tr if t["phase"] == 1)
    assert s_start >= f_end - 1.0
    assert np.isfinite([t["t1_us"] for t in tr]).all()
    plan.close()
