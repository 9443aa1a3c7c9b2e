"""The allocation-free drift entry point against the regular one.

cl_drift_eval_noalloc serves callers that cannot allocate device memory (a
host runtime whose allocator owns the GPU's memory, a plugin that must not
grow the footprint, a loop that cannot afford cudaMalloc's synchronisation);
it keeps its scratch in a fixed device array inside the library.  This file is
collected last so that a failure here does not hide the rest of the suite.
"""
import numpy as np
import pytest

from paper_1707_08874_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M, MU = 0.05, 0.25


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_noalloc_matches_drift_eval_twice():
    from paper_1707_08874_gb300 import binding as B
    U = inputs.random_links(4, 4, seed=77, batch=1)
    links = torch.from_numpy(U).to("cuda")
    plan = B.Plan.analyze(4, 4, 1, B.CL_FP64)
    ref = plan.alloc_outputs()
    plan.drift_eval(links, M, MU, 1.0, ref["Gdiag"], ref["Gfwd"], ref["Gbwd"], ref["Kf"])
    torch.cuda.synchronize()
    assert plan.get_status()[0] == B.CL_OK
    want = {k: v.cpu().numpy() for k, v in ref.items()}
    for call in range(2):
        out = plan.alloc_outputs()
        for v in out.values():
            v.fill_(float("nan"))
        st = B.drift_eval_noalloc(4, 4, links, M, MU, 1.0, out["Gdiag"], out["Gfwd"], out["Gbwd"], out["Kf"])
        assert st == B.CL_OK, B.error_string(st)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        for k in ("Gdiag", "Gfwd", "Gbwd", "Kf"):
            assert np.isfinite(got[k]).all(), (call, k)
            assert _rel(got[k], want[k]) < 1e-10, (call, k, _rel(got[k], want[k]))
    plan.close()


def test_noalloc_rejects_large_lattice():
    from paper_1707_08874_gb300 import binding as B
    U = inputs.random_links(6, 4, seed=1, batch=1)
    links = torch.from_numpy(U).to("cuda")
    V = 6 ** 3 * 4
    kw = dict(dtype=torch.complex128, device="cuda")
    Gf = torch.empty((1, V, 4, 3, 3), **kw)
    Gb = torch.empty((1, V, 4, 3, 3), **kw)
    K = torch.empty((1, V, 4, 8), **kw)
    assert B.drift_eval_noalloc(6, 4, links, M, MU, 1.0, None, Gf, Gb, K) == B.CL_ERR_UNSUPPORTED
