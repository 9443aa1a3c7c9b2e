"""GPU parity of the stochastic estimator of the drift (Eq. 7, the paper's
comparison path): the row-vector solves w = eta^dag D^{-1} from the factors of
cl_factor, the estimated selected blocks and the estimated drift against the
oracle's literal Eq. 7 for the same noise vectors, the complete-basis case
that makes the estimator exact, and a ragged plan."""
import numpy as np
import pytest

import oracle
from paper_1707_08874_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M, MU = 0.05, 0.25


def _B():
    from paper_1707_08874_gb300 import binding as B
    return B


def _z4(rng, shape):
    return rng.choice(np.array([1.0, 1j, -1.0, -1j]), size=shape)


def _run(plan, U, eta):
    links = torch.from_numpy(np.ascontiguousarray(U).reshape((1, -1, 4, 3, 3))).to("cuda")
    e = torch.from_numpy(np.ascontiguousarray(eta)).to("cuda")
    w = torch.empty_like(e)
    out = plan.alloc_outputs()
    work = plan.stochastic_drift(links, M, MU, 1.0, e, w, out["Gdiag"], out["Gfwd"], out["Gbwd"], out["Kf"])
    torch.cuda.synchronize()
    del work
    st, _ = plan.get_status()
    return w.cpu().numpy(), {k: v.cpu().numpy().reshape((-1,) + v.shape[2:]) for k, v in out.items()}, st


@pytest.mark.parametrize("prec", ["fp64_emu", "fp64"])
def test_left_solve_and_estimate_match_oracle(prec):
    B = _B()
    ns, nt = 6, 4
    V = ns ** 3 * nt
    U = inputs.random_links(ns, nt, seed=81)
    eta = _z4(np.random.default_rng(2), (4, V, 3))
    plan = B.Plan.analyze(ns, nt, 1, B.CL_FP64_EMU if prec == "fp64_emu" else B.CL_FP64)
    w, out, st = _run(plan, U, eta)
    assert st == B.CL_OK
    D = oracle.dirac_dense(ns, nt, U, M, MU)
    G = oracle.inverse(*oracle.lu(D)[:2])
    # the FP64 path's bar; the plain-FP64 tensor-pipe path's factors carry its
    # static-pivoting bound max(1e-10, 1e-13 kappa(D)) (as its selected blocks)
    bar = 1e-10
    if prec == "fp64":
        sv = np.linalg.svd(D, compute_uv=False)
        bar = max(bar, 1e-13 * sv[0] / sv[-1])
    want = (eta.reshape(4, 3 * V).conj() @ G).reshape(4, V, 3)
    assert np.abs(w - want).max() < bar * np.abs(want).max()
    K = oracle.stochastic_drift(ns, nt, U, M, MU, eta)
    assert np.abs(out["Kf"] - K).max() < bar * np.abs(K).max()
    # the estimated blocks are averages of outer products eta w^T
    up = oracle.neighbour_table(ns, nt)
    Pf = np.einsum("ixa,ixnb->xnab", eta, w[:, up]) / 4
    assert np.abs(out["Gfwd"] - Pf).max() < 1e-12 * np.abs(Pf).max()
    plan.close()


def test_complete_basis_gives_the_exact_drift():
    """With the N unit vectors (random phases, scaled by sqrt(N)) as noise the
    estimator is the exact drift: the GPU estimate equals the selected-
    inversion drift and the oracle's drift at 1e-10."""
    B = _B()
    ns, nt = 4, 4
    V = ns ** 3 * nt
    N = 3 * V
    U = inputs.random_links(ns, nt, seed=82)
    phase = np.exp(2j * np.pi * np.random.default_rng(4).random(N))
    eta = (np.sqrt(N) * phase[:, None] * np.eye(N)).reshape(N, V, 3)
    plan = B.Plan.analyze(ns, nt, 1, B.CL_FP64_EMU)
    w, out, st = _run(plan, U, eta)
    assert st == B.CL_OK
    ref = oracle.drift_eval(ns, nt, U, M, MU)
    for key in ("Gdiag", "Gfwd", "Gbwd"):
        assert np.abs(out[key] - ref[key]).max() < 1e-10 * np.abs(ref[key]).max(), key
    assert np.abs(out["Kf"] - ref["Kf"]).max() < 1e-10 * np.abs(ref["Kf"]).max()
    plan.close()


def test_estimator_statistics_and_ragged_plan():
    """A ragged plan (two shapes): each lattice's left solutions match the
    oracle; with 64 Z4 noise vectors the estimate lies within a few standard
    errors of the exact drift, and one vector alone is far from it."""
    B = _B()
    shapes = [(4, 4, 2), (4, 6, 1)]
    lat = [(ns, nt) for ns, nt, c in shapes for _ in range(c)]
    Us = [inputs.random_links(ns, nt, seed=90 + i) for i, (ns, nt) in enumerate(lat)]
    sites = sum(ns ** 3 * nt for ns, nt in lat)
    n = 64
    eta = _z4(np.random.default_rng(9), (n, sites, 3))
    plan = B.Plan.analyze_ragged(shapes, B.CL_FP64_EMU)
    links = np.concatenate([U.reshape((-1, 4, 3, 3)) for U in Us])
    w, out, st = _run(plan, links, eta)
    assert st == B.CL_OK
    s0 = 0
    for (ns, nt), U in zip(lat, Us):
        V = ns ** 3 * nt
        D = oracle.dirac_dense(ns, nt, U, M, MU)
        G = oracle.inverse(*oracle.lu(D)[:2])
        e = eta[:, s0:s0 + V]
        want = (e.reshape(n, 3 * V).conj() @ G).reshape(n, V, 3)
        assert np.abs(w[:, s0:s0 + V] - want).max() < 1e-10 * np.abs(want).max()
        samples = oracle.stochastic_drift(ns, nt, U, M, MU, e, per_vector=True)
        K = out["Kf"][s0:s0 + V]
        assert np.abs(K - samples.mean(0)).max() < 1e-10 * np.abs(K).max()
        exact = oracle.drift_eval(ns, nt, U, M, MU)["Kf"]
        se = np.sqrt(samples.real.var(0) + samples.imag.var(0)) / np.sqrt(n)
        z = np.abs(K - exact) / se
        assert np.percentile(z, 99) < 4.0 and z.max() < 8.0
        s0 += V
    plan.close()
