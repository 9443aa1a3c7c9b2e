"""GPU parity: the CUDA selected inversion and drift against the CPU oracle.

Tolerance (FP64 path).  The oracle is a dense LU with partial pivoting; the
multifrontal factorisation may pivot only inside each supernode's panels
(static ordering, as in every supernodal selected inversion).  Its rounding
error is therefore bounded by the condition number of D times a growth factor
of the static ordering: on the paper's link distribution the measured ratio
err / kappa(D) is about 1e-14.  The bar is the 1e-10 normwise target wherever
kappa(D) allows it and 1e-13 * kappa(D) above (kappa from the oracle's own
dense D), for the G blocks (max_b |dG_b|_F / max_b |G_b|_F) and for the drift
(max |dK| / max |K|).
"""
import numpy as np
import pytest

import oracle
from paper_1707_08874_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M, MU = 0.05, 0.25


def _binding():
    from paper_1707_08874_gb300 import binding as B
    return B


def _tol(D):
    sv = np.linalg.svd(D, compute_uv=False)
    kappa = sv[0] / sv[-1]
    return max(1e-10, 1e-13 * kappa), kappa


def _blockwise(a, b):
    da = np.sqrt((np.abs(a - b) ** 2).sum((-1, -2)))
    nb = np.sqrt((np.abs(b) ** 2).sum((-1, -2)))
    return da.max() / nb.max()


def _run(plan, U, m=M, mu=MU, nf=1.0):
    B = _binding()
    links = torch.from_numpy(np.ascontiguousarray(U)).to("cuda")
    if links.dim() == 4:
        links = links.unsqueeze(0)
    out = plan.alloc_outputs()
    plan.drift_eval(links.contiguous(), m, mu, nf, out["Gdiag"], out["Gfwd"], out["Gbwd"], out["Kf"])
    torch.cuda.synchronize()
    st, detail = plan.get_status()
    return {k: v.cpu().numpy() for k, v in out.items()}, st


PRECS = ["fp64", "fp64_emu"]


def _prec(B, name):
    return {"fp64": B.CL_FP64, "fp64_emu": B.CL_FP64_EMU, "mixed": B.CL_MIXED_FP32}[name]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("ns,nt,seed", [(4, 4, 1707), (4, 4, 1), (6, 4, 1707), (4, 6, 3)])
def test_fp64_parity_small(ns, nt, seed, prec):
    """FP64 fronts, and FP64 fronts whose GEMMs are exact BF16 digit products
    (CL_FP64_EMU): both held to the FP64 bar."""
    B = _binding()
    U = inputs.random_links(ns, nt, seed=seed)
    ref = oracle.drift_eval(ns, nt, U, M, MU)
    tol, kappa = _tol(oracle.dirac_dense(ns, nt, U, M, MU))
    plan = B.Plan.analyze(ns, nt, 1, _prec(B, prec))
    got, st = _run(plan, U)
    assert st == B.CL_OK
    for name, key in (("Gdiag", "Gdiag"), ("Gfwd", "Gfwd"), ("Gbwd", "Gbwd")):
        err = _blockwise(got[key][0], ref[key])
        assert err < tol, (name, err, tol, kappa)
    kerr = np.abs(got["Kf"][0] - ref["Kf"]).max() / np.abs(ref["Kf"]).max()
    assert kerr < tol, (kerr, tol, kappa)
    plan.close()



_REF64 = {}


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("panel", [12, 27, 30, 48])
def test_fp64_parity_panel_widths(panel, prec):
    """Every width instantiation of the panel inverse (24-, 32- and 48-wide
    blocks); 27 and 30 leave a ragged last panel in most supernodes, 30 is the
    widest panel whose products stay single-chunk digit GEMMs."""
    B = _binding()
    U = inputs.random_links(6, 4, seed=1707)
    if not _REF64:
        _REF64["ref"] = oracle.drift_eval(6, 4, U, M, MU)
        _REF64["tol"] = _tol(oracle.dirac_dense(6, 4, U, M, MU))
    ref, (tol, kappa) = _REF64["ref"], _REF64["tol"]
    plan = B.Plan.analyze_ex(6, 4, 1, _prec(B, prec), panel)
    assert plan.info["panel"] == panel
    got, st = _run(plan, U)
    assert st == B.CL_OK
    for key in ("Gdiag", "Gfwd", "Gbwd"):
        err = _blockwise(got[key][0], ref[key])
        assert err < tol, (key, err, tol, kappa)
    kerr = np.abs(got["Kf"][0] - ref["Kf"]).max() / np.abs(ref["Kf"]).max()
    assert kerr < tol, (kerr, tol, kappa)
    plan.close()

def test_fp64_free_field_and_su3():
    """U = 1 (free field) and SU(3) links at mu = 0 (real drift)."""
    B = _binding()
    plan = B.Plan.analyze(4, 4, 1, B.CL_FP64)
    U = inputs.unit_links(4, 4)
    ref = oracle.drift_eval(4, 4, U, M, MU)
    got, st = _run(plan, U)
    assert st == B.CL_OK
    assert _blockwise(got["Gfwd"][0], ref["Gfwd"]) < 1e-11
    U = inputs.random_links(4, 4, seed=9, sigma_im=0.0)
    ref = oracle.drift_eval(4, 4, U, M, 0.0)
    got, st = _run(plan, U, mu=0.0)
    assert np.abs(got["Kf"][0] - ref["Kf"]).max() < 1e-10 * np.abs(ref["Kf"]).max()
    assert np.abs(got["Kf"][0].imag).max() < 1e-10 * np.abs(got["Kf"][0]).max()
    plan.close()


@pytest.mark.parametrize("prec", PRECS)
def test_fp64_batch_replicas_independent(prec):
    """A batch of replicas gives each replica's own result (no cross-talk)."""
    B = _binding()
    U = inputs.random_links(4, 4, seed=40, batch=3)
    plan = B.Plan.analyze(4, 4, 3, _prec(B, prec))
    got, st = _run(plan, U)
    assert st == B.CL_OK
    for b in range(3):
        ref = oracle.drift_eval(4, 4, U[b], M, MU)
        tol, _ = _tol(oracle.dirac_dense(4, 4, U[b], M, MU))
        assert _blockwise(got["Gbwd"][b], ref["Gbwd"]) < tol
        assert np.abs(got["Kf"][b] - ref["Kf"]).max() < tol * np.abs(ref["Kf"]).max()
    plan.close()


@pytest.mark.parametrize("prec", PRECS)
def test_fp64_repeatable_bitwise(prec):
    """Two evaluations of the same links give identical bits (no atomics)."""
    B = _binding()
    U = inputs.random_links(6, 4, seed=5)
    plan = B.Plan.analyze(6, 4, 1, _prec(B, prec))
    a, _ = _run(plan, U)
    b, _ = _run(plan, U)
    assert np.array_equal(a["Kf"], b["Kf"]) and np.array_equal(a["Gfwd"], b["Gfwd"])
    plan.close()


def test_free_chain_sms_bitwise(monkeypatch):
    """The SMs the bulk digit GEMMs leave to the panel chain only change which
    persistent CTA computes which output tile: bitwise identical results."""
    B = _binding()
    U = inputs.random_links(6, 4, seed=9)
    outs = []
    for free in ("0", "2", "24"):
        monkeypatch.setenv("CLSELINV_CHAIN_SMS", free)
        plan = B.Plan.analyze(6, 4, 1, B.CL_FP64_EMU)
        got, st = _run(plan, U)
        assert st == B.CL_OK
        outs.append(got)
        plan.close()
    for got in outs[1:]:
        for key in ("Gdiag", "Gfwd", "Gbwd", "Kf"):
            assert np.array_equal(got[key], outs[0][key]), key


def test_nonfinite_status():
    """A NaN link is reported through the status word, not a fault."""
    B = _binding()
    U = inputs.random_links(4, 4, seed=2)
    U[17, 2, 1, 1] = np.nan
    plan = B.Plan.analyze(4, 4, 1, B.CL_FP64)
    got, st = _run(plan, U)
    assert st in (B.CL_ERR_NONFINITE, B.CL_ERR_SINGULAR)
    U = inputs.random_links(4, 4, seed=2)
    got, st = _run(plan, U)
    assert st == B.CL_OK
    plan.close()


@pytest.fixture(scope="module")
def full_size():
    ns, nt = 8, 4
    U = inputs.random_links(ns, nt, seed=1707)
    D = oracle.dirac_dense(ns, nt, U, M, MU)
    tol, kappa = _tol(D)
    LU, piv, info = oracle.lu(D)
    assert info == 0
    return U, D, tol, LU, piv


@pytest.mark.parametrize("prec", PRECS)
def test_fp64_full_size_sampled(prec, full_size):
    """8^3 x 4 (the benchmark workload, batch 1): sampled columns of D^{-1} from
    the oracle's LU, every selected block touching them, the drift of the links
    whose both blocks are known, and D G = 1 on every site."""
    B = _binding()
    ns, nt = 8, 4
    V = ns ** 3 * nt
    U, D, tol, LU, piv = full_size
    plan = B.Plan.analyze(ns, nt, 1, _prec(B, prec))
    got, st = _run(plan, U)
    assert st == B.CL_OK
    Gd, Gf, Gb, K = got["Gdiag"][0], got["Gfwd"][0], got["Gbwd"][0], got["Kf"][0]
    # D G = 1 on the diagonal blocks, from the selected blocks only
    up = inputs.shift_table(ns, nt)
    dn = np.empty_like(up)
    for nu in range(4):
        dn[up[:, nu], nu] = np.arange(V)
    Db = D.reshape(V, 3, V, 3).transpose(0, 2, 1, 3)
    x = np.arange(V)
    dg = M * Gd
    for nu in range(4):
        dg = dg + Db[x, up[:, nu]] @ Gb[:, nu] + Db[x, dn[:, nu]] @ Gf[dn[:, nu], nu]
    gnorm = np.sqrt((np.abs(Gf) ** 2).sum((-1, -2))).max()
    assert np.abs(dg - np.eye(3)).max() < 10 * tol * gnorm
    # sampled columns
    rng = np.random.default_rng(0)
    ys = rng.choice(V, 6, replace=False)
    sites = sorted(set(int(y) for y in ys) | {int(up[y, nu]) for y in ys for nu in range(4)})
    cols = np.array([3 * s + a for s in sites for a in range(3)])
    X = oracle.solve_unit_columns(LU, piv, cols)
    col = {s: X[:, 3 * i:3 * i + 3] for i, s in enumerate(sites)}
    scale = np.sqrt((np.abs(Gf) ** 2).sum((-1, -2))).max()
    Gf_ref = np.zeros_like(Gf)
    Gb_ref = np.zeros_like(Gb)
    for y in ys:
        blk = lambda x: col[int(y)][3 * x:3 * x + 3]
        assert np.linalg.norm(Gd[y] - blk(y)) < tol * scale
        for nu in range(4):
            yp = int(up[y, nu])
            assert np.linalg.norm(Gb[y, nu] - blk(yp)) < tol * scale          # G_{y+nu,y}
            assert np.linalg.norm(Gf[dn[y, nu], nu] - blk(int(dn[y, nu]))) < tol * scale  # G_{y-nu,y}
            Gb_ref[y, nu] = blk(yp)
            Gf_ref[y, nu] = col[yp][3 * y:3 * y + 3]                          # G_{y,y+nu}
            assert np.linalg.norm(Gf[y, nu] - Gf_ref[y, nu]) < tol * scale
    Kref = oracle.fermion_drift(ns, nt, U, Gf_ref, Gb_ref, MU)
    kmax = np.abs(K).max()
    assert np.abs(K[ys] - Kref[ys]).max() < tol * kmax
    plan.close()


@pytest.mark.parametrize("prec", PRECS)
def test_singular_panel_reported(prec):
    """m = 0, mu = 0 and one temporal link of -1 on the ring of sites
    (1,1,1,t): the ring's holonomy cancels the antiperiodic sign, so that leaf's
    pivot block has an exact zero mode (static pivoting cannot avoid it) and the
    status word names the supernode; a regular configuration clears it."""
    B = _binding()
    plan = B.Plan.analyze(4, 4, 1, _prec(B, prec))
    leaf = [i for i in range(plan.info["n_supernodes"]) if 21 in plan.node(i)["sep"]][0]
    U = inputs.unit_links(4, 4)
    U[21, 3] = -np.eye(3)
    links = torch.from_numpy(U[None].copy()).to("cuda")
    out = plan.alloc_outputs()
    plan.drift_eval(links, 0.0, 0.0, 1.0, out["Gdiag"], out["Gfwd"], out["Gbwd"], out["Kf"])
    st, detail = plan.get_status()
    assert st == B.CL_ERR_SINGULAR and detail[0] == leaf
    got, st = _run(plan, inputs.random_links(4, 4, seed=8))
    assert st == B.CL_OK
    plan.close()
