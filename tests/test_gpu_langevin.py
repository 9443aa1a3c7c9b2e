"""GPU parity of the Langevin pieces (Eq. 3-5, Sec. 4.1) against the oracle:
gauge drift, link update with the shared Philox noise, gauge cooling,
observables, and whole steps with the fermion drift from the selected
inversion."""
import numpy as np
import pytest

import oracle
from oracle import langevin as L
from paper_1707_08874_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NS, NT = 4, 4


def _B():
    from paper_1707_08874_gb300 import binding as B
    return B


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def plan():
    B = _B()
    p = B.Plan.analyze(NS, NT, 2, B.CL_FP64)
    yield p
    p.close()


@pytest.fixture(scope="module")
def links2():
    return inputs.random_links(NS, NT, seed=500, batch=2)


def test_gauge_drift(plan, links2):
    V = NS ** 3 * NT
    Kg = torch.empty((2, V, 4, 8), dtype=torch.complex128, device="cuda")
    plan.gauge_drift(_dev(links2), 5.0, Kg)
    got = Kg.cpu().numpy()
    for b in range(2):
        want = L.gauge_drift(links2[b], 5.0, NS, NT)
        assert _rel(got[b], want) < 1e-12


def test_link_update_shared_noise(plan, links2):
    V = NS ** 3 * NT
    rng = np.random.default_rng(1)
    K = rng.normal(size=(2, V, 4, 8)) + 1j * rng.normal(size=(2, V, 4, 8))
    U = _dev(links2)
    plan.link_update(U, _dev(K), 1e-3, 99, 7)
    got = U.cpu().numpy()
    for b in range(2):
        want = L.link_update(links2[b], K[b], 1e-3, L.noise(99, 7, V, replica=b))
        assert _rel(got[b], want) < 1e-13


def test_gauge_cooling(plan, links2):
    U = _dev(links2)
    plan.gauge_cool(U, 3, 0.05)
    got = U.cpu().numpy()
    for b in range(2):
        want = L.gauge_cool(links2[b], 3, 0.05, NS, NT)
        assert _rel(got[b], want) < 1e-12
        assert L.unitarity_norm(got[b]) < L.unitarity_norm(links2[b])


def test_observables(plan, links2):
    B = _B()
    V = NS ** 3 * NT
    res = [oracle.drift_eval(NS, NT, links2[b], 0.05, 0.25) for b in range(2)]
    Gd = np.stack([r["Gdiag"] for r in res])
    Gf = np.stack([r["Gfwd"] for r in res])
    Gb = np.stack([r["Gbwd"] for r in res])
    obs = torch.zeros((2, 20), dtype=torch.float64, device="cuda")
    plan.observables(_dev(links2), _dev(Gd), _dev(Gf), _dev(Gb), 0.25, 1.0, obs)
    o = obs.cpu().numpy()
    for b in range(2):
        got = B.obs_dict(o[b])
        want = L.observables_full(links2[b], NS, NT, res[b], 0.25)
        for k in ("plaq_s", "plaq_t", "poly", "poly_inv", "condensate", "density"):
            assert abs(got[k] - want[k]) < 1e-12 * max(1.0, abs(want[k])), k
        assert abs(got["unitarity"] - want["unitarity"]) < 1e-12 * max(1.0, want["unitarity"])


@pytest.mark.parametrize("kappa,n_cool", [(0.0, 0), (2e-3, 2)])
def test_langevin_steps_match_oracle(plan, links2, kappa, n_cool):
    """Two full steps (fermion drift by selected inversion + gauge drift,
    adaptive step, noise, cooling) on both replicas."""
    B = _B()
    prm = dict(beta=5.0, m=0.05, mu=0.25, nf=1.0, eps_max=1e-3, kappa=kappa, alpha_cool=0.05, seed=2024,
               n_cool=n_cool, fermions=1)
    U = _dev(links2)
    state = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    obs = torch.zeros((2, 20), dtype=torch.float64, device="cuda")
    ref = [links2[0].copy(), links2[1].copy()]
    t = [0.0, 0.0]
    for step in range(2):
        plan.langevin_step(U, prm, state, obs)
        torch.cuda.synchronize()
        assert plan.get_status()[0] == B.CL_OK
        o = obs.cpu().numpy()
        for b in range(2):
            ref[b], ro, eps = L.langevin_step(ref[b], prm, step, NS, NT, replica=b)
            t[b] += eps
            go = B.obs_dict(o[b])
            assert abs(go["eps"] - eps) < 1e-9 * eps  # eps = kappa / K_max inherits the drift error
            assert abs(go["kmax"] - ro["kmax"]) < 1e-9 * ro["kmax"]
            for k in ("plaq_s", "plaq_t", "poly", "poly_inv", "condensate", "density"):
                assert abs(go[k] - ro[k]) < 1e-9 * max(1.0, abs(ro[k])), (step, b, k)
            assert go["step"] == step + 1 and abs(go["t"] - t[b]) < 1e-9 * t[b]
    got = U.cpu().numpy()
    for b in range(2):
        assert _rel(got[b], ref[b]) < 1e-11


def test_langevin_step_renorm_det(plan, links2):
    """The optional determinant renormalisation: links scaled off SL(3,C)
    come back to det U = 1 after one full step, matching the oracle step."""
    B = _B()
    prm = dict(beta=5.0, m=0.05, mu=0.25, nf=1.0, eps_max=1e-3, kappa=0.0, alpha_cool=0.05, seed=77,
               n_cool=1, fermions=1, renorm_det=1)
    U0 = links2 * (1.05 * np.exp(0.2j))
    U = _dev(U0)
    state = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    obs = torch.zeros((2, 20), dtype=torch.float64, device="cuda")
    plan.langevin_step(U, prm, state, obs)
    torch.cuda.synchronize()
    assert plan.get_status()[0] == B.CL_OK
    got = U.cpu().numpy()
    for b in range(2):
        ref, _, _ = L.langevin_step(U0[b].copy(), prm, 0, NS, NT, replica=b)
        assert _rel(got[b], ref) < 1e-11
        assert np.abs(np.linalg.det(got[b]) - 1).max() < 1e-12


def test_langevin_step_reunitarize(plan, links2):
    """The optional SU(3) reunitarisation (Sec. 4.2): after one full step at
    mu = 0 the links are in SU(3) to rounding and match the oracle step."""
    B = _B()
    prm = dict(beta=5.0, m=0.05, mu=0.0, nf=1.0, eps_max=1e-3, kappa=0.0, alpha_cool=0.05, seed=78,
               n_cool=0, fermions=1, renorm_det=0, reunit=1)
    U0 = links2
    U = _dev(U0)
    state = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    obs = torch.zeros((2, 20), dtype=torch.float64, device="cuda")
    plan.langevin_step(U, prm, state, obs)
    torch.cuda.synchronize()
    assert plan.get_status()[0] == B.CL_OK
    got = U.cpu().numpy()
    for b in range(2):
        ref, _, _ = L.langevin_step(U0[b].copy(), prm, 0, NS, NT, replica=b)
        assert _rel(got[b], ref) < 1e-11
        assert np.abs(got[b] @ np.conj(np.swapaxes(got[b], -1, -2)) - np.eye(3)).max() < 1e-13
        assert np.abs(np.linalg.det(got[b]) - 1).max() < 1e-13


def test_pure_gauge_su3_stays_unitary():
    """beta > 0, no fermions, SU(3) start: real drift and real noise keep the
    links in SU(3) (no excursion without a complex action)."""
    B = _B()
    p = B.Plan.analyze(NS, NT, 1, B.CL_FP64)
    U = _dev(inputs.random_links(NS, NT, seed=3, sigma_im=0.0, batch=1))
    prm = dict(beta=5.5, m=0.05, mu=0.0, nf=1.0, eps_max=1e-2, kappa=0.0, alpha_cool=0.05, seed=1,
               n_cool=0, fermions=0)
    state = torch.zeros((1, 4), dtype=torch.float64, device="cuda")
    obs = torch.zeros((1, 20), dtype=torch.float64, device="cuda")
    for _ in range(20):
        p.langevin_step(U, prm, state, obs)
    torch.cuda.synchronize()
    u = U.cpu().numpy()[0]
    I3 = np.conj(np.swapaxes(u, -1, -2)) @ u
    assert np.abs(I3 - np.eye(3)).max() < 1e-12
    assert B.obs_dict(obs.cpu().numpy()[0])["unitarity"] < 1e-12
    p.close()


def test_checkpoint_resume_bitwise(tmp_path):
    """4 steps straight == 2 steps, checkpoint, reload into fresh buffers, 2
    steps: the noise of step n depends only on (seed, n, link, replica)."""
    B = _B()
    from paper_1707_08874_gb300 import checkpoint
    prm = dict(beta=5.0, m=0.05, mu=0.25, nf=1.0, eps_max=1e-3, kappa=2e-3, alpha_cool=0.05, seed=77,
               n_cool=1, fermions=1)
    U0 = inputs.random_links(NS, NT, seed=12, batch=2)
    p = B.Plan.analyze(NS, NT, 2, B.CL_FP64_EMU)

    def run(U, state, n):
        obs = torch.zeros((2, 20), dtype=torch.float64, device="cuda")
        for _ in range(n):
            p.langevin_step(U, prm, state, obs)
        torch.cuda.synchronize()

    Ua = _dev(U0)
    sa = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    run(Ua, sa, 4)
    Ub = _dev(U0)
    sb = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    run(Ub, sb, 2)
    path = str(tmp_path / "ck.npz")
    checkpoint.save(path, Ub, sb, prm)
    U2, s2, prm2 = checkpoint.load(path)
    assert prm2 == prm
    Uc, sc = _dev(U2), _dev(s2)
    run(Uc, sc, 2)
    assert np.array_equal(Ua.cpu().numpy(), Uc.cpu().numpy())
    assert np.array_equal(sa.cpu().numpy(), sc.cpu().numpy())
    p.close()
