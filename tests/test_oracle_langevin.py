"""Pins of the oracle's Langevin pieces (Eq. 3-5, Sec. 4.1): counter-based
noise against published known-answer vectors and its moments, the gauge drift
against finite differences of the Wilson action, exactness of the SL(3,C)
update, gauge cooling (invariants, monotone unitarity norm) and observables."""
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import langevin as L
from paper_1707_08874_gb300 import inputs

NS, NT = 4, 4
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    n = 0
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out = L.philox4x32_10(np.array([w[:4]], np.uint64), (w[4], w[5]))[0]
        assert [int(x) for x in out] == w[6:10]
        n += 1
    assert n == 3


def test_noise_moments():
    """<eta_a> = 0 and <eta_a eta_b> = 2 delta_ab (standard CL normalisation)."""
    V = 8 ** 3 * 4
    eta = np.concatenate([L.noise(1234, s, V).reshape(-1, 8) for s in range(4)])
    n = eta.shape[0]
    assert np.abs(eta.mean(0)).max() < 5 * np.sqrt(2.0 / n)
    C = eta.T @ eta / n
    np.testing.assert_allclose(np.diag(C), 2.0, atol=5 * 2 * np.sqrt(2.0 / n))
    off = C - np.diag(np.diag(C))
    assert np.abs(off).max() < 5 * 2 / np.sqrt(n)
    # distinct steps, replicas and seeds give distinct streams
    a = L.noise(1, 0, 16)
    assert not np.allclose(a, L.noise(1, 1, 16))
    assert not np.allclose(a, L.noise(1, 0, 16, replica=1))
    assert not np.allclose(a, L.noise(2, 0, 16))


@pytest.fixture(scope="module")
def links():
    return inputs.random_links(NS, NT, seed=31)


def test_gauge_drift_finite_differences(links):
    """K^g_a = -d/dh S_g(e^{i h lambda_a} U_{x,nu}) at h = 0."""
    U = links
    beta = 5.0
    K = L.gauge_drift(U, beta, NS, NT)
    lam = inputs._GM
    h = 1e-5
    kmax = np.abs(K).max()
    for (s, nu) in ((0, 0), (45, 3), (130, 1), (255, 2)):
        for a in range(8):
            Up = U.copy()
            Um = U.copy()
            Up[s, nu] = scipy.linalg.expm(1j * h * lam[a]) @ U[s, nu]
            Um[s, nu] = scipy.linalg.expm(-1j * h * lam[a]) @ U[s, nu]
            fd = -(L.gauge_action(Up, beta, NS, NT) - L.gauge_action(Um, beta, NS, NT)) / (2 * h)
            assert abs(fd - K[s, nu, a]) < 1e-7 * kmax, (s, nu, a)


def test_gauge_drift_real_for_su3():
    U = inputs.random_links(NS, NT, seed=8, sigma_im=0.0)
    K = L.gauge_drift(U, 5.0, NS, NT)
    assert np.abs(K.imag).max() < 1e-12 * np.abs(K).max()
    # unit links: every plaquette is 1, the drift vanishes
    assert np.abs(L.gauge_drift(inputs.unit_links(NS, NT), 5.0, NS, NT)).max() < 1e-14


def test_link_update_exact(links):
    U = links
    V = U.shape[0]
    rng = np.random.default_rng(0)
    K = rng.normal(size=(V, 4, 8)) + 1j * rng.normal(size=(V, 4, 8))
    eta = L.noise(5, 0, V)
    U2 = L.link_update(U, K, 1e-3, eta)
    R = U2 @ np.linalg.inv(U)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-13)
    # real drift + real noise keep SU(3) links unitary (Eq. 4 with real K)
    Us = inputs.random_links(NS, NT, seed=2, sigma_im=0.0)
    U3 = L.link_update(Us, K.real, 1e-3, eta)
    I3 = np.conj(np.swapaxes(U3, -1, -2)) @ U3
    np.testing.assert_allclose(I3, np.broadcast_to(np.eye(3), I3.shape), atol=1e-13)
    # R = exp(X) against a high-order Taylor series
    X = L.algebra(1e-3 * K[0, 0] + np.sqrt(1e-3) * eta[0, 0])
    T = np.eye(3, dtype=complex)
    term = np.eye(3, dtype=complex)
    for n in range(1, 30):
        term = term @ X / n
        T = T + term
    np.testing.assert_allclose(L.expm_batch(X[None])[0], T, atol=1e-15)


def test_step_size_rule():
    K = np.zeros((4, 4, 8), complex)
    K[1, 2, 3] = 3 + 4j
    eps, km = L.step_size(K, 1e-3, 1e-3)
    assert km == 5.0 and eps == pytest.approx(2e-4)
    eps, km = L.step_size(K, 1e-3, 0.0)
    assert eps == 1e-3


def test_cooling_invariants(links):
    U = links
    n0 = L.unitarity_norm(U)
    o0 = L.observables(U, NS, NT)
    prev = n0
    Uc = U
    for _ in range(3):
        Uc = L.gauge_cool(Uc, 1, 0.05, NS, NT)
        n = L.unitarity_norm(Uc)
        assert n <= prev + 1e-12
        prev = n
    assert prev < n0
    o1 = L.observables(Uc, NS, NT)
    for k in ("plaq_s", "plaq_t", "poly", "poly_inv"):
        assert abs(o1[k] - o0[k]) < 1e-12, k
    np.testing.assert_allclose(np.linalg.det(Uc), 1.0, atol=1e-12)
    # det D and hence the physics are unchanged by the gauge transformation
    a = oracle.drift_eval(NS, NT, U, 0.05, 0.25)["logdet"]
    b = oracle.drift_eval(NS, NT, Uc, 0.05, 0.25)["logdet"]
    assert abs(a.real - b.real) < 1e-10 * abs(a.real)


def test_cooling_gradient_is_the_norm_gradient(links):
    """The cooling direction (Sec. 4.1, gauge cooling) is the gradient of the
    unitarity norm under gauge transformations.  A transformation exp(h X) at
    one site x (X traceless) changes N_U at the rate (2 / 4V) Re Tr(X f_x);
    checked by central differences at several sites and directions, which
    fixes the sign and both neighbour terms of f.  f is also Hermitian and
    traceless, and the norm, which is 0 on SU(3) links, has f = 0 there."""
    U = links
    V = U.shape[0]
    f = L.cooling_gradient(U, NS, NT)
    np.testing.assert_allclose(f, np.conj(np.swapaxes(f, -1, -2)), atol=1e-12)
    assert np.abs(np.trace(f, axis1=1, axis2=2)).max() < 1e-12
    rng = np.random.default_rng(17)
    h = 1e-5
    for x in (0, 37, V - 1):
        for _ in range(2):
            X = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
            X -= np.trace(X) / 3 * np.eye(3)
            n = []
            for sgn in (1, -1):
                om = np.broadcast_to(np.eye(3, dtype=complex), (V, 3, 3)).copy()
                om[x] = scipy.linalg.expm(sgn * h * X)
                n.append(L.unitarity_norm(inputs.gauge_transform(U, om, NS, NT)))
            fd = (n[0] - n[1]) / (2 * h)
            want = 2.0 / (4 * V) * np.trace(X @ f[x]).real
            assert abs(fd - want) < 1e-6 * abs(want) + 1e-12, (x, fd, want)
    su3 = inputs.unit_links(NS, NT)
    assert abs(L.unitarity_norm(su3)) < 1e-15
    assert np.abs(L.cooling_gradient(su3, NS, NT)).max() < 1e-15


def test_observables_unit_and_gauge_invariant(links):
    o = L.observables(inputs.unit_links(NS, NT), NS, NT)
    for k in ("plaq_s", "plaq_t", "poly", "poly_inv"):
        assert abs(o[k] - 1) < 1e-15
    assert abs(o["unitarity"]) < 1e-15
    Om = inputs.random_gauge(NS, NT, seed=9)
    U2 = inputs.gauge_transform(links, Om, NS, NT)
    a = L.observables(links, NS, NT)
    b = L.observables(U2, NS, NT)
    for k in ("plaq_s", "plaq_t", "poly", "poly_inv"):
        assert abs(a[k] - b[k]) < 1e-12, k


def test_renorm_det_pins():
    """Determinant renormalisation: det U = 1 afterwards; SL(3,C) links are
    left as they are; a positive real factor on U is removed exactly (the
    principal cube root of c^3 det U is c det(U)^{1/3})."""
    rng = np.random.default_rng(12)
    U = inputs.random_links(4, 4, seed=31)
    A = U * (1.3 * np.exp(0.4j))
    R = L.renorm_det(A)
    assert np.abs(np.linalg.det(R) - 1).max() < 1e-13
    assert np.abs(L.renorm_det(U) - U).max() < 1e-13 * np.abs(U).max()
    c = rng.uniform(0.5, 2.0)
    assert np.abs(L.renorm_det(c * A) - R).max() < 1e-13 * np.abs(R).max()


def _sl3(rng):
    """a random SL(3,C) matrix (non-unitary, non-diagonal)"""
    A = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3)) + 2 * np.eye(3)
    return A / np.linalg.det(A) ** (1.0 / 3.0)


def test_observables_closed_form_planes_and_time_order():
    """Links with a closed-form answer that tells the plaquette planes and the
    time order of the Polyakov product apart (c10).  All spatial links are one
    diagonal SL(3,C) matrix Dg (they commute, so every spatial plaquette is the
    identity), the temporal links of time slice t are one non-diagonal
    SL(3,C) matrix W_t, constant in space.  Then
      plaq_s = 1,
      plaq_t = (1/3) mean_t Tr(Dg W_t Dg^{-1} W_t^{-1})      (path x -> x+mu -> x+mu+t -> x+t),
      P  = (1/3) Tr(W_0 W_1 ... W_{Nt-1}),  P' = (1/3) Tr((W_0 ... W_{Nt-1})^{-1}),
      N_U = (1/4) [3 (Tr Dg Dg^dag - 3) + mean_t (Tr W_t W_t^dag - 3)].
    Swapping the spatial and temporal sets, or multiplying the temporal links
    in the reverse time order, changes these values (checked below)."""
    rng = np.random.default_rng(2024)
    ns, nt = 4, 4
    vs = ns ** 3
    d = np.exp(1j * rng.normal(size=3) * 0.7 + rng.normal(size=3) * 0.3)
    Dg = np.diag(d / np.prod(d) ** (1.0 / 3.0))
    W = [_sl3(rng) for _ in range(nt)]
    U = np.empty((vs * nt, 4, 3, 3), np.complex128)
    for t in range(nt):
        U[t * vs:(t + 1) * vs, :3] = Dg
        U[t * vs:(t + 1) * vs, 3] = W[t]
    o = L.observables(U, ns, nt)
    Di = np.linalg.inv(Dg)
    pt = np.mean([np.trace(Dg @ w @ Di @ np.linalg.inv(w)) for w in W]) / 3
    line = np.linalg.multi_dot(W)
    rev = np.linalg.multi_dot(W[::-1])
    nu = 0.25 * (3 * (np.trace(Dg @ Dg.conj().T).real - 3) +
                 np.mean([np.trace(w @ w.conj().T).real - 3 for w in W]))
    assert abs(o["plaq_s"] - 1) < 1e-13
    assert abs(o["plaq_t"] - pt) < 1e-13
    assert abs(o["poly"] - np.trace(line) / 3) < 1e-13
    assert abs(o["poly_inv"] - np.trace(np.linalg.inv(line)) / 3) < 1e-13
    assert abs(o["unitarity"] - nu) < 1e-12
    # the pins separate the readings: temporal plaquettes differ from 1, the
    # reversed product has another trace, and the inverse loop is not conj(P)
    assert abs(pt - 1) > 1e-2
    assert abs(np.trace(rev) - np.trace(line)) > 1e-2
    assert abs(np.trace(np.linalg.inv(line)) - np.conj(np.trace(line))) > 1e-2


def test_reunitarize_pins():
    """SU(3) projection: the result is unitary with det 1 for SL(3,C) input;
    SU(3) links are left as they are; the first row keeps its direction and
    the second row stays in the span of the first two input rows (the
    defining properties of Gram-Schmidt)."""
    U = inputs.random_links(4, 4, seed=33)
    R = L.reunitarize(U)
    eye = np.eye(3)
    assert np.abs(R @ np.conj(np.swapaxes(R, -1, -2)) - eye).max() < 1e-13
    assert np.abs(np.linalg.det(R) - 1).max() < 1e-13
    S = inputs.random_links(4, 4, seed=34, sigma_im=0.0)
    assert np.abs(L.reunitarize(S) - S).max() < 1e-13
    r0 = U[..., 0, :]
    assert np.abs(R[..., 0, :] - r0 / np.linalg.norm(r0, axis=-1, keepdims=True)).max() < 1e-14
    # R[1] is a combination of U[0], U[1]: orthogonal to the cross product of U[0], U[1]
    n = np.cross(U[..., 0, :], U[..., 1, :])
    assert np.abs(np.sum(n * R[..., 1, :], axis=-1)).max() < 1e-12
    # R[2] is orthogonal to both input rows in the hermitian sense
    for j in range(2):
        assert np.abs(np.sum(np.conj(U[..., j, :]) * R[..., 2, :], axis=-1)).max() < 1e-12
