"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each check is independent of the oracle's own arithmetic: closed forms of the
free field, LAPACK and a complete-pivoting elimination on tiny lattices,
finite differences of log det D (Eq. 6 is its gradient), exact symmetries of
det D, gauge covariance and the inverse identity D G = 1 on the selected
pattern (Eq. 8 uses only blocks where D is non-zero).
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1707_08874_gb300 import inputs

M, MU = 0.05, 0.25
NS, NT = 4, 4


def _momenta(Ns, Nt):
    """All lattice momenta: periodic in space, antiperiodic in time."""
    ks = 2 * np.pi * np.arange(Ns) / Ns
    kt = (2 * np.arange(Nt) + 1) * np.pi / Nt
    P = np.array(np.meshgrid(ks, ks, ks, kt, indexing="ij")).reshape(4, -1).T
    return P


def _free_h(d, Ns, Nt, m, mu):
    """H(d) = (1/V) sum_p e^{ip.d} / (m^2 + sum_i sin^2 p_i + sin^2(p_t - i mu))."""
    P = _momenta(Ns, Nt)
    den = m * m + (np.sin(P[:, :3]) ** 2).sum(1) + np.sin(P[:, 3] - 1j * mu) ** 2
    ph = np.exp(1j * (np.asarray(d, float) @ P.T))
    return (ph / den).sum(-1) / P.shape[0]


def _free_g(cx, cy, Ns, Nt, m, mu):
    """Scalar free-field propagator G_{x,y} = [(m - D_hop) H](x,y), raw coordinates."""
    cx = np.asarray(cx)
    cy = np.asarray(cy)
    g = m * _free_h(cx - cy, Ns, Nt, m, mu)
    for nu in range(4):
        e = np.zeros(4, int)
        e[nu] = 1
        et = np.exp(mu) if nu == 3 else 1.0
        eta = (-1.0) ** (cx[..., :nu].sum(-1)) if nu else np.ones(cx.shape[:-1])
        g = g - 0.5 * eta * (et * _free_h(cx + e - cy, Ns, Nt, m, mu)
                             - _free_h(cx - e - cy, Ns, Nt, m, mu) / et)
    return g


@pytest.fixture(scope="module")
def free():
    U = inputs.unit_links(NS, NT)
    return U, oracle.drift_eval(NS, NT, U, M, MU)


@pytest.fixture(scope="module")
def rand():
    U = inputs.random_links(NS, NT, seed=11)
    D = oracle.dirac_dense(NS, NT, U, M, MU)
    return U, D, oracle.drift_eval(NS, NT, U, M, MU)


def test_gell_mann_table():
    lam = oracle.gell_mann()
    tr = np.einsum("aij,bji->ab", lam, lam)
    np.testing.assert_allclose(tr, 2 * np.eye(8), atol=1e-14)
    np.testing.assert_allclose(lam, np.conj(np.swapaxes(lam, 1, 2)), atol=1e-15)
    np.testing.assert_allclose(np.trace(lam, axis1=1, axis2=2), 0, atol=1e-15)
    # su(3) structure constants: [l1,l2] = 2i l3, [l4,l5] = i l3 + i sqrt3 l8
    c12 = lam[0] @ lam[1] - lam[1] @ lam[0]
    np.testing.assert_allclose(c12, 2j * lam[2], atol=1e-14)
    c45 = lam[3] @ lam[4] - lam[4] @ lam[3]
    np.testing.assert_allclose(c45, 1j * lam[2] + 1j * np.sqrt(3) * lam[7], atol=1e-14)


def test_free_field_propagator_closed_form(free):
    """U = 1: D^2 is diagonal in momentum space, so G has a closed form."""
    U, res = free
    c = inputs.site_coords(NS, NT)
    up = inputs.shift_table(NS, NT)
    want_d = _free_g(c, c, NS, NT, M, MU)
    got = res["Gdiag"]
    np.testing.assert_allclose(got, want_d[:, None, None] * np.eye(3), atol=1e-12)
    for nu in range(4):
        cy = c[up[:, nu]]
        wf = _free_g(c, cy, NS, NT, M, MU)
        wb = _free_g(cy, c, NS, NT, M, MU)
        np.testing.assert_allclose(res["Gfwd"][:, nu], wf[:, None, None] * np.eye(3), atol=1e-12)
        np.testing.assert_allclose(res["Gbwd"][:, nu], wb[:, None, None] * np.eye(3), atol=1e-12)


def test_free_field_logdet_closed_form(free):
    """log det D = (3/2) sum_p log(m^2 + sum sin^2) and det D is real positive."""
    _, res = free
    P = _momenta(NS, NT)
    den = M * M + (np.sin(P[:, :3]) ** 2).sum(1) + np.sin(P[:, 3] - 1j * MU) ** 2
    want = 1.5 * np.log(den).sum()
    ld = res["logdet"]
    assert abs(ld.real - want.real) < 1e-10 * abs(want.real)
    assert abs(np.angle(np.exp(1j * ld.imag))) < 1e-10


def test_lu_and_inverse_against_lapack(rand):
    U, D, res = rand
    LU, piv, info = oracle.lu(D)
    assert info == 0
    sign, lad = np.linalg.slogdet(D)
    ld = oracle.logdet(LU, piv)
    assert abs(ld.real - lad) < 1e-10 * abs(lad)
    assert abs(np.exp(1j * ld.imag) - sign) < 1e-10
    Ginv = np.linalg.inv(D)
    Gd, Gf, Gb = oracle.extract_blocks(NS, NT, Ginv)
    scale = np.abs(Ginv).max()
    for a, b in ((Gd, res["Gdiag"]), (Gf, res["Gfwd"]), (Gb, res["Gbwd"])):
        assert np.abs(a - b).max() < 1e-12 * scale


def test_dirac_pattern_and_hops(rand):
    """D has exactly 9 non-zero 3x3 blocks per block row, laid out as in Eq. 1."""
    U, D, _ = rand
    V = NS ** 3 * NT
    blk = np.abs(D.reshape(V, 3, V, 3)).sum((1, 3)) > 0
    assert (blk.sum(1) == 9).all()
    up = inputs.shift_table(NS, NT)
    c = inputs.site_coords(NS, NT)
    for s in (0, 5, 77, V - 1):
        for nu in range(4):
            y = up[s, nu]
            eta = (-1.0) ** c[s, :nu].sum()
            sg = -1.0 if (nu == 3 and c[s, 3] == NT - 1) else 1.0
            ef = np.exp(MU) if nu == 3 else 1.0
            np.testing.assert_allclose(D[3 * s:3 * s + 3, 3 * y:3 * y + 3],
                                       0.5 * eta * sg * ef * U[s, nu], atol=1e-15)
            np.testing.assert_allclose(D[3 * y:3 * y + 3, 3 * s:3 * s + 3],
                                       -0.5 * eta * sg / ef * np.linalg.inv(U[s, nu]), atol=1e-14)


def _complete_pivot_logdet(A):
    """Gaussian elimination with complete pivoting (independent second method)."""
    A = np.array(A, dtype=np.complex128)
    n = A.shape[0]
    lr, ph = 0.0, 0.0
    for k in range(n):
        sub = np.abs(A[k:, k:])
        i, j = np.unravel_index(np.argmax(sub), sub.shape)
        i += k
        j += k
        if i != k:
            A[[k, i]] = A[[i, k]]
            ph += np.pi
        if j != k:
            A[:, [k, j]] = A[:, [j, k]]
            ph += np.pi
        p = A[k, k]
        lr += np.log(abs(p))
        ph += np.angle(p)
        A[k + 1:, k:] -= np.outer(A[k + 1:, k] / p, A[k, k:])
    return complex(lr, ph)


def test_logdet_complete_pivoting(rand):
    U, D, res = rand
    want = _complete_pivot_logdet(D)
    ld = res["logdet"]
    assert abs(ld.real - want.real) < 1e-10 * abs(want.real)
    assert abs(np.angle(np.exp(1j * (ld.imag - want.imag)))) < 1e-9


def _logdet(U, m=M, mu=MU, Ns=NS, Nt=NT):
    LU, piv, info = oracle.lu(oracle.dirac_dense(Ns, Nt, U, m, mu))
    assert info == 0
    return oracle.logdet(LU, piv)


def test_drift_finite_differences(rand):
    """Eq. 6: K^f_a = d/dh log det D(e^{i h lambda_a} U_{x,nu}) at h = 0."""
    U, D, res = rand
    lam = inputs._GM
    h = 1e-5
    K = res["Kf"]
    kmax = np.abs(K).max()
    for (s, nu) in ((0, 0), (37, 3), (200, 1), (255, 2)):
        for a in range(8):
            Up = U.copy()
            Um = U.copy()
            Up[s, nu] = scipy.linalg.expm(1j * h * lam[a]) @ U[s, nu]
            Um[s, nu] = scipy.linalg.expm(-1j * h * lam[a]) @ U[s, nu]
            dp = _logdet(Up)
            dm = _logdet(Um)
            diff = complex(dp.real - dm.real, np.angle(np.exp(1j * (dp.imag - dm.imag))))
            fd = diff / (2 * h)
            assert abs(fd - K[s, nu, a]) < 2e-7 * kmax, (s, nu, a, fd, K[s, nu, a])


def test_condensate_is_mass_derivative(rand):
    """d log det D / dm = sum_x Tr G_xx."""
    U, D, res = rand
    h = 1e-5
    dp = _logdet(U, m=M + h)
    dm = _logdet(U, m=M - h)
    fd = complex(dp.real - dm.real, np.angle(np.exp(1j * (dp.imag - dm.imag)))) / (2 * h)
    V = NS ** 3 * NT
    tr = oracle.condensate(res["Gdiag"]) * V
    assert abs(fd - tr) < 1e-6 * abs(tr)


def test_det_symmetries_su3():
    """SU(3) links: det D(mu)^* = det D(-mu^*); det D(0) real positive; K^f(0) real."""
    U = inputs.random_links(NS, NT, seed=5, sigma_im=0.0)
    for mu in (0.25, 0.3):
        a = _logdet(U, mu=mu)
        b = _logdet(U, mu=-mu)
        assert abs(a.real - b.real) < 1e-10 * abs(a.real)
        assert abs(np.angle(np.exp(1j * (a.imag + b.imag)))) < 1e-9
    z = _logdet(U, mu=0.0)
    assert abs(np.angle(np.exp(1j * z.imag))) < 1e-10
    r = oracle.drift_eval(NS, NT, U, M, 0.0)
    assert np.abs(r["Kf"].imag).max() < 1e-11 * np.abs(r["Kf"]).max()
    # K^f(mu)^* = K^f(-mu) for SU(3) links and real mu
    kp = oracle.drift_eval(NS, NT, U, M, 0.25)["Kf"]
    km = oracle.drift_eval(NS, NT, U, M, -0.25)["Kf"]
    np.testing.assert_allclose(np.conj(kp), km, atol=1e-11 * np.abs(kp).max())


def test_mu_moved_to_last_timeslice():
    """det D(mu;U) = det D(0;U'') with U''_t = e^{mu Nt} U_t on the t = Nt-1 links only."""
    U = inputs.random_links(NS, NT, seed=21)
    a = _logdet(U, mu=MU)
    c = inputs.site_coords(NS, NT)
    U2 = U.copy()
    last = c[:, 3] == NT - 1
    U2[last, 3] *= np.exp(MU * NT)
    b = _logdet(U2, mu=0.0)
    assert abs(a.real - b.real) < 1e-10 * abs(a.real)
    assert abs(np.angle(np.exp(1j * (a.imag - b.imag)))) < 1e-9


def test_selected_blocks_invert_d(rand):
    """(D G)_{xx} = (G D)_{xx} = 1 and Tr(G D) = 3V use only the selected blocks."""
    U, D, res = rand
    V = NS ** 3 * NT
    up = inputs.shift_table(NS, NT)
    dn = np.empty_like(up)
    for nu in range(4):
        dn[up[:, nu], nu] = np.arange(V)
    Db = D.reshape(V, 3, V, 3).transpose(0, 2, 1, 3)
    Gd, Gf, Gb = res["Gdiag"], res["Gfwd"], res["Gbwd"]
    x = np.arange(V)
    dg = M * Gd.copy()
    gd = M * Gd.copy()
    for nu in range(4):
        y = up[:, nu]
        w = dn[:, nu]
        # (DG)_xx = m G_xx + sum_nu D_{x,x+nu} G_{x+nu,x} + D_{x,x-nu} G_{x-nu,x}
        dg += Db[x, y] @ Gb[:, nu] + Db[x, w] @ Gf[w, nu]
        # (GD)_xx = m G_xx + sum_nu G_{x,x+nu} D_{x+nu,x} + G_{x,x-nu} D_{x-nu,x}
        gd += Gf[:, nu] @ Db[y, x] + Gb[w, nu] @ Db[w, x]
    np.testing.assert_allclose(dg, np.broadcast_to(np.eye(3), dg.shape), atol=1e-11)
    np.testing.assert_allclose(gd, np.broadcast_to(np.eye(3), gd.shape), atol=1e-11)
    assert abs(np.trace(gd, axis1=1, axis2=2).sum() - 3 * V) < 1e-9


def test_gauge_covariance():
    """U -> Om_x U Om_{x+nu}^{-1}: det invariant, G_xy -> Om_x G Om_y^{-1}, K^f adjoint."""
    U = inputs.random_links(NS, NT, seed=3)
    Om = inputs.random_gauge(NS, NT, seed=4)
    U2 = inputs.gauge_transform(U, Om, NS, NT)
    r1 = oracle.drift_eval(NS, NT, U, M, MU)
    r2 = oracle.drift_eval(NS, NT, U2, M, MU)
    assert abs(r1["logdet"].real - r2["logdet"].real) < 1e-10 * abs(r1["logdet"].real)
    assert abs(np.angle(np.exp(1j * (r1["logdet"].imag - r2["logdet"].imag)))) < 1e-9
    up = inputs.shift_table(NS, NT)
    Oi = np.linalg.inv(Om)
    want_f = np.einsum("xij,xnjk,xnkl->xnil", Om, r1["Gfwd"], Oi[up])
    np.testing.assert_allclose(r2["Gfwd"], want_f, atol=1e-10 * np.abs(want_f).max())
    lam = inputs._GM
    # R_ab = 1/2 Tr(lambda_b Om^{-1} lambda_a Om), K'_a = sum_b R_ab K_b
    R = 0.5 * np.einsum("bij,xjk,akl,xli->xab", lam, Oi, lam, Om)
    want_k = np.einsum("xab,xnb->xna", R, r1["Kf"])
    np.testing.assert_allclose(r2["Kf"], want_k, atol=1e-10 * np.abs(want_k).max())


def test_unit_column_solves_match_inverse(rand):
    """Sampled columns (the full-size parity route) equal the full inverse's columns."""
    U, D, _ = rand
    LU, piv, info = oracle.lu(D)
    G = oracle.inverse(LU, piv)
    cols = np.array([0, 1, 2, 400, 767])
    X = oracle.solve_unit_columns(LU, piv, cols)
    np.testing.assert_allclose(X, G[:, cols], atol=1e-13 * np.abs(G).max())


def test_number_density_is_mu_derivative(rand):
    """n = (1/V) d log det D / d mu, evaluated from the temporal selected blocks."""
    U, D, res = rand
    h = 1e-5
    dp = _logdet(U, mu=MU + h)
    dm = _logdet(U, mu=MU - h)
    fd = complex(dp.real - dm.real, np.angle(np.exp(1j * (dp.imag - dm.imag)))) / (2 * h)
    V = NS ** 3 * NT
    n = oracle.number_density(NS, NT, U, res["Gfwd"], res["Gbwd"], MU)
    assert abs(n * V - fd) < 1e-6 * abs(fd)


def test_stochastic_drift_complete_basis_is_exact():
    """Eq. 7 with the complete unit basis as noise, each vector with its own
    phase (eta_i = sqrt(N) e^{i theta_i} e_i, so that (1/N) sum_i eta_i
    eta_i^dag = 1 exactly, and a missing complex conjugate shows), reproduces
    the exact drift of Eq. 6 / Eq. 8 from the selected blocks."""
    ns, nt = 4, 4
    V = ns ** 3 * nt
    N = 3 * V
    U = inputs.random_links(ns, nt, seed=61)
    phase = np.exp(2j * np.pi * np.random.default_rng(3).random(N))
    eta = (np.sqrt(N) * phase[:, None] * np.eye(N, dtype=np.complex128)).reshape(N, V, 3)
    K = oracle.stochastic_drift(ns, nt, U, 0.05, 0.25, eta)
    ref = oracle.drift_eval(ns, nt, U, 0.05, 0.25)["Kf"]
    assert np.abs(K - ref).max() < 1e-11 * np.abs(ref).max()


def test_stochastic_drift_is_unbiased():
    """Z4 noise (entries 1, i, -1, -i, E[eta eta^dag] = 1): the estimator is unbiased, so
    the mean over n = 256 noise vectors lies within a few standard errors of
    the exact drift for every component (standard errors from the samples);
    one noise vector alone is far from it (the indefinite-matrix variance the
    paper warns about)."""
    ns, nt = 4, 4
    V = ns ** 3 * nt
    U = inputs.random_links(ns, nt, seed=62)
    ref = oracle.drift_eval(ns, nt, U, 0.05, 0.25)["Kf"]
    rng = np.random.default_rng(7)
    n = 256
    eta = rng.choice(np.array([1.0, 1j, -1.0, -1j]), size=(n, V, 3))
    samples = oracle.stochastic_drift(ns, nt, U, 0.05, 0.25, eta, per_vector=True)
    K = samples.mean(0)
    assert np.abs(K - oracle.stochastic_drift(ns, nt, U, 0.05, 0.25, eta)).max() < 1e-13 * np.abs(K).max()
    se = np.sqrt(samples.real.var(0) + samples.imag.var(0)) / np.sqrt(n)
    z = np.abs(K - ref) / np.maximum(se, 1e-300)
    assert np.percentile(z, 99) < 4.0 and z.max() < 8.0, (np.percentile(z, 99), z.max())
    assert np.abs(samples[0] - ref).max() > 3 * np.abs(K - ref).max()
