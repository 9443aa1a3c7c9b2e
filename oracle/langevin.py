"""Oracle for the complex-Langevin step (Sec. 2, Eq. 3-5; Sec. 4.1): gauge
drift, adaptive step, link update with Gaussian noise, gauge cooling and the
observables.  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Plain numpy in FP64, vectorised over links; 3x3 exponentials by scipy's expm.
Readings of what the paper leaves open (shared with the CUDA library):
  S_g = beta sum_P [1 - (Tr U_P + Tr U_P^{-1}) / 6]                  (c9)
  K^g_a = -d_a S_g = (i beta/6) sum_staples Tr[lambda_a (U A - A^{-1} U^{-1})]
  eta_a real Gaussian with <eta_a eta_b> = 2 delta_ab, drawn from Philox4x32-10
    (Salmon et al. 2011) with counter (link, half, step, replica), key = seed,
    and Box-Muller on u = (x + 1/2) 2^-32                                  (c6)
  eps = min(eps_max, kappa / K_max), K_max = max_link |K|_2 (kappa <= 0: eps_max) (c7)
  cooling: f_x = sum_nu [U_x U_x^dag - U_{x-nu}^dag U_{x-nu}] (traceless part),
    alpha = alpha0 / max_x |f_x|_F, Omega_x = exp(-alpha f_x),
    U_{x,nu} -> Omega_x U Omega_{x+nu}^{-1}                                (c8)
  unitarity norm N_U = (1/4V) sum [Tr U U^dag - 3]; plaquettes (1/3) Tr U_P
  averaged over spatial / temporal planes; Polyakov loop and its inverse
  (1/(3 Ns^3)) sum Tr prod_t U_t^{+-1}                                     (c10)
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import gell_mann

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon et al., SC'11).  ctr [...,4], key (k0, k1)."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.uint64(key[0]) & _MASK
    k1 = np.uint64(key[1]) & _MASK
    for _ in range(10):
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return np.stack(c, axis=-1).astype(np.uint32)


def noise(seed: int, step: int, V: int, replica: int = 0) -> np.ndarray:
    """eta[V,4,8]: for link l = 4 s + nu and half h, Philox(l, h, step, replica; seed)
    gives 4 words -> two Box-Muller pairs -> eta_{4h..4h+3}; <eta eta> = 2."""
    L = 4 * V
    ctr = np.zeros((L, 2, 4), np.uint64)
    ctr[:, :, 0] = np.arange(L)[:, None]
    ctr[:, :, 1] = np.arange(2)[None, :]
    ctr[:, :, 2] = step
    ctr[:, :, 3] = replica
    w = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)).astype(np.float64)
    u = (w + 0.5) * 2.0 ** -32
    r1 = np.sqrt(-2.0 * np.log(u[..., 0]))
    r2 = np.sqrt(-2.0 * np.log(u[..., 2]))
    z = np.stack([r1 * np.cos(2 * np.pi * u[..., 1]), r1 * np.sin(2 * np.pi * u[..., 1]),
                  r2 * np.cos(2 * np.pi * u[..., 3]), r2 * np.sin(2 * np.pi * u[..., 3])], axis=-1)
    return (np.sqrt(2.0) * z).reshape(V, 4, 8)


def shifts(Ns: int, Nt: int):
    V = Ns ** 3 * Nt
    s = np.arange(V)
    c = np.stack([s % Ns, (s // Ns) % Ns, (s // Ns ** 2) % Ns, s // Ns ** 3], 1)
    L = np.array([Ns, Ns, Ns, Nt])

    def idx(d):
        return ((d[:, 3] * Ns + d[:, 2]) * Ns + d[:, 1]) * Ns + d[:, 0]
    up = np.empty((V, 4), np.int64)
    dn = np.empty((V, 4), np.int64)
    for nu in range(4):
        d = c.copy()
        d[:, nu] = (d[:, nu] + 1) % L[nu]
        up[:, nu] = idx(d)
        d = c.copy()
        d[:, nu] = (d[:, nu] - 1) % L[nu]
        dn[:, nu] = idx(d)
    return up, dn, c


def _traces(M):
    """Tr(lambda_a M) for the eight Gell-Mann matrices: [..., 8]."""
    lam = gell_mann()
    return np.einsum("aij,...ji->...a", lam, M)


def staples(U, Ns, Nt):
    """For every link: S = sum of the six staples A with Tr U_P = Tr(U A), and
    T = sum of their inverses."""
    up, dn, _ = shifts(Ns, Nt)
    Ui = np.linalg.inv(U)
    V = U.shape[0]
    S = np.zeros((V, 4, 3, 3), np.complex128)
    T = np.zeros_like(S)
    for nu in range(4):
        for mu in range(4):
            if mu == nu:
                continue
            xn = up[:, nu]
            # upper: x -> x+nu -> x+nu+mu -> x+mu -> x
            A = U[xn, mu] @ Ui[up[:, mu], nu] @ Ui[:, mu]
            # lower: x -> x+nu -> x+nu-mu -> x-mu -> x
            xm = dn[:, mu]
            B = Ui[dn[xn, mu], mu] @ Ui[xm, nu] @ U[xm, mu]
            S[:, nu] += A + B
            T[:, nu] += np.linalg.inv(A) + np.linalg.inv(B)
    return S, T


def gauge_drift(U, beta, Ns, Nt):
    """K^g[V,4,8] = (i beta/6) sum_A Tr[lambda_a (U A - A^{-1} U^{-1})] (Eq. 5 with S_g)."""
    S, T = staples(U, Ns, Nt)
    M = U @ S - T @ np.linalg.inv(U)
    return 1j * beta / 6.0 * _traces(M)


def plaquette_fields(U, Ns, Nt):
    """dict (mu, nu) -> U_P[V,3,3] for mu < nu."""
    up, _, _ = shifts(Ns, Nt)
    Ui = np.linalg.inv(U)
    out = {}
    for mu in range(4):
        for nu in range(mu + 1, 4):
            out[(mu, nu)] = U[:, mu] @ U[up[:, mu], nu] @ Ui[up[:, nu], mu] @ Ui[:, nu]
    return out


def gauge_action(U, beta, Ns, Nt):
    S = 0.0 + 0.0j
    for P in plaquette_fields(U, Ns, Nt).values():
        S += (1.0 - (np.trace(P, axis1=1, axis2=2) + np.trace(np.linalg.inv(P), axis1=1, axis2=2)) / 6.0).sum()
    return beta * S


def expm_batch(X):
    flat = X.reshape(-1, 3, 3)
    try:
        out = scipy.linalg.expm(flat)
    except (ValueError, TypeError):
        out = np.stack([scipy.linalg.expm(m) for m in flat])
    return out.reshape(X.shape)


def algebra(c):
    """i sum_a c_a lambda_a for coefficient arrays [..., 8] (complex allowed)."""
    return 1j * np.einsum("...a,aij->...ij", c, gell_mann())


def kmax(K):
    return float(np.sqrt((np.abs(K) ** 2).sum(-1)).max())


def step_size(K, eps_max, kappa):
    km = kmax(K)
    if kappa <= 0 or km == 0:
        return eps_max, km
    return min(eps_max, kappa / km), km


def link_update(U, K, eps, eta):
    """Eq. 3-4: U <- exp(i sum_a lambda_a (eps K_a + sqrt(eps) eta_a)) U."""
    R = expm_batch(algebra(eps * K + np.sqrt(eps) * eta))
    return R @ U


def renorm_det(U):
    """Optional determinant renormalisation, off by default as in the paper
    (Sec. 4.2 keeps the links free rather than reunitarising): U <- U /
    det(U)^{1/3} with the principal cube root |d|^{1/3} exp(i arg(d) / 3),
    arg in (-pi, pi]."""
    d = np.linalg.det(U)
    c = np.abs(d) ** (1.0 / 3.0) * np.exp(1j * np.angle(d) / 3.0)
    return U / c[..., None, None]


def reunitarize(U):
    """Optional projection onto SU(3) after an update (Sec. 4.2 names it as the
    remedy of the wrong mu = 0 results; off by default, as in the paper's
    runs): Gram-Schmidt on the first two rows, u = r0/|r0|, v = (r1 - (u^dag
    r1) u) / |...|, and the third row the complex conjugate of the cross
    product u x v (which makes det = 1)."""
    U = np.array(U, dtype=np.complex128)
    r0, r1 = U[..., 0, :], U[..., 1, :]
    u = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    v = r1 - np.sum(u.conj() * r1, axis=-1, keepdims=True) * u
    v = v / np.linalg.norm(v, axis=-1, keepdims=True)
    w = np.conj(np.cross(u, v))
    return np.stack([u, v, w], axis=-2)


def cooling_gradient(U, Ns, Nt):
    _, dn, _ = shifts(Ns, Nt)
    Uh = np.conj(np.swapaxes(U, -1, -2))
    f = np.zeros((U.shape[0], 3, 3), np.complex128)
    for nu in range(4):
        f += U[:, nu] @ Uh[:, nu] - Uh[dn[:, nu], nu] @ U[dn[:, nu], nu]
    f -= np.trace(f, axis1=1, axis2=2)[:, None, None] / 3.0 * np.eye(3)
    return f


def gauge_cool(U, n_cool, alpha0, Ns, Nt):
    up, _, _ = shifts(Ns, Nt)
    for _ in range(n_cool):
        f = cooling_gradient(U, Ns, Nt)
        fmax = np.sqrt((np.abs(f) ** 2).sum((1, 2))).max()
        if fmax == 0:
            break
        alpha = alpha0 / fmax
        Om = expm_batch(-alpha * f)
        Oi = expm_batch(alpha * f)
        U = np.einsum("xij,xnjk,xnkl->xnil", Om, U, Oi[up])
    return U


def unitarity_norm(U):
    Uh = np.conj(np.swapaxes(U, -1, -2))
    return float((np.trace(U @ Uh, axis1=-2, axis2=-1).real - 3.0).sum() / U.shape[0] / 4)


def observables(U, Ns, Nt, Gdiag=None, nf=1.0):
    P = plaquette_fields(U, Ns, Nt)
    ps = np.mean([np.trace(P[(mu, nu)], axis1=1, axis2=2).mean() for (mu, nu) in P if nu < 3]) / 3.0
    pt = np.mean([np.trace(P[(mu, nu)], axis1=1, axis2=2).mean() for (mu, nu) in P if nu == 3]) / 3.0
    V = U.shape[0]
    vs = Ns ** 3
    line = np.broadcast_to(np.eye(3), (vs, 3, 3)).copy()
    for t in range(Nt):
        line = line @ U[t * vs:(t + 1) * vs, 3]
    poly = np.trace(line, axis1=1, axis2=2).mean() / 3.0
    polyi = np.trace(np.linalg.inv(line), axis1=1, axis2=2).mean() / 3.0
    out = dict(plaq_s=complex(ps), plaq_t=complex(pt), poly=complex(poly), poly_inv=complex(polyi),
               unitarity=unitarity_norm(U))
    if Gdiag is not None:
        out["condensate"] = complex(nf * np.trace(Gdiag, axis1=1, axis2=2).sum() / V)
    return out


def observables_full(U, Ns, Nt, blocks, mu, nf=1.0):
    """observables() plus the quark-number density from the selected blocks."""
    from . import number_density
    out = observables(U, Ns, Nt, blocks["Gdiag"], nf)
    out["density"] = number_density(Ns, Nt, U, blocks["Gfwd"], blocks["Gbwd"], mu, nf)
    return out


def langevin_step(U, prm: dict, step: int, Ns: int, Nt: int, replica: int = 0):
    """One stochastic Euler step (Eq. 3-5) in the order of the library's step:
    K = K^g (+ K^f), eps from K_max, observables of the configuration before the
    update, update with noise(seed, step), cooling.  Returns (U', obs, eps)."""
    from . import drift_eval
    V = U.shape[0]
    K = gauge_drift(U, prm["beta"], Ns, Nt)
    Gd = None
    if prm.get("fermions", 1):
        r = drift_eval(Ns, Nt, U, prm["m"], prm["mu"], prm.get("nf", 1.0))
        K = K + r["Kf"]
        Gd = r["Gdiag"]
    eps, km = step_size(K, prm["eps_max"], prm.get("kappa", 0.0))
    obs = observables(U, Ns, Nt, Gd, prm.get("nf", 1.0))
    if Gd is not None:
        from . import number_density
        obs["density"] = number_density(Ns, Nt, U, r["Gfwd"], r["Gbwd"], prm["mu"], prm.get("nf", 1.0))
    obs["kmax"] = km
    obs["eps"] = eps
    eta = noise(prm["seed"], step, V, replica)
    U2 = link_update(U, K, eps, eta)
    if prm.get("renorm_det", 0):
        U2 = renorm_det(U2)
    if prm.get("reunit", 0):
        U2 = reunitarize(U2)
    if prm.get("n_cool", 0) > 0:
        U2 = gauge_cool(U2, prm["n_cool"], prm["alpha_cool"], Ns, Nt)
    return U2, obs, eps
