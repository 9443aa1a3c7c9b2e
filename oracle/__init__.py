"""CPU FP64 oracle for the selected-inversion fermion drift (arXiv:1707.08874).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The product library never imports this package.

The heavy dense algebra (Dirac matrix, LU with partial pivoting, column solves,
drift traces) lives in ``cl_oracle.c``; the Langevin pieces are in
``langevin.py`` (plain numpy, per-link loops over 3x3 matrices).

Nothing here shares code with the CUDA library: the oracle builds the dense
matrix D and evaluates the definitions of Sec. 2-3 literally.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``cl_oracle.c`` with gcc (OpenMP) into ``_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "cl_oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                           "-D_DEFAULT_SOURCE", src, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        _lib.or_dirac_dense.argtypes = [I, I, P, D, D, P]
        _lib.or_lu.argtypes = [I, P, P]
        _lib.or_lu.restype = I
        _lib.or_lu_steps.argtypes = [I, P, P, I]
        _lib.or_lu_steps.restype = I
        _lib.or_solve_unit_columns.argtypes = [I, P, P, I, P, P]
        _lib.or_inverse.argtypes = [I, P, P, P]
        _lib.or_logdet.argtypes = [I, P, P, P, P]
        _lib.or_extract_blocks.argtypes = [I, I, P, P, P, P]
        _lib.or_fermion_drift.argtypes = [I, I, P, P, P, D, D, P]
        _lib.or_drift_eval.argtypes = [I, I, P, D, D, D, P, P, P, P, P, P]
        _lib.or_drift_eval.restype = I
        _lib.or_gell_mann.argtypes = [P]
    return _lib


def _c128(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def volume(Ns: int, Nt: int) -> int:
    return Ns * Ns * Ns * Nt


def gell_mann() -> np.ndarray:
    """The oracle's table of the eight Gell-Mann matrices, shape [8,3,3]."""
    out = np.zeros((8, 3, 3), np.complex128)
    _load().or_gell_mann(_ptr(out))
    return out


def dirac_dense(Ns: int, Nt: int, links, m: float, mu: float) -> np.ndarray:
    """Dense staggered D(m;mu) of order 3V (Eq. 1), row-major complex128."""
    U = _c128(links).reshape(-1)
    N = 3 * volume(Ns, Nt)
    D = np.empty((N, N), np.complex128)
    _load().or_dirac_dense(Ns, Nt, _ptr(U), float(m), float(mu), _ptr(D))
    return D


def lu(A: np.ndarray):
    """Textbook LU with partial pivoting; returns (LU, piv, info)."""
    LU = np.array(A, dtype=np.complex128, order="C", copy=True)
    N = LU.shape[0]
    piv = np.empty(N, np.int32)
    info = _load().or_lu(N, _ptr(LU), _ptr(piv))
    return LU, piv, int(info)


def lu_steps(A: np.ndarray, nsteps: int):
    """Only the first ``nsteps`` elimination steps of ``lu`` (timing samples)."""
    LU = np.array(A, dtype=np.complex128, order="C", copy=True)
    N = LU.shape[0]
    piv = np.empty(N, np.int32)
    info = _load().or_lu_steps(N, _ptr(LU), _ptr(piv), int(nsteps))
    return LU, piv, int(info)


def solve_unit_columns(LU, piv, cols) -> np.ndarray:
    """Columns ``cols`` of A^{-1} from the factorisation, shape [N, len(cols)]."""
    N = LU.shape[0]
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    X = np.empty((N, len(cols)), np.complex128)
    _load().or_solve_unit_columns(N, _ptr(LU), _ptr(piv), len(cols), _ptr(cols), _ptr(X))
    return X


def inverse(LU, piv) -> np.ndarray:
    N = LU.shape[0]
    X = np.empty((N, N), np.complex128)
    _load().or_inverse(N, _ptr(LU), _ptr(piv), _ptr(X))
    return X


def logdet(LU, piv) -> complex:
    """log det from the LU factors; imaginary part unwrapped (sum of arguments)."""
    N = LU.shape[0]
    re = ctypes.c_double()
    im = ctypes.c_double()
    _load().or_logdet(N, _ptr(LU), _ptr(piv), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def extract_blocks(Ns: int, Nt: int, Ginv: np.ndarray):
    """Selected 3x3 blocks of a full inverse: Gdiag [V,3,3], Gfwd/Gbwd [V,4,3,3]."""
    V = volume(Ns, Nt)
    Gd = np.empty((V, 3, 3), np.complex128)
    Gf = np.empty((V, 4, 3, 3), np.complex128)
    Gb = np.empty((V, 4, 3, 3), np.complex128)
    G = _c128(Ginv)
    _load().or_extract_blocks(Ns, Nt, _ptr(G), _ptr(Gd), _ptr(Gf), _ptr(Gb))
    return Gd, Gf, Gb


def fermion_drift(Ns: int, Nt: int, links, Gfwd, Gbwd, mu: float, nf: float = 1.0) -> np.ndarray:
    """K^f[V,4,8] from the selected blocks (Eq. 6 via Eq. 8)."""
    V = volume(Ns, Nt)
    U = _c128(links)
    Gf = _c128(Gfwd)
    Gb = _c128(Gbwd)
    K = np.empty((V, 4, 8), np.complex128)
    _load().or_fermion_drift(Ns, Nt, _ptr(U), _ptr(Gf), _ptr(Gb), float(mu), float(nf), _ptr(K))
    return K


def drift_eval(Ns: int, Nt: int, links, m: float, mu: float, nf: float = 1.0):
    """One complete drift evaluation through the dense inverse.

    Returns dict(Gdiag, Gfwd, Gbwd, Kf, logdet).
    """
    V = volume(Ns, Nt)
    U = _c128(links)
    Gd = np.empty((V, 3, 3), np.complex128)
    Gf = np.empty((V, 4, 3, 3), np.complex128)
    Gb = np.empty((V, 4, 3, 3), np.complex128)
    K = np.empty((V, 4, 8), np.complex128)
    re = ctypes.c_double()
    im = ctypes.c_double()
    info = _load().or_drift_eval(Ns, Nt, _ptr(U), float(m), float(mu), float(nf), _ptr(Gd),
                                 _ptr(Gf), _ptr(Gb), _ptr(K), ctypes.byref(re),
                                 ctypes.byref(im))
    if info != 0:
        raise RuntimeError("oracle: singular Dirac matrix (info=%d)" % info)
    return dict(Gdiag=Gd, Gfwd=Gf, Gbwd=Gb, Kf=K, logdet=complex(re.value, im.value))


def condensate(Gdiag, nf: float = 1.0) -> complex:
    """(nf/V) sum_x Tr G_xx."""
    Gd = np.asarray(Gdiag)
    V = Gd.shape[0]
    return complex(nf * np.trace(Gd, axis1=-2, axis2=-1).sum() / V)


def number_density(Ns: int, Nt: int, links, Gfwd, Gbwd, mu: float, nf: float = 1.0) -> complex:
    """n = (nf/V) Tr(G dD/dmu) = (nf/V) d log det D / d mu from the temporal blocks:
    dD_{x,x+t}/dmu = D_{x,x+t}, dD_{x+t,x}/dmu = -D_{x+t,x}  (Sec. 3: the fermionic
    observables need only G where D is non-zero)."""
    U = _c128(links)
    V = volume(Ns, Nt)
    s = np.arange(V)
    x = s % Ns
    y = (s // Ns) % Ns
    z = (s // (Ns * Ns)) % Ns
    t = s // (Ns ** 3)
    eta = (-1.0) ** (x + y + z)
    sg = np.where(t == Nt - 1, -1.0, 1.0)
    ph = 0.5 * eta * sg
    Df = ph[:, None, None] * np.exp(mu) * U[:, 3]
    Db = -ph[:, None, None] * np.exp(-mu) * np.linalg.inv(U[:, 3])
    tr = np.einsum("xij,xji->x", Gbwd[:, 3], Df) - np.einsum("xij,xji->x", Gfwd[:, 3], Db)
    return complex(nf * tr.sum() / V)


def neighbour_table(Ns: int, Nt: int) -> np.ndarray:
    """up[s, nu] = index of s + nu-hat (periodic), plain integer geometry."""
    V = volume(Ns, Nt)
    s = np.arange(V)
    x = s % Ns
    y = (s // Ns) % Ns
    z = (s // (Ns * Ns)) % Ns
    t = s // (Ns * Ns * Ns)
    up = np.empty((V, 4), np.int64)
    up[:, 0] = ((t * Ns + z) * Ns + y) * Ns + (x + 1) % Ns
    up[:, 1] = ((t * Ns + z) * Ns + (y + 1) % Ns) * Ns + x
    up[:, 2] = ((t * Ns + (z + 1) % Ns) * Ns + y) * Ns + x
    up[:, 3] = ((((t + 1) % Nt) * Ns + z) * Ns + y) * Ns + x
    return up


def derivative_blocks(Ns: int, Nt: int, links, mu: float):
    """The two non-zero 3x3 blocks of d_{a x nu} D for every link (the left Lie
    derivative d_a U = i lambda_a U, d_a U^{-1} = -i U^{-1} lambda_a applied to
    Eq. 1 with the readings of the library's header):
        F[x, nu, a] = d_a D_{x, x+nu} = +1/2 eta_nu(x) s_nu(x) e^{+mu d_{nu,t}} i lambda_a U_{x,nu}
        B[x, nu, a] = d_a D_{x+nu, x} = -1/2 eta_nu(x) s_nu(x) e^{-mu d_{nu,t}} (-i U_{x,nu}^{-1} lambda_a)
    Returns F, B of shape [V, 4, 8, 3, 3]."""
    U = _c128(links)
    V = volume(Ns, Nt)
    s = np.arange(V)
    c = np.stack([s % Ns, (s // Ns) % Ns, (s // Ns ** 2) % Ns, s // Ns ** 3], 1)
    lam = gell_mann()
    Ui = np.linalg.inv(U)
    F = np.empty((V, 4, 8, 3, 3), np.complex128)
    Bk = np.empty_like(F)
    for nu in range(4):
        eta = (-1.0) ** c[:, :nu].sum(1)
        sgn = np.where((nu == 3) & (c[:, 3] == Nt - 1), -1.0, 1.0)
        ph = 0.5 * eta * sgn
        ef, eb = (np.exp(mu), np.exp(-mu)) if nu == 3 else (1.0, 1.0)
        F[:, nu] = (ph * ef)[:, None, None, None] * 1j * np.einsum("aij,xjk->xaik", lam, U[:, nu])
        Bk[:, nu] = (-ph * eb)[:, None, None, None] * (-1j) * np.einsum("xij,ajk->xaik", Ui[:, nu], lam)
    return F, Bk


def stochastic_drift(Ns: int, Nt: int, links, m: float, mu: float, eta, nf: float = 1.0,
                     per_vector: bool = False) -> np.ndarray:
    """The stochastic estimator of the fermion drift, Eq. 7, written out:
        K^f_{a x nu} ~ nf (1/n) sum_i eta_i^dag D^{-1} (d_{a x nu} D) eta_i
    for noise vectors eta [n, V, 3] (normalised so that E[eta eta^dag] = 1).
    d_{a x nu} D has two non-zero blocks, so with w_i = eta_i^dag D^{-1} (a row
    vector, from the dense inverse) each term is
        w_i[x] F_a eta_i[x+nu] + w_i[x+nu] B_a eta_i[x].
    Returns K [V, 4, 8] (with per_vector: the n single-vector estimates, [n, V, 4, 8])."""
    V = volume(Ns, Nt)
    eta = _c128(eta).reshape(-1, V, 3)
    D = dirac_dense(Ns, Nt, links, m, mu)
    LU, piv, info = lu(D)
    if info != 0:
        raise RuntimeError("oracle: singular Dirac matrix (info=%d)" % info)
    G = inverse(LU, piv)
    w = (eta.reshape(len(eta), 3 * V).conj() @ G).reshape(len(eta), V, 3)
    F, Bk = derivative_blocks(Ns, Nt, links, mu)
    up = neighbour_table(Ns, Nt)
    K = np.zeros((len(eta), V, 4, 8), np.complex128)
    for nu in range(4):
        y = up[:, nu]
        K[:, :, nu] = (np.einsum("ixj,xajk,ixk->ixa", w, F[:, nu], eta[:, y]) +
                       np.einsum("ixj,xajk,ixk->ixa", w[:, y], Bk[:, nu], eta))
    return nf * K if per_vector else nf * K.mean(0)
