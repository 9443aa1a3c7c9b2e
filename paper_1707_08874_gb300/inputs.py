"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds only input generation (random numbers and their shaping into
link fields); none of the method's arithmetic.  Stand-in for the paper's own
Langevin ensembles, which are not available: links
U = exp(i sum_a c_a lambda_a) with c_a = N(0, 0.5) + i N(0, 0.1) drawn per link
and per generator (the 8^3x4, mu/T = 1, m = 0.05 set-up of Sec. 4.1).

Layout of a link field: complex128 array [B][V][4][3][3] (or [V][4][3][3]),
site index s = ((t*Ns + z)*Ns + y)*Ns + x, direction 0..3 = x, y, z, t.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

# Generators used only to shape random numbers into group elements.
_GM = np.zeros((8, 3, 3), np.complex128)
_GM[0][0, 1] = _GM[0][1, 0] = 1
_GM[1][0, 1] = -1j
_GM[1][1, 0] = 1j
_GM[2][0, 0] = 1
_GM[2][1, 1] = -1
_GM[3][0, 2] = _GM[3][2, 0] = 1
_GM[4][0, 2] = -1j
_GM[4][2, 0] = 1j
_GM[5][1, 2] = _GM[5][2, 1] = 1
_GM[6][1, 2] = -1j
_GM[6][2, 1] = 1j
_GM[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)

BASE_SEED = 1707


def volume(Ns: int, Nt: int) -> int:
    return Ns * Ns * Ns * Nt


def random_algebra(rng: np.random.Generator, shape, sigma_re: float, sigma_im: float):
    """Coefficients c_a (complex) for a field of traceless generators."""
    c = rng.normal(0.0, sigma_re, size=tuple(shape) + (8,))
    if sigma_im > 0:
        c = c + 1j * rng.normal(0.0, sigma_im, size=tuple(shape) + (8,))
    return c.astype(np.complex128)


def exp_of_algebra(c: np.ndarray) -> np.ndarray:
    """exp(i sum_a c_a lambda_a) for an array of coefficient 8-vectors."""
    H = np.einsum("...a,aij->...ij", c, _GM)
    flat = (1j * H).reshape(-1, 3, 3)
    try:
        out = scipy.linalg.expm(flat)
    except (ValueError, TypeError):  # older scipy: no batched expm
        out = np.stack([scipy.linalg.expm(m) for m in flat])
    return out.reshape(H.shape)


def random_links(Ns: int, Nt: int, seed: int = BASE_SEED, sigma_re: float = 0.5,
                 sigma_im: float = 0.1, batch: int | None = None) -> np.ndarray:
    """SL(3,C) links (SU(3) when sigma_im == 0); shape [V,4,3,3] or [B,V,4,3,3].

    Replica b of a batch uses seed + b.
    """
    V = volume(Ns, Nt)
    if batch is None:
        rng = np.random.default_rng(seed)
        return exp_of_algebra(random_algebra(rng, (V, 4), sigma_re, sigma_im))
    return np.stack([random_links(Ns, Nt, seed + b, sigma_re, sigma_im) for b in range(batch)])


def random_gauge(Ns: int, Nt: int, seed: int, sigma_re: float = 0.4, sigma_im: float = 0.1):
    """Site field Omega_x in SL(3,C), shape [V,3,3]."""
    rng = np.random.default_rng(seed)
    return exp_of_algebra(random_algebra(rng, (volume(Ns, Nt),), sigma_re, sigma_im))


def unit_links(Ns: int, Nt: int) -> np.ndarray:
    V = volume(Ns, Nt)
    U = np.zeros((V, 4, 3, 3), np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def site_coords(Ns: int, Nt: int) -> np.ndarray:
    """[V,4] integer coordinates (x,y,z,t) of every site."""
    s = np.arange(volume(Ns, Nt))
    return np.stack([s % Ns, (s // Ns) % Ns, (s // (Ns * Ns)) % Ns, s // (Ns ** 3)], axis=1)


def shift_table(Ns: int, Nt: int) -> np.ndarray:
    """[V,4] index of the forward neighbour s + nu-hat (periodic)."""
    c = site_coords(Ns, Nt)
    L = np.array([Ns, Ns, Ns, Nt])
    up = np.empty((c.shape[0], 4), np.int64)
    for nu in range(4):
        d = c.copy()
        d[:, nu] = (d[:, nu] + 1) % L[nu]
        up[:, nu] = ((d[:, 3] * Ns + d[:, 2]) * Ns + d[:, 1]) * Ns + d[:, 0]
    return up


def gauge_transform(links: np.ndarray, omega: np.ndarray, Ns: int, Nt: int) -> np.ndarray:
    """U_{x,nu} -> Omega_x U_{x,nu} Omega_{x+nu}^{-1} (input preparation for tests)."""
    up = shift_table(Ns, Nt)
    oinv = np.linalg.inv(omega)
    return np.einsum("xij,xnjk,xnkl->xnil", omega, links, oinv[up])
