"""Checkpoint / resume of complex-Langevin runs.

A checkpoint holds the links, the Langevin state (time, step count, last
step size) and the run parameters.  The noise of step n is a pure function of
(seed, n, link, replica) (counter-based Philox), so a run resumed from a
checkpoint continues bitwise identically to an uninterrupted one.
"""
from __future__ import annotations

import json

import numpy as np


def save(path: str, links, state, params: dict) -> None:
    """links: complex128 tensor/array [B][V][4][3][3]; state: float64 [B][4]."""
    U = links.cpu().numpy() if hasattr(links, "cpu") else np.asarray(links)
    S = state.cpu().numpy() if hasattr(state, "cpu") else np.asarray(state)
    with open(path, "wb") as f:
        np.savez(f, links=U, state=S, params=json.dumps(params))


def load(path: str):
    """Returns (links ndarray, state ndarray, params dict)."""
    with np.load(path, allow_pickle=False) as z:
        return z["links"], z["state"], json.loads(str(z["params"]))
