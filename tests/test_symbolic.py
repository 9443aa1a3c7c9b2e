"""Host-side logic of the library (no GPU): C-ABI exports and the symbolic
analysis (nested dissection, supernodes, boundaries) against a brute-force
symbolic elimination of the lattice graph."""
import ctypes
import re
import os

import numpy as np
import pytest

from paper_1707_08874_gb300 import binding as B
from paper_1707_08874_gb300 import build as libbuild
from paper_1707_08874_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return B.load()


def test_header_symbols_exported(lib):
    hdr = open(os.path.join(ROOT, "include", "clselinv.h")).read()
    names = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(cl_\w+)\s*\(", hdr, re.M))
    assert len(names) >= 10
    handle = ctypes.CDLL(B.lib_path())
    for n in sorted(names):
        assert hasattr(handle, n), n
    assert set(B.EXPORTS) <= names


def test_error_strings(lib):
    assert B.error_string(B.CL_OK) == "success"
    assert "singular" in B.error_string(B.CL_ERR_SINGULAR)


@pytest.mark.parametrize("ns,nt", [(4, 3), (5, 4), (2, 4)])
def test_invalid_shapes_rejected(lib, ns, nt):
    with pytest.raises(B.CLError) as e:
        B.Plan.analyze_symbolic(ns, nt)
    assert e.value.code == B.CL_ERR_INVALID_ARG


def _nodes(plan):
    return [plan.node(i) for i in range(plan.info["n_supernodes"])]


@pytest.mark.parametrize("ns,nt", [(4, 4), (6, 4), (8, 4), (4, 6)])
def test_tree_partitions_sites(lib, ns, nt):
    p = B.Plan.analyze_symbolic(ns, nt)
    nodes = _nodes(p)
    V = ns ** 3 * nt
    allsep = np.concatenate([n["sep"] for n in nodes])
    assert np.array_equal(np.sort(allsep), np.arange(V))
    assert nodes[-1]["parent"] == -1 and len(nodes[-1]["bnd"]) == 0
    for i, n in enumerate(nodes[:-1]):
        par = nodes[n["parent"]]
        assert n["parent"] > i  # postorder
        front = np.concatenate([par["sep"], par["bnd"]])
        pos = {s: q for q, s in enumerate(front)}
        # boundary inside the parent's front, in the parent's front order
        assert all(s in pos for s in n["bnd"])
        assert np.all(np.diff([pos[s] for s in n["bnd"]]) > 0)
        assert par["level"] > n["level"]
    info = p.info
    assert info["max_front"] == max(3 * (len(n["sep"]) + len(n["bnd"])) for n in nodes)
    p.close()


def _brute_force_fill(ns, nt, order):
    """Symbolic elimination of the site graph in `order`: for each eliminated
    site the set of not-yet-eliminated sites it is coupled to (filled graph)."""
    V = ns ** 3 * nt
    up = inputs.shift_table(ns, nt)
    adj = [set() for _ in range(V)]
    for s in range(V):
        for nu in range(4):
            y = int(up[s, nu])
            adj[s].add(y)
            adj[y].add(s)
    done = np.zeros(V, bool)
    later = {}
    for s in order:
        nb = {y for y in adj[s] if not done[y]}
        later[s] = nb
        for a in nb:
            adj[a] |= nb - {a}
        done[s] = True
    return later


@pytest.mark.parametrize("ns,nt", [(4, 4), (6, 4)])
def test_fronts_contain_symbolic_fill(lib, ns, nt):
    """Every fill entry of the elimination in supernode order lies inside the
    front of the supernode that eliminates it, so the multifrontal fronts hold
    the exact sparse LU."""
    p = B.Plan.analyze_symbolic(ns, nt)
    nodes = _nodes(p)
    order = np.concatenate([n["sep"] for n in nodes])
    later = _brute_force_fill(ns, nt, order)
    owner = {}
    for i, n in enumerate(nodes):
        for s in n["sep"]:
            owner[int(s)] = i
    for s, nb in later.items():
        n = nodes[owner[s]]
        front = set(int(v) for v in n["sep"]) | set(int(v) for v in n["bnd"])
        assert nb <= front, (s, nb - front)
    p.close()


def test_flop_counts_scale(lib):
    """Factor + selected-inverse flops grow more slowly than N^3 (Sec. 3)."""
    f = {}
    for ns, nt in [(4, 4), (8, 4), (12, 6)]:
        p = B.Plan.analyze_symbolic(ns, nt)
        f[3 * ns ** 3 * nt] = p.info["factor_flops"] + p.info["selinv_flops"]
        p.close()
    n = sorted(f)
    slope = np.log(f[n[-1]] / f[n[0]]) / np.log(n[-1] / n[0])
    assert 1.5 < slope < 3.0


@pytest.mark.parametrize("panel", [1, 4, 50, -3])
def test_invalid_panel_width_rejected(lib, panel):
    """cl_analyze_ex validates the panel width on the host before any device work."""
    h = ctypes.c_void_p()
    assert lib.cl_analyze_ex(4, 4, 1, B.CL_FP64, panel, ctypes.byref(h)) == B.CL_ERR_INVALID_ARG
