"""Host execution of a plan's schedule (no GPU).

The analyser turns the nested dissection into op lists over descriptor tables
(front offsets, masks, transposed operands, look-ahead strips, write-backs,
extend-add and gather maps).  Here those tables, read through
cl_plan_export, are executed in list order in FP64 on the host, each kernel
reduced to its definition (panel inverse = a dense inverse of the block,
GEMM = C <- beta C -/+ A B on the unmasked entries, ...), with the dense D of
the oracle assembled into the fronts.  The extracted blocks must equal the
oracle's blocks of D^{-1} to the FP64 parity bar: this checks the
arithmetic of the schedule itself, independently of the CUDA kernels (the
race check covers the ordering of its two streams).  The factorisation is
also executed in other orders its two streams may run in, which must leave
the same arena bit for bit, while dropping any group of its waits must not.
"""
import numpy as np
import pytest

import oracle
from paper_1707_08874_gb300 import binding as B
from paper_1707_08874_gb300 import build as libbuild
from paper_1707_08874_gb300 import inputs

OP_ZERO, OP_ASSEMBLE, OP_EXTADD, OP_PANEL, OP_GEMM, OP_COPY, OP_GATHER, OP_EXTRACT, OP_SWAP, OP_UNPERM = range(10)
M, MU = 0.05, 0.25


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return B.load()


def _site(x, y, z, t, Ns):
    return ((t * Ns + z) * Ns + y) * Ns + x


def _fwd(s, nu, Ns, Nt):
    x, r = s % Ns, s // Ns
    y, r = r % Ns, r // Ns
    z, t = r % Ns, r // Ns
    c = [x, y, z, t]
    c[nu] = (c[nu] + 1) % (Nt if nu == 3 else Ns)
    return _site(*c, Ns)


def _hit(m, idx):
    return ((idx >= m[0]) & (idx < m[1])) | ((idx >= m[2]) & (idx < m[3]))


def _grid(base, rows, cols, ld, trans=False):
    """element indices of a rows x cols operand: (i, j) at base + i ld + j,
    or at base + j ld + i when stored transposed"""
    i = np.arange(rows, dtype=np.int64)[:, None]
    j = np.arange(cols, dtype=np.int64)[None, :]
    return base + (j * ld + i if trans else i * ld + j)


def _copies(A, descs):
    """(indices, values) of the copy descriptors' unmasked entries."""
    out = []
    for src, dst, lds, ldd, rows, cols, *mk in descs:
        keep = ~_hit(mk[0:4], np.arange(rows))[:, None] & ~_hit(mk[4:8], np.arange(cols))[None, :]
        out.append((_grid(dst, rows, cols, ldd)[keep], A[_grid(src, rows, cols, lds)][keep]))
    return out


def _pivot_rows(T, bp):
    """Local permutation of the nc candidate rows of a panel (rows of T): the
    bp rows that partial pivoting on T (magnitude max(|re|, |im|), ties to the
    lowest row) makes pivots take the panel positions, the chosen rows of the
    panel keeping theirs and the displaced rows taking the places of the
    incoming ones; position i then holds candidate row lperm[i]."""
    T = T.copy()
    nc = T.shape[0]
    live = list(range(nc))
    chosen = []
    for c in range(bp):
        mags = np.maximum(np.abs(T[live, c].real), np.abs(T[live, c].imag))
        j = live[int(np.argmax(mags))]
        chosen.append(j)
        live.remove(j)
        for r in live:
            T[r, c:] -= T[r, c] / T[j, c] * T[j, c:]
    incoming = [j for j in chosen if j >= bp]
    vacated = [i for i in range(bp) if i not in chosen]
    lperm = np.arange(nc)
    for i, j in zip(vacated, incoming):
        lperm[i], lperm[j] = j, i
    return lperm


def legal_order(ops, mode, rng=None, waits=True):
    """An order of a factor op list that the device could run it in: each
    stream's ops in list order, every op after the op it waits for (the
    op lists' waits point backwards, so the walk never gets stuck).  mode:
    0 / 1 runs that stream as far ahead as it can go, "random" switches
    streams after bursts of random length.  waits=False drops the
    cross-stream waits (an order the device must not run)."""
    per = [[i for i in range(len(ops)) if ops[i][5] == s] for s in (0, 1)]
    pos, done, out, cur = [0, 0], set(), [], 0
    while len(out) < len(ops):
        ready = [s for s in (0, 1) if pos[s] < len(per[s]) and
                 (not waits or ops[per[s][pos[s]]][6] < 0 or ops[per[s][pos[s]]][6] in done)]
        assert ready
        if mode == "random":
            if cur not in ready or rng.random() < 0.3:
                cur = ready[int(rng.integers(len(ready)))]
        else:
            cur = mode if mode in ready else ready[0]
        i = per[cur][pos[cur]]
        pos[cur] += 1
        done.add(i)
        out.append(i)
    return out


def execute(t, D, Ns=None, Nt=None, phases=("factor_ops", "selinv_ops"), arena_out=None, perm_out=None,
            factor_order=None):
    """Run the plan's op lists in order on a host arena.  D: the dense Dirac
    matrix of the one lattice of a single-shape plan, or the list of the dense
    matrices of every lattice of a ragged plan (shape order, replicas in
    order).  factor_order: the factorisation's ops in this order of their
    indices instead of list order.  Returns the extracted blocks, one dict
    per lattice for a list."""
    segs = t["segments"]
    Ds = D if isinstance(D, list) else [D]
    assert len(Ds) == int(segs[:, 3].sum())
    meta = t["meta"][0]
    pool, n_arena = int(meta[6]), int(meta[8])
    A = np.full(n_arena, np.nan + 0j)  # the workspace is never read before it is written
    perm = np.zeros(int(meta[10]), dtype=np.int64)  # the permutation workspace (pi per supernode)
    node_k = {}
    for _, _, bp, node, c0, *_ in t["panel"]:
        node_k[node] = max(node_k.get(node, 0), int(c0 + bp))
    off, ld, maps = t["off"], t["ld"], t["maps"]
    lattices = []  # (Ns, Nt, V, arena base, table base) per lattice
    for sNs, sNt, V, count, pbase, rstride, tbase, _ in segs:
        for r in range(count):
            lattices.append((int(sNs), int(sNt), int(V), int(pbase + r * rstride), int(tbase)))
    outs = [dict() for _ in lattices]
    for ph in phases:
        ops = t[ph]
        if ph == "factor_ops" and factor_order is not None:
            assert sorted(factor_order) == list(range(len(ops)))
            ops = ops[factor_order]
        for row in ops:
            kind, d0, d1, blocks = row[:4]
            x0, x1 = row[9], row[10]
            if blocks == 0 and kind != OP_ZERO:
                continue
            writes = []  # (indices, values): every descriptor reads the state before the op
            if kind == OP_ZERO:
                writes.append((np.arange(pool), np.zeros(pool)))
            elif kind == OP_ASSEMBLE:
                for (ns, nt, V, base, tb), Dl in zip(lattices, Ds):
                    for s in range(V):
                        blocks3 = [(s, s, off[tb + s], ld[tb + s])]
                        for nu in range(4):
                            y = _fwd(s, nu, ns, nt)
                            j = tb + V + 4 * s + nu
                            blocks3.append((s, y, off[j], ld[j]))
                            blocks3.append((y, s, off[j + 4 * V], ld[j + 4 * V]))
                        for a, b, o, l in blocks3:
                            writes.append((_grid(base + o, 3, 3, l), Dl[3 * a:3 * a + 3, 3 * b:3 * b + 3]))
            elif kind == OP_EXTADD:
                for parent, nfp, nchild, c0, c1, f0, f1, k0, k1, m0, m1 in t["extadd"][d0:d1]:
                    acc = np.zeros((nfp, nfp), complex)
                    hit = np.zeros((nfp, nfp), bool)
                    I = np.arange(nfp)
                    for child, nfc, kc, mp in ((c0, f0, k0, m0), (c1, f1, k1, m1))[:nchild]:
                        ci = maps[mp + I // 3]
                        ok = ci >= 0
                        pos = kc + 3 * ci + I % 3
                        sel = np.ix_(I[ok], I[ok])
                        acc[sel] += A[child + pos[ok][:, None] * nfc + pos[ok][None, :]]
                        hit[sel] = True
                    idx = _grid(parent, nfp, nfp, nfp)
                    writes.append((idx[hit], A[idx][hit] + acc[hit]))
            elif kind == OP_PANEL:
                for idx, val in _copies(A, t["copy"][x0:x1]):  # launched with the panels, before them
                    A[idx] = val
                for a, l, bp, node, c0, nc, lp, pi, _ in t["panel"][d0:d1]:
                    if c0 == 0:  # a supernode's first panel: its rows in their original order
                        perm[pi:pi + node_k[node]] = np.arange(node_k[node])
                    # pivots among the nc candidate rows; the rows are exchanged on
                    # every column at once (the device swaps the panel's columns in
                    # the panel launch and the others in the swap op after it)
                    first = a - c0  # column 0 of the candidate rows
                    R = A[first + np.arange(nc)[:, None] * l + np.arange(l)[None, :]]
                    lperm = _pivot_rows(R[:, c0:c0 + bp], bp)
                    A[first + np.arange(nc)[:, None] * l + np.arange(l)[None, :]] = R[lperm]
                    perm[pi + c0:pi + c0 + nc] = perm[pi + c0 + lperm]
                    idx = _grid(a, bp, bp, l)
                    writes.append((idx, np.linalg.inv(A[idx])))
            elif kind == OP_SWAP:
                pass  # applied with the panel op above
            elif kind == OP_UNPERM:
                for front, nf, k, p0, npn, _ in t["unperm"][d0:d1]:
                    pi = t["panel"][t["node_panels"][p0]][7]  # the supernode's running permutation
                    F = A[front:front + nf * nf].reshape(nf, nf).copy()
                    G = F.copy()
                    G[:, perm[pi:pi + k]] = F[:, :k]
                    writes.append((np.arange(front, front + nf * nf), G.reshape(-1)))
            elif kind == OP_COPY:
                writes += _copies(A, t["copy"][d0:d1])
            elif kind == OP_GEMM:
                for (a, b, c, lda, ldb, ldc, Mg, Ng, Kg, neg, beta, *mk) in t["gemm"][d0:d1]:
                    rm, cm, tr = mk[0:4], mk[4:8], mk[8]
                    P = A[_grid(a, Mg, Kg, lda, tr & 1)] @ A[_grid(b, Kg, Ng, ldb, tr & 2)]
                    idx = _grid(c, Mg, Ng, ldc, tr & 4)
                    val = (A[idx] if beta else 0) + (-P if neg else P)
                    keep = ~_hit(rm, np.arange(Mg))[:, None] & ~_hit(cm, np.arange(Ng))[None, :]
                    writes.append((idx[keep], val[keep]))
            elif kind == OP_GATHER:
                for child, parent, nfc, kc, nfp, rs, mp in t["gather"][d0:d1]:
                    I = np.arange(3 * rs)
                    pi = 3 * maps[mp + I // 3] + I % 3
                    writes.append((child + (kc + I[:, None]) * nfc + kc + I[None, :],
                                   A[parent + pi[:, None] * nfp + pi[None, :]]))
            elif kind == OP_EXTRACT:
                for (ns, nt, V, base, tb), out in zip(lattices, outs):
                    blk = lambda j: A[_grid(base + off[j], 3, 3, ld[j])]
                    out["Gdiag"] = np.array([blk(tb + s) for s in range(V)])
                    out["Gfwd"] = np.array([[blk(tb + V + 4 * s + nu) for nu in range(4)] for s in range(V)])
                    out["Gbwd"] = np.array([[blk(tb + 5 * V + 4 * s + nu) for nu in range(4)] for s in range(V)])
            for idx, val in writes:
                A[idx] = val
    if arena_out is not None:
        arena_out.append(A)
    if perm_out is not None:
        perm_out.append(perm)
    return outs if isinstance(D, list) else outs[0]


def left_solve(t, A, eta, perm):
    """The row-vector solves w = eta^dag D^{-1} of cl_left_solve executed from
    the exported front-vector tables on a factorised host arena A (forward
    over the levels, then backward), for a plan with one replica per shape
    segment row; eta [n, sites, 3]."""
    vn, vs, maps = t["vnodes"], t["vsites"], t["maps"]
    n, sites = eta.shape[0], eta.shape[1]
    ne = int((vn[:, 1] + vn[:, 3]).max())
    R = np.zeros((n, ne), complex)
    W = np.zeros((n, ne), complex)
    w = np.zeros_like(eta)
    levels = sorted(set(vn[:, 6]))
    front = lambda x: A[x[0]:x[0] + x[3] * x[3]].reshape(x[3], x[3])
    for h in levels:  # forward
        for x in vn[vn[:, 6] == h]:
            fr, vec, pvec, nf, k, r, lv, nch, cv0, cv1, ck0, ck1, em0, em1, gm, s0, p0, npn = x
            v = np.zeros((n, nf), complex)
            e = np.arange(k)
            v[:, :k] = eta[:, vs[s0 + e // 3], e % 3].conj()
            for cv, ck, em in ((cv0, ck0, em0), (cv1, ck1, em1))[:nch]:
                E = np.arange(nf)
                m = maps[em + E // 3]
                ok = m >= 0
                v[:, ok] += R[:, cv + ck + 3 * m[ok] + E[ok] % 3]
            F = front(x)
            v[:, k:] -= v[:, :k] @ F[:k, k:]
            R[:, vec:vec + nf] = v
    for h in levels[::-1]:  # backward
        for x in vn[vn[:, 6] == h]:
            fr, vec, pvec, nf, k, r, lv, nch, cv0, cv1, ck0, ck1, em0, em1, gm, s0, p0, npn = x
            pi = t["panel"][t["node_panels"][p0]][7] if npn else 0
            F = front(x)
            S = np.arange(r)
            wS = W[:, pvec + 3 * maps[gm + S // 3] + S % 3] if r else np.zeros((n, 0), complex)
            wJ = R[:, vec:vec + k] @ F[:k, :k] + wS @ F[k:, :k]
            # the factors are those of the row-permuted supernode: entry i of wJ
            # belongs to the supernode's unknown pi[i]
            e = perm[pi:pi + k] if k else np.zeros(0, dtype=np.int64)
            W[:, vec + e] = wJ
            W[:, vec + k:vec + nf] = wS
            w[:, vs[s0 + e // 3], e % 3] = wJ
    return w


def _blockwise(a, b):
    da = np.sqrt((np.abs(a - b) ** 2).sum((-1, -2)))
    nb = np.sqrt((np.abs(b) ** 2).sum((-1, -2)))
    return da.max() / nb.max()


_REF = {}


def _reference(Ns, Nt):
    if (Ns, Nt) not in _REF:
        U = inputs.random_links(Ns, Nt, seed=1707)
        D = oracle.dirac_dense(Ns, Nt, U, M, MU)
        sv = np.linalg.svd(D, compute_uv=False)
        _REF[(Ns, Nt)] = (D, oracle.drift_eval(Ns, Nt, U, M, MU), max(1e-10, 1e-13 * sv[0] / sv[-1]))
    return _REF[(Ns, Nt)]


@pytest.mark.parametrize("ns,nt,prec,panel", [
    (4, 4, B.CL_FP64, 48), (4, 4, B.CL_FP64_EMU, 30), (4, 4, B.CL_MIXED_FP32, 30), (4, 4, B.CL_FP64_EMU, 12),
    (4, 4, B.CL_FP64_EMU, 24), (4, 4, B.CL_FP64_EMU, 27), (4, 4, B.CL_FP64, 3), (4, 6, B.CL_FP64_EMU, 30),
    (6, 4, B.CL_FP64_EMU, 30), (6, 4, B.CL_FP64, 48)])
def test_schedule_reproduces_dense_inverse(ns, nt, prec, panel):
    D, ref, tol = _reference(ns, nt)
    tables = B.Plan.analyze_symbolic(ns, nt, prec, panel).export_tables()
    assert int(tables["meta"][0][5]) == panel
    if prec == B.CL_FP64_EMU:  # the panel products with few rows are issued transposed
        assert (tables["gemm"][:, 19] == 7).any()
    got = execute(tables, D, ns, nt)
    for key in ("Gdiag", "Gfwd", "Gbwd"):
        err = _blockwise(got[key], ref[key])
        assert err < tol, (key, err, tol)


def test_schedule_executor_sees_a_broken_table():
    """The check has teeth: one dropped bulk update (a GEMM descriptor of the
    factorisation turned into a no-op) must spoil the result."""
    D, ref, tol = _reference(4, 4)
    tables = B.Plan.analyze_symbolic(4, 4, B.CL_FP64_EMU, 30).export_tables()
    bulk = [i for i, row in enumerate(tables["gemm"]) if row[10] == 1 and row[6] > 64 and row[7] > 64]
    assert bulk
    tables["gemm"][bulk[0], 8] = 0  # K = 0: the product adds nothing
    got = execute(tables, D, 4, 4)
    assert _blockwise(got["Gfwd"], ref["Gfwd"]) > 1e3 * tol


@pytest.mark.parametrize("ns,nt,prec,panel", [(4, 4, B.CL_FP64_EMU, 12), (4, 4, B.CL_FP64, 24),
                                              (4, 6, B.CL_FP64_EMU, 30)])
def test_schedule_same_in_every_legal_order(ns, nt, prec, panel):
    """The factorisation's two streams may interleave in any way that keeps
    each stream's order and the cross-stream waits.  Executed in such orders
    (each stream as far ahead as it can go, and random bursts), the schedule
    leaves the same arena, bit for bit, as in list order: a check of the
    race check by execution.  The same walk with the waits dropped changes
    the result."""
    D, _, _ = _reference(ns, nt)
    t = B.Plan.analyze_symbolic(ns, nt, prec, panel).export_tables()
    ops = t["factor_ops"]
    assert (ops[:, 5] == 1).any() and (ops[:, 6] >= 0).any()

    def run(order):
        arena = []
        got = execute(t, D, ns, nt, arena_out=arena, factor_order=order)
        return arena[0], got

    A0, g0 = run(None)
    rng = np.random.default_rng(1707)
    orders = [legal_order(ops, m, rng) for m in (0, 1, "random", "random")]
    assert len({tuple(o) for o in orders}) == len(orders)
    for order in orders:
        A, g = run(order)
        assert np.array_equal(A, A0, equal_nan=True)
        for key in g0:
            assert np.array_equal(g[key], g0[key]), key
    with np.errstate(invalid="ignore", divide="ignore"):  # reads of unwritten (NaN) entries
        A, _ = run(legal_order(ops, 1, waits=False))
    assert not np.array_equal(A, A0, equal_nan=True)


def test_ragged_schedule_same_in_every_legal_order():
    """The merged schedule of a ragged plan (two 4^4 lattices and one 4^3 x 6
    lattice, fronts of different pivot counts in every launch) leaves the same
    arena in the extreme and random interleavings of its two streams."""
    shapes = [(4, 4, 2), (4, 6, 1)]
    t = B.Plan.analyze_ragged(shapes, B.CL_FP64_EMU, 0, symbolic=True).export_tables()
    Us = [inputs.random_links(4, 4, seed=1707 + r) for r in range(2)] + [inputs.random_links(4, 6, seed=3)]
    Ds = [oracle.dirac_dense(4, 4, Us[0], M, MU), oracle.dirac_dense(4, 4, Us[1], M, MU),
          oracle.dirac_dense(4, 6, Us[2], M, MU)]
    ops = t["factor_ops"]
    arena = []
    execute(t, Ds, phases=("factor_ops",), arena_out=arena)
    A0 = arena[0]
    rng = np.random.default_rng(11)
    for mode in (0, 1, "random"):
        arena = []
        execute(t, Ds, phases=("factor_ops",), arena_out=arena, factor_order=legal_order(ops, mode, rng))
        assert np.array_equal(arena[0], A0, equal_nan=True), mode


def test_each_dropped_wait_changes_some_order():
    """Every group of cross-stream waits is needed: with the waits of one
    (op kind, stream) group dropped, one of the two extreme interleavings
    (either stream as far ahead as it can go) leaves another arena than
    list order."""
    D, _, _ = _reference(4, 4)
    t = B.Plan.analyze_symbolic(4, 4, B.CL_FP64_EMU, 12).export_tables()
    ops = t["factor_ops"]
    arena = []
    execute(t, D, 4, 4, arena_out=arena)
    A0 = arena[0]
    groups = sorted({(int(o[0]), int(o[5])) for o in ops if o[6] >= 0})
    assert len(groups) >= 3
    for kind, stream in groups:
        o2 = ops.copy()
        o2[(o2[:, 0] == kind) & (o2[:, 5] == stream), 6] = -1
        t2 = dict(t, factor_ops=o2)
        changed = []
        for mode in (0, 1):
            arena = []
            with np.errstate(invalid="ignore", divide="ignore"):  # reads of unwritten (NaN) entries
                execute(t2, D, 4, 4, arena_out=arena, factor_order=legal_order(o2, mode))
            changed.append(not np.array_equal(arena[0], A0, equal_nan=True))
        assert any(changed), (kind, stream)


def test_ragged_schedule_reproduces_dense_inverses():
    """A ragged plan (two 4^4 lattices and one 4^3 x 6 lattice in one merged
    schedule: each level's panels, products, copies, extend-adds and gathers
    over the fronts of all three lattices at once) reproduces every lattice's
    blocks of D^{-1}."""
    shapes = [(4, 4, 2), (4, 6, 1)]
    plan = B.Plan.analyze_ragged(shapes, B.CL_FP64_EMU, 0, symbolic=True)
    tables = plan.export_tables()
    segs = tables["segments"]
    assert segs.shape == (2, 8) and list(segs[:, 3]) == [2, 1]
    assert plan.info["batch"] == 3 and plan.info["V"] == 2 * 256 + 384 and plan.info["n_shapes"] == 2
    Us = [inputs.random_links(4, 4, seed=1707 + r) for r in range(2)] + [inputs.random_links(4, 6, seed=3)]
    Ds = [oracle.dirac_dense(4, 4, Us[0], M, MU), oracle.dirac_dense(4, 4, Us[1], M, MU),
          oracle.dirac_dense(4, 6, Us[2], M, MU)]
    got = execute(tables, Ds)
    for (ns, nt), U, g in zip([(4, 4), (4, 4), (4, 6)], Us, got):
        ref = oracle.drift_eval(ns, nt, U, M, MU)
        for key in ("Gdiag", "Gfwd", "Gbwd"):
            assert _blockwise(g[key], ref[key]) < 1e-10, key
    # one launch per step across all lattices: the level-0 panel inverses of
    # the three lattices share launches, and the GEMM problems of a launch
    # span the lattices' fronts
    ops = tables["factor_ops"]
    panel_ops = ops[ops[:, 0] == OP_PANEL]
    assert panel_ops[:, 3].max() >= 3 * 4  # >= 4 leaves per 4^4 lattice, three lattices


@pytest.mark.parametrize("shapes", [[(4, 4, 1)], [(4, 4, 2), (4, 6, 1)]])
def test_left_solve_tables(shapes):
    """The front-vector tables of the row-vector solves (cl_left_solve), run on
    the host on the factorised fronts, give w = eta^dag D^{-1} for every
    lattice of a single-shape and of a ragged plan."""
    if len(shapes) == 1:
        ns, nt, _ = shapes[0]
        tables = B.Plan.analyze_symbolic(ns, nt, B.CL_FP64_EMU, 30).export_tables()
    else:
        tables = B.Plan.analyze_ragged(shapes, B.CL_FP64_EMU, 0, symbolic=True).export_tables()
    lat = [(ns, nt) for ns, nt, c in shapes for _ in range(c)]
    Us = [inputs.random_links(ns, nt, seed=70 + i) for i, (ns, nt) in enumerate(lat)]
    Ds = [oracle.dirac_dense(ns, nt, U, M, MU) for (ns, nt), U in zip(lat, Us)]
    arena, perm = [], []
    execute(tables, Ds if len(Ds) > 1 else Ds[0], phases=("factor_ops",), arena_out=arena, perm_out=perm)
    sites = sum(ns ** 3 * nt for ns, nt in lat)
    rng = np.random.default_rng(5)
    eta = rng.normal(size=(3, sites, 3)) + 1j * rng.normal(size=(3, sites, 3))
    w = left_solve(tables, arena[0], eta, perm[0])
    s0 = 0
    for (ns, nt), D in zip(lat, Ds):
        V = ns ** 3 * nt
        e = eta[:, s0:s0 + V].reshape(3, 3 * V)
        want = (e.conj() @ np.linalg.inv(D)).reshape(3, V, 3)
        got = w[:, s0:s0 + V]
        assert np.abs(got - want).max() < 1e-10 * np.abs(want).max()
        s0 += V
