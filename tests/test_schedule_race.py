"""Race check of the two-stream factor schedule (host only, no GPU).

The factorisation's panel chain and bulk updates run on two streams ordered
only by the events the schedule names.  cl_plan_check_schedule replays the
ops with vector clocks and counts unordered conflicting accesses element by
element; every plan shape, precision and panel width must be race-free, and
the same check with the cross-stream waits dropped must find races (so the
check can see them)."""
import pytest

from paper_1707_08874_gb300 import binding as B
from paper_1707_08874_gb300 import build as libbuild


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return B.load()


CASES = [(4, 4, B.CL_FP64, 12), (4, 4, B.CL_FP64, 24), (4, 4, B.CL_FP64, 48),
         (4, 4, B.CL_FP64_EMU, 12), (4, 4, B.CL_FP64_EMU, 24), (4, 4, B.CL_FP64_EMU, 48),
         (4, 4, B.CL_MIXED_FP32, 48), (6, 4, B.CL_FP64, 48), (6, 4, B.CL_FP64_EMU, 24),
         (4, 6, B.CL_FP64_EMU, 24), (4, 8, B.CL_FP64, 24), (6, 6, B.CL_FP64_EMU, 48),
         (4, 4, B.CL_FP64_EMU, 30), (6, 4, B.CL_FP64_EMU, 30), (6, 4, B.CL_FP64, 27), (8, 4, B.CL_FP64_EMU, 30)]


@pytest.mark.parametrize("ns,nt,prec,panel", CASES)
def test_factor_schedule_race_free(ns, nt, prec, panel):
    p = B.Plan.analyze_symbolic(ns, nt, prec, panel)
    conflicts, first = p.check_schedule()
    assert conflicts == 0, first
    p.close()


@pytest.mark.parametrize("ns,nt,prec,panel", [(4, 4, B.CL_FP64, 48), (4, 6, B.CL_FP64_EMU, 24)])
def test_check_finds_races_without_waits(ns, nt, prec, panel):
    p = B.Plan.analyze_symbolic(ns, nt, prec, panel)
    conflicts, first = p.check_schedule(ignore_waits=True)
    assert conflicts > 0 and "unordered" in first
    p.close()


@pytest.mark.parametrize("prec", [B.CL_FP64_EMU, B.CL_MIXED_BF16X3, B.CL_FP64])
def test_ragged_schedule_race_free(prec):
    """The merged schedule of a ragged plan (fronts of three lattice shapes in
    the same launches, trees of different heights) is race-free as well, and
    the check still finds races when its waits are dropped."""
    p = B.Plan.analyze_ragged([(4, 4, 2), (6, 4, 1), (4, 6, 1)], prec, 0, symbolic=True)
    conflicts, first = p.check_schedule()
    assert conflicts == 0, first
    conflicts, first = p.check_schedule(ignore_waits=True)
    assert conflicts > 0
    p.close()


@pytest.mark.parametrize("ns,nt,prec,panel", [(6, 4, B.CL_FP64_EMU, 30), (4, 4, B.CL_FP64, 12),
                                              (8, 4, B.CL_FP64_EMU, 30)])
def test_row_swaps_wait_for_no_bulk_update(ns, nt, prec, panel):
    """The row swap of a step exchanges rows of its panel and of the next one,
    which the previous step updated in its strips on the chain stream: every
    swap runs on that stream with no cross-stream wait, the bulk updates leave
    out the rows of the next two panels, and the schedule stays race-free."""
    p = B.Plan.analyze_symbolic(ns, nt, prec, panel)
    t = p.export_tables()
    ops, gemm = t["factor_ops"], t["gemm"]
    swaps = [op for op in ops if op[0] == 8]
    assert swaps and all(op[5] == 0 and op[6] < 0 for op in swaps)
    b = p.info["panel"]
    bulk = [g for op in ops if op[0] == 4 and op[5] == 1 for g in gemm[op[1]:op[2]]]
    assert bulk
    for g in bulk:
        rm, cm = g[11:15], g[15:19]
        # rows left out: panel p, then panels p+1 and p+2; columns: panels p and p+1
        assert tuple(rm[:3]) == tuple(cm[:3]) and rm[3] - rm[2] <= 2 * b and cm[3] - cm[2] <= b
    assert any(g[14] - g[13] > b for g in bulk)
    conflicts, first = p.check_schedule()
    assert conflicts == 0, first
    p.close()
