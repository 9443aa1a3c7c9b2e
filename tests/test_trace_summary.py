"""Host logic of the timeline summary (paper_1707_08874_gb300.trace) on
synthetic records: spans, per-stream busy time, root-front medians."""
from paper_1707_08874_gb300.trace import summarise


def _rec(name, phase, op, stream, level, t0, t1):
    return dict(name=name, phase=phase, op=op, stream=stream, level=level, t0_us=t0, t1_us=t1)


def test_summary_of_synthetic_timeline():
    tr = [
        _rec("assemble", 0, 0, 0, -1, 0.0, 5.0),
        _rec("panel_inverse", 0, 1, 0, 1, 6.0, 16.0),
        _rec("gemm", 0, 2, 0, 1, 17.0, 20.0),
        _rec("gemm", 0, 3, 1, 1, 20.5, 40.0),
        _rec("panel_inverse", 0, 4, 0, 1, 21.0, 33.0),
        _rec("copy", 0, 5, 1, 1, 40.5, 41.5),
        _rec("gemm", 1, 0, 0, 1, 42.0, 50.0),
        _rec("extract", 1, 1, 0, -1, 50.0, 51.0),
        _rec("drift", -1, -1, 0, -1, 51.0, 52.0),
    ]
    s = summarise(tr)
    assert set(s["levels"]) == {-1, 1}
    lv = s["levels"][1]
    assert lv["span_us"] == 41.5 - 6.0
    assert lv["chain_busy_us"] == 10.0 + 3.0 + 12.0 and lv["chain_launches"] == 3
    assert lv["bulk_busy_us"] == 19.5 + 1.0 and lv["bulk_launches"] == 2
    assert s["root_median_us"]["panel_inverse/stream0"] == dict(launches=2, median=11.0)
    assert s["root_median_us"]["gemm/stream1"]["launches"] == 1
    assert s["selinv_span_us"] == 51.0 - 42.0
    assert s["total_us"] == 52.0


def test_merge_takes_medians():
    from paper_1707_08874_gb300.trace import merge
    sums = [summarise([_rec("panel_inverse", 0, 1, 0, 2, 0.0, x), _rec("gemm", 1, 0, 0, 2, x, x + 1.0)])
            for x in (3.0, 5.0, 4.0)]
    m = merge(sums)
    assert m["reps"] == 3
    assert m["levels"][2]["span_us"] == 4.0 and m["levels"][2]["chain_launches"] == 1
    assert m["root_median_us"]["panel_inverse/stream0"] == dict(launches=1, median=4.0)
    assert m["selinv_span_us"] == 1.0 and m["total_us"] == 5.0
