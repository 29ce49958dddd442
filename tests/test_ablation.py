"""The parameter-study driver (paper_2312_04876_gb300.ablation) on CPU: its grid of settings, the
measurement protocol and the relative runtime / modularity it reports, with a fake runner in place
of the CUDA path (which the study itself requires)."""
from __future__ import annotations

import math
from types import SimpleNamespace

import pytest

from paper_2312_04876_gb300 import ablation as A


def test_each_setting_changes_one_control_from_its_default():
    import paper_2312_04876_gb300 as lv
    d = lv.default_params()
    s = A.settings()
    assert s[0] == ("defaults", {})
    labels = [lab for lab, _ in s]
    assert len(set(labels)) == len(labels)
    for lab, ov in s[1:]:
        (name, value), = ov.items()
        assert getattr(d, name) != value, lab
    # the paper's comparisons are all present
    for name, value in (("max_iterations", 100), ("tolerance_drop", 1.0), ("tolerance", 1e-6),
                        ("aggregation_tolerance", 1.0), ("pruning", 0)):
        assert {name: value} in [ov for _, ov in s]


def test_measure_discards_the_first_run_and_takes_median_time_and_mean_q():
    calls = []
    seq = iter([(100.0, 0.0), (5.0, 0.30), (7.0, 0.32), (6.0, 0.34)])

    def timed_run():
        ms, q = next(seq)
        calls.append(ms)
        return ms, SimpleNamespace(modularity=q, passes=2, total_iterations=5)

    m = A.measure(timed_run, 3)
    assert calls == [100.0, 5.0, 7.0, 6.0]
    assert m["ms"] == 6.0 and m["reps"] == 3
    assert m["q"] == pytest.approx(0.32) and m["passes"] == 2 and m["iterations"] == 5


def test_summary_is_geometric_in_time_and_arithmetic_in_q():
    res = {"a": {"defaults": {"ms": 10.0, "q": 0.5}, "pruning=0": {"ms": 20.0, "q": 0.5}},
           "b": {"defaults": {"ms": 10.0, "q": 0.4}, "pruning=0": {"ms": 5.0, "q": 0.2}}}
    rows = dict((lab, (rt, rq)) for lab, rt, rq in A.summarise(res))
    assert rows["defaults"] == (1.0, 1.0)
    rt, rq = rows["pruning=0"]
    assert rt == pytest.approx(math.sqrt(2.0 * 0.5)) and rq == pytest.approx((1.0 + 0.5) / 2)


def test_study_runs_every_setting_on_every_workload_and_reports_them():
    seen = []

    def make(graph, ov):
        seen.append((graph, tuple(ov.items())))
        t = 10.0 * (2.0 if ov.get("pruning") == 0 else 1.0)
        return lambda: (t, SimpleNamespace(modularity=0.4, passes=1, total_iterations=3))

    res = A.study({"g1": "G1", "g2": "G2"}, make, reps=2)
    # every setting once per workload, and the defaults a second time at the end
    assert len(seen) == 2 * (len(A.settings()) + 1)
    assert seen[len(A.settings())] == ("G1", ())
    assert set(res) == {"g1", "g2"} and all(len(v) == len(A.settings()) for v in res.values())
    md = A.markdown(res, "fast", "python -m paper_2312_04876_gb300.ablation --reps 2")
    for lab, _ in A.settings():
        assert f"| {lab} |" in md
    assert "| pruning=0 | 2.000 | 1.0000 |" in md


def test_study_needs_a_cuda_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is visible")
    with pytest.raises(SystemExit):
        A.main(["--workloads", "sbm10k", "--reps", "1"])


def test_study_keeps_the_faster_of_the_two_default_measurements():
    calls = {"n": 0}

    def make(graph, ov):
        def run():
            calls["n"] += 1
            slow = not ov and calls["n"] <= 4  # the defaults' first measure(): a stalled start
            return (70.0 if slow else 10.0), SimpleNamespace(modularity=0.4, passes=1, total_iterations=3)
        return run

    res = A.study({"g": "G"}, make, reps=3)
    assert res["g"]["defaults"]["ms"] == 10.0
    md = A.markdown(res, "fast", "cmd")
    assert "| max_iterations=100 | 1.000 |" in md


def test_a_failing_setting_is_recorded_not_fatal():
    def make(graph, ov):
        def run():
            if ov.get("table_factor") == 1:
                raise RuntimeError("hash table overflow")
            return 10.0, SimpleNamespace(modularity=0.4, passes=1, total_iterations=3)
        return run

    res = A.study({"g": "G"}, make, reps=1)
    assert "error" in res["g"]["table_factor=1"] and "overflow" in res["g"]["table_factor=1"]["error"]
    md = A.markdown(res, "fast", "cmd")
    assert "| table_factor=1 | nan | nan | failed |" in md
    assert "| max_iterations=100 | 1.000 |" in md
