"""The phase / pass split driver (paper_2312_04876_gb300.phases) on CPU with fake runs: shares by
phase and by pass, the median run's choice and the per-arc runtime in the report."""
from __future__ import annotations

import pytest

from paper_2312_04876_gb300 import phases as P


def _pass(c, m, a, o):
    return {"ms_colour": c, "ms_move": m, "ms_aggregate": a, "ms_other": o}


def test_split_by_phase_and_by_pass():
    sp = P.split([_pass(0.0, 6.0, 2.0, 2.0), _pass(0.0, 3.0, 1.0, 1.0), _pass(0.0, 0.5, 0.0, 0.5)])
    assert sp["ms"] == pytest.approx(16.0)
    assert sp["phase_ms"]["ms_move"] == pytest.approx(9.5)
    assert sp["phase_share"]["ms_move"] == pytest.approx(9.5 / 16.0)
    assert sum(sp["phase_share"].values()) == pytest.approx(1.0)
    assert sp["pass_share"] == pytest.approx([10 / 16, 5 / 16, 1 / 16])
    assert P.split([])["ms"] == 0.0


def test_profile_uses_the_median_run_after_a_warm_up():
    seq = iter([(99.0, [_pass(0, 99, 0, 0)]), (12.0, [_pass(0, 12, 0, 0)]), (10.0, [_pass(0, 10, 0, 0)]),
                (11.0, [_pass(1, 9, 1, 0)])])
    r = P.profile(lambda: next(seq), n_arcs=2_000_000, reps=3)
    assert r["ms"] == 11.0 and r["split"]["phase_ms"]["ms_colour"] == 1
    md = P.markdown({"g": r}, "deterministic", "python -m paper_2312_04876_gb300.phases --reps 3")
    assert "| g | 2,000,000 | 11.00 | 5.500 |" in md  # 11 ms / 2M arcs = 5.5 ns per arc
    assert "81.8%" in md  # local moving 9 of 11 ms


def test_report_needs_a_cuda_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is visible")
    with pytest.raises(SystemExit):
        P.main(["--workloads", "sbm10k", "--reps", "1"])
