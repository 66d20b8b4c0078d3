"""The benchmark's algorithmic work model (operations per event, the numerator of the
`alu` roofline) gives explicit leap 538, implicit leap 1,049.6 (4.3 Newton iterations), SSA firing
126.5 and rejected leap 520 operations for the dimerisation, and on the
single-reaction pure-decay network the counts a hand tally gives: propensity 2 (one
factor, one rate product), SSA firing 2 + 70 (Philox) + 6 (two uniforms) + 15 (log) + 1 +
2 + 2 + 2 + 1 = 101, explicit leap 132, one Newton iteration 19, implicit leap
132 + 4.3 x 19 + 12 = 225.7, rejected leap 132 - 2 - 1 = 129."""
import pytest

import bench
from paper_1608_07058_gb300 import workloads as W


def test_dimerisation_work_model():
    m = bench.work_model(W.dimerisation())
    assert m["explicit_leap"] == 538 and m["ssa_firing"] == pytest.approx(126.5)
    assert m["implicit_leap"] == pytest.approx(1049.6) and m["rejected_leap"] == 520


def test_pure_decay_hand_tally():
    m = bench.work_model(W.pure_decay())
    assert m["ssa_firing"] == pytest.approx(101.0)
    assert m["explicit_leap"] == 132 and m["rejected_leap"] == 129
    assert m["implicit_leap"] == pytest.approx(225.7)


def test_ops_from_counts_is_linear():
    m = bench.work_model(W.dimerisation())
    total = bench.ops_from_counts(m, [1, 2, 3, 4])
    assert total == pytest.approx(538 + 2 * 1049.6 + 3 * 126.5 + 4 * 520)
