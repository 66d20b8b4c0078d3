"""Pins for the count limits of the oracle: a trajectory whose counts would leave the
range where int64 arithmetic is exact stops with status OVERFLOW (64) instead of wrapping.
The limits: a count or firing total above 2^62 at the start of a step; a Poisson mean, or
an implicit firing count, above 2^48 in a leap (so that x + nu^T K, with at most 128
reactions and |nu| <= 127, stays below 2^63)."""
import numpy as np

from paper_1608_07058_gb300 import workloads as W

ST_OVERFLOW = 64
LIMIT = 2 ** 62


def test_count_above_limit_stops_at_once(oracle):
    crn = W.pure_decay(1e-30)
    out = oracle.simulate(crn, 3, [LIMIT + 1], [1.0])
    assert (out["status"] == ST_OVERFLOW).all()
    assert (out["X"][:, 0] == LIMIT + 1).all() and (out["r"] == 0).all()
    assert (out["G"] == 0).all()
    out = oracle.simulate(crn, 3, [LIMIT], [1.0])     # the limit itself is allowed
    assert (out["status"] == 0).all()


def test_autocatalysis_stops_before_wrapping(oracle):
    """A -> 2A at rate 85 from one molecule grows like e^(85 t): by T = 0.3 about 1e11
    (no limit reached), by T = 0.5 about 3e18, where an int64 sum would soon wrap.  Leaps
    there have tau = eps / 85 and Poisson means 0.03 x, so the leap limit 2^48 stops each
    trajectory once x passes 2^48 / 0.03 = 9.4e15, with X(T) = x0 + nu^T r exact."""
    crn = W._crn("autocatalysis", 1, [({0: 1}, {0: 2}, 85.0)])
    out = oracle.simulate(crn, 200, [1], [0.3], seed=1)
    assert (out["status"] == 0).all()
    out = oracle.simulate(crn, 200, [1], [0.5], seed=1)
    assert (out["status"] == ST_OVERFLOW).all()
    X, r = out["X"][:, 0], out["r"][:, 0]
    assert np.array_equal(X, 1 + r)
    assert (X > 2 ** 48 / 0.03 * 0.9).all() and (X < 2 ** 48 / 0.03 * 1.1).all()


def test_poisson_mean_above_leap_limit_stops(oracle):
    """A <-> B at 2^40 molecules each with rates 1000: the pair is in partial equilibrium,
    the leap runs to T = 1 and each reaction's mean is about 1.1e15 > 2^48."""
    crn = W.isomerisation(1000.0, 1000.0)
    out = oracle.simulate(crn, 3, [2 ** 40, 2 ** 40], [1.0])
    assert (out["status"] == ST_OVERFLOW).all()
    assert (out["X"] == 2 ** 40).all() and (out["r"] == 0).all()
    crn = W.isomerisation(1.0, 1.0)                     # means 2^40: allowed
    out = oracle.simulate(crn, 3, [2 ** 40, 2 ** 40], [1.0])
    assert (out["status"] == 0).all()
    assert np.array_equal(out["X"], 2 ** 40 + out["r"] @ crn.stoich)


def test_implicit_count_saturates(oracle):
    assert oracle.implicit_count(1e300, 1.0, 0.0, 0.0) == LIMIT
    assert oracle.implicit_count(float("nan"), 1.0, 0.0, 0.0) == LIMIT
    assert oracle.implicit_count(2.0 ** 61, 1.0, 0.0, 0.0) == 2 ** 61
