"""Property tests of two oracle functions on random inputs.

Systematic resampling: with the oracle's quantized weights q_i = floor(exp(logw_i - max)
2^40) (NaN as 0) and Q = sum q_i, ancestors are sorted and in range, particle i is kept
floor(n q_i / Q) or ceil(n q_i / Q) times, and a zero weight is never kept.
KL of two integer samples: equal to scipy's entropy of the half-count-smoothed histograms
on the pooled range with bin width ceil(range / max_bins)."""
import math

import numpy as np
import pytest
from scipy import stats

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")

logw_values = st.one_of(st.floats(-60.0, 30.0), st.just(-math.inf), st.just(math.nan))


@hyp.settings(max_examples=150, deadline=None)
@hyp.given(st.lists(logw_values, min_size=1, max_size=300), st.integers(0, 2**64 - 1),
           st.integers(0, 2**32 - 1))
def test_resampling_guarantees(oracle, logw, seed, base):
    logw = np.array(logw, np.float64)
    finite = logw[np.isfinite(logw)]
    hyp.assume(finite.size > 0)
    mx = finite.max()
    w = np.where(np.isnan(logw), 0.0, np.exp(np.where(np.isnan(logw), -np.inf, logw) - mx))
    q = np.floor(w * 2.0 ** 40).astype(object)
    Q = sum(q)
    hyp.assume(Q > 0)
    n = logw.size
    anc = oracle.resample_systematic(logw, seed=seed, id_base=base)
    assert (np.diff(anc) >= 0).all() and anc.min() >= 0 and anc.max() < n
    counts = np.bincount(anc, minlength=n)
    for i in range(n):
        lo, hi = (n * q[i]) // Q, -((-n * q[i]) // Q)
        assert lo <= counts[i] <= hi, (i, counts[i], lo, hi)
        if q[i] == 0:
            assert counts[i] == 0


@hyp.settings(max_examples=150, deadline=None)
@hyp.given(st.lists(st.integers(-10**6, 10**6), min_size=1, max_size=200),
           st.lists(st.integers(-10**6, 10**6), min_size=1, max_size=200),
           st.integers(1, 4096))
def test_kl_matches_scipy(oracle, a, b, max_bins):
    a, b = np.array(a, np.int64), np.array(b, np.int64)
    lo, hi = min(a.min(), b.min()), max(a.max(), b.max())
    w = -(-(hi - lo + 1) // max_bins)
    nb = (hi - lo) // w + 1
    ca = np.bincount((a - lo) // w, minlength=nb) + 0.5
    cb = np.bincount((b - lo) // w, minlength=nb) + 0.5
    ref = stats.entropy(ca, cb)
    assert oracle.kl_sample(a, b, max_bins) == pytest.approx(ref, rel=1e-11, abs=1e-13)
