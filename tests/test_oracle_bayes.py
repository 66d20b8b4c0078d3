"""Pins for the oracle's Bayesian step (Section 1: the rate constant's posterior given a
path is Gamma(alpha + r, beta + G)): the Gamma sampler against scipy's Gamma law, the
posterior draws against their Gamma laws, and systematic resampling against its exact
defining properties."""
import numpy as np
import pytest
from scipy import stats


@pytest.mark.parametrize("shape", [0.05, 0.3, 1.0, 2.5, 10.0, 1e3, 1e5])
def test_gamma_sampler_law(oracle, shape):
    rate, n = 2.0, 40_000
    x = np.array([oracle.gamma(shape, rate, seed=3, traj_id=i, stream=5)[0] for i in range(n)])
    mean, var = shape / rate, shape / rate**2
    assert abs(x.mean() - mean) < 5 * np.sqrt(var / n)
    m4 = 3 * shape * (shape + 2) / rate**4  # fourth central moment of Gamma
    assert abs(x.var() - var) < 5 * np.sqrt((m4 - var * var) / n)
    assert stats.kstest(x, stats.gamma(a=shape, scale=1 / rate).cdf).pvalue > 1e-3


def test_gamma_invalid_arguments(oracle):
    assert np.isnan(oracle.gamma(0.0, 1.0)[0]) and np.isnan(oracle.gamma(1.0, -1.0)[0])


def test_posterior_sample_law(oracle):
    # the same (r, G) for every row: each column is a sample of Gamma(alpha + r, beta + G)
    n, M = 20_000, 3
    alpha, beta = np.array([2.0, 0.5, 10.0]), np.array([1.0, 3.0, 0.1])
    r = np.tile([5, 0, 1000], (n, 1))
    G = np.tile([0.5, 7.0, 12.5], (n, 1))
    th, st = oracle.posterior_sample(alpha, beta, r, G, seed=11)
    assert (st == 0).all()
    for j in range(M):
        a, b = alpha[j] + r[0, j], beta[j] + G[0, j]
        assert stats.kstest(th[:, j], stats.gamma(a=a, scale=1 / b).cdf).pvalue > 1e-3
    # per-trajectory hyperparameters are honoured
    th2, _ = oracle.posterior_sample(np.tile(alpha, (n, 1)), beta, r, G, seed=11)
    assert np.array_equal(th, th2)


def test_systematic_resampling_properties(oracle):
    rng = np.random.default_rng(0)
    n = 1000
    logw = rng.normal(0, 2, n)
    logw[::7] = -np.inf                      # some particles with zero weight
    w = np.exp(logw - logw.max())
    wn = w / w.sum()
    anc = oracle.resample_systematic(logw, seed=4)
    assert (np.diff(anc) >= 0).all() and anc.min() >= 0 and anc.max() < n
    counts = np.bincount(anc, minlength=n)
    # systematic resampling: every particle is copied floor or ceil of n w_i times
    assert ((counts >= np.floor(n * wn) - 1e-9) & (counts <= np.ceil(n * wn) + 1e-9)).all()
    assert (counts[::7] == 0).all()
    # equal weights reproduce every particle once
    assert np.array_equal(oracle.resample_systematic(np.zeros(n), seed=9), np.arange(n))
    # unbiased: the mean count over seeds is n w_i
    tot = np.zeros(n)
    for s in range(400):
        tot += np.bincount(oracle.resample_systematic(logw, seed=100 + s), minlength=n)
    assert np.abs(tot / 400 - n * wn).max() < 0.15


def test_systematic_resampling_rejects_degenerate_weights(oracle):
    with pytest.raises(ValueError):
        oracle.resample_systematic(np.full(5, -np.inf))
    # NaN log-weights count as weight zero
    assert list(oracle.resample_systematic(np.array([0.0, np.nan, 0.0]), seed=2)) in ([0, 2, 2], [0, 0, 2])
