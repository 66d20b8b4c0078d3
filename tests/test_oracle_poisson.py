"""Pins for the oracle's Poisson sampler (inversion below mean 10, Hoermann's PTRS
from 10 on) against scipy.stats.poisson: chi-square on binned counts, exact mean and
variance within 5 standard errors, across the switch point and large means."""
import numpy as np
import pytest
from scipy import stats

MUS = [1e-3, 0.5, 3.0, 9.99, 10.0, 10.01, 37.0, 1e3, 1e5, 1e7]


def _chi2_pvalue(draws, mu):
    lo, hi = stats.poisson.ppf(1e-4, mu), stats.poisson.ppf(1 - 1e-4, mu)
    edges = np.unique(np.round(np.linspace(lo, hi + 1, 41)))
    obs = np.histogram(draws, bins=np.concatenate([[-np.inf], edges[1:-1], [np.inf]]))[0]
    cdf = stats.poisson.cdf(edges[1:-1] - 1, mu)
    probs = np.diff(np.concatenate([[0.0], cdf, [1.0]]))
    exp = probs * draws.size
    keep = exp > 5
    obs_k, exp_k = obs[keep], exp[keep]
    exp_k = exp_k * obs_k.sum() / exp_k.sum()
    return stats.chisquare(obs_k, exp_k).pvalue if keep.sum() > 1 else 1.0


@pytest.mark.parametrize("mu", MUS)
def test_poisson_distribution(oracle, mu):
    n = 200_000
    d = oracle.poisson_batch(mu, n, seed=42)
    se_mean = np.sqrt(mu / n)
    assert abs(d.mean() - mu) < 5 * se_mean
    se_var = np.sqrt((mu + 3 * mu * mu) / n - mu * mu / n)  # Var of the sample variance
    assert abs(d.var() - mu) < 5 * se_var + 1e-12
    if mu >= 0.5:
        assert _chi2_pvalue(d, mu) > 1e-4


def test_poisson_small_mean_exact_probabilities(oracle):
    # mu = 1e-3: P(0) = e^-mu exactly known; P(k>=2) ~ mu^2/2
    n = 400_000
    d = oracle.poisson_batch(1e-3, n, seed=1)
    p0 = np.exp(-1e-3)
    assert abs((d == 0).mean() - p0) < 5 * np.sqrt(p0 * (1 - p0) / n)


def test_poisson_zero_mean_draws_nothing(oracle):
    assert oracle.poisson(0.0)[0] == 0
    assert oracle.poisson(-1.0)[0] == 0
