"""Pins for the whole oracle method: per-trajectory invariants, closed-form laws of
linear networks, exact chemical-master-equation distributions in SSA mode, Gamma
conjugacy of the (r, G) statistics, and the paper's observation that implicit leaping
underestimates the variance of the fast dimerisation species (Section 3)."""
import numpy as np
import pytest
from scipy import linalg, stats

from paper_1608_07058_gb300 import workloads as W

SSA, EXPL, ADAPT = 2, 1, 0


def _check_invariants(crn, out, x0):
    X, r, G = out["X"], out["r"], out["G"]
    x0 = np.broadcast_to(np.asarray(x0, np.int64), X.shape)
    assert np.array_equal(X, x0 + r @ crn.stoich)      # X(T) = x0 + nu^T r exactly
    assert (r >= 0).all() and (X >= 0).all() and (G >= 0).all()
    assert np.isfinite(G).all()


@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_invariants_configs(oracle, cfg):
    w = W.config(cfg, n_traj=300)
    out = oracle.simulate(w.crn, w.n_traj, w.x0, w.T, w.theta)
    _check_invariants(w.crn, out, w.x0)
    assert (out["status"] == 0).all()


def test_invariants_random_crn_short(oracle):
    w = W.config(3, n_traj=3)
    out = oracle.simulate(w.crn, 3, w.x0, [0.02], None)
    _check_invariants(w.crn, out, w.x0)


@pytest.mark.parametrize("mode", [SSA, EXPL, ADAPT])
def test_invariants_modes_small_counts(oracle, mode):
    # small counts exercise critical reactions and the negativity check
    crn = W.dimerisation()
    out = oracle.simulate(crn, 500, [12, 5, 0], [1.0], params=oracle.Params(mode=mode))
    _check_invariants(crn, out, [12, 5, 0])


def test_immigration_death_closed_form(oracle):
    """0 -> A (10), A -> 0 (0.1), x0 = 0, T = 100: X(T) ~ Poisson(100 (1 - e^-10)),
    r_1 ~ Poisson(1000), G_1 = T, E[G_2] = 100 (100 - 10 (1 - e^-10)), E[r_2] = 0.1 E[G_2]."""
    n = 10_000
    w = W.config(0, n_traj=n)
    out = oracle.simulate(w.crn, n, w.x0, w.T, None)
    X = out["X"][:, 0].astype(float)
    lam = 100 * (1 - np.exp(-10))
    assert abs(X.mean() - lam) < 4 * np.sqrt(lam / n)
    assert abs(X.var() - lam) < 4 * np.sqrt((lam + 2 * lam**2) / n)
    r1 = out["r"][:, 0].astype(float)
    assert abs(r1.mean() - 1000) < 4 * np.sqrt(1000 / n)
    assert np.allclose(out["G"][:, 0], 100.0, rtol=1e-11)
    G2 = out["G"][:, 1]
    EG2 = 100 * (100 - 10 * (1 - np.exp(-10)))
    assert abs(G2.mean() - EG2) < 4 * G2.std() / np.sqrt(n)
    d = out["r"][:, 1] - 0.1 * G2
    assert abs(d.mean()) < 4 * d.std() / np.sqrt(n)
    # whole distribution: chi-square against Poisson(lam)
    edges = np.arange(70, 132, 3)
    obs = np.histogram(X, np.concatenate([[-1], edges, [1e9]]))[0]
    cdf = stats.poisson.cdf(np.concatenate([edges - 1, [1e9]]), lam)
    p = np.diff(np.concatenate([[0.0], cdf]))
    assert stats.chisquare(obs, p * n).pvalue > 1e-3


def _bias(oracle, crn, x0, T, eps, n, mode, exact_mean):
    out = oracle.simulate(crn, n, x0, [T], params=oracle.Params(eps=eps, mode=mode))
    return out["X"][:, 0].mean() - exact_mean, out


def test_pure_decay_binomial_and_leap_consistency(oracle):
    """A -> 0 (k = 1), x0 = 2000, T = 1: X ~ Bin(2000, e^-1).  Explicit leaping has an
    O(eps) weak error: at eps = 0.03 the mean is within eps of the exact one, and the
    error shrinks as eps does."""
    crn, n, x0 = W.pure_decay(1.0), 20_000, 2000
    p = np.exp(-1.0)
    mean = x0 * p
    b03, out = _bias(oracle, crn, [x0], 1.0, 0.03, n, EXPL, mean)
    b005, _ = _bias(oracle, crn, [x0], 1.0, 0.005, n, EXPL, mean)
    assert abs(b03) < 0.03 * mean
    assert abs(b005) < abs(b03) / 2 + 4 * np.sqrt(x0 * p * (1 - p) / n)
    assert (out["counters"][:, 0] > 10).all()          # it really leapt
    var = out["X"][:, 0].var()
    assert abs(var - x0 * p * (1 - p)) < 0.15 * x0 * p * (1 - p)


def test_isomerisation_explicit_binomial(oracle):
    """A <-> B (k1 = 1, k2 = 2), (A, B)(0) = (1000, 0): A(T) ~ Bin(1000, q),
    q = k2/(k1+k2) + k1/(k1+k2) e^{-(k1+k2) T}."""
    k1, k2, T, n0, n = 1.0, 2.0, 0.7, 1000, 20_000
    q = k2 / (k1 + k2) + k1 / (k1 + k2) * np.exp(-(k1 + k2) * T)
    v = n0 * q * (1 - q)
    out = oracle.simulate(W.isomerisation(k1, k2), n, [n0, 0], [T],
                          params=oracle.Params(mode=EXPL))
    A = out["X"][:, 0]
    # explicit leaping near equilibrium inflates the variance by O(eps) (about 13% at
    # eps = 0.03); the error vanishes as eps shrinks
    assert abs(A.mean() - n0 * q) < 0.01 * n0 * q
    assert abs(A.var() - v) < 0.25 * v
    fine = oracle.simulate(W.isomerisation(k1, k2), n, [n0, 0], [T],
                           params=oracle.Params(mode=EXPL, eps=0.01))["X"][:, 0]
    assert abs(fine.mean() - n0 * q) < 4 * np.sqrt(v / n) + 0.002 * n0 * q
    assert abs(fine.var() - v) < 0.06 * v


def test_ssa_isomerisation_exact(oracle):
    k1, k2, T, n0, n = 1.0, 2.0, 0.5, 20, 20_000
    q = k2 / (k1 + k2) + k1 / (k1 + k2) * np.exp(-(k1 + k2) * T)
    out = oracle.simulate(W.isomerisation(k1, k2), n, [n0, 0], [T],
                          params=oracle.Params(mode=SSA))
    obs = np.bincount(out["X"][:, 0], minlength=n0 + 1)
    exp = stats.binom.pmf(np.arange(n0 + 1), n0, q) * n
    keep = exp > 5
    obs_k = np.concatenate([obs[keep], [obs[~keep].sum()]])
    exp_k = np.concatenate([exp[keep], [exp[~keep].sum()]])
    assert stats.chisquare(obs_k, exp_k * obs_k.sum() / exp_k.sum()).pvalue > 1e-3


def _cme_dimerisation(x0, c, T):
    """Exact distribution of the dimerisation network by the master equation on the
    finite set s1 + 2 s2 + 2 s3 <= s1(0) + 2 s2(0) + 2 s3(0)."""
    tot = x0[0] + 2 * x0[1] + 2 * x0[2]
    states = [(a, b, d) for a in range(tot + 1) for b in range(tot // 2 + 1)
              for d in range(tot // 2 + 1) if a + 2 * b + 2 * d <= tot]
    idx = {s: i for i, s in enumerate(states)}
    Q = np.zeros((len(states), len(states)))
    for s, i in idx.items():
        a, b, d = s
        moves = [((a - 1, b, d), c[0] * a), ((a - 2, b + 1, d), c[1] * a * (a - 1) / 2),
                 ((a + 2, b - 1, d), c[2] * b), ((a, b - 1, d + 1), c[3] * b)]
        for t, rate in moves:
            if rate > 0:
                Q[i, idx[t]] += rate
                Q[i, i] -= rate
    p0 = np.zeros(len(states))
    p0[idx[tuple(x0)]] = 1.0
    return states, p0 @ linalg.expm(Q * T)


def test_ssa_dimerisation_matches_master_equation(oracle):
    x0, c, T, n = (6, 3, 0), (1.0, 10.0, 1000.0, 0.1), 0.3, 20_000
    states, pT = _cme_dimerisation(x0, c, T)
    out = oracle.simulate(W.dimerisation(c), n, list(x0), [T], params=oracle.Params(mode=SSA))
    idx = {s: i for i, s in enumerate(states)}
    obs = np.bincount([idx[tuple(v)] for v in out["X"]], minlength=len(states))
    exp = pT * n
    keep = exp > 5
    obs_k = np.concatenate([obs[keep], [obs[~keep].sum()]])
    exp_k = np.concatenate([exp[keep], [exp[~keep].sum()]])
    assert stats.chisquare(obs_k, exp_k).pvalue > 1e-3


def test_ssa_immigration_death_transient_exact(oracle):
    n, T = 20_000, 5.0
    lam = 100 * (1 - np.exp(-0.1 * T))
    out = oracle.simulate(W.immigration_death(), n, [0], [T], params=oracle.Params(mode=SSA))
    X = out["X"][:, 0]
    edges = np.arange(int(lam - 25), int(lam + 25), 3)
    obs = np.histogram(X, np.concatenate([[-1], edges, [1e9]]))[0]
    cdf = stats.poisson.cdf(np.concatenate([edges - 1, [1e9]]), lam)
    assert stats.chisquare(obs, np.diff(np.concatenate([[0.0], cdf])) * n).pvalue > 1e-3


def test_gamma_conjugacy_calibration(oracle):
    """theta_j ~ Gamma(alpha_j, beta_j); the posterior given the exact path statistics is
    Gamma(alpha_j + r_j, beta_j + G_j) (Section 1), so the posterior CDF at the true
    theta_j is Uniform(0, 1) across replicates (simulation-based calibration)."""
    n = 4000
    alpha = np.array([5.0, 5.0])
    beta = np.array([0.5, 50.0])
    rng = np.random.default_rng(9)
    theta = rng.gamma(alpha, 1.0 / beta, size=(n, 2))
    out = oracle.simulate(W.immigration_death(), n, [0], [10.0], theta=theta,
                          params=oracle.Params(mode=SSA))
    for j in range(2):
        u = stats.gamma.cdf(theta[:, j], a=alpha[j] + out["r"][:, j],
                            scale=1.0 / (beta[j] + out["G"][:, j]))
        assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_dimerisation_implicit_underestimates_fast_variance(oracle):
    """Section 3: on the stiff dimerisation model the implicit leap underestimates the
    variance of the two fast species; SSA mode does not."""
    w = W.config(1, n_traj=1)
    ad = oracle.simulate(w.crn, 2000, w.x0, w.T)
    ss = oracle.simulate(w.crn, 60, w.x0, w.T, params=oracle.Params(mode=SSA), traj_id_base=5000)
    assert ad["counters"][:, 1].mean() > 5            # implicit leaps were taken
    v_ad = ad["X"][:, 0].var()
    v_ss = ss["X"][:, 0].var(ddof=1)
    assert v_ad < 0.6 * v_ss
    # the slow species S3 is unaffected: means agree
    assert abs(ad["X"][:, 2].mean() - ss["X"][:, 2].mean()) < 4 * np.sqrt(ss["X"][:, 2].var() / 60 + ad["X"][:, 2].var() / 2000)
