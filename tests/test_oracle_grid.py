"""Pins for the oracle's time-grid output and its KL accuracy metric (Section 3, Table 1:
KL divergence from exact SSA averaged over time points and species).

Grid: X(t_k) is the right-continuous path's state.  Pinned by exact transient laws at
every grid point (immigration-death Poisson means in SSA mode, the dimerisation master
equation at three times), conservation and monotonicity along the grid, the special cases
t_k = 0 (x0), t_k = T and t_k > T (the final state, with the whole run unchanged when the
only point is T), and the leap error of adaptive mode on pure decay at every point.
KL: zero for equal samples, equal to scipy's entropy of the histogrammed samples, and the
closed form lambda1 log(lambda1/lambda2) + lambda2 - lambda1 for Poisson samples in both
directions."""
import numpy as np
import pytest
from scipy import stats

from paper_1608_07058_gb300 import workloads as W
from tests.test_oracle_laws import _cme_dimerisation

SSA, EXPL, ADAPT = 2, 1, 0


def _chi2_poisson(x, lam):
    """Chi-square of integer sample x against Poisson(lam), consecutive counts merged until
    each group expects at least 5."""
    x = np.asarray(x, np.int64)
    top = int(lam + 8 * np.sqrt(lam) + 10)
    pmf = stats.poisson.pmf(np.arange(top), lam)
    pmf[-1] += stats.poisson.sf(top - 1, lam)
    obs = np.bincount(np.minimum(x, top - 1), minlength=top)
    go, ge, o, e = [], [], 0, 0.0
    for k in range(top):
        o, e = o + obs[k], e + pmf[k] * x.size
        if e >= 5:
            go.append(o); ge.append(e); o, e = 0, 0.0
    go[-1] += o; ge[-1] += e
    return stats.chisquare(go, np.asarray(ge) * sum(go) / sum(ge)).pvalue


def test_grid_ssa_immigration_death_poisson_at_every_point(oracle):
    """0 -> A (10), A -> 0 (0.1), x0 = 0: X(t) ~ Poisson(100 (1 - e^{-0.1 t})).  A grid
    point recorded after the next firing instead of before it shifts the early means."""
    n = 20_000
    t_obs = np.array([0.0, 0.3, 1.0, 5.0, 20.0, 60.0])
    out = oracle.simulate(W.immigration_death(), n, [0], [60.0], params=oracle.Params(mode=SSA),
                          t_obs=t_obs)
    Xo = out["X_obs"][:, :, 0]
    assert (Xo[:, 0] == 0).all()
    for k in range(1, t_obs.size):
        lam = 100 * (1 - np.exp(-0.1 * t_obs[k]))
        x = Xo[:, k].astype(float)
        assert abs(x.mean() - lam) < 4 * np.sqrt(lam / n), (t_obs[k], x.mean(), lam)
        assert _chi2_poisson(x, lam) > 1e-3, t_obs[k]
    assert np.array_equal(Xo[:, -1], out["X"][:, 0])


def test_grid_ssa_dimerisation_master_equation_at_three_times(oracle):
    x0, c, n = (6, 3, 0), (1.0, 10.0, 1000.0, 0.1), 20_000
    t_obs = np.array([0.05, 0.3, 1.2])
    out = oracle.simulate(W.dimerisation(c), n, list(x0), [1.2], params=oracle.Params(mode=SSA),
                          t_obs=t_obs)
    for k, t in enumerate(t_obs):
        states, pT = _cme_dimerisation(x0, c, t)
        idx = {s: i for i, s in enumerate(states)}
        obs = np.bincount([idx[tuple(v)] for v in out["X_obs"][:, k]], minlength=len(states))
        exp = pT * n
        keep = exp > 5
        obs_k = np.concatenate([obs[keep], [obs[~keep].sum()]])
        exp_k = np.concatenate([exp[keep], [exp[~keep].sum()]])
        assert stats.chisquare(obs_k, exp_k).pvalue > 1e-3, t


def test_grid_point_at_horizon_leaves_the_run_unchanged(oracle):
    w = W.config(1, n_traj=200)
    base = oracle.simulate(w.crn, 200, w.x0, w.T, seed=4)
    T = float(w.T[0])
    g = oracle.simulate(w.crn, 200, w.x0, w.T, seed=4, t_obs=[0.0, T, T, 2 * T, 1e9])
    for key in ("X", "r", "G", "status", "counters"):
        assert np.array_equal(g[key], base[key]), key
    Xo = g["X_obs"]
    assert (Xo[:, 0] == np.asarray(w.x0)).all()
    for k in (1, 2, 3, 4):
        assert np.array_equal(Xo[:, k], base["X"])


def test_grid_invariants_along_the_path(oracle):
    """Isomerisation conserves A + B at every grid point; pure decay never increases."""
    t_obs = np.linspace(0.0, 1.0, 11)
    iso = oracle.simulate(W.isomerisation(1.0, 2.0), 500, [300, 100], [1.0], t_obs=t_obs)
    assert (iso["X_obs"].sum(axis=2) == 400).all()
    dec = oracle.simulate(W.pure_decay(1.0), 500, [2000], [1.0], t_obs=t_obs)
    d = dec["X_obs"][:, :, 0]
    assert (np.diff(d, axis=1) <= 0).all() and (d[:, 0] == 2000).all()


def test_grid_adaptive_pure_decay_means(oracle):
    """A -> 0 (k = 1), x0 = 2000: E X(t) = 2000 e^{-t} at every point within the leap
    error O(eps) (eps = 0.03); the leaps end exactly on the grid."""
    n, t_obs = 10_000, np.array([0.1, 0.25, 0.5, 1.0, 2.0])
    out = oracle.simulate(W.pure_decay(1.0), n, [2000], [2.0], t_obs=t_obs,
                          params=oracle.Params(mode=ADAPT))
    for k, t in enumerate(t_obs):
        m = 2000 * np.exp(-t)
        assert abs(out["X_obs"][:, k, 0].mean() - m) < 0.03 * m + 4 * np.sqrt(m / n)
    assert (out["counters"][:, 0] >= t_obs.size).all()


def test_grid_rejects_malformed_times(oracle):
    crn = W.pure_decay(1.0)
    for bad in ([0.5, 0.2], [-0.1], [np.nan], [np.inf]):
        with pytest.raises(ValueError):
            oracle.simulate(crn, 2, [10], [1.0], t_obs=bad)


# ---- KL metric ---------------------------------------------------------------------

def _kl_scipy(a, b, max_bins):
    lo, hi = min(a.min(), b.min()), max(a.max(), b.max())
    w = -(-(hi - lo + 1) // max_bins)
    nb = (hi - lo) // w + 1
    ca = np.bincount((a - lo) // w, minlength=nb) + 0.5
    cb = np.bincount((b - lo) // w, minlength=nb) + 0.5
    return stats.entropy(ca, cb)


def test_kl_identical_samples_is_zero(oracle):
    a = np.random.default_rng(0).poisson(30, 5000)
    assert oracle.kl_sample(a, a) == 0.0
    assert oracle.kl_sample(a, np.random.default_rng(1).permutation(a)) == 0.0


@pytest.mark.parametrize("max_bins", [1024, 37, 5, 1])
def test_kl_equals_scipy_entropy_of_smoothed_histograms(oracle, max_bins):
    rng = np.random.default_rng(max_bins)
    a = rng.poisson(300, 4000)
    b = rng.negative_binomial(30, 30 / 330, 3000)
    assert np.isclose(oracle.kl_sample(a, b, max_bins), _kl_scipy(a, b, max_bins),
                      rtol=1e-12, atol=1e-15)


def test_kl_poisson_closed_form_both_directions(oracle):
    rng = np.random.default_rng(7)
    n = 400_000
    p5, p10 = rng.poisson(5.0, n), rng.poisson(10.0, n)
    exact = lambda l1, l2: l1 * np.log(l1 / l2) + l2 - l1
    assert abs(oracle.kl_sample(p5, p10) - exact(5.0, 10.0)) < 0.01
    # Poisson(10)'s upper tail lands in bins that Poisson(5) leaves empty; the half count
    # there understates log(p/q), so this direction reads about 0.012 low
    assert abs(oracle.kl_sample(p10, p5) - exact(10.0, 5.0)) < 0.02
    assert oracle.kl_sample(p10, p5) - oracle.kl_sample(p5, p10) > 0.3  # not symmetric
    assert abs(oracle.kl_sample(rng.poisson(20.0, n), rng.poisson(22.0, n))
               - exact(20.0, 22.0)) < 0.003


def test_kl_grid_layout_and_mean(oracle):
    rng = np.random.default_rng(3)
    Xa = rng.poisson(20, size=(3000, 4, 3))
    Xb = rng.poisson(21, size=(2000, 4, 3))
    Xb[:, 0, :] = Xa[:2000, 0, :]  # point 0: similar samples
    kl, mean = oracle.kl_grid(Xa, Xb)
    for k in range(4):
        for s in range(3):
            assert kl[k, s] == oracle.kl_sample(Xa[:, k, s], Xb[:, k, s])
    assert np.isclose(mean, kl.mean(), rtol=1e-14)
    assert (kl >= 0).all() and kl[0].max() < kl[1:].min()
