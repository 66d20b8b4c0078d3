"""The Bayesian step on the GPU against the CPU oracle, through the C ABI.

Posterior draws theta ~ Gamma(alpha + r, beta + G) (Section 1) and systematic resampling
are FP64 on both sides with the same Philox counters and operation order, so every draw
and every ancestor index must be identical, including NaN results for invalid posterior
parameters and the all -1 answer for degenerate weights.  The last test chains a whole
particle-filter step (simulate, draw from the posterior, weight, resample, simulate
again) and checks each stage bit for bit."""
import numpy as np
import pytest

from paper_1608_07058_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ml():
    import torch
    from paper_1608_07058_gb300 import build, matleap
    assert torch.cuda.is_available()
    build.build()
    matleap.lib()
    return matleap


def dev(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype), device="cuda")


def gpu_posterior(ml, alpha, beta, r, G, seed, base):
    import torch
    th, st = ml.ml_posterior_sample(dev(alpha, np.float64), dev(beta, np.float64),
                                    dev(r, np.int64), dev(G, np.float64), seed=seed,
                                    traj_id_base=base)
    torch.cuda.synchronize()
    return th.cpu().numpy(), st.cpu().numpy().astype(np.uint32)


def oracle_posterior(oracle, alpha, beta, r, G, seed, base):
    return oracle.posterior_sample(alpha, beta, r, G, seed=seed, traj_id_base=base)


def assert_same_draws(g, o):
    assert np.array_equal(g[0], o[0], equal_nan=True), \
        f"{np.count_nonzero(~((g[0] == o[0]) | (np.isnan(g[0]) & np.isnan(o[0]))))} draws differ"
    assert np.array_equal(g[1], o[1])


def test_posterior_shared_prior_bit_exact(ml, oracle):
    rng = np.random.default_rng(1)
    n, M = 6000, 5
    alpha = np.array([0.3, 1.0, 2.5, 40.0, 1e6])
    beta = np.array([0.5, 2.0, 1e-3, 10.0, 3.0])
    r = rng.integers(0, 1000, size=(n, M))
    r[rng.random((n, M)) < 0.2] = 0  # shape alpha_j < 1 for some of the first reaction
    G = rng.exponential(50.0, size=(n, M))
    G[rng.random((n, M)) < 0.1] = 0.0
    assert_same_draws(gpu_posterior(ml, alpha, beta, r, G, 7, 0),
                      oracle_posterior(oracle, alpha, beta, r, G, 7, 0))


def test_posterior_per_trajectory_prior_and_invalid(ml, oracle):
    rng = np.random.default_rng(2)
    n, M = 3000, 3
    alpha = rng.gamma(1.0, 1.0, size=(n, M))
    beta = rng.gamma(1.0, 1.0, size=(n, M))
    r = rng.integers(0, 20, size=(n, M))
    G = rng.uniform(0.0, 5.0, size=(n, M))
    alpha[5, 0], r[5, 0] = 0.0, 0              # shape 0: NaN
    beta[6, 1], G[6, 1] = -2.0, 1.0            # negative rate: NaN
    alpha[7, 2] = np.nan                       # NaN shape: NaN
    alpha[8, 0], r[8, 0] = 1e-3, 0             # tiny shape: boost path
    alpha[9, 1] = 1e12                         # huge shape
    g = gpu_posterior(ml, alpha, beta, r, G, 2**40 + 11, 12345)
    o = oracle_posterior(oracle, alpha, beta, r, G, 2**40 + 11, 12345)
    assert_same_draws(g, o)
    assert np.isnan(g[0][5, 0]) and np.isnan(g[0][6, 1]) and np.isnan(g[0][7, 2])
    assert g[0][8, 0] >= 0.0 and np.isfinite(g[0][9, 1])


def test_posterior_ids_are_independent_of_batching(ml):
    """Trajectory i of a batch with base b draws what trajectory 0 of a batch with base
    b + i draws: the counter carries the trajectory id, not the batch position."""
    rng = np.random.default_rng(3)
    n, M = 257, 4
    alpha, beta = np.full(M, 2.0), np.full(M, 1.0)
    r = rng.integers(0, 50, size=(n, M))
    G = rng.uniform(0.0, 9.0, size=(n, M))
    full = gpu_posterior(ml, alpha, beta, r, G, 5, 1000)[0]
    tail = gpu_posterior(ml, alpha, beta, r[100:], G[100:], 5, 1100)[0]
    assert np.array_equal(full[100:], tail)


def test_posterior_argument_errors(ml):
    import torch
    r = torch.zeros((4, 2), dtype=torch.int64, device="cuda")
    G = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    a = torch.ones(2, dtype=torch.float64, device="cuda")
    with pytest.raises(ml.MatleapError):
        ml.ml_posterior_sample(a, a, r, G, traj_id_base=2**32 - 2)  # ids past 2^32
    with pytest.raises(ml.MatleapError):
        ml.ml_posterior_sample(a.cpu(), a, r, G)                    # host pointer


@pytest.mark.parametrize("n", [1, 7, 1023, 1024, 1025, 5000, 300_001])
def test_resampling_bit_exact(ml, oracle, n):
    import torch
    rng = np.random.default_rng(n)
    logw = rng.normal(0.0, 3.0, size=n)
    if n > 10:
        logw[rng.random(n) < 0.05] = -np.inf
        logw[rng.random(n) < 0.01] = np.nan
        logw[rng.integers(0, n)] = 2.0 + np.nanmax(logw)  # a dominant particle
    for seed, base in ((0, 0), (99, 17)):
        g = ml.ml_resample_systematic(dev(logw, np.float64), seed=seed, id_base=base)
        torch.cuda.synchronize()
        o = oracle.resample_systematic(logw, seed=seed, id_base=base)
        assert np.array_equal(g.cpu().numpy(), o)


def test_resampling_degenerate_weights(ml, oracle):
    import torch
    for logw in (np.full(100, -np.inf), np.full(5, np.nan),
                 np.array([0.0, np.inf, 1.0]), np.array([np.nan, -np.inf])):
        g = ml.ml_resample_systematic(dev(logw, np.float64), seed=1)
        torch.cuda.synchronize()
        assert (g.cpu().numpy() == -1).all()
        with pytest.raises(ValueError):
            oracle.resample_systematic(logw, seed=1)


def test_resampling_workspace_and_size_errors(ml):
    import torch
    n = 5000
    need = ml.ml_resample_workspace_bytes(n)
    assert need >= 8 * n
    logw = torch.zeros(n, dtype=torch.float64, device="cuda")
    small = torch.empty(need - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ml.MatleapError):
        ml.ml_resample_systematic(logw, workspace=small)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    a1 = ml.ml_resample_systematic(logw, seed=3, workspace=ws).clone()
    a2 = ml.ml_resample_systematic(logw, seed=3, workspace=ws)  # workspace reuse
    torch.cuda.synchronize()
    assert torch.equal(a1, a2)
    # equal weights: systematic resampling keeps every particle exactly once
    assert torch.equal(torch.sort(a1).values, torch.arange(n, device="cuda"))


def test_particle_filter_step_chain(ml, oracle):
    """simulate -> posterior draw -> weight -> resample -> simulate with the resampled
    draws, on the gene-expression network with per-trajectory rate constants; every stage
    bit-identical to the oracle."""
    import torch
    n = 2048
    w = W.config(2, n_traj=n)
    T = np.full(n, 20.0)
    model = ml.model_from_crn(w.crn)
    p = ml.ml_default_params(max_steps=200_000)
    out = ml.ml_simulate(model, n, dev(w.x0, np.int64), dev(T, np.float64),
                         dev(w.theta, np.float64), params=p, seed=31)
    alpha = np.full(w.crn.n_reactions, 2.0)
    beta = np.full(w.crn.n_reactions, 2.0) / np.asarray(W.GENE_THETA_TRUE)
    th_g, st_g = ml.ml_posterior_sample(dev(alpha, np.float64), dev(beta, np.float64),
                                        out["r"], out["G"], seed=32)
    torch.cuda.synchronize()
    o = oracle.simulate(w.crn, n, w.x0, T, w.theta, params=oracle.Params(max_steps=200_000),
                        seed=31)
    assert np.array_equal(out["X"].cpu().numpy(), o["X"])
    assert np.array_equal(out["r"].cpu().numpy(), o["r"])
    th_o, st_o = oracle.posterior_sample(alpha, beta, o["r"], out["G"].cpu().numpy(), seed=32)
    assert_same_draws((th_g.cpu().numpy(), st_g.cpu().numpy().astype(np.uint32)), (th_o, st_o))
    # Gaussian observation of the protein count, log-weights from the simulated X(T)
    X = o["X"][:, 2].astype(np.float64)
    logw = -0.5 * ((X - np.median(X)) / (0.3 * np.std(X) + 1.0)) ** 2
    anc_g = ml.ml_resample_systematic(dev(logw, np.float64), seed=33).cpu().numpy()
    anc_o = oracle.resample_systematic(logw, seed=33)
    assert np.array_equal(anc_g, anc_o)
    theta2 = th_o[anc_o]
    out2 = ml.ml_simulate(model, n, dev(w.x0, np.int64), dev(T, np.float64),
                          dev(theta2, np.float64), params=p, seed=34, traj_id_base=n)
    torch.cuda.synchronize()
    o2 = oracle.simulate(w.crn, n, w.x0, T, theta2, params=oracle.Params(max_steps=200_000),
                         seed=34, traj_id_base=n)
    assert np.array_equal(out2["X"].cpu().numpy(), o2["X"])
    assert np.array_equal(out2["r"].cpu().numpy(), o2["r"])
