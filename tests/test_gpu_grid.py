"""Time-grid output and the KL accuracy metric on the GPU against the CPU oracle, through
the C ABI.

Reference precision: X_obs and every other output bit-identical to the oracle with the
same grid (leaps ending on grid points, SSA firings unmoved, points past the end), in
every mode, both thread drivers, both launch forms and the warp kernel.  Fast precision:
the marginals at every grid point agree statistically (4-SE mean and variance, KS, Holm).
KL: bit-identical to the oracle's binned, half-count-smoothed divergence.  Last, the
paper's accuracy comparison (Section 3, Table 1) in miniature: on the stiff dimerisation
the adaptive method's KL from exact SSA is well above the KL of one SSA sample from
another, and fully explicit leaping is much closer to SSA."""
import numpy as np
import pytest

from paper_1608_07058_gb300 import workloads as W
from tests import stats_util
from tests.test_gpu_parity import assert_bit_parity

pytestmark = pytest.mark.gpu

MAX_STEPS = 200_000


@pytest.fixture(scope="module")
def ml():
    import torch
    from paper_1608_07058_gb300 import build, matleap
    assert torch.cuda.is_available()
    build.build()
    matleap.lib()
    return matleap


def dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype), device="cuda")


def run_gpu_grid(ml, crn, n, x0, T, t_obs, theta=None, seed=0, base=0, **pkw):
    import torch
    pkw.setdefault("max_steps", MAX_STEPS)
    model = ml.model_from_crn(crn)
    out = ml.ml_simulate_grid(model, n, dev(x0, np.int64), dev(np.atleast_1d(T), np.float64),
                              dev(t_obs, np.float64),
                              None if theta is None else dev(theta, np.float64),
                              params=ml.ml_default_params(**pkw), seed=seed, traj_id_base=base)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["status"] = res["status"].astype(np.uint32)
    return res


def run_oracle_grid(oracle, crn, n, x0, T, t_obs, theta=None, seed=0, base=0, **pkw):
    pkw.setdefault("max_steps", MAX_STEPS)
    okw = {k: v for k, v in pkw.items() if k in oracle.Params.__dataclass_fields__}
    return oracle.simulate(crn, n, x0, T, theta, params=oracle.Params(**okw), seed=seed,
                           traj_id_base=base, t_obs=t_obs)


def assert_grid_parity(g, o, label):
    assert_bit_parity(g, o, label)
    bad = np.flatnonzero((g["X_obs"] != o["X_obs"]).any(axis=(1, 2)))
    assert bad.size == 0, f"{label}: X_obs differs on {bad.size} trajectories, first {bad[:5]}"


@pytest.mark.parametrize("cfg,n,grid", [
    (0, 3000, [0.0, 0.5, 3.0, 10.0, 50.0, 100.0, 150.0]),
    (1, 2000, [0.0, 0.01, 0.05, 0.05, 0.1, 0.2, 0.3]),
    (2, 600, [0.0, 5.0, 25.0, 60.0, 120.0, 400.0]),
])
def test_ref_grid_bit_parity_configs(ml, oracle, cfg, n, grid):
    w = W.config(cfg, n_traj=n)
    g = run_gpu_grid(ml, w.crn, n, w.x0, w.T, grid, w.theta, seed=cfg + 3, base=77)
    o = run_oracle_grid(oracle, w.crn, n, w.x0, w.T, grid, w.theta, seed=cfg + 3, base=77)
    assert_grid_parity(g, o, f"config {cfg}")


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_ref_grid_bit_parity_modes_small_counts(ml, oracle, mode):
    """Small counts: critical reactions, rejections and SSA bursts all meet grid points."""
    crn = W.dimerisation()
    grid = np.linspace(0.0, 1.0, 9)
    g = run_gpu_grid(ml, crn, 1500, [12, 5, 0], [1.0], grid, seed=5, mode=mode)
    o = run_oracle_grid(oracle, crn, 1500, [12, 5, 0], [1.0], grid, seed=5, mode=mode)
    assert_grid_parity(g, o, f"mode {mode}")


@pytest.mark.parametrize("shape,form", [(1, 0), (1, 1), (4, 0), (4, 1), (2, 0), (2, 1)])
def test_ref_grid_bit_parity_shapes_and_forms(ml, oracle, shape, form):
    w = W.config(1, n_traj=1200)
    grid = [0.02, 0.07, 0.13, 0.2]
    g = run_gpu_grid(ml, w.crn, 1200, w.x0, w.T, grid, seed=11, shape=shape, form=form)
    o = run_oracle_grid(oracle, w.crn, 1200, w.x0, w.T, grid, seed=11)
    assert_grid_parity(g, o, f"shape {shape} form {form}")


def test_ref_grid_bit_parity_random_crn_warp(ml, oracle):
    w = W.config(3, n_traj=32)
    grid = [0.0, 0.004, 0.011, 0.02]
    g = run_gpu_grid(ml, w.crn, 32, w.x0, [0.02], grid, seed=9)
    o = run_oracle_grid(oracle, w.crn, 32, w.x0, [0.02], grid, seed=9)
    assert_grid_parity(g, o, "random 50 x 100")


def test_ref_grid_per_trajectory_horizons_and_step_limit(ml, oracle):
    """Per-trajectory T below, at and above grid points; a step limit that stops some
    trajectories early (their remaining points get the state at the stop)."""
    rng = np.random.default_rng(4)
    n = 1000
    T = rng.uniform(0.01, 0.3, n)
    grid = [0.0, 0.05, 0.1, 0.2, 0.25]
    crn = W.dimerisation()
    for max_steps in (MAX_STEPS, 12):
        g = run_gpu_grid(ml, crn, n, [400, 798, 0], T, grid, seed=2, max_steps=max_steps)
        o = run_oracle_grid(oracle, crn, n, [400, 798, 0], T, grid, seed=2,
                            max_steps=max_steps)
        assert_grid_parity(g, o, f"max_steps {max_steps}")
    assert (g["status"] & 1).any()


def test_grid_without_points_is_ml_simulate(ml):
    import torch
    w = W.config(1, n_traj=4000)
    model = ml.model_from_crn(w.crn)
    x0, T = dev(w.x0, np.int64), dev(w.T, np.float64)
    a = ml.ml_simulate(model, 4000, x0, T, seed=3)
    b = ml.ml_simulate_grid(model, 4000, x0, T, torch.empty(0, dtype=torch.float64,
                                                            device="cuda"), seed=3)
    torch.cuda.synchronize()
    for k in ("X", "r", "G", "status", "counters"):
        assert torch.equal(a[k], b[k]), k


def test_malformed_grid_is_bad_input(ml):
    w = W.config(0, n_traj=64)
    for grid in ([0.5, 0.2], [-1.0], [np.nan, 1.0], [1.0, np.inf]):
        g = run_gpu_grid(ml, w.crn, 64, w.x0, w.T, grid)
        assert (g["status"] & 16).all()
        assert (g["X_obs"] == 0).all() and (g["X"] == 0).all()


def test_grid_argument_errors(ml):
    import torch
    w = W.config(0, n_traj=8)
    model = ml.model_from_crn(w.crn)
    with pytest.raises(ml.MatleapError):  # host grid
        ml.ml_simulate_grid(model, 8, dev(w.x0, np.int64), dev(w.T, np.float64),
                            torch.tensor([1.0, 2.0], dtype=torch.float64))


def test_fast_grid_statistics(ml, oracle):
    """Fast precision: marginals at every grid point match the oracle's (Holm at 0.01)."""
    w = W.config(1, n_traj=20000)
    grid = [0.01, 0.05, 0.1, 0.2]
    g = run_gpu_grid(ml, w.crn, w.n_traj, w.x0, w.T, grid, seed=21,
                     precision=ml.ML_PREC_FAST_FP32, form=ml.ML_FORM_PERSISTENT)
    o = run_oracle_grid(oracle, w.crn, w.n_traj, w.x0, w.T, grid, seed=21)
    n, K, N = g["X_obs"].shape
    rows = stats_util.compare({"X_obs": g["X_obs"].reshape(n, K * N)},
                              {"X_obs": o["X_obs"].reshape(n, K * N)}, keys=("X_obs",))
    s = stats_util.summary(rows)
    assert s["holm_pass_0.01"], s


# ---- KL metric -----------------------------------------------------------------------

@pytest.mark.parametrize("max_bins", [4096, 1024, 37, 1])
def test_kl_bit_exact_random_samples(ml, oracle, max_bins):
    import torch
    rng = np.random.default_rng(max_bins)
    Xa = rng.poisson(rng.uniform(1, 3000, size=(1, 7, 3)), size=(5000, 7, 3))
    Xb = rng.negative_binomial(20, 0.02, size=(3001, 7, 3))
    Xa[:, 0, 0] = 5          # a constant marginal
    Xb[:, 0, 0] = 5
    Xa[:, 1, 2] = rng.integers(0, 10**9, 5000)  # a wide range
    kl_g, mean_g = ml.ml_kl_divergence(dev(Xa, np.int64), dev(Xb, np.int64), max_bins)
    torch.cuda.synchronize()
    kl_o, mean_o = oracle.kl_grid(Xa, Xb, max_bins)
    assert np.array_equal(kl_g.cpu().numpy(), kl_o)
    assert mean_g.item() == mean_o
    assert kl_o[0, 0] == 0.0


def test_kl_argument_errors(ml):
    import torch
    x = torch.zeros((4, 2, 3), dtype=torch.int64, device="cuda")
    for bins in (0, 4097):
        with pytest.raises(ml.MatleapError):
            ml.ml_kl_divergence(x, x, bins)
    with pytest.raises(ml.MatleapError):
        ml.ml_kl_divergence(x.cpu(), x)


def test_accuracy_table_dimerisation(ml):
    """Section 3, Table 1 in miniature (10^4 trajectories per method, 20 time points, the
    stiff dimerisation): exact SSA against an independent SSA sample gives the estimator's
    floor; the adaptive method, which leaps implicitly over the fast pair and underestimates
    the fast species' variance, sits well above it; fully explicit leaping stays close."""
    import torch
    w = W.config(1, n_traj=10_000)
    grid = np.linspace(0.01, 0.2, 20)
    kw = dict(precision=ml.ML_PREC_FAST_FP32, form=ml.ML_FORM_PERSISTENT)
    ssa = run_gpu_grid(ml, w.crn, w.n_traj, w.x0, w.T, grid, seed=100, mode=2, **kw)
    ssa2 = run_gpu_grid(ml, w.crn, w.n_traj, w.x0, w.T, grid, seed=200, mode=2, **kw)
    ada = run_gpu_grid(ml, w.crn, w.n_traj, w.x0, w.T, grid, seed=300, mode=0, **kw)
    exp = run_gpu_grid(ml, w.crn, w.n_traj, w.x0, w.T, grid, seed=400, mode=1, **kw)
    ref = dev(ssa["X_obs"], np.int64)
    kl = {}
    for name, r in (("ssa", ssa2), ("adaptive", ada), ("explicit", exp)):
        _, m = ml.ml_kl_divergence(ref, dev(r["X_obs"], np.int64))
        torch.cuda.synchronize()
        kl[name] = m.item()
    assert kl["adaptive"] > 3 * kl["ssa"], kl
    assert kl["explicit"] < kl["adaptive"], kl

