"""GPU path against the CPU oracle, through the C ABI.

Reference precision: every trajectory bit-identical in X(T), r and status and G within
1e-12 relative (here equal), with the same RNG keys, across the paper's workload shapes,
small counts (critical reactions, rejections), every mode, the padded generic variant,
and a full-size launch sampled by trajectory id.  Fast precision: ensemble statistics
within 4 standard errors and KS p > 0.01 (Holm-corrected) against the oracle."""
import numpy as np
import pytest

from paper_1608_07058_gb300 import workloads as W
from tests import stats_util

pytestmark = pytest.mark.gpu

MAX_STEPS = 200_000
G_RTOL = 1e-12


@pytest.fixture(scope="module")
def ml():
    import torch
    from paper_1608_07058_gb300 import build, matleap
    assert torch.cuda.is_available()
    build.build()
    matleap.lib()
    return matleap


def run_gpu(ml, crn, n, x0, T, theta=None, seed=0, base=0, model=None, **pkw):
    import torch
    d = torch.device("cuda")
    model = model or ml.model_from_crn(crn)
    x0t = torch.as_tensor(np.asarray(x0, np.int64), device=d)
    Tt = torch.as_tensor(np.atleast_1d(np.asarray(T, np.float64)), device=d)
    tht = None if theta is None else torch.as_tensor(np.asarray(theta, np.float64), device=d)
    pkw.setdefault("max_steps", MAX_STEPS)
    out = ml.ml_simulate(model, n, x0t, Tt, tht, params=ml.ml_default_params(**pkw), seed=seed,
                         traj_id_base=base)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["status"] = res["status"].astype(np.uint32)
    return res


def run_oracle(oracle, crn, n, x0, T, theta=None, seed=0, base=0, **pkw):
    pkw.setdefault("max_steps", MAX_STEPS)
    okw = {k: v for k, v in pkw.items() if k in oracle.Params.__dataclass_fields__}
    return oracle.simulate(crn, n, x0, T, theta, params=oracle.Params(**okw), seed=seed,
                           traj_id_base=base)


def assert_bit_parity(g, o, label=""):
    bad = np.flatnonzero((g["X"] != o["X"]).any(1) | (g["r"] != o["r"]).any(1))
    assert bad.size == 0, f"{label}: {bad.size} trajectories differ, first {bad[:5]}"
    assert np.array_equal(g["status"], o["status"]), label
    assert np.array_equal(g["counters"], o["counters"]), label
    den = np.maximum(np.abs(o["G"]), 1e-300)
    rel = np.max(np.abs(g["G"] - o["G"]) / den) if o["G"].size else 0.0
    assert rel <= G_RTOL, f"{label}: G rel err {rel}"


def _generic_network():
    # 5 species, 9 reactions, orders up to 3, a reversible pair: runs on the padded
    # (8 species, 16 reactions) variant
    return W._crn("generic5", 5, [
        ({0: 1}, {1: 1}, 2.0), ({1: 1}, {0: 1}, 1.5),          # A <-> B
        ({1: 2}, {2: 1}, 0.01), ({2: 1, 0: 1}, {3: 1}, 0.002),  # 2B -> C, A + C -> D
        ({0: 3}, {4: 1}, 1e-5), ({0: 2, 1: 1}, {4: 2}, 1e-5),  # 3A -> E, 2A + B -> 2E
        ({4: 1}, {}, 0.3), ({}, {0: 1}, 50.0), ({3: 1}, {0: 1, 2: 1}, 0.5),
    ])


CASES = {
    "immigration_death": lambda: (W.config(0, n_traj=3000), {}),
    "dimerisation": lambda: (W.config(1, n_traj=4000), {}),
    "gene_expression": lambda: (W.config(2, n_traj=400), {}),
}


@pytest.mark.parametrize("name", list(CASES))
def test_ref_bit_parity_configs(ml, oracle, name):
    w, kw = CASES[name]()
    g = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, w.theta, seed=3, **kw)
    o = run_oracle(oracle, w.crn, w.n_traj, w.x0, w.T, w.theta, seed=3, **kw)
    assert_bit_parity(g, o, name)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("x0", [(12, 5, 0), (60, 20, 0)])
def test_ref_bit_parity_small_counts_modes(ml, oracle, mode, x0):
    crn = W.dimerisation()
    g = run_gpu(ml, crn, 1500, list(x0), [1.5], seed=11, mode=mode)
    o = run_oracle(oracle, crn, 1500, list(x0), [1.5], seed=11, mode=mode)
    assert_bit_parity(g, o, f"mode{mode}")


@pytest.mark.parametrize("mode", [0, 1])
def test_ref_bit_parity_rejections(ml, oracle, mode):
    # without critical reactions (n_c = 0) and without the SSA switch (ssa_factor = 0)
    # small counts make leaps overshoot: the negativity check rejects and halves tau
    crn = W.dimerisation()
    kw = dict(mode=mode, n_c=0, ssa_factor=0.0)
    g = run_gpu(ml, crn, 2000, [12, 5, 0], [1.5], seed=13, **kw)
    o = run_oracle(oracle, crn, 2000, [12, 5, 0], [1.5], seed=13, **kw)
    assert_bit_parity(g, o, f"reject mode{mode}")
    assert g["counters"][:, 3].sum() > 0


def test_ref_bit_parity_generic_variant(ml, oracle):
    crn = _generic_network()
    for x0, T in (([200, 100, 5, 0, 3], 2.0), ([20000, 10000, 500, 0, 300], 0.5)):
        g = run_gpu(ml, crn, 1500, x0, [T], seed=5)
        o = run_oracle(oracle, crn, 1500, x0, [T], seed=5)
        assert_bit_parity(g, o, f"generic5 {x0}")
        assert g["counters"].sum(0)[:3].sum() > 0


def test_ref_bit_parity_per_traj_inputs_and_offsets(ml, oracle):
    w = W.config(1, n_traj=700)
    rng = np.random.default_rng(2)
    x0 = rng.integers(0, 500, size=(700, 3))
    T = rng.uniform(0.0, 0.3, size=700)
    T[:5] = 0.0
    theta = np.abs(w.crn.rates * rng.gamma(2.0, 0.5, size=(700, 4)))
    g = run_gpu(ml, w.crn, 700, x0, T, theta, seed=2**40 + 9, base=123456)
    o = run_oracle(oracle, w.crn, 700, x0, T, theta, seed=2**40 + 9, base=123456)
    assert_bit_parity(g, o, "per-traj")


def test_ref_full_size_sampled(ml, oracle):
    """The full 100,000-trajectory dimerisation launch, sampled by trajectory id."""
    w = W.config(1)
    g = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, seed=1)
    ids = np.unique(np.concatenate([np.arange(0, w.n_traj, 197), [w.n_traj - 1]]))
    for i in ids:
        o = run_oracle(oracle, w.crn, 1, w.x0, w.T, seed=1, base=int(i))
        sub = {k: v[i:i + 1] for k, v in g.items()}
        assert_bit_parity(sub, o, f"id {i}")
    assert (g["status"] == 0).all()


def test_persistent_graph_and_host_paths_identical(ml):
    import torch
    w = W.config(2, n_traj=3000)
    model = ml.model_from_crn(w.crn)
    base = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, w.theta, seed=4, model=model)
    pers = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, w.theta, seed=4, model=model,
                   form=ml.ML_FORM_PERSISTENT, block_size=64, ctas_per_sm=2)
    graph1 = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, w.theta, seed=4, model=model,
                     form=ml.ML_FORM_PERSISTENT, use_graph=1)
    graph2 = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, w.theta, seed=4, model=model,
                     form=ml.ML_FORM_PERSISTENT, use_graph=1)
    host = ml.ml_simulate_host(model, w.n_traj, w.x0, w.T, w.theta,
                               params=ml.ml_default_params(max_steps=MAX_STEPS), seed=4)
    host["status"] = host["status"].astype(np.uint32)
    for name, other in (("persistent", pers), ("graph1", graph1), ("graph2", graph2), ("host", host)):
        for k in ("X", "r", "G", "status", "counters"):
            assert np.array_equal(base[k], other[k]), (name, k)


def test_zero_and_tiny_batches(ml, oracle):
    import torch
    crn = W.immigration_death()
    m = ml.model_from_crn(crn)
    x0 = torch.zeros(1, dtype=torch.int64, device="cuda")
    T = torch.full((1,), 5.0, dtype=torch.float64, device="cuda")
    out = ml.ml_simulate(m, 0, x0, T)
    assert out["X"].shape == (0, 1)
    for n in (1, 31, 33, 257):
        g = run_gpu(ml, crn, n, [0], [5.0], seed=8, model=m)
        o = run_oracle(oracle, crn, n, [0], [5.0], seed=8)
        assert_bit_parity(g, o, f"n={n}")


def test_fast_statistics_dimerisation(ml, oracle):
    w = W.config(1, n_traj=20000)
    g = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, seed=21, precision=ml.ML_PREC_FAST_FP32,
                form=ml.ML_FORM_PERSISTENT, use_graph=1)
    o = run_oracle(oracle, w.crn, w.n_traj, w.x0, w.T, seed=21)
    rows = stats_util.compare(g, o, g_res=stats_util.G_RESOLUTION_FAST)
    s = stats_util.summary(rows)
    assert s["holm_pass_0.01"], (s, sorted(rows, key=lambda r: r[2])[:5])
    assert (g["status"] == 0).all()


def test_fast_statistics_immigration_death_and_gene(ml, oracle):
    for cfg, n in ((0, 10000), (2, 3000)):
        w = W.config(cfg, n_traj=n)
        g = run_gpu(ml, w.crn, n, w.x0, w.T, w.theta, seed=31, precision=ml.ML_PREC_FAST_FP32)
        o = run_oracle(oracle, w.crn, n, w.x0, w.T, w.theta, seed=31)
        rows = stats_util.compare(g, o, g_res=stats_util.G_RESOLUTION_FAST)
        s = stats_util.summary(rows)
        assert s["holm_pass_0.01"], (cfg, s, sorted(rows, key=lambda r: r[2])[:5])


def test_autotune_picks_a_valid_shape(ml):
    import torch
    w = W.config(1, n_traj=20000)
    model = ml.model_from_crn(w.crn)
    d = torch.device("cuda")
    x0 = torch.as_tensor(w.x0, device=d)
    T = torch.as_tensor(w.T, device=d)
    best = ml.ml_autotune(model, w.n_traj, x0, T, None,
                          params=ml.ml_default_params(precision=ml.ML_PREC_FAST_FP32,
                                                      form=ml.ML_FORM_PERSISTENT),
                          n_sample=8192)
    assert best.shape in (1, 2, 3, 4, 5)
    assert best.block_size in (64, 128, 256)


# ---- one trajectory per warp ------------------------------------------------------

@pytest.mark.parametrize("name", ["immigration_death", "dimerisation", "gene_expression"])
def test_ref_warp_shape_bit_parity_small_networks(ml, oracle, name):
    """The warp kernel keeps the same canonical order, so it matches the same oracle."""
    w, kw = CASES[name]()
    n = min(w.n_traj, 1000)
    th = None if w.theta is None else w.theta[:n]
    T = w.T[:n] if w.T.size > 1 else w.T
    g = run_gpu(ml, w.crn, n, w.x0, T, th, seed=3, shape=ml.ML_SHAPE_WARP)
    o = run_oracle(oracle, w.crn, n, w.x0, T, th, seed=3)
    assert_bit_parity(g, o, name + " warp")


def test_ref_warp_generic_and_small_counts(ml, oracle):
    crn = _generic_network()
    x0 = [20000, 10000, 500, 0, 300]
    g = run_gpu(ml, crn, 600, x0, [0.5], seed=5, shape=ml.ML_SHAPE_WARP)
    o = run_oracle(oracle, crn, 600, x0, [0.5], seed=5)
    assert_bit_parity(g, o, "generic5 warp")
    crn = W.dimerisation()
    for mode, n_c, f in ((0, 10, 10.0), (1, 0, 0.0), (0, 0, 0.0), (2, 10, 10.0)):
        g = run_gpu(ml, crn, 800, [12, 5, 0], [1.5], seed=13, mode=mode, n_c=n_c,
                    ssa_factor=f, shape=ml.ML_SHAPE_WARP)
        o = run_oracle(oracle, crn, 800, [12, 5, 0], [1.5], seed=13, mode=mode, n_c=n_c,
                       ssa_factor=f)
        assert_bit_parity(g, o, f"dimer warp mode{mode}")


def test_ref_random_crn_50x100(ml, oracle):
    """The large random network (50 species, 100 reactions, 10 reversible pairs) on a short
    horizon: explicit, implicit (50x50 Newton) and SSA steps, bit-identical."""
    w = W.config(3, n_traj=48)
    g = run_gpu(ml, w.crn, 48, w.x0, [0.05], seed=9, base=1000)
    o = run_oracle(oracle, w.crn, 48, w.x0, [0.05], seed=9, base=1000)
    assert_bit_parity(g, o, "random_crn")
    c = g["counters"].sum(0)
    assert c[1] > 0 and c[2] > 0  # implicit leaps and SSA firings both occurred


def test_fast_warp_statistics_dimerisation(ml, oracle):
    w = W.config(1, n_traj=20000)
    g = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, seed=22, precision=ml.ML_PREC_FAST_FP32,
                shape=ml.ML_SHAPE_WARP, form=ml.ML_FORM_PERSISTENT)
    o = run_oracle(oracle, w.crn, w.n_traj, w.x0, w.T, seed=22)
    s = stats_util.summary(stats_util.compare(g, o, g_res=stats_util.G_RESOLUTION_FAST))
    assert s["holm_pass_0.01"], s


def test_fast_random_crn_statistics(ml, oracle):
    w = W.config(3, n_traj=400)
    g = run_gpu(ml, w.crn, 400, w.x0, [0.02], seed=23, precision=ml.ML_PREC_FAST_FP32,
                form=ml.ML_FORM_PERSISTENT)
    o = run_oracle(oracle, w.crn, 400, w.x0, [0.02], seed=23)
    s = stats_util.summary(stats_util.compare(g, o, g_res=stats_util.G_RESOLUTION_FAST))
    assert s["holm_pass_0.01"], s


@pytest.mark.parametrize("shape", [1, 2])
def test_ref_bit_parity_analytic_jacobian(ml, oracle, shape):
    """The exact (symbolic) Jacobian option: bit-identical to the oracle's exact
    Jacobian, in both kernel shapes."""
    w = W.config(1, n_traj=3000)
    g = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, seed=17, jacobian=1, shape=shape)
    o = run_oracle(oracle, w.crn, w.n_traj, w.x0, w.T, seed=17, jacobian=1)
    assert_bit_parity(g, o, f"analytic shape{shape}")
    assert g["counters"][:, 1].sum() > 0
    crn = _generic_network()
    x0 = [20000, 10000, 500, 0, 300]
    g = run_gpu(ml, crn, 600, x0, [0.5], seed=5, jacobian=1, shape=shape)
    o = run_oracle(oracle, crn, 600, x0, [0.5], seed=5, jacobian=1)
    assert_bit_parity(g, o, f"generic analytic shape{shape}")


def test_ref_random_crn_analytic_jacobian(ml, oracle):
    w = W.config(3, n_traj=32)
    g = run_gpu(ml, w.crn, 32, w.x0, [0.05], seed=19, jacobian=1)
    o = run_oracle(oracle, w.crn, 32, w.x0, [0.05], seed=19, jacobian=1)
    assert_bit_parity(g, o, "random_crn analytic")


@pytest.mark.parametrize("mu", [3.0, 9.5, 50.0, 1.2e4, 1e6, 3e7])
def test_fast_poisson_sampler_law(ml, oracle, mu):
    """0 -> A at rate mu over T = 1 from A = 0: no species bounds the leap, so each
    trajectory is one leap to T and X(T) is a single Poisson(mu) draw of the kernel's
    sampler (inversion below 10, PTRS above).  Fast precision against scipy's Poisson law."""
    from scipy import stats
    crn = W._crn("source", 1, [({}, {0: 1}, mu)])
    n = 100_000
    for shape in (1, 2):
        g = run_gpu(ml, crn, n, [0], [1.0], seed=29, precision=ml.ML_PREC_FAST_FP32,
                    shape=shape, form=ml.ML_FORM_PERSISTENT)
        assert (g["counters"][:, 0] == 1).all()
        X = g["X"][:, 0].astype(np.float64)
        assert abs(X.mean() - mu) < 5 * np.sqrt(mu / n)
        se_var = np.sqrt((mu + 2 * mu * mu) / n)
        assert abs(X.var() - mu) < 5 * se_var
        lo, hi = stats.poisson.ppf([1e-4, 1 - 1e-4], mu)
        edges = np.unique(np.round(np.linspace(lo, hi + 1, 30)))
        obs = np.histogram(X, np.concatenate([[-np.inf], edges[1:-1], [np.inf]]))[0]
        p = np.diff(np.concatenate([[0.0], stats.poisson.cdf(edges[1:-1] - 1, mu), [1.0]]))
        keep = p * n > 5
        assert stats.chisquare(obs[keep], p[keep] * n * obs[keep].sum() / (p[keep] * n).sum()).pvalue > 1e-4


@pytest.mark.parametrize("shape", [1, 4])
@pytest.mark.parametrize("cfg,n", [(1, 3000), (2, 500)])
def test_ref_bit_parity_thread_drivers(ml, oracle, shape, cfg, n):
    """Both thread drivers (round-based and sequential per lane) in both launch forms run
    the same per-lane arithmetic: bit-identical to the oracle."""
    w = W.config(cfg, n_traj=n)
    o = run_oracle(oracle, w.crn, n, w.x0, w.T, w.theta, seed=41)
    for form in (0, 1):
        g = run_gpu(ml, w.crn, n, w.x0, w.T, w.theta, seed=41, shape=shape, form=form)
        assert_bit_parity(g, o, f"shape{shape} form{form}")


@pytest.mark.parametrize("shape,newton,jac", [
    (4, 0, 0), (4, 0, 1), (4, 1, 1), (5, 0, 0), (5, 1, 1), (1, 0, 0), (3, 0, 1),
    (2, 0, 0), (2, 1, 0)])
def test_fast_statistics_dimerisation_newton_forms(ml, oracle, shape, newton, jac):
    """Fast precision with the FP64 Newton solve (forward-difference or exact Jacobian) and
    with the FP32 one, in every thread driver/build and the warp kernel: the ensemble of
    20,000 stiff-dimerisation trajectories (about 14 implicit leaps each) matches the
    oracle's statistics."""
    w = W.config(1, n_traj=20000)
    g = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, seed=41 + shape, precision=ml.ML_PREC_FAST_FP32,
                form=ml.ML_FORM_PERSISTENT, shape=shape, newton_precision=newton, jacobian=jac)
    o = run_oracle(oracle, w.crn, w.n_traj, w.x0, w.T, seed=41 + shape, jacobian=jac)
    assert (g["counters"][:, 1] > 0).mean() > 0.99
    s = stats_util.summary(stats_util.compare(g, o, g_res=stats_util.G_RESOLUTION_FAST))
    assert s["holm_pass_0.01"], s
    assert (g["status"] == 0).all()
