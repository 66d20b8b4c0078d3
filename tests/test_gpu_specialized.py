"""Model-specialized kernels (ml_sim_params.specialize = 1): the thread-per-trajectory
drivers compiled at run time with the model's tables as constants.  They run the same
lane state machine as the precompiled kernels, so in reference precision every
trajectory must be bit-identical to the oracle and to the precompiled kernels, in every
driver, mode and feature (critical reactions, rejections, partial equilibrium and the
implicit Newton solve with either Jacobian, the padded generic variant); in fast
precision the ensemble statistics must match the oracle's."""
import numpy as np
import pytest

from paper_1608_07058_gb300 import workloads as W
from tests import stats_util
from tests.test_gpu_parity import _generic_network, assert_bit_parity, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

KEYS = ("X", "r", "G", "status", "counters")


@pytest.fixture(scope="module")
def ml():
    import torch
    from paper_1608_07058_gb300 import build, matleap
    assert torch.cuda.is_available()
    build.build()
    matleap.lib()
    return matleap


def drivers(ml):
    """(name, parameters) of every thread driver the specialized kernels serve."""
    P = ml.ML_FORM_PERSISTENT
    return [("plain", dict(form=ml.ML_FORM_PLAIN)),
            ("rounds", dict(form=P, shape=ml.ML_SHAPE_THREAD)),
            ("sequential", dict(form=P, shape=ml.ML_SHAPE_THREAD_SEQ, use_graph=1)),
            ("pool", dict(form=P, shape=ml.ML_SHAPE_THREAD_POOL, use_graph=1))]


@pytest.mark.parametrize("cfg,n", [(0, 3000), (1, 4000), (2, 500)])
def test_specialized_ref_bit_parity_configs(ml, oracle, cfg, n):
    w = W.config(cfg, n_traj=n)
    o = run_oracle(oracle, w.crn, n, w.x0, w.T, w.theta, seed=3)
    model = ml.model_from_crn(w.crn)
    for name, kw in drivers(ml):
        g = run_gpu(ml, w.crn, n, w.x0, w.T, w.theta, seed=3, model=model, specialize=1, **kw)
        assert_bit_parity(g, o, f"specialized {name} cfg{cfg}")


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_specialized_ref_small_counts_modes_and_rejections(ml, oracle, mode):
    crn = W.dimerisation()
    model = ml.model_from_crn(crn)
    for kw in ({}, {"n_c": 0, "ssa_factor": 0.0}):
        o = run_oracle(oracle, crn, 1500, [12, 5, 0], [1.5], seed=11, mode=mode, **kw)
        g = run_gpu(ml, crn, 1500, [12, 5, 0], [1.5], seed=11, model=model, specialize=1,
                    mode=mode, form=ml.ML_FORM_PERSISTENT, **kw)
        assert_bit_parity(g, o, f"specialized mode{mode} {kw}")


@pytest.mark.parametrize("jac", [0, 1])
def test_specialized_ref_implicit_leaps(ml, oracle, jac):
    """The stiff dimerisation takes implicit leaps (one reversible pair in partial
    equilibrium): the specialized kernel keeps the Newton solve, with either Jacobian."""
    w = W.config(1, n_traj=3000)
    o = run_oracle(oracle, w.crn, w.n_traj, w.x0, w.T, seed=9, jacobian=jac)
    assert o["counters"][:, 1].sum() > 0
    g = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, seed=9, specialize=1, jacobian=jac,
                form=ml.ML_FORM_PERSISTENT, shape=ml.ML_SHAPE_THREAD_SEQ)
    assert_bit_parity(g, o, f"specialized implicit jac{jac}")


def test_specialized_ref_generic_variant_and_per_traj_inputs(ml, oracle):
    crn = _generic_network()
    for x0, T in (([200, 100, 5, 0, 3], 2.0), ([20000, 10000, 500, 0, 300], 0.5)):
        g = run_gpu(ml, crn, 1500, x0, [T], seed=5, specialize=1, form=ml.ML_FORM_PERSISTENT,
                    shape=ml.ML_SHAPE_THREAD_POOL, block_size=256)
        o = run_oracle(oracle, crn, 1500, x0, [T], seed=5)
        assert_bit_parity(g, o, f"specialized generic5 {x0}")
    w = W.config(1, n_traj=700)
    rng = np.random.default_rng(2)
    x0 = rng.integers(0, 500, size=(700, 3))
    T = rng.uniform(0.0, 0.3, size=700)
    theta = np.abs(w.crn.rates * rng.gamma(2.0, 0.5, size=(700, 4)))
    g = run_gpu(ml, w.crn, 700, x0, T, theta, seed=2**40 + 9, base=123456, specialize=1)
    o = run_oracle(oracle, w.crn, 700, x0, T, theta, seed=2**40 + 9, base=123456)
    assert_bit_parity(g, o, "specialized per-traj")
    crn = W.immigration_death()
    for n in (1, 31, 33, 257):
        g = run_gpu(ml, crn, n, [0], [5.0], seed=8, specialize=1, form=ml.ML_FORM_PERSISTENT)
        o = run_oracle(oracle, crn, n, [0], [5.0], seed=8)
        assert_bit_parity(g, o, f"specialized n={n}")


def test_specialized_equals_precompiled_reference(ml):
    w = W.config(2, n_traj=3000)
    model = ml.model_from_crn(w.crn)
    for name, kw in drivers(ml):
        a = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, w.theta, seed=4, model=model, **kw)
        b = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, w.theta, seed=4, model=model, specialize=1,
                    **kw)
        for k in KEYS:
            assert np.array_equal(a[k], b[k]), (name, k)


@pytest.mark.parametrize("cfg,n", [(0, 10000), (1, 20000), (2, 3000)])
def test_specialized_fast_statistics(ml, oracle, cfg, n):
    w = W.config(cfg, n_traj=n)
    o = run_oracle(oracle, w.crn, n, w.x0, w.T, w.theta, seed=31)
    model = ml.model_from_crn(w.crn)
    for name, kw in drivers(ml)[1:]:
        for occ in (False, True):
            kw2 = dict(kw)
            if occ:
                kw2["shape"] = {ml.ML_SHAPE_THREAD: ml.ML_SHAPE_THREAD_OCC,
                                ml.ML_SHAPE_THREAD_SEQ: ml.ML_SHAPE_THREAD_SEQ_OCC,
                                ml.ML_SHAPE_THREAD_POOL: ml.ML_SHAPE_THREAD_POOL_OCC}[kw["shape"]]
            g = run_gpu(ml, w.crn, n, w.x0, w.T, w.theta, seed=31, model=model, specialize=1,
                        precision=ml.ML_PREC_FAST_FP32, **kw2)
            rows = stats_util.compare(g, o, g_res=stats_util.G_RESOLUTION_FAST)
            s = stats_util.summary(rows)
            assert s["holm_pass_0.01"], (cfg, name, occ, s, sorted(rows, key=lambda r: r[2])[:5])
            assert (g["status"] == 0).all()
