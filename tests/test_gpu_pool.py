"""The pool driver (ML_SHAPE_THREAD_POOL, _OCC): each warp keeps 64 trajectories in shared
memory and runs one phase for 32 of them per round.  Trajectories are keyed by id and the
arithmetic is the lane state machine's, so in reference precision every result must be
bit-identical to the oracle (and to the other drivers), whatever the pool's schedule; in
fast precision the ensemble statistics must match the oracle's."""
import numpy as np
import pytest

from paper_1608_07058_gb300 import workloads as W
from tests import stats_util
from tests.test_gpu_parity import _generic_network, assert_bit_parity, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ml():
    import torch
    from paper_1608_07058_gb300 import build, matleap
    assert torch.cuda.is_available()
    build.build()
    matleap.lib()
    return matleap


def pool_kw(ml, **kw):
    return dict(form=ml.ML_FORM_PERSISTENT, shape=ml.ML_SHAPE_THREAD_POOL, **kw)


@pytest.mark.parametrize("cfg,n", [(0, 3000), (1, 4000), (2, 500)])
@pytest.mark.parametrize("block", [64, 256])
def test_pool_ref_bit_parity_configs(ml, oracle, cfg, n, block):
    w = W.config(cfg, n_traj=n)
    g = run_gpu(ml, w.crn, n, w.x0, w.T, w.theta, seed=3, **pool_kw(ml, block_size=block))
    o = run_oracle(oracle, w.crn, n, w.x0, w.T, w.theta, seed=3)
    assert_bit_parity(g, o, f"pool cfg{cfg} block{block}")


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_pool_ref_bit_parity_small_counts_modes(ml, oracle, mode):
    crn = W.dimerisation()
    g = run_gpu(ml, crn, 1500, [12, 5, 0], [1.5], seed=11, **pool_kw(ml, mode=mode))
    o = run_oracle(oracle, crn, 1500, [12, 5, 0], [1.5], seed=11, mode=mode)
    assert_bit_parity(g, o, f"pool mode{mode}")


def test_pool_ref_bit_parity_rejections_and_generic(ml, oracle):
    crn = W.dimerisation()
    kw = dict(n_c=0, ssa_factor=0.0)
    g = run_gpu(ml, crn, 2000, [12, 5, 0], [1.5], seed=13, **pool_kw(ml, **kw))
    o = run_oracle(oracle, crn, 2000, [12, 5, 0], [1.5], seed=13, **kw)
    assert_bit_parity(g, o, "pool rejections")
    assert g["counters"][:, 3].sum() > 0
    # the padded (8 species, 16 reactions) variant; 256 threads per CTA are cut to what
    # the shared-memory records allow
    crn = _generic_network()
    for x0, T in (([200, 100, 5, 0, 3], 2.0), ([20000, 10000, 500, 0, 300], 0.5)):
        g = run_gpu(ml, crn, 1500, x0, [T], seed=5, **pool_kw(ml, block_size=256))
        o = run_oracle(oracle, crn, 1500, x0, [T], seed=5)
        assert_bit_parity(g, o, f"pool generic5 {x0}")


def test_pool_ref_per_traj_inputs_offsets_and_tiny_batches(ml, oracle):
    w = W.config(1, n_traj=700)
    rng = np.random.default_rng(2)
    x0 = rng.integers(0, 500, size=(700, 3))
    T = rng.uniform(0.0, 0.3, size=700)
    T[:5] = 0.0
    theta = np.abs(w.crn.rates * rng.gamma(2.0, 0.5, size=(700, 4)))
    g = run_gpu(ml, w.crn, 700, x0, T, theta, seed=2**40 + 9, base=123456, **pool_kw(ml))
    o = run_oracle(oracle, w.crn, 700, x0, T, theta, seed=2**40 + 9, base=123456)
    assert_bit_parity(g, o, "pool per-traj")
    crn = W.immigration_death()
    for n in (1, 31, 33, 65, 257):
        g = run_gpu(ml, crn, n, [0], [5.0], seed=8, **pool_kw(ml))
        o = run_oracle(oracle, crn, n, [0], [5.0], seed=8)
        assert_bit_parity(g, o, f"pool n={n}")


def test_pool_equals_round_based_reference(ml):
    w = W.config(2, n_traj=3000)
    model = ml.model_from_crn(w.crn)
    a = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, w.theta, seed=4, model=model,
                form=ml.ML_FORM_PERSISTENT, shape=ml.ML_SHAPE_THREAD)
    b = run_gpu(ml, w.crn, w.n_traj, w.x0, w.T, w.theta, seed=4, model=model,
                **pool_kw(ml, use_graph=1))
    for k in ("X", "r", "G", "status", "counters"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("shape_name", ["ML_SHAPE_THREAD_POOL", "ML_SHAPE_THREAD_POOL_OCC"])
def test_pool_fast_statistics(ml, oracle, shape_name):
    for cfg, n in ((1, 20000), (2, 3000), (0, 10000)):
        w = W.config(cfg, n_traj=n)
        g = run_gpu(ml, w.crn, n, w.x0, w.T, w.theta, seed=31, precision=ml.ML_PREC_FAST_FP32,
                    form=ml.ML_FORM_PERSISTENT, shape=getattr(ml, shape_name), use_graph=1)
        o = run_oracle(oracle, w.crn, n, w.x0, w.T, w.theta, seed=31)
        rows = stats_util.compare(g, o, g_res=stats_util.G_RESOLUTION_FAST)
        s = stats_util.summary(rows)
        assert s["holm_pass_0.01"], (cfg, shape_name, s, sorted(rows, key=lambda r: r[2])[:5])
        assert (g["status"] == 0).all()
