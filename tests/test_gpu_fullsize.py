"""Full-size launches of the benchmark workloads, checked on every trajectory by properties
that hold at any size and on sampled trajectory ids against the oracle.

- Gene expression, 1,000,000 trajectories in the launch configuration the benchmark times
  (fast precision, persistent form, CUDA graph, kernels compiled for the model, pool
  driver -- the shape the benchmark's whole-batch autotuning picks on GB300): X(T) =
  x0 + nu^T r exactly and nothing negative on all of them; the ensemble statistics of
  3,000 ids spread over the batch agree with the oracle run on the same ids (4-SE mean and
  variance, KS, Holm at 0.01).  The same launch in reference precision: 200 ids spread
  over the batch bit-identical to the oracle.
- Random 50 x 100 network, its full batch of 65,536 trajectories (one per warp) over a
  short horizon, reference precision: the same invariants on all, and 64 sampled ids
  bit-identical to the oracle."""
import numpy as np
import pytest

from paper_1608_07058_gb300 import workloads as W
from tests import stats_util
from tests.test_gpu_parity import assert_bit_parity

pytestmark = pytest.mark.gpu

MAX_STEPS = 1_000_000


@pytest.fixture(scope="module")
def ml():
    import torch
    from paper_1608_07058_gb300 import build, matleap
    assert torch.cuda.is_available()
    build.build()
    matleap.lib()
    return matleap


def _device_run(ml, w, T, params, seed):
    import torch
    d = torch.device("cuda")
    model = ml.model_from_crn(w.crn)
    x0 = torch.as_tensor(w.x0, device=d)
    Tt = torch.as_tensor(np.atleast_1d(T), device=d)
    th = None if w.theta is None else torch.as_tensor(w.theta, device=d)
    if params.form == ml.ML_FORM_PERSISTENT and params.block_size == 0:
        best = ml.ml_autotune(model, w.n_traj, x0, Tt, th, params=params, n_sample=8_192)
        params.shape, params.block_size, params.ctas_per_sm = (best.shape, best.block_size,
                                                               best.ctas_per_sm)
    out = ml.ml_simulate(model, w.n_traj, x0, Tt, th, params=params, seed=seed)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["status"] = res["status"].astype(np.uint32)
    return res


def _invariants(w, g):
    x0 = np.broadcast_to(np.asarray(w.x0, np.int64), g["X"].shape)
    assert np.array_equal(g["X"], x0 + g["r"] @ w.crn.stoich.astype(np.int64))
    assert (g["X"] >= 0).all() and (g["r"] >= 0).all()
    assert np.isfinite(g["G"]).all() and (g["G"] >= 0).all()


def test_gene_expression_full_batch_fast(ml, oracle):
    w = W.config(2)
    assert w.n_traj == 1_000_000
    p = ml.ml_default_params(precision=ml.ML_PREC_FAST_FP32, form=ml.ML_FORM_PERSISTENT,
                             use_graph=1, max_steps=MAX_STEPS, specialize=1,
                             shape=ml.ML_SHAPE_THREAD_POOL, block_size=128)
    g = _device_run(ml, w, w.T, p, seed=77)
    _invariants(w, g)
    assert (g["status"] & ~np.uint32(2 | 8) == 0).all()
    ids = np.linspace(0, w.n_traj - 1, 3000).astype(np.int64)
    o = {k: [] for k in ("X", "r", "G")}
    for i in ids:
        oi = oracle.simulate(w.crn, 1, w.x0, w.T[i:i + 1], w.theta[i:i + 1],
                             params=oracle.Params(max_steps=MAX_STEPS), seed=77,
                             traj_id_base=int(i))
        for k in o:
            o[k].append(oi[k][0])
    o = {k: np.array(v) for k, v in o.items()}
    sub = {k: g[k][ids] for k in ("X", "r", "G")}
    s = stats_util.summary(stats_util.compare(sub, o, g_res=stats_util.G_RESOLUTION_FAST))
    assert s["holm_pass_0.01"], s


def test_gene_expression_full_batch_ref_specialized_sampled(ml, oracle):
    w = W.config(2)
    p = ml.ml_default_params(form=ml.ML_FORM_PERSISTENT, use_graph=1, max_steps=MAX_STEPS,
                             specialize=1, shape=ml.ML_SHAPE_THREAD_POOL, block_size=128)
    g = _device_run(ml, w, w.T, p, seed=78)
    _invariants(w, g)
    ids = np.unique(np.concatenate([np.linspace(0, w.n_traj - 1, 199).astype(np.int64),
                                    [w.n_traj - 1]]))
    for i in ids:
        oi = oracle.simulate(w.crn, 1, w.x0, w.T[i:i + 1], w.theta[i:i + 1],
                             params=oracle.Params(max_steps=MAX_STEPS), seed=78,
                             traj_id_base=int(i))
        assert_bit_parity({k: v[i:i + 1] for k, v in g.items()}, oi, f"id {i}")


def test_random_crn_full_batch_ref_sampled(ml, oracle):
    w = W.config(3)
    assert w.n_traj == 65_536
    T = 0.004
    p = ml.ml_default_params(max_steps=MAX_STEPS, form=ml.ML_FORM_PERSISTENT, block_size=128)
    g = _device_run(ml, w, T, p, seed=5)
    _invariants(w, g)
    assert (g["status"] == 0).all()
    ids = np.unique(np.concatenate([np.linspace(0, w.n_traj - 1, 63).astype(np.int64),
                                    [w.n_traj - 1]]))
    for i in ids:
        oi = oracle.simulate(w.crn, 1, w.x0, [T], None,
                             params=oracle.Params(max_steps=MAX_STEPS), seed=5,
                             traj_id_base=int(i))
        assert_bit_parity({k: v[i:i + 1] for k, v in g.items()}, oi, f"id {i}")
