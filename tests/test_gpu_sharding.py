"""The product path sharded by trajectory id on one GPU: any partition of a batch into
id ranges (matleap.shard_bounds, rows sliced, traj_id_base = the range's first id) gives
exactly the results of one call over the whole batch, in both precisions and through
both the device-buffer and the host-buffer entry points.  This is what lets ranks of a
multi-GPU job simulate disjoint id ranges with no exchange step."""
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


KEYS = ("X", "r", "G", "status", "counters")


@pytest.mark.parametrize("precision", [0, 1])
def test_id_ranges_concatenate_to_one_call(ml, precision):
    import torch
    d = torch.device("cuda")
    n = 5003
    w = W.config(2, n_traj=n)
    model = ml.model_from_crn(w.crn)
    x0 = torch.as_tensor(w.x0, device=d)
    T = torch.as_tensor(w.T, device=d)
    theta = torch.as_tensor(w.theta, device=d)
    p = ml.ml_default_params(precision=precision, form=ml.ML_FORM_PERSISTENT, use_graph=1,
                             max_steps=200_000)
    whole = ml.ml_simulate(model, n, x0, T, theta, params=p, seed=13, traj_id_base=1000)
    whole = {k: v.cpu().numpy() for k, v in whole.items()}
    for world in (2, 3):
        parts = []
        for rank in range(world):
            lo, hi = ml.shard_bounds(n, rank, world)
            o = ml.ml_simulate(model, hi - lo, x0, T[lo:hi], theta[lo:hi], params=p, seed=13,
                               traj_id_base=1000 + lo)
            parts.append({k: v.cpu().numpy() for k, v in o.items()})
        for k in KEYS:
            assert np.array_equal(np.concatenate([q[k] for q in parts]), whole[k]), (world, k)


def test_host_entry_point_shards(ml):
    import torch
    n = 3001
    w = W.config(1, n_traj=n)
    model = ml.model_from_crn(w.crn)
    p = ml.ml_default_params(precision=ml.ML_PREC_FAST_FP32, form=ml.ML_FORM_PERSISTENT)
    whole = ml.ml_simulate_host(model, n, w.x0, w.T, params=p, seed=14)
    parts = []
    for rank in range(2):
        lo, hi = ml.shard_bounds(n, rank, 2)
        parts.append(ml.ml_simulate_host(model, hi - lo, w.x0, w.T, params=p, seed=14,
                                         traj_id_base=lo))
    for k in KEYS:
        assert np.array_equal(np.concatenate([q[k] for q in parts]), whole[k]), k
