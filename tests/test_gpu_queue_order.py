"""The persistent form's work-queue order (ml_sim_params.queue_order): trajectories are
keyed by id, so handing them out in any order -- reversed, shuffled, longest first by a
previous call's event counts -- leaves every result bit-identical, in both precisions and
kernel shapes and through the host-buffer entry point.  Entries outside [0, n) are passed
over by the kernels' bounds check."""
import numpy as np
import pytest

from paper_1608_07058_gb300 import workloads as W

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


@pytest.mark.parametrize("precision,shape,cfg,n", [(1, 1, 2, 20000), (1, 4, 2, 5000), (0, 1, 1, 3000),
                                                   (1, 2, 1, 2000)])
def test_queue_order_does_not_change_results(ml, precision, shape, cfg, n):
    import torch
    d = torch.device("cuda")
    w = W.config(cfg, n_traj=n)
    model = ml.model_from_crn(w.crn)
    x0 = torch.as_tensor(w.x0, device=d)
    T = torch.as_tensor(w.T, device=d)
    theta = None if w.theta is None else torch.as_tensor(w.theta, device=d)
    p = ml.ml_default_params(precision=precision, form=ml.ML_FORM_PERSISTENT, shape=shape,
                             max_steps=1_000_000)
    base = ml.ml_simulate(model, n, x0, T, theta, params=p, seed=19)
    base = {k: v.cpu().numpy() for k, v in base.items()}
    cost = 8 * base["counters"][:, :2].sum(1) + base["counters"][:, 2]
    g = torch.Generator().manual_seed(3)
    orders = {"reversed": torch.arange(n - 1, -1, -1), "shuffled": torch.randperm(n, generator=g),
              "longest first": torch.as_tensor(np.argsort(-cost, kind="stable"))}
    for name, o in orders.items():
        od = o.to(torch.int64).to(d).contiguous()
        q = ml.ml_default_params(precision=precision, form=ml.ML_FORM_PERSISTENT, shape=shape,
                                 max_steps=1_000_000, use_graph=1, queue_order=od.data_ptr())
        got = ml.ml_simulate(model, n, x0, T, theta, params=q, seed=19)
        torch.cuda.synchronize()
        for k in KEYS:
            assert np.array_equal(got[k].cpu().numpy(), base[k]), (name, k)


def test_queue_order_host_path_and_out_of_range_entries(ml):
    import torch
    d = torch.device("cuda")
    n = 3000
    w = W.config(1, n_traj=n)
    model = ml.model_from_crn(w.crn)
    p = ml.ml_default_params(precision=1, form=ml.ML_FORM_PERSISTENT)
    base = ml.ml_simulate_host(model, n, w.x0, w.T, params=p, seed=23)
    order = np.ascontiguousarray(np.arange(n)[::-1], np.int64)
    q = ml.ml_default_params(precision=1, form=ml.ML_FORM_PERSISTENT, queue_order=order.ctypes.data)
    got = ml.ml_simulate_host(model, n, w.x0, w.T, params=q, seed=23)
    for k in KEYS:
        assert np.array_equal(got[k], base[k]), k
    # an order with entries outside [0, n): those are passed over, the rest run as usual
    bad = np.arange(n, dtype=np.int64)
    bad[:10] = [-1, n, n + 7, -(2 ** 40), 2 ** 40, 0, 1, 2, 3, 4]   # ids 0..4 still present
    bad_d = torch.as_tensor(bad, device=d)
    N, M = model.N, model.M
    out = {"X": torch.full((n, N), -7, dtype=torch.int64, device=d),
           "r": torch.full((n, M), -7, dtype=torch.int64, device=d),
           "G": torch.full((n, M), -7.0, dtype=torch.float64, device=d),
           "status": torch.full((n,), -7, dtype=torch.int32, device=d),
           "counters": torch.full((n, 4), -7, dtype=torch.int64, device=d)}
    q = ml.ml_default_params(precision=1, form=ml.ML_FORM_PERSISTENT, queue_order=bad_d.data_ptr())
    ml.ml_simulate(model, n, torch.as_tensor(w.x0, device=d), torch.as_tensor(w.T, device=d),
                   params=q, seed=23, out=out)
    torch.cuda.synchronize()
    ran = np.r_[0:5, 10:n]
    skipped = np.r_[5:10]
    for k in KEYS:
        v = out[k].cpu().numpy()
        assert np.array_equal(v[ran].astype(base[k].dtype), base[k][ran]), k
        assert (v[skipped] == -7).all(), k
