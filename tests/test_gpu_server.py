"""The continuous-batching server: requests of different models and sizes admitted as
slots and device memory free up, running concurrently, each with exactly the results it
gets alone; admission never exceeds the device-memory budget; bounded waits; shutdown
with queued requests."""
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


@pytest.fixture(scope="module")
def models(ml):
    return {m: ml.model_from_crn(W.config(m, n_traj=1).crn) for m in (0, 1, 2, 3)}


@pytest.mark.parametrize("precision", [0, 1])
def test_mix_equals_standalone(ml, models, precision):
    p = ml.ml_default_params(precision=precision, form=ml.ML_FORM_PERSISTENT, max_steps=200_000)
    reqs = W.serving_requests(24, seed=3, min_traj=100, max_traj=4000)
    srv = ml.ml_server(256 << 20, 6, p)
    handles = []
    for q in reqs:
        wl = q["workload"]
        handles.append(srv.submit(models[q["model_index"]], wl.n_traj, wl.x0, wl.T, wl.theta,
                                  seed=wl.seed, traj_id_base=wl.traj_id_base))
    for h in handles:
        assert h.wait(300_000)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["peak_inflight"] > 1
    for q, h in zip(reqs, handles):
        wl = q["workload"]
        got = h.result()
        alone = ml.ml_simulate_host(models[q["model_index"]], wl.n_traj, wl.x0, wl.T, wl.theta,
                                    params=p, seed=wl.seed, traj_id_base=wl.traj_id_base)
        for k in ("X", "r", "G", "counters"):
            assert np.array_equal(got[k], alone[k]), (wl.name, k)
        assert np.array_equal(got["status"], alone["status"].astype(np.uint32))
        assert got["latency_s"] >= got["queue_s"] >= 0
        h.free()
    srv.close()


def test_admission_respects_budget(ml, models):
    budget = 4 << 20
    srv = ml.ml_server(budget, 8, ml.ml_default_params(precision=1))
    w = W.config(1, n_traj=20_000)  # about 2.6 MB of device buffers each
    hs = [srv.submit(models[1], w.n_traj, w.x0, w.T, seed=s, traj_id_base=0) for s in range(6)]
    for h in hs:
        assert h.wait(120_000)
    st = srv.stats()
    assert st["peak_bytes"] <= budget and st["peak_inflight"] == 1 and st["completed"] == 6
    for h in hs:
        h.free()
    srv.close()


def test_oversized_request_and_timeout(ml, models):
    srv = ml.ml_server(2 << 20, 2, ml.ml_default_params(precision=1))
    w = W.config(1, n_traj=100_000)
    with pytest.raises(ml.MatleapError) as e:
        srv.submit(models[1], w.n_traj, w.x0, w.T)
    assert e.value.code == ml.ML_ERR_BUSY
    w = W.config(2, n_traj=5000)
    h = srv.submit(models[2], w.n_traj, w.x0, w.T, w.theta)
    assert h.wait(0) in (False, True)   # a zero timeout returns at once
    assert h.wait(300_000)
    assert h.result()["X"].shape == (5000, 3)
    h.free()
    srv.close()


def test_destroy_with_queued_requests(ml, models):
    srv = ml.ml_server(64 << 20, 1, ml.ml_default_params(precision=1))
    w = W.config(1, n_traj=50_000)
    hs = [srv.submit(models[1], w.n_traj, w.x0, w.T, seed=s) for s in range(4)]
    srv.close()                    # returns once the running request is done
    for h in hs:
        h.server.handle = None
        h.free()
