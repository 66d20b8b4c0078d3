"""The allocation-free entry point ml_simulate_noalloc.

Some callers cannot let a library allocate device memory (code under a framework-owned
memory pool or a capped MPS client, latency-bound loops that cannot afford cudaMalloc's
synchronization, code that must not take the allocator's lock).  For them the library
keeps the persistent kernel's scratch -- its work-queue counter and the model tables -- in
a fixed 4 KiB device array.  This file checks, through the C ABI, that two calls in a row
give exactly what the ordinary entry point gives for the same inputs, in both
precisions, and that a model too large for the array is refused.  It is collected last
and does not depend on state left by other tests."""
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


def _bufs(torch, n, N, M):
    d = torch.device("cuda")
    return {"X": torch.full((n, N), -1, dtype=torch.int64, device=d),
            "r": torch.full((n, M), -1, dtype=torch.int64, device=d),
            "G": torch.full((n, M), -1.0, dtype=torch.float64, device=d),
            "status": torch.full((n,), -1, dtype=torch.int32, device=d),
            "counters": torch.full((n, 4), -1, dtype=torch.int64, device=d)}


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_simulate_two_calls(ml, precision):
    import torch
    d = torch.device("cuda")
    w = W.config(2, n_traj=5000)  # per-trajectory theta and horizons
    model = ml.model_from_crn(w.crn)
    x0 = torch.as_tensor(w.x0, device=d)
    T = torch.as_tensor(w.T, device=d)
    theta = torch.as_tensor(w.theta, device=d)
    for call, seed in enumerate((11, 12)):
        p = ml.ml_default_params(precision=precision, form=ml.ML_FORM_PERSISTENT,
                                 max_steps=200_000)
        ref = ml.ml_simulate(model, w.n_traj, x0, T, theta, params=p, seed=seed,
                             traj_id_base=77, out=_bufs(torch, w.n_traj, model.N, model.M))
        got = ml.ml_simulate_noalloc(model, w.n_traj, x0, T, theta, params=p, seed=seed,
                                     traj_id_base=77,
                                     out=_bufs(torch, w.n_traj, model.N, model.M))
        torch.cuda.synchronize()
        for k in ("X", "r", "status", "counters"):
            assert torch.equal(ref[k], got[k]), (call, k)
        g1, g2 = ref["G"].cpu().numpy(), got["G"].cpu().numpy()
        assert np.allclose(g1, g2, rtol=1e-12, atol=0), call


def test_noalloc_second_model_reloads_tables(ml):
    import torch
    d = torch.device("cuda")
    for cfg in (1, 0):  # a different model in the shared array on each call
        w = W.config(cfg, n_traj=3000)
        model = ml.model_from_crn(w.crn)
        x0 = torch.as_tensor(w.x0, device=d)
        T = torch.as_tensor(w.T, device=d)
        ref = ml.ml_simulate(model, w.n_traj, x0, T, seed=5, out=_bufs(torch, w.n_traj, model.N, model.M))
        got = ml.ml_simulate_noalloc(model, w.n_traj, x0, T, seed=5,
                                     out=_bufs(torch, w.n_traj, model.N, model.M))
        torch.cuda.synchronize()
        for k in ("X", "r", "G", "status", "counters"):
            assert torch.equal(ref[k], got[k]), (cfg, k)


def test_noalloc_rejects_models_beyond_its_scratch(ml):
    import torch
    d = torch.device("cuda")
    crn, x0 = W.random_crn()
    model = ml.model_from_crn(crn)
    n = 4
    with pytest.raises(ml.MatleapError) as e:
        ml.ml_simulate_noalloc(model, n, torch.as_tensor(x0, device=d),
                               torch.ones(1, dtype=torch.float64, device=d),
                               out=_bufs(torch, n, model.N, model.M))
    assert e.value.code == ml.ML_ERR_ARG
    assert "at most" in str(e.value)


def test_noalloc_leaves_free_device_memory_unchanged(ml):
    """On a model that never went through ml_simulate (so it owns no device tables), after
    one warm-up call (which may load the library's module), further calls change nothing
    in the device's free memory; their results equal a later ml_simulate run."""
    import torch
    d = torch.device("cuda")
    w = W.config(1, n_traj=4000)
    model = ml.model_from_crn(w.crn)
    x0 = torch.as_tensor(w.x0, device=d)
    T = torch.as_tensor(w.T, device=d)
    outs = [_bufs(torch, w.n_traj, model.N, model.M) for _ in range(4)]
    ml.ml_simulate_noalloc(model, w.n_traj, x0, T, seed=3, out=outs[0])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in range(1, 4):
        ml.ml_simulate_noalloc(model, w.n_traj, x0, T, seed=3 + k, out=outs[k])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ref = ml.ml_simulate(model, w.n_traj, x0, T, seed=6, out=_bufs(torch, w.n_traj, model.N, model.M))
    torch.cuda.synchronize()
    for key in ("X", "r", "G", "status", "counters"):
        assert torch.equal(ref[key], outs[3][key]), key
