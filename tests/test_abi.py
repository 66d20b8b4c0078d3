"""Host-side checks of the C ABI (no GPU needed): the library loads and exports every
function include/matleap.h declares; model creation validates its input and finds the
reversible pairs; a simulate call without a usable device fails with an error code."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1608_07058_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ml():
    from paper_1608_07058_gb300 import build, matleap
    build.build()
    matleap.lib()
    return matleap


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ml_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(ml):
    declared = _declared()
    assert {"ml_model_create", "ml_simulate", "ml_simulate_host"} <= declared
    L = C.CDLL(ml.LIB_PATH)
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing


def test_default_params(ml):
    p = ml.ml_default_params()
    assert p.eps == 0.03 and p.n_c == 10 and p.ssa_factor == 10.0
    assert p.mode == ml.ML_MODE_ADAPTIVE and p.precision == ml.ML_PREC_REF_FP64


@pytest.mark.parametrize("cfg,pairs", [(0, 0), (1, 1), (2, 0)])
def test_pairs_found(ml, cfg, pairs):
    crn = W.config(cfg, n_traj=1).crn
    m = ml.model_from_crn(crn)
    assert ml.ml_model_num_pairs(m) == pairs


def test_random_crn_pairs(ml):
    crn, _ = W.random_crn()
    assert ml.ml_model_num_pairs(ml.model_from_crn(crn)) >= 10


@pytest.mark.parametrize("bad", ["neg_order", "order4", "overconsume", "neg_rate", "nan_rate", "dims"])
def test_model_validation(ml, bad):
    o = np.array([[1, 0], [0, 1]], np.int32)
    s = np.array([[-1, 1], [1, -1]], np.int32)
    r = np.array([1.0, 2.0])
    if bad == "neg_order":
        o[0, 0] = -1
    elif bad == "order4":
        o[0, 0] = 4
        s[0, 0] = -4
    elif bad == "overconsume":
        s[0, 0] = -2
    elif bad == "neg_rate":
        r[1] = -1.0
    elif bad == "nan_rate":
        r[0] = np.nan
    elif bad == "dims":
        o = np.zeros((200, 2), np.int32)
        s = np.zeros((200, 2), np.int32)
        r = np.ones(200)
    with pytest.raises(ml.MatleapError) as e:
        ml.ml_model_create(o, s, r)
    assert e.value.code == ml.ML_ERR_ARG


def test_simulate_rejects_host_pointers(ml):
    import torch
    crn = W.immigration_death()
    m = ml.model_from_crn(crn)
    x0 = torch.zeros(1, dtype=torch.int64)
    T = torch.ones(1, dtype=torch.float64)
    out = {"X": torch.empty((4, 1), dtype=torch.int64), "r": torch.empty((4, 2), dtype=torch.int64),
           "G": torch.empty((4, 2), dtype=torch.float64), "status": torch.empty(4, dtype=torch.int32)}
    with pytest.raises(ml.MatleapError) as e:
        ml.ml_simulate(m, 4, x0, T, out=out)
    assert e.value.code in (ml.ML_ERR_ARG, ml.ML_ERR_CUDA)


def test_simulate_rejects_bad_params(ml):
    import torch
    m = ml.model_from_crn(W.immigration_death())
    x0 = torch.zeros(1, dtype=torch.int64)
    T = torch.ones(1, dtype=torch.float64)
    for kw in ({"eps": 0.0}, {"eps": 1.5}, {"n_ssa_explicit": 0}, {"mode": 7}, {"precision": 3},
               {"block_size": 48}, {"newton_maxit": 0}, {"specialize": 2},
               {"shape": ml.ML_SHAPE_THREAD_POOL},  # the pool driver needs the persistent form
               {"shape": ml.ML_SHAPE_THREAD_POOL_OCC, "form": ml.ML_FORM_PERSISTENT},  # fast only
               {"shape": 8}):
        with pytest.raises(ml.MatleapError) as e:
            ml.ml_simulate(m, 4, x0, T, params=ml.ml_default_params(**kw))
        assert e.value.code == ml.ML_ERR_ARG


def test_trajectory_id_range(ml):
    import torch
    m = ml.model_from_crn(W.immigration_death())
    x0 = torch.zeros(1, dtype=torch.int64)
    T = torch.ones(1, dtype=torch.float64)
    with pytest.raises(ml.MatleapError) as e:
        ml.ml_simulate(m, 10, x0, T, traj_id_base=2**32 - 5)
    assert e.value.code == ml.ML_ERR_ARG


def test_server_without_device_fails_cleanly(ml):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(ml.MatleapError) as e:
        ml.ml_server(16 << 20, 2)
    assert e.value.code in (ml.ML_ERR_CUDA, ml.ML_ERR_OOM)


def test_bayes_argument_errors_without_device(ml):
    """The Bayesian-step entry points validate sizes on the host before any launch."""
    L = ml.lib()
    assert L.ml_resample_workspace_bytes(0) == 0
    assert L.ml_resample_workspace_bytes(5000) >= 8 * 5000
    assert L.ml_resample_systematic(0, None, 0, 0, None, None, 0, None) == ml.ML_ERR_ARG
    assert L.ml_resample_systematic(1 << 24, None, 0, 0, None, None, 0, None) == ml.ML_ERR_ARG
    assert L.ml_posterior_sample(4, 0, None, 0, None, 0, None, None, 0, 0, None, None,
                                 None) == ml.ML_ERR_ARG
    assert L.ml_posterior_sample(0, 3, None, 0, None, 0, None, None, 0, 0, None, None,
                                 None) == ml.ML_OK  # empty batch: no-op
    assert L.ml_posterior_sample(4, 3, None, 0, None, 0, None, None, 0, 2**32 - 2, None, None,
                                 None) == ml.ML_ERR_ARG
    # host pointers where device memory is required
    a = np.ones(12)
    p = a.ctypes.data
    assert L.ml_posterior_sample(4, 3, p, 0, p, 0, p, p, 0, 0, p, None, None) == ml.ML_ERR_ARG
    assert "device memory" in ml.ml_last_error()


def test_grid_kl_and_peaks_argument_errors_without_device(ml):
    """The time-grid, KL and pipe-peak entry points reject malformed arguments on the host
    before touching a device."""
    import ctypes as C
    L = ml.lib()
    m = ml.model_from_crn(W.config(0, n_traj=1).crn)
    p = ml.ml_default_params()
    args = lambda K, tobs, xobs: (C.c_void_p(m.handle), 4, None, None, 0, None, 0, C.byref(p),
                                  0, 0, tobs, K, xobs, None, None, None, None, None, None)
    assert L.ml_simulate_grid(*args(-1, None, None)) == ml.ML_ERR_ARG
    assert L.ml_simulate_grid(*args(3, None, None)) == ml.ML_ERR_ARG      # K > 0, no grid
    host = np.zeros(8)
    assert L.ml_simulate_grid(*args(3, host.ctypes.data, host.ctypes.data)) == ml.ML_ERR_ARG
    assert "device memory" in ml.ml_last_error()
    kl = lambda n1, n2, K, N, b: L.ml_kl_divergence(n1, None, n2, None, K, N, b, None, None, None)
    assert kl(0, 5, 1, 1, 16) == ml.ML_ERR_ARG
    assert kl(5, 5, 0, 1, 16) == ml.ML_ERR_ARG
    assert kl(5, 5, 1, 1, 0) == ml.ML_ERR_ARG and kl(5, 5, 1, 1, 4097) == ml.ML_ERR_ARG
    assert kl(5, 5, 1, 1, 16) == ml.ML_ERR_ARG                          # NULL buffers
    assert L.ml_measure_pipe_peaks(None, None) == ml.ML_ERR_ARG
