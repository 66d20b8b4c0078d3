"""The random 50 x 100 network at its full horizon T = 10: about 1.8 M SSA firings and
4,000 implicit leaps (50 x 50 FP64 Newton systems, forward-difference Jacobian) per
trajectory.  32 trajectory ids in four blocks spread over the 65,536-trajectory batch run
through the warp kernel in reference precision and must be bit-identical to the oracle
(run in spawned host processes, which share nothing with this process's CUDA context)."""
import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_1608_07058_gb300 import workloads as W
from tests.test_gpu_parity import assert_bit_parity

pytestmark = pytest.mark.gpu

T_FULL = 10.0
MAX_STEPS = 10_000_000
BLOCKS = [0, 21840, 43680, 65528]   # first ids of four blocks of 8
PER_BLOCK = 8


def _oracle_one(task):
    tid, seed = task
    from oracle import oracle as O
    w = W.config(3, n_traj=1)
    out = O.simulate(w.crn, 1, w.x0, [T_FULL], None,
                     params=O.Params(max_steps=MAX_STEPS, jacobian=0), seed=seed,
                     traj_id_base=tid)
    return tid, out


@pytest.fixture(scope="module")
def ml():
    import torch
    from paper_1608_07058_gb300 import build, matleap
    assert torch.cuda.is_available()
    build.build()
    matleap.lib()
    return matleap


def test_random_crn_full_horizon_sampled_ids_bit_exact(ml):
    import torch
    seed = 17
    ids = [b + k for b in BLOCKS for k in range(PER_BLOCK)]
    pool = mp.get_context("spawn").Pool(min(len(ids), os.cpu_count() or 1))
    pending = pool.map_async(_oracle_one, [(i, seed) for i in ids])
    w = W.config(3, n_traj=1)
    model = ml.model_from_crn(w.crn)
    d = torch.device("cuda")
    x0 = torch.as_tensor(w.x0, device=d)
    T = torch.tensor([T_FULL], dtype=torch.float64, device=d)
    p = ml.ml_default_params(precision=ml.ML_PREC_REF_FP64, shape=ml.ML_SHAPE_WARP,
                             jacobian=ml.ML_JAC_FD, max_steps=MAX_STEPS)
    gpu = {}
    for b in BLOCKS:
        out = ml.ml_simulate(model, PER_BLOCK, x0, T, params=p, seed=seed, traj_id_base=b)
        torch.cuda.synchronize()
        for k in range(PER_BLOCK):
            gpu[b + k] = {key: v[k:k + 1].cpu().numpy() for key, v in out.items()}
    ref = dict(pending.get(timeout=3000))
    pool.close()
    pool.join()
    for i in ids:
        g = gpu[i]
        g["status"] = g["status"].astype(np.uint32)
        assert_bit_parity(g, ref[i], f"id {i}")
    c = np.concatenate([gpu[i]["counters"] for i in ids])
    assert (c[:, 1] > 1000).all() and (c[:, 2] > 500_000).all()
