"""Multi-rank sharding on CPU (gloo, 2 ranks).  Trajectories are independent and their
random numbers are keyed by the global trajectory id, so rank k simulating ids
[k B, (k+1) B) with traj_id_base = k B and gathering gives exactly the single-process
result; there is no exchange step on the data path."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, result_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_1608_07058_gb300 import workloads as W
    w = W.config(2, n_traj=n)
    B = n // world
    lo, hi = rank * B, (rank + 1) * B
    out = O.simulate(w.crn, B, w.x0, w.T[lo:hi], w.theta[lo:hi], seed=5, traj_id_base=lo)
    parts = [None] * world
    dist.all_gather_object(parts, {k: out[k] for k in ("X", "r", "G", "status")})
    if rank == 0:
        np.savez(result_path, **{k: np.concatenate([p[k] for p in parts]) for k in parts[0]})
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_concatenate_to_single_run(tmp_path, oracle):
    from paper_1608_07058_gb300 import workloads as W
    n, world = 64, 2
    path = str(tmp_path / "gathered.npz")
    mp.spawn(_worker, args=(world, _free_port(), n, path), nprocs=world, join=True)
    got = np.load(path)
    w = W.config(2, n_traj=n)
    ref = oracle.simulate(w.crn, n, w.x0, w.T, w.theta, seed=5)
    for k in ("X", "r", "status"):
        assert np.array_equal(got[k], ref[k]), k
    assert np.array_equal(got["G"], ref["G"])
