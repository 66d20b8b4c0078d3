"""Multi-rank sharding on CPU (gloo, 2 ranks).  Trajectories are independent and their
random numbers are keyed by the global trajectory id, so rank k simulating ids
[k B, (k+1) B) with traj_id_base = k B and gathering gives exactly the single-process
result; there is no exchange step on the data path.  The same holds for the time-grid
output and the posterior draws.  (Resampling is the one global step: its weights span all
particles, so it runs on the gathered log-weights.)"""
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


def _worker_grid_bayes(rank, world, port, n, result_path):
    """Each rank: simulate its id range with a time grid, draw the posterior of its
    trajectories; gather X_obs and theta."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_1608_07058_gb300 import workloads as W
    w = W.config(1, n_traj=n)
    B = n // world
    lo = rank * B
    t_obs = [0.0, 0.05, 0.1, 0.2]
    out = O.simulate(w.crn, B, w.x0, w.T, None, seed=6, traj_id_base=lo, t_obs=t_obs)
    alpha = np.full(w.crn.n_reactions, 2.0)
    beta = np.full(w.crn.n_reactions, 0.5)
    theta, st = O.posterior_sample(alpha, beta, out["r"], out["G"], seed=7, traj_id_base=lo)
    parts = [None] * world
    dist.all_gather_object(parts, {"X_obs": out["X_obs"], "theta": theta, "st": st})
    if rank == 0:
        np.savez(result_path, **{k: np.concatenate([p[k] for p in parts]) for k in parts[0]})
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_grid_and_posterior_shards(tmp_path, oracle):
    """Time-grid output and posterior draws are keyed by the global trajectory id too, so
    the gathered shards equal one run over all ids."""
    from paper_1608_07058_gb300 import workloads as W
    n, world = 48, 2
    path = str(tmp_path / "gathered_grid.npz")
    mp.spawn(_worker_grid_bayes, args=(world, _free_port(), n, path), nprocs=world, join=True)
    got = np.load(path)
    w = W.config(1, n_traj=n)
    ref = oracle.simulate(w.crn, n, w.x0, w.T, None, seed=6, t_obs=[0.0, 0.05, 0.1, 0.2])
    theta, st = oracle.posterior_sample(np.full(4, 2.0), np.full(4, 0.5), ref["r"], ref["G"],
                                        seed=7)
    assert np.array_equal(got["X_obs"], ref["X_obs"])
    assert np.array_equal(got["theta"], theta) and np.array_equal(got["st"], st)


def _worker_uneven(rank, world, port, n, result_path):
    """The package's partition (matleap.shard_bounds, uneven sizes) with the oracle as the
    simulator on each rank."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_1608_07058_gb300 import workloads as W
    from paper_1608_07058_gb300.matleap import shard_bounds
    w = W.config(2, n_traj=n)
    lo, hi = shard_bounds(n, rank, world)
    out = O.simulate(w.crn, hi - lo, w.x0, w.T[lo:hi], w.theta[lo:hi], seed=9, traj_id_base=lo)
    parts = [None] * world
    dist.all_gather_object(parts, {k: out[k] for k in ("X", "r", "G", "status")})
    if rank == 0:
        np.savez(result_path, **{k: np.concatenate([p[k] for p in parts]) for k in parts[0]})
    dist.barrier()
    dist.destroy_process_group()


def test_shard_bounds_partition():
    from paper_1608_07058_gb300.matleap import shard_bounds
    for n in (0, 1, 5, 64, 67, 1000):
        for world in (1, 2, 3, 7):
            rng = [shard_bounds(n, k, world) for k in range(world)]
            assert rng[0][0] == 0 and rng[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rng, rng[1:]))
            sizes = [hi - lo for lo, hi in rng]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_bounds(10, 2, 2)


def test_three_rank_uneven_shards_concatenate_to_single_run(tmp_path, oracle):
    from paper_1608_07058_gb300 import workloads as W
    n, world = 67, 3
    path = str(tmp_path / "gathered_uneven.npz")
    mp.spawn(_worker_uneven, args=(world, _free_port(), n, path), nprocs=world, join=True)
    got = np.load(path)
    w = W.config(2, n_traj=n)
    ref = oracle.simulate(w.crn, n, w.x0, w.T, w.theta, seed=9)
    for k in ("X", "r", "G", "status"):
        assert np.array_equal(got[k], ref[k]), k
