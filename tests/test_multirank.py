"""The N > 1 path on the host with world-size-2 ``gloo`` process groups.

The path shards by rays (every ray is independent from sampling to the
grid adjoint); the only cross-rank quantities are the parameter and grid
gradients, whose sum over ray shards must equal the gradient of the whole
batch, and the benchmark's whole-job timing (max over ranks, samples summed
over ranks).  Both are checked here with 2 CPU ranks, the first with the
FP64 oracle (spawned processes)."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

N_RAYS = 48


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _scene():
    from paper_2206_05085_gb300 import synth
    cfg = synth.CFG1
    rp = synth.render_params(cfg)
    o, d = synth.rays(cfg, seed=3, n_rays=N_RAYS)
    t = synth.target_rgb(cfg, seed=3, n_rays=N_RAYS)
    return cfg, rp, synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params(), o, d, t


def _flat(fb):
    return np.concatenate([fb["g_params"].ravel(), fb["g_density"].ravel(), fb["g_feature"].ravel(),
                           [fb["loss"][2]]])


def _shard_worker(rank, world, port, out):
    import oracle_step
    _init(rank, world, port)
    cfg, rp, D, F, P, o, d, t = _scene()
    per = N_RAYS // world
    sl = slice(rank * per, (rank + 1) * per)
    fb = oracle_step.forward_backward(cfg, rp, D, F, P, o[sl], d[sl], t[sl])
    # this shard's gradient with the whole batch's 1/R normalisation
    g = torch.from_numpy(_flat(fb) * (per / N_RAYS))
    dist.all_reduce(g)
    if rank == 0:
        np.save(out, g.numpy())
    dist.destroy_process_group()


def test_ray_sharded_gradients_sum_to_the_full_batch(orc):
    import oracle_step
    cfg, rp, D, F, P, o, d, t = _scene()
    ref = _flat(oracle_step.forward_backward(cfg, rp, D, F, P, o, d, t))
    with tempfile.TemporaryDirectory() as tmp:
        out = os.path.join(tmp, "sharded.npy")
        mp.spawn(_shard_worker, args=(2, _free_port(), out), nprocs=2, join=True)
        got = np.load(out)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def _reduce_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    _init(rank, world, port)
    res = bench.reduce_over_ranks(10.0 + rank, 20.0 - rank, 100.0 * (rank + 1), "cpu")
    if rank == 0:
        np.save(out, np.array(res))
    dist.destroy_process_group()


def test_bench_whole_job_figures_over_two_ranks():
    with tempfile.TemporaryDirectory() as tmp:
        out = os.path.join(tmp, "res.npy")
        mp.spawn(_reduce_worker, args=(2, _free_port(), out), nprocs=2, join=True)
        total_ms, e2e_ms, samples = np.load(out)
    assert (total_ms, e2e_ms, samples) == (11.0, 20.0, 300.0)


def test_bench_figures_unchanged_without_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(3.0, 4.0, 5.0, "cpu") == (3.0, 4.0, 5.0)
