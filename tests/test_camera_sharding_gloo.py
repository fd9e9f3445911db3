"""Camera sharding of the normal equations (the multi-GPU layout: every rank holds the scene,
takes a subset of the cameras, and one sum-reduction of (G, b, w) precedes the per-Gaussian solve,
Eq. 12-14). Two gloo ranks on the CPU, each folding the FP64 oracle's sums of its own cameras, must
reproduce the single-process solution. No GPU is involved."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_2604_17155_gb300 import workloads as W


def _problem():
    sc = W.uniform_scene(60, 77, box=0.6, log_scale_mean=-2.6, log_scale_std=0.3)
    cams = W.hemisphere_cameras(10, 3.0, 40, 40, 50.0)
    t = np.random.default_rng(78).uniform(0, 1, (cams.n, 40, 40, 3))
    return sc, cams, t


def _rank_main(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc, cams, t = _problem()
        mine = np.arange(rank, cams.n, world)  # round-robin camera shard
        sub = cams.subset(mine)
        V, S, _, _, _ = O.accumulate(sc, sub, t[mine], threads=1)
        G, b, w = O.fold(V, S, O.view_basis(sc, sub, 3))
        parts = [torch.from_numpy(np.ascontiguousarray(x)) for x in (G, b, w)]
        for p in parts:
            dist.all_reduce(p, op=dist.ReduceOp.SUM)
        c, status, _ = O.solve(parts[0].numpy(), parts[1].numpy(), parts[2].numpy(), O.paper_lambda(3))
        if rank == 0:
            np.save(out_path, c)
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_rank_camera_shards_reproduce_single_process(tmp_path):
    out = str(tmp_path / "c.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    c_sharded = np.load(out)
    sc, cams, t = _problem()
    ref = O.colorize(sc, cams, t, 3)["c"]
    seen = np.abs(ref).reshape(ref.shape[0], -1).max(1) > 0
    assert seen.sum() > 30
    err = O.relative_errors(c_sharded[seen], ref[seen])
    assert err.max() < 1e-10


def _oracle_accumulate(sc, cams, t, L, lam, precision):
    V, S, _, _, _ = O.accumulate(sc, cams, t.numpy(), threads=1)
    G, b, w = O.fold(V, S, O.view_basis(sc, cams, L))
    return tuple(torch.from_numpy(np.ascontiguousarray(x)) for x in (G, b, w))


def _oracle_solve(G, b, w, L, lam, precision):
    c, status, _ = O.solve(G.numpy(), b.numpy(), w.numpy(), O.paper_lambda(L) if lam is None else np.asarray(lam))
    return c


def _rank_sharded(rank, world, port, out_path):
    """The library's colorize_sharded (camera partition, all-reduce of G, b, w, solve) with the
    oracle standing in for the GPU accumulate and solve."""
    from paper_2604_17155_gb300 import icgs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc, cams, t = _problem()
        c = icgs.colorize_sharded(sc, cams, torch.from_numpy(t), 3, rank, world,
                                  accumulate_fn=_oracle_accumulate, solve_fn=_oracle_solve)
        np.save(out_path.replace(".npy", f"_{rank}.npy"), c)
    finally:
        dist.destroy_process_group()


def test_colorize_sharded_host_logic_two_ranks(tmp_path):
    out = str(tmp_path / "c.npy")
    mp.start_processes(_rank_sharded, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    sc, cams, t = _problem()
    ref = O.colorize(sc, cams, t, 3)["c"]
    seen = np.abs(ref).reshape(ref.shape[0], -1).max(1) > 0
    for rank in range(2):
        c = np.load(out.replace(".npy", f"_{rank}.npy"))
        assert O.relative_errors(c[seen], ref[seen]).max() < 1e-10


def test_shard_partition_covers_every_camera_once():
    from paper_2604_17155_gb300 import icgs
    for n_cams, world in ((10, 2), (7, 3), (3, 4), (100, 8)):
        parts = [icgs.shard_cameras(n_cams, r, world) for r in range(world)]
        allc = np.sort(np.concatenate(parts))
        assert np.array_equal(allc, np.arange(n_cams))
