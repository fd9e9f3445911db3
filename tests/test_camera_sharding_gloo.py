"""Camera sharding of the normal equations (the multi-GPU layout: every rank holds the scene,
takes a subset of the cameras, and one sum-reduction of the packed (G, b, w) precedes the
per-Gaussian solve, Eq. 12-14). Two or three gloo ranks on the CPU, each folding the FP64 oracle's
sums of its own cameras, must reproduce the single-process solution: an all-reduce of the full
sums, and the library's colorize_sharded (reduce-scatter over Gaussian ranges, a solve per range,
an all-gather of the coefficients). No GPU is involved."""
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


def _pack(G, b, w):
    """The library's packed layout of the normal equations (icgs_normal_size): the upper triangle
    of G row by row, then b [B,K] row-major, then w."""
    B = G.shape[1]
    r, c = np.triu_indices(B)
    return np.concatenate([G[:, r, c], b.reshape(len(w), -1), w[:, None]], axis=1)


def _unpack(sums, L):
    B = (L + 1) ** 2
    P = B * (B + 1) // 2
    n = sums.shape[0]
    K = (sums.shape[1] - P - 1) // B
    G = np.zeros((n, B, B))
    r, c = np.triu_indices(B)
    G[:, r, c] = sums[:, :P]
    G[:, c, r] = sums[:, :P]
    return G, sums[:, P:P + B * K].reshape(n, B, K), sums[:, -1]


def _oracle_accumulate(sc, cams, t, L, lam, precision):
    V, S, _, _, _ = O.accumulate(sc, cams, t.numpy(), threads=1)
    G, b, w = O.fold(V, S, O.view_basis(sc, cams, L))
    return torch.from_numpy(np.ascontiguousarray(_pack(G, b, w)))


def _oracle_solve(sums, L, lam, precision):
    G, b, w = _unpack(sums.numpy(), L)
    c, status, _ = O.solve(G, b, w, O.paper_lambda(L) if lam is None else np.asarray(lam))
    return torch.from_numpy(c), torch.from_numpy(status), None


def _rank_sharded(rank, world, port, out_path, gather):
    """The library's colorize_sharded (camera partition, reduce-scatter of the packed sums over
    Gaussian ranges, a solve per range, optional all-gather) with the oracle standing in for the
    GPU accumulate and solve."""
    from paper_2604_17155_gb300 import icgs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc, cams, t = _problem()
        out = icgs.colorize_sharded(sc, cams, torch.from_numpy(t), 3, rank, world, gather=gather,
                                    accumulate_fn=_oracle_accumulate, solve_fn=_oracle_solve)
        np.save(out_path.replace(".npy", f"_{rank}.npy"), out["coeffs"].numpy())
        np.save(out_path.replace(".npy", f"_{rank}_range.npy"), np.array(out["range"]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,gather", [(2, True), (3, False)])
def test_colorize_sharded_host_logic(tmp_path, world, gather):
    """60 Gaussians over 2 ranks (ranges of 30) or 3 ranks (20 each): every rank solves its own
    range; with the all-gather every rank holds every coefficient."""
    out = str(tmp_path / "c.npy")
    mp.start_processes(_rank_sharded, args=(world, _free_port(), out, gather), nprocs=world, join=True,
                       start_method="spawn")
    sc, cams, t = _problem()
    ref = O.colorize(sc, cams, t, 3)["c"]
    seen = np.abs(ref).reshape(ref.shape[0], -1).max(1) > 0
    covered = np.zeros(sc.n, bool)
    for rank in range(world):
        c = np.load(out.replace(".npy", f"_{rank}.npy"))
        lo, hi = np.load(out.replace(".npy", f"_{rank}_range.npy"))
        covered[lo:hi] = True
        if gather:
            assert c.shape[0] == sc.n
            assert O.relative_errors(c[seen], ref[seen]).max() < 1e-10
        else:
            assert c.shape[0] == hi - lo
            sl = seen[lo:hi]
            assert O.relative_errors(c[sl], ref[lo:hi][sl]).max() < 1e-10
    assert covered.all()


def test_packed_layout_round_trip():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((7, 9, 9))
    G = A + np.transpose(A, (0, 2, 1))
    b = rng.standard_normal((7, 9, 4))
    w = rng.uniform(1, 2, 7)
    G2, b2, w2 = _unpack(_pack(G, b, w), 2)
    assert np.array_equal(G2, G) and np.array_equal(b2, b) and np.array_equal(w2, w)


def test_shard_partition_covers_every_camera_and_gaussian_once():
    from paper_2604_17155_gb300 import icgs
    for n_cams, world in ((10, 2), (7, 3), (3, 4), (100, 8)):
        parts = [icgs.shard_cameras(n_cams, r, world) for r in range(world)]
        allc = np.sort(np.concatenate(parts))
        assert np.array_equal(allc, np.arange(n_cams))
    for n, world in ((60, 2), (61, 3), (5, 8), (200000, 8)):
        ranges = [icgs.shard_gaussians(n, r, world) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        assert all(ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))
