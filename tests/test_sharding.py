"""Multi-rank host logic on the CPU: world-size-2 gloo ranks shard frames
without overlap, regenerate the same frames a single process would, and
reduce time (max) and totals (sum) exactly."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1903_10107_gb300 import inputs, sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = inputs.WORKLOADS["n4096_r075_q02"]
        first, count = sharding.weak_shard(6, rank, world)
        xa, yb, q = w.frames(count, first)
        vmax, vsum = sharding.reduce_max_sum([1.0 + rank, 10.0 * rank], [float(count), float(xa.sum())], dist)
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), xa=xa, yb=yb, first=first, vmax=vmax, vsum=vsum)
    finally:
        dist.destroy_process_group()


def test_weak_and_strong_shards_cover_without_overlap():
    for world in (1, 2, 3, 8):
        spans = [sharding.strong_shard(1000, r, world) for r in range(world)]
        assert sum(c for _, c in spans) == 1000
        assert [f for f, _ in spans] == sorted(f for f, _ in spans)
        assert all(spans[i][0] + spans[i][1] == spans[i + 1][0] for i in range(world - 1))
        w = [sharding.weak_shard(7, r, world) for r in range(world)]
        assert w == [(7 * r, 7) for r in range(world)]


def test_two_gloo_ranks_shard_frames_and_reduce(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = np.load(tmp_path / "r0.npz")
    r1 = np.load(tmp_path / "r1.npz")
    w = inputs.WORKLOADS["n4096_r075_q02"]
    xa_all, yb_all, _ = w.frames(12, 0)   # what one process would draw for 12 frames
    assert np.array_equal(np.concatenate([r0["xa"], r1["xa"]]), xa_all)
    assert np.array_equal(np.concatenate([r0["yb"], r1["yb"]]), yb_all)
    for r in (r0, r1):
        assert np.array_equal(r["vmax"], [2.0, 10.0])
        assert r["vsum"][0] == 12 and r["vsum"][1] == float(xa_all.sum())
