"""Sharding a frame by contiguous cluster ranges (host side, no GPU).

Each shard is estimated with its clusters' original indices (the oracle's
subset mode; rvh's first_cluster), so the shards' merged results equal the
whole frame's.  The two-rank test exchanges shard results over gloo."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2012_12618_gb300 import partition, synth


def test_balanced_ranges_cover_and_balance():
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w, n_clusters=1000, gen_seed=13)
    for parts in (1, 2, 3, 7, 16):
        r = partition.balanced_ranges(f.offsets, w.num_hypotheses, parts)
        assert r[0][0] == 0 and r[-1][1] == f.n_clusters
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        cost = np.diff(f.offsets).astype(np.int64) * w.num_hypotheses + partition.CLUSTER_OVERHEAD
        loads = [cost[c0:c1].sum() for c0, c1 in r]
        assert max(loads) <= cost.sum() / parts + cost.max()
    assert partition.balanced_ranges(np.array([0], np.int32), 8, 4) == [(0, 0)] * 4


def test_shard_slices_and_rebases():
    off = np.array([0, 3, 3, 7, 12], np.int32)
    az = np.arange(12, dtype=np.float32)
    a, d, o, e, (p0, p1) = partition.shard(az, az * 2, off, 1, 3)
    assert (p0, p1) == (3, 7) and list(o) == [0, 0, 4] and list(a) == [3, 4, 5, 6] and e is None


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w = synth.WORKLOADS["frame64"]
    f = synth.make_frame(w, n_clusters=48, gen_seed=17)
    ranges = partition.balanced_ranges(f.offsets, w.num_hypotheses, world)
    c0, c1 = ranges[rank]
    mine = oracle.estimate(f.azimuth, f.doppler, f.offsets, num_hypotheses=w.num_hypotheses, tau=w.tau,
                           seed=w.seed, subset=np.arange(c0, c1))
    p0, p1 = int(f.offsets[c0]), int(f.offsets[c1])
    mine["inlier_mask"] = mine["inlier_mask"][p0:p1]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        merged = partition.merge(gathered, ranges, f.offsets)
        whole = oracle.estimate(f.azimuth, f.doppler, f.offsets, num_hypotheses=w.num_hypotheses, tau=w.tau,
                                seed=w.seed)
        ok = all(np.array_equal(merged[k], whole[k], equal_nan=True) for k in whole)
        with open(out_path, "w") as fh:
            fh.write("ok" if ok else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo_merge_equals_whole(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    out = tmp_path / "result.txt"
    mp.spawn(_rank_main, args=(2, _free_port(), str(out)), nprocs=2, join=True)
    assert out.read_text() == "ok"
