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


def test_shard_with_first_cluster_equals_whole_frame_subset():
    """A shard's rebased arrays estimated with first_cluster = c0 give the
    whole frame's results for clusters [c0, c1): the draws follow the frame
    index (reading G16 of the random minimal sets)."""
    w = synth.WORKLOADS["frame64"]
    f = synth.make_frame(w, n_clusters=40, gen_seed=19)
    sh = partition.rank_shard(f.azimuth, f.doppler, f.offsets, w.num_hypotheses, 1, 3)
    assert sh.c0 > 0 and sh.n_clusters > 0
    part = oracle.estimate(sh.azimuth, sh.doppler, sh.offsets, num_hypotheses=w.num_hypotheses, tau=w.tau,
                           seed=w.seed, first_cluster=sh.c0)
    whole = oracle.estimate(f.azimuth, f.doppler, f.offsets, num_hypotheses=w.num_hypotheses, tau=w.tau,
                            seed=w.seed, subset=np.arange(sh.c0, sh.c1))
    for k in part:
        a = part[k]
        b = whole[k] if k != "inlier_mask" else whole[k][sh.p0:sh.p1]
        assert np.array_equal(a, b, equal_nan=True), k
    # without the offset the draws differ
    plain = oracle.estimate(sh.azimuth, sh.doppler, sh.offsets, num_hypotheses=w.num_hypotheses, tau=w.tau,
                            seed=w.seed)
    assert not np.array_equal(plain["best_hypothesis"], part["best_hypothesis"])


def _rank_main_rank_shard(rank, world, port, out_path):
    """Each rank takes its shard with partition.rank_shard, as bench.py
    --strong does on the GPUs, and estimates it with first_cluster = c0."""
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w, n_clusters=96, gen_seed=23)
    sh = partition.rank_shard(f.azimuth, f.doppler, f.offsets, 256, rank, world)
    mine = oracle.estimate(sh.azimuth, sh.doppler, sh.offsets, num_hypotheses=256, tau=w.tau, seed=w.seed,
                           first_cluster=sh.c0)
    gathered = [None] * world
    dist.all_gather_object(gathered, (sh.c0, sh.c1, mine))
    if rank == 0:
        ranges = [(c0, c1) for c0, c1, _ in gathered]
        merged = partition.merge([m for _, _, m in gathered], ranges, f.offsets)
        whole = oracle.estimate(f.azimuth, f.doppler, f.offsets, num_hypotheses=256, tau=w.tau, seed=w.seed)
        ok = ranges[0][0] == 0 and ranges[-1][1] == f.n_clusters and \
            all(np.array_equal(merged[k], whole[k], equal_nan=True) for k in whole)
        with open(out_path, "w") as fh:
            fh.write("ok" if ok else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo_rank_shards_equal_whole(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    out = tmp_path / "result.txt"
    mp.spawn(_rank_main_rank_shard, args=(2, _free_port(), str(out)), nprocs=2, join=True)
    assert out.read_text() == "ok"

