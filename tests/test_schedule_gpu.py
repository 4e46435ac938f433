"""Autotuner, CUDA-graph replay and the direct (no work list) launch (GPU).

Whatever the schedule, the launch form or the replay, results stay those of
the oracle (every schedule computes the same exact counts)."""
import ctypes
import os

import numpy as np
import pytest

from paper_2012_12618_gb300 import rvh, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _device_frame(torch, f):
    dev = torch.device("cuda", 0)
    t = [None if x is None else torch.from_numpy(x).to(dev) for x in (f.azimuth, f.elevation, f.doppler, f.offsets)]
    return t, rvh.make_frame(t[0], t[2], t[3], t[1])


def _np(outs, n):
    d = {k: v.cpu().numpy() for k, v in outs.items()}
    d["inlier_mask"] = d["inlier_mask"][:n]
    return d


def test_autotune_and_cache(torch, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("RVH_TUNE_CACHE", str(cache))
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w, n_clusters=256, gen_seed=61)
    keep, frame = _device_frame(torch, f)
    params = rvh.make_params(2, 1024, w.tau, 3)
    dev = torch.device("cuda", 0)
    outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
    ctx = rvh.Context(0)
    try:
        best = rvh.rvh_schedule()
        ctx.check(rvh.rvh_autotune(ctx.handle, frame, params, rvh.make_result(outs), 2, best), "autotune")
        assert best.points_per_warp in (1, 8, 32) and best.hyps_per_lane in (4, 8) and best.kernel_ms > 0
        ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, rvh.make_result(outs), None), "estimate")
        torch.cuda.synchronize()
        st = rvh.rvh_stats()
        ctx.check(rvh.rvh_get_stats(ctx.handle, st), "stats")
        assert (st.points_per_warp, st.hyps_per_lane) == (best.points_per_warp, best.hyps_per_lane)
        g = _np(outs, f.n_points)
    finally:
        ctx.close()
    o = G.run_oracle(f.azimuth, f.doppler, f.offsets, H=1024, tau=w.tau, seed=3)
    rep = G.compare(g, o, f.offsets)
    assert not rep["mismatch"], rep["mismatch"][:10]
    text = cache.read_text()
    assert f"|2|10 {best.points_per_warp} {best.hyps_per_lane} " in text
    # a new context picks the cached choice up
    ctx2 = rvh.Context(0)
    try:
        ctx2.check(rvh.rvh_estimate(ctx2.handle, frame, params, rvh.make_result(outs), None), "estimate")
        st = rvh.rvh_stats()
        ctx2.check(rvh.rvh_get_stats(ctx2.handle, st), "stats")
        assert (st.points_per_warp, st.hyps_per_lane) == (best.points_per_warp, best.hyps_per_lane)
    finally:
        ctx2.close()


def test_graph_replay_with_rotating_buffers(torch):
    """A pipeline that rotates its input and output buffers: four frames of
    different sizes (one needs the work list, three do not), each in buffers
    of its own, go through rvh_estimate three times over.  The first call
    builds the graph of the 2D launch and every later call replays it with
    the new addresses and sizes; a 3D frame builds the 3D graph once.  Every
    result equals the oracle's."""
    dev = torch.device("cuda", 0)
    w = synth.WORKLOADS["dense2d"]
    frames = [synth.make_frame(w, n_clusters=nc, gen_seed=90 + k) for k, nc in enumerate((100, 900, 37, 300))]
    bufs = []
    for k, f in enumerate(frames):
        keep, frame = _device_frame(torch, f)
        outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
        bufs.append((keep, frame, outs, rvh.make_params(2, 512, w.tau, 20 + k)))
    s = torch.cuda.Stream(dev)
    sptr = ctypes.c_void_p(s.cuda_stream)
    torch.cuda.synchronize()
    ctx = rvh.Context(0)
    try:
        st = rvh.rvh_stats()
        calls = 0
        for rnd in range(3):
            if rnd == 2:  # the last round must rewrite every output
                s.synchronize()
                for _, _, outs, _ in bufs:
                    for v in outs.values():
                        v.zero_()
                torch.cuda.synchronize()
            for k, (keep, frame, outs, params) in enumerate(bufs):
                ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, rvh.make_result(outs), sptr), "estimate")
                calls += 1
        s.synchronize()
        ctx.check(rvh.rvh_get_stats(ctx.handle, st), "stats")
        assert st.graph_builds == 1 and st.graph_replays == calls - 1, (st.graph_builds, st.graph_replays, calls)
        got = [_np(outs, f.n_points) for f, (_, _, outs, _) in zip(frames, bufs)]
        # a 3D frame: one more graph, then replays again
        w3 = synth.WORKLOADS["dense3d"]
        f3 = synth.make_frame(w3, n_clusters=64, gen_seed=99)
        keep3, frame3 = _device_frame(torch, f3)
        outs3 = rvh.alloc_outputs(f3.n_clusters, f3.n_points, dev)
        p3 = rvh.make_params(3, 256, w3.tau, 7)
        for _ in range(2):
            ctx.check(rvh.rvh_estimate(ctx.handle, frame3, p3, rvh.make_result(outs3), sptr), "estimate 3D")
        s.synchronize()
        ctx.check(rvh.rvh_get_stats(ctx.handle, st), "stats")
        assert st.graph_builds == 2 and st.graph_replays == calls, (st.graph_builds, st.graph_replays)
        g3 = _np(outs3, f3.n_points)
    finally:
        ctx.close()
    for k, (f, g) in enumerate(zip(frames, got)):
        o = G.run_oracle(f.azimuth, f.doppler, f.offsets, H=512, tau=w.tau, seed=20 + k)
        G.check_parity(G.compare(g, o, f.offsets), tau=w.tau, label=f"rotating buffers, frame {k}")
    o3 = G.run_oracle(f3.azimuth, f3.doppler, f3.offsets, el=f3.elevation, H=256, tau=w3.tau, seed=7)
    G.check_parity(G.compare(g3, o3, f3.offsets), tau=w3.tau, label="rotating buffers, 3D frame")


@pytest.mark.parametrize("name", ["dense2d", "dense3d"])
def test_shards_equal_whole(torch, name):
    """Contiguous cluster ranges estimated separately with first_cluster give
    exactly the whole frame's results (the multi-GPU sharding rule)."""
    from paper_2012_12618_gb300 import partition
    w = synth.WORKLOADS[name]
    f = synth.make_frame(w, n_clusters=300, gen_seed=71)
    H = 512
    dev = torch.device("cuda", 0)

    def run(az, dop, off, el, first):
        t = [None if x is None else torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (az, el, dop, off)]
        frame = rvh.make_frame(t[0], t[2], t[3], t[1])
        params = rvh.make_params(w.model_dim, H, w.tau, 4, first_cluster=first)
        outs = rvh.alloc_outputs(off.shape[0] - 1, az.shape[0], dev)
        ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, rvh.make_result(outs), None), "estimate")
        torch.cuda.synchronize()
        return _np(outs, az.shape[0])

    ctx = rvh.Context(0)
    try:
        whole = run(f.azimuth, f.doppler, f.offsets, f.elevation, 0)
        ranges = partition.balanced_ranges(f.offsets, H, 3)
        parts = []
        for c0, c1 in ranges:
            az, dop, off, el, _ = partition.shard(f.azimuth, f.doppler, f.offsets, c0, c1, f.elevation)
            parts.append(run(az, dop, off, el, c0))
    finally:
        ctx.close()
    merged = partition.merge(parts, ranges, f.offsets)
    for k in whole:
        assert np.array_equal(merged[k], whole[k], equal_nan=True), k


@pytest.mark.parametrize("dim", [2, 3])
def test_every_schedule_same_result(torch, dim):
    """Both scoring passes (tiled shared-memory rows, float4 global rows) under
    every schedule: cluster sizes 2..2600 cover ragged quads (N mod 4 != 0),
    single tiles and clusters above the shared-memory capacity."""
    w = synth.WORKLOADS["dense2d" if dim == 2 else "dense3d"]
    sizes = np.array([2, 3, 5, 7, 31, 33, 64, 101, 257, 1000, 1535, 1536, 1537, 2049, 2600], np.int64)
    f = synth.make_frame(w, sizes=sizes, gen_seed=63)
    keep, frame = _device_frame(torch, f)
    H = 512
    params = rvh.make_params(dim, H, w.tau, 9)
    dev = torch.device("cuda", 0)
    ctx = rvh.Context(0)
    results = {}
    try:
        for pw in (1, 8, 32):
            for hpl in (4, 8):
                ctx.check(rvh.rvh_set_schedule(ctx.handle, pw, hpl), "schedule")
                outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
                ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, rvh.make_result(outs), None), "estimate")
                torch.cuda.synchronize()
                results[(pw, hpl)] = _np(outs, f.n_points)
    finally:
        ctx.close()
    first = results[(1, 4)]
    for key, r in results.items():
        for k in ("inlier_mask", "inlier_count", "best_hypothesis", "status", "vx", "vy", "vz", "heading"):
            assert np.array_equal(r[k], first[k], equal_nan=True), (key, k)
    o = G.run_oracle(f.azimuth, f.doppler, f.offsets, el=f.elevation, H=H, tau=w.tau, seed=9)
    rep = G.compare(first, o, f.offsets)
    assert not rep["mismatch"], rep["mismatch"][:10]


def test_cta_row_slots_equal_per_point_rows(torch, monkeypatch):
    """FP64 rows kept in the CTA's own slot (clusters that fit shared memory)
    or in per-point scratch (RVH_CTA_ROWS=0): identical results, in 3D
    (rows stored) and under the line model (normalised points stored)."""
    dev = torch.device("cuda", 0)
    cases = [(synth.WORKLOADS["dense3d"], 700, {}), (synth.WORKLOADS["dense2d"], 300, {"hypothesis_model": 1})]
    results = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("RVH_CTA_ROWS", flag)
        ctx = rvh.Context(0)
        try:
            for k, (w, nc, kw) in enumerate(cases):
                f = synth.make_frame(w, n_clusters=nc, gen_seed=71 + k)
                keep, frame = _device_frame(torch, f)
                outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev, threshold=True)
                params = rvh.make_params(w.model_dim, 512, w.tau, 3, **kw)
                ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, rvh.make_result(outs), None), "estimate")
                torch.cuda.synchronize()
                results[(flag, k)] = _np(outs, f.n_points)
        finally:
            ctx.close()
    for k in range(len(cases)):
        for key in results[("1", k)]:
            assert np.array_equal(results[("1", k)][key], results[("0", k)][key], equal_nan=True), (k, key)



@pytest.mark.parametrize("case", ["dense2d", "stress2d", "dense3d", "adaptive", "local_opt", "paper_line"])
def test_pruning_same_result(torch, case):
    """The staged scoring pass with exact pruning (the default) and the plain
    pass give identical outputs -- masks, counts, winners, status,
    velocities and headings bit for bit -- while the pruned one evaluates
    fewer (trial, point) pairs.  Sizes 2..2600 include clusters around the
    staging threshold (512 points), ragged quads and clusters beyond the
    shared-memory capacity (never staged); 3D runs two chunks of trials."""
    ext = {"adaptive": {"confidence": 0.99, "trial_block": 128}, "local_opt": {"refine_iterations": 2},
           "paper_line": {"hypothesis_model": rvh.RVH_MODEL_PAPER_LINE}}.get(case, {})
    w = synth.WORKLOADS[case if case in ("dense2d", "stress2d", "dense3d") else "dense2d"]
    rng = np.random.default_rng(5)
    sizes = np.concatenate([[2, 3, 255, 256, 257, 383, 511, 512, 513, 1000, 1535, 1536, 2047, 2048, 2049, 2600],
                            rng.integers(200, 2048, 180)]).astype(np.int64)
    f = synth.make_frame(w, sizes=sizes, gen_seed=81)
    keep, frame = _device_frame(torch, f)
    H = 2048 if w.model_dim == 3 else 1024
    params = rvh.make_params(w.model_dim, H, w.tau, 13, **ext)
    dev = torch.device("cuda", 0)
    ctx = rvh.Context(0)
    out, scored = {}, {}
    try:
        for on in (1, 0):
            ctx.check(rvh.rvh_set_pruning(ctx.handle, on), "pruning")
            outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev, threshold=True)
            ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, rvh.make_result(outs), None), "estimate")
            torch.cuda.synchronize()
            out[on] = _np(outs, f.n_points)
            st = rvh.rvh_stats()
            ctx.check(rvh.rvh_get_stats(ctx.handle, st), "stats")
            scored[on] = st.pairs_scored
        assert rvh.rvh_set_pruning(ctx.handle, 2) == rvh.RVH_EINVAL
    finally:
        ctx.close()
    for k in out[1]:
        assert np.array_equal(out[1][k], out[0][k], equal_nan=True), k
    # the adaptive count scores blocks of 128 trials, under the lanes-over-points
    # schedule, which the staged pass does not take
    assert 0 < scored[1] <= scored[0] if case == "adaptive" else 0 < scored[1] < scored[0], scored
    if not ext:
        n = np.diff(f.offsets)
        assert scored[0] == int(n[n >= w.model_dim].sum()) * H, scored
        print(f"pruning {case}: {scored[1] / scored[0]:.3f} of the pairs scored")


@pytest.mark.parametrize("name", ["dense2d", "dense3d"])
def test_pruning_with_tied_counts(torch, name):
    """Noise-free clusters without outliers: nearly every trial counts every
    point, so the winner is decided by the lowest index among equal counts.
    The staged pass's lead and drops compare (count, index) keys; pruned
    and unpruned runs agree bit for bit and both equal the oracle."""
    import dataclasses
    w = dataclasses.replace(synth.WORKLOADS[name], outlier_frac=0.0, noise_sigma=0.0)
    sizes = np.random.default_rng(17).integers(512, 1600, 24).astype(np.int64)
    f = synth.make_frame(w, sizes=sizes, gen_seed=91)
    keep, frame = _device_frame(torch, f)
    H = 1024
    params = rvh.make_params(w.model_dim, H, w.tau, 21)
    dev = torch.device("cuda", 0)
    ctx = rvh.Context(0)
    out = {}
    try:
        for on in (1, 0):
            ctx.check(rvh.rvh_set_pruning(ctx.handle, on), "pruning")
            outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
            ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, rvh.make_result(outs), None), "estimate")
            torch.cuda.synchronize()
            out[on] = _np(outs, f.n_points)
    finally:
        ctx.close()
    for k in out[1]:
        assert np.array_equal(out[1][k], out[0][k], equal_nan=True), k
    assert (out[1]["inlier_count"] == np.diff(f.offsets)).mean() > 0.9  # the ties are real
    o = G.run_oracle(f.azimuth, f.doppler, f.offsets, el=f.elevation, H=H, tau=w.tau, seed=21)
    rep = G.compare(out[1], o, f.offsets)
    assert not rep["mismatch"], rep["mismatch"][:10]
