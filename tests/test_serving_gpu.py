"""Serving: rvh_submit / rvh_poll / rvh_wait with continuous batching (GPU).

The central property: a frame's result does not depend on which other frames
share its batch or step -- it equals the result of rvh_estimate on the frame
alone (bit-exact masks, counts, winners and status; identical velocities).
"""
import ctypes

import numpy as np
import pytest

from paper_2012_12618_gb300 import rvh, serving, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _frames():
    spec = synth.ServingSpec(clusters_lo=20, clusters_hi=160)
    out = []
    for radar, k in ((0, 0), (40, 0), (1, 3), (33, 1), (2, 5), (50, 2), (3, 1)):
        f, w = synth.serving_frame(spec, radar, k)
        out.append((f, w, synth.radar_frame_seed(radar, k)))
    return out


def _np(outs, n_points):
    d = {k: v.cpu().numpy().copy() for k, v in outs.items()}
    d["inlier_mask"] = d["inlier_mask"][:n_points]
    return d


def _same(a, b):
    for k in ("inlier_mask", "inlier_count", "best_hypothesis", "status", "vx", "vy", "vz", "heading"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k


def test_results_same_alone_and_in_the_mix(torch):
    dev = torch.device("cuda", 0)
    frames = _frames()
    ctx = rvh.Context(0)
    try:
        inputs, alone = [], []
        for f, w, seed in frames:
            t = [torch.from_numpy(x).to(dev) if x is not None else None
                 for x in (f.azimuth, f.elevation, f.doppler, f.offsets)]
            frame = rvh.make_frame(t[0], t[2], t[3], t[1])
            params = rvh.make_params(w.model_dim, w.num_hypotheses, w.tau, seed)
            outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
            ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, rvh.make_result(outs), None), "estimate")
            torch.cuda.synchronize()
            alone.append(_np(outs, f.n_points))
            inputs.append((t, frame, params))
        for order in (list(range(len(frames))), list(reversed(range(len(frames))))):
            tickets, results = [], []
            for i in order:
                f, w, seed = frames[i]
                # alternate device outputs and host outputs, device inputs and host inputs
                if i % 2:
                    outs = rvh.alloc_outputs(f.n_clusters, f.n_points, "cpu")
                    frame = rvh.make_frame(f.azimuth, f.doppler, f.offsets, f.elevation)
                else:
                    outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
                    frame = inputs[i][1]
                tk = ctypes.c_uint64(0)
                ctx.check(rvh.rvh_submit(ctx.handle, frame, inputs[i][2], rvh.make_result(outs), tk), "submit")
                tickets.append((i, tk.value, outs, frame))
            for i, tk, outs, _ in tickets:
                assert rvh.rvh_wait(ctx.handle, tk, 30_000_000) == rvh.RVH_OK, rvh.rvh_last_error(None)
                torch.cuda.synchronize()
                _same(_np(outs, frames[i][0].n_points), alone[i])
    finally:
        ctx.close()


def test_serving_frames_equal_the_oracle(torch):
    """Frames of the 64-radar serving load at its full sizes (50..2000
    clusters of 8..2048 points; 2D radars with 256 trials, 3D radars with
    2048), submitted together through rvh_submit so that they share
    batches, each compared on every cluster with the oracle."""
    dev = torch.device("cuda", 0)
    spec = synth.ServingSpec()
    picks = [(0, 0), (32, 0), (5, 2), (40, 1), (17, 3), (63, 4)]
    ctx = rvh.Context(0)
    try:
        held, tickets = [], []
        for radar, k in picks:
            f, w = synth.serving_frame(spec, radar, k)
            t = [None if x is None else torch.from_numpy(x).to(dev) for x in (f.azimuth, f.doppler, f.offsets,
                                                                               f.elevation)]
            frame = rvh.make_frame(*t)
            params = rvh.make_params(w.model_dim, w.num_hypotheses, w.tau, synth.radar_frame_seed(radar, k))
            outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
            tk = ctypes.c_uint64(0)
            ctx.check(rvh.rvh_submit(ctx.handle, frame, params, rvh.make_result(outs), tk), "submit")
            held.append(t)
            tickets.append((radar, k, f, w, tk.value, outs))
        assert sum(1 for r, *_ in tickets if r >= 32) >= 2 and sum(1 for r, *_ in tickets if r < 32) >= 2
        for radar, k, f, w, tk, outs in tickets:
            assert rvh.rvh_wait(ctx.handle, tk, 60_000_000) == rvh.RVH_OK, rvh.rvh_last_error(None)
        torch.cuda.synchronize()
        for radar, k, f, w, tk, outs in tickets:
            g = _np(outs, f.n_points)
            o = G.run_oracle_parallel(f.azimuth, f.doppler, f.offsets, el=f.elevation, H=w.num_hypotheses,
                                      tau=w.tau, seed=synth.radar_frame_seed(radar, k))
            G.check_parity(G.compare(g, o, f.offsets), tau=w.tau,
                           label=f"serving radar {radar} frame {k} ({w.model_dim}D, {f.n_clusters} clusters)")
    finally:
        ctx.close()


def test_serving_steps_replay_graphs(torch):
    """Serving steps launch through CUDA graphs: a slot's graph for a kernel
    instantiation and node list is built once and replayed by later steps
    with their own batches, and results stay those of the frames alone."""
    dev = torch.device("cuda", 0)
    frames = _frames()
    ctx = rvh.Context(0)
    try:
        inputs, alone = [], []
        for f, w, seed in frames:
            t = [None if x is None else torch.from_numpy(x).to(dev) for x in (f.azimuth, f.doppler, f.offsets,
                                                                               f.elevation)]
            frame = rvh.make_frame(*t)
            params = rvh.make_params(w.model_dim, w.num_hypotheses, w.tau, seed)
            outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
            ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, rvh.make_result(outs), None), "estimate")
            torch.cuda.synchronize()
            alone.append(_np(outs, f.n_points))
            inputs.append((t, frame, params))
        for wave in range(8):
            tickets = []
            for i in (wave % len(frames), (wave + 3) % len(frames)):
                f = frames[i][0]
                outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
                tk = ctypes.c_uint64(0)
                ctx.check(rvh.rvh_submit(ctx.handle, inputs[i][1], inputs[i][2], rvh.make_result(outs), tk), "submit")
                tickets.append((i, tk.value, outs))
            for i, tk, outs in tickets:
                assert rvh.rvh_wait(ctx.handle, tk, 30_000_000) == rvh.RVH_OK, rvh.rvh_last_error(None)
                torch.cuda.synchronize()
                _same(_np(outs, frames[i][0].n_points), alone[i])
        st = rvh.rvh_stats()
        ctx.check(rvh.rvh_get_stats(ctx.handle, st), "stats")
        # at most one graph per slot (3) x dimension (2) x work list or not (2) is built
        assert st.serving_steps >= 8 and st.serving_graph_replays >= st.serving_steps - 12, \
            (st.serving_steps, st.serving_graph_replays)
    finally:
        ctx.close()


def test_extension_frames_same_alone_and_in_the_mix(torch):
    """Frames that use the extensions (local optimisation, adaptive trial
    count, Alg. 1's line model) batched with plain frames: a batch holding
    any of them runs the extension instantiation of the kernel for all its
    frames, and every result must still equal the frame's result alone."""
    dev = torch.device("cuda", 0)
    frames = _frames()
    ext = {0: dict(refine_iterations=2), 1: dict(confidence=0.99, trial_block=64),
           2: dict(hypothesis_model=rvh.RVH_MODEL_PAPER_LINE), 5: dict(confidence=0.999, refine_iterations=1)}
    ctx = rvh.Context(0)
    try:
        inputs, alone = [], []
        for i, (f, w, seed) in enumerate(frames):
            kw = ext.get(i, {})
            if kw.get("hypothesis_model") and w.model_dim != 2:
                kw = {}
            t = [torch.from_numpy(x).to(dev) if x is not None else None
                 for x in (f.azimuth, f.elevation, f.doppler, f.offsets)]
            frame = rvh.make_frame(t[0], t[2], t[3], t[1])
            params = rvh.make_params(w.model_dim, w.num_hypotheses, w.tau, seed, **kw)
            outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
            ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, rvh.make_result(outs), None), "estimate")
            torch.cuda.synchronize()
            alone.append(_np(outs, f.n_points))
            inputs.append((frame, params, t))  # t keeps the device inputs alive
        tickets = []
        for i in range(len(frames)):
            f = frames[i][0]
            outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
            tk = ctypes.c_uint64(0)
            ctx.check(rvh.rvh_submit(ctx.handle, inputs[i][0], inputs[i][1], rvh.make_result(outs), tk), "submit")
            tickets.append((i, tk.value, outs))
        for i, tk, outs in tickets:
            assert rvh.rvh_wait(ctx.handle, tk, 30_000_000) == rvh.RVH_OK, rvh.rvh_last_error(None)
            torch.cuda.synchronize()
            _same(_np(outs, frames[i][0].n_points), alone[i])
    finally:
        ctx.close()


def test_poll_semantics(torch):
    dev = torch.device("cuda", 0)
    f, w, seed = _frames()[0]
    ctx = rvh.Context(0)
    try:
        assert rvh.rvh_poll(ctx.handle, 12345) == rvh.RVH_EINVAL
        outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
        frame = rvh.make_frame(f.azimuth, f.doppler, f.offsets)
        params = rvh.make_params(2, w.num_hypotheses, w.tau, seed)
        tk = ctypes.c_uint64(0)
        ctx.check(rvh.rvh_submit(ctx.handle, frame, params, rvh.make_result(outs), tk), "submit")
        rc = rvh.rvh_wait(ctx.handle, tk.value, 0)
        assert rc in (rvh.RVH_OK, rvh.RVH_ETIMEDOUT)
        if rc != rvh.RVH_OK:
            assert rvh.rvh_wait(ctx.handle, tk.value, -1) == rvh.RVH_OK
        # a completed ticket is released by the call that reported it
        assert rvh.rvh_poll(ctx.handle, tk.value) == rvh.RVH_EINVAL
        # invalid frames are refused at submission
        bad = np.array([0, 5, 3], np.int32)
        fr = rvh.make_frame(f.azimuth[:3], f.doppler[:3], bad)
        assert rvh.rvh_submit(ctx.handle, fr, params, rvh.make_result(outs), tk) == rvh.RVH_EINVAL
    finally:
        ctx.close()


def test_backpressure_and_recovery(torch):
    """A small budget fills up: submissions get RVH_EAGAIN (or a frame too big
    for the pool RVH_ENOMEM) and succeed again once earlier frames complete."""
    dev = torch.device("cuda", 0)
    ctx = rvh.Context(0, mem_budget_bytes=96 << 20)
    try:
        w = synth.WORKLOADS["dense3d"]
        f = synth.make_frame(w, n_clusters=1500, gen_seed=3)
        t = [torch.from_numpy(x).to(dev) for x in (f.azimuth, f.elevation, f.doppler, f.offsets)]
        frame = rvh.make_frame(t[0], t[2], t[3], t[1])
        params = rvh.make_params(3, 2048, 0.1, 1)
        held, saw_eagain = [], False
        for _ in range(64):
            outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
            tk = ctypes.c_uint64(0)
            rc = rvh.rvh_submit(ctx.handle, frame, params, rvh.make_result(outs), tk)
            if rc == rvh.RVH_EAGAIN:
                saw_eagain = True
                break
            assert rc == rvh.RVH_OK, rvh.rvh_last_error(None)
            held.append((tk.value, outs))
        for tk, _ in held:
            assert rvh.rvh_wait(ctx.handle, tk, 60_000_000) == rvh.RVH_OK
        outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
        tk = ctypes.c_uint64(0)
        assert rvh.rvh_submit(ctx.handle, frame, params, rvh.make_result(outs), tk) == rvh.RVH_OK
        assert rvh.rvh_wait(ctx.handle, tk.value, 60_000_000) == rvh.RVH_OK
        assert saw_eagain or len(held) == 64
        big = synth.make_frame(synth.WORKLOADS["dense2d"], n_clusters=16384, gen_seed=4)
        bframe = rvh.make_frame(big.azimuth, big.doppler, big.offsets)
        bouts = rvh.alloc_outputs(big.n_clusters, big.n_points, "cpu")
        rc = rvh.rvh_submit(ctx.handle, bframe, rvh.make_params(2, 64, 0.1, 1), rvh.make_result(bouts), tk)
        assert rc == rvh.RVH_ENOMEM
    finally:
        ctx.close()


def test_short_load(torch):
    dev = torch.device("cuda", 0)
    spec = synth.ServingSpec(n_radars=16, duration_s=0.6, warmup_s=0.2, clusters_lo=50, clusters_hi=400)
    ctx = rvh.Context(0)
    try:
        res = serving.run_load(ctx, spec, dev, pool_frames=2)
    finally:
        ctx.close()
    s = res.summary()
    assert res.frames > 50 and s["p99_ms"] is not None and s["p99_ms"] < 1000.0, s
