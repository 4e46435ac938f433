"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar: inlier masks, inlier counts, winning hypothesis indices and status bits
bit-exact; vx, vy, vz within 1e-6 m/s; heading within 1e-6 rad (where
|v| >= 1e-3 m/s).  Full-size workloads are compared on sampled clusters the
oracle computes one by one (the RNG is keyed per cluster, so any subset is
well defined).
"""
import ctypes

import numpy as np
import pytest

from paper_2012_12618_gb300 import synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_12618_gb300 import rvh
    c = rvh.Context(0)
    yield c
    c.close()


def _check(rep, tau=0.1):
    G.check_parity(rep, tau=tau)


def _run_pair(ctx, f, w, *, H=None, seed=None, subset=None, baseline=False, tau=None):
    H = H or w.num_hypotheses
    seed = w.seed if seed is None else seed
    tau = w.tau if tau is None else tau
    g = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, el=f.elevation, H=H, tau=tau, seed=seed,
                  baseline=baseline)
    o = G.run_oracle(f.azimuth, f.doppler, f.offsets, el=f.elevation, H=H, tau=tau, seed=seed, subset=subset)
    return g, o


def test_frame64_full(ctx):
    w = synth.WORKLOADS["frame64"]
    f = synth.make_frame(w)
    g, o = _run_pair(ctx, f, w)
    _check(G.compare(g, o, f.offsets))


@pytest.mark.parametrize("name,nc", [("dense2d", 192), ("stress2d", 256), ("dense3d", 96)])
def test_small_full(ctx, name, nc):
    w = synth.WORKLOADS[name]
    f = synth.make_frame(w, n_clusters=nc, gen_seed=w.gen_seed + 100)
    g, o = _run_pair(ctx, f, w)
    _check(G.compare(g, o, f.offsets))


@pytest.mark.parametrize("name", ["dense2d", "stress2d", "dense3d"])
def test_full_frames(ctx, name):
    """Every cluster of the full-size frame (4096 / 16384 / 8192 clusters), in
    the launch configuration bench.py times: device-resident inputs on a
    stream of its own, the autotuned scoring schedule, CUDA-graph replay.
    The oracle runs over all host cores (spawned processes)."""
    import torch
    from paper_2012_12618_gb300 import rvh
    w = synth.WORKLOADS[name]
    f = synth.make_frame(w)
    dev = torch.device("cuda", 0)
    ins = [None if a is None else torch.from_numpy(a).to(dev) for a in (f.azimuth, f.doppler, f.offsets, f.elevation)]
    frame = rvh.make_frame(*ins)
    params = rvh.make_params(w.model_dim, w.num_hypotheses, w.tau, w.seed)
    outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
    res = rvh.make_result(outs)
    stream = torch.cuda.Stream(dev)
    sptr = ctypes.c_void_p(stream.cuda_stream)
    tuned = rvh.rvh_schedule()
    try:
        ctx.check(rvh.rvh_autotune(ctx.handle, frame, params, res, 3, tuned), "rvh_autotune")
        for _ in range(2):  # the second call replays the captured graph
            ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, res, sptr), "rvh_estimate")
        stream.synchronize()
    finally:
        ctx.check(rvh.rvh_set_schedule(ctx.handle, 0, 0), "rvh_set_schedule")
    g = {k: v.cpu().numpy() for k, v in outs.items()}
    g["inlier_mask"] = g["inlier_mask"][:f.n_points]
    o = G.run_oracle_parallel(f.azimuth, f.doppler, f.offsets, el=f.elevation, H=w.num_hypotheses, tau=w.tau,
                              seed=w.seed)
    _check(G.compare(g, o, f.offsets))


def test_noise_free_band(ctx):
    """Noise-free inliers plus band points at tau +- 2e-5: many points fall in
    the FP32 error band and are decided in FP64."""
    import dataclasses
    w = dataclasses.replace(synth.WORKLOADS["stress2d"], noise_sigma=0.0)
    f = synth.make_frame(w, n_clusters=256, gen_seed=77)
    g, o = _run_pair(ctx, f, w)
    _check(G.compare(g, o, f.offsets))


def test_baseline_parity(ctx):
    for name, nc in (("frame64", 64), ("dense3d", 24)):
        w = synth.WORKLOADS[name]
        f = synth.make_frame(w, n_clusters=nc, gen_seed=5)
        H = 256
        g, o = _run_pair(ctx, f, w, H=H, baseline=True)
        _check(G.compare(g, o, f.offsets))


@pytest.mark.parametrize("pw,hpl", [(1, 4), (1, 8), (8, 4), (8, 8), (32, 4), (32, 8)])
def test_schedules_agree(ctx, pw, hpl):
    from paper_2012_12618_gb300 import rvh
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w, n_clusters=128, gen_seed=9)
    assert rvh.rvh_set_schedule(ctx.handle, pw, hpl) == 0
    try:
        g, o = _run_pair(ctx, f, w, H=640)
    finally:
        rvh.rvh_set_schedule(ctx.handle, 0, 0)
    _check(G.compare(g, o, f.offsets))


def test_edge_cases(ctx):
    rng = np.random.default_rng(3)
    sizes = [0, 1, 2, 3, 5, 40, 2047, 2048, 2049, 5000, 17]
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w, sizes=np.array(sizes), gen_seed=8)
    az = f.azimuth.copy()
    dop = f.doppler.copy()
    off = f.offsets
    # cluster 4 (5 points): every point at one azimuth -> all minimal sets singular
    az[off[4]:off[5]] = np.float32(0.25)
    # cluster 10: duplicated points and a NaN Doppler
    s = off[10]
    az[s + 1] = az[s]
    dop[s + 1] = dop[s]
    dop[s + 3] = np.nan
    for H, tau in ((1, 0.1), (1500, 0.1), (64, 0.0), (300, 5.0)):
        g = G.run_rvh(ctx, az, dop, off, H=H, tau=tau, seed=11)
        o = G.run_oracle(az, dop, off, H=H, tau=tau, seed=11)
        _check(G.compare(g, o, off), tau=tau)
    st = g["status"]
    assert st[0] & 1 and st[1] & 1 and st[2] == 0 or st[2] & 4


def test_3d_edge_cases(ctx):
    w = synth.WORKLOADS["dense3d"]
    f = synth.make_frame(w, sizes=np.array([0, 2, 3, 4, 9, 1500, 2100, 100]), gen_seed=12)
    for H in (1, 100, 1100):
        g = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, el=f.elevation, H=H, tau=0.1, seed=2)
        o = G.run_oracle(f.azimuth, f.doppler, f.offsets, el=f.elevation, H=H, tau=0.1, seed=2)
        _check(G.compare(g, o, f.offsets))


def test_empty_frame(ctx):
    g = G.run_rvh(ctx, np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(1, np.int32), H=8, tau=0.1, seed=1)
    assert g["vx"].shape == (0,)


def test_host_and_device_pointers_agree(ctx):
    w = synth.WORKLOADS["frame64"]
    f = synth.make_frame(w, n_clusters=40, gen_seed=21)
    a = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=256, tau=0.1, seed=4, device="cuda")
    b = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=256, tau=0.1, seed=4, device="cpu")
    for k in G.OUT_KEYS:
        assert np.array_equal(a[k], b[k], equal_nan=True), k


def test_seeds_change_draws(ctx):
    w = synth.WORKLOADS["frame64"]
    f = synth.make_frame(w, n_clusters=32, gen_seed=31)
    bests = []
    for seed in (1, 2, 0xFFFFFFFF00000001):
        g, o = _run_pair(ctx, f, w, seed=seed)
        _check(G.compare(g, o, f.offsets))
        bests.append(g["best_hypothesis"])
    assert not np.array_equal(bests[0], bests[1])


def _far_objects(n_clusters, gen_seed):
    """Clusters of far objects: a few metres across at hundreds of metres span
    0.1-0.6 deg of azimuth, so every minimal set is ill-conditioned
    (|det| = |sin(t1 - t0)| < 0.01) and most trials take the 2D refinement
    pass.  Doppler follows the velocity profile with N(0, 0.05) noise; 20%
    are outliers."""
    rng = np.random.default_rng(gen_seed)
    az, dop, off = [], [], [0]
    for c in range(n_clusters):
        n = int(rng.integers(16, 400))
        t0 = rng.uniform(-1.0, 1.0)
        half = [0.001, 0.0025, 0.005][c % 3]
        t = t0 + rng.uniform(-half, half, n)
        vx, vy = rng.uniform(-30.0, 30.0, 2)
        d = vx * np.cos(t) + vy * np.sin(t) + rng.normal(0.0, 0.05, n)
        out = rng.random(n) < 0.2
        d[out] = rng.uniform(-40.0, 40.0, out.sum())
        az.append(t)
        dop.append(d)
        off.append(off[-1] + n)
    return (np.concatenate(az).astype(np.float32), np.concatenate(dop).astype(np.float32),
            np.asarray(off, np.int32))


def test_narrow_azimuth_far_objects(ctx):
    from paper_2012_12618_gb300 import rvh
    import ctypes
    az, dop, off = _far_objects(60, 41)
    g = G.run_rvh(ctx, az, dop, off, H=1024, tau=0.1, seed=5)
    st = rvh.rvh_stats()
    assert rvh.load().rvh_get_stats(ctx.handle, ctypes.byref(st)) == rvh.RVH_OK
    assert st.refined_hypotheses > 0  # the queued 2D refinement ran
    o = G.run_oracle(az, dop, off, H=1024, tau=0.1, seed=5)
    _check(G.compare(g, o, off))


@pytest.mark.parametrize("name,nc,kw", [("dense2d", 400, {}), ("dense3d", 160, {}),
                                        ("stress2d", 300, {"hypothesis_model": 1}),
                                        ("dense2d", 256, {"first_cluster": 77, "refine_iterations": 1}),
                                        ("dense2d", 700, {"confidence": 0.99, "trial_block": 64})])
def test_host_frames_equal_device_frames(ctx, name, nc, kw):
    """A frame and its results in host memory give every output, the
    threshold array included, exactly as the same frame in device memory:
    page-locked buffers (read and written in place by the kernels) and
    pageable ones (staged through the context's scratch), mixed with device
    buffers too; with extensions and a first_cluster offset."""
    import torch
    from paper_2012_12618_gb300 import rvh
    w = synth.WORKLOADS[name]
    f = synth.make_frame(w, n_clusters=nc, gen_seed=w.gen_seed + 1300)
    dim = 3 if f.elevation is not None else 2
    params = rvh.make_params(dim, 256, w.tau, 9, **kw)
    dev = torch.device("cuda", 0)

    def place(t, where):
        return t.to(dev) if where == "device" else (t.pin_memory() if where == "pinned" else t)

    results = []
    for w_in, w_out in (("device", "device"), ("pinned", "pinned"), ("pageable", "pageable"),
                        ("pinned", "device"), ("device", "pinned"), ("pinned", "pageable")):
        # the frame holds raw pointers: keep its tensors alive until the call is done
        ins = [None if a is None else place(torch.from_numpy(a.copy()), w_in)
               for a in (f.azimuth, f.doppler, f.offsets, f.elevation)]
        frame = rvh.make_frame(*ins)
        outs = {k: place(v, w_out) for k, v in rvh.alloc_outputs(f.n_clusters, f.n_points, "cpu",
                                                                 threshold=True).items()}
        for v in outs.values():
            v.fill_(7)
        ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, rvh.make_result(outs), None), "estimate")
        torch.cuda.synchronize()
        results.append({k: v.cpu().numpy() for k, v in outs.items()})
    for r in results[1:]:
        for k in results[0]:
            assert np.array_equal(results[0][k][:f.n_points if k == "inlier_mask" else None],
                                  r[k][:f.n_points if k == "inlier_mask" else None], equal_nan=True), k
