"""GPU parity of Alg. 1 as printed (hypothesis_model = RVH_MODEL_PAPER_LINE:
line fits in the normalised (azimuth, Doppler) plane, perpendicular
distance, MAD threshold) against the FP64 oracle.  Every decision is made
from the same FP64 formulas on both sides (no trigonometry enters them), so
masks, counts, winners and status must be bit-exact with no rounding ties;
the least-squares velocity within 1e-6 m/s, heading within 1e-6 rad."""
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


def _pair(ctx, az, dop, off, *, H, seed, conf=0.0, block=0, subset=None):
    g = G.run_rvh(ctx, az, dop, off, H=H, tau=0.1, seed=seed, line_model=True, confidence=conf, trial_block=block)
    o = G.run_oracle(az, dop, off, H=H, tau=0.1, seed=seed, subset=subset, line_model=True, confidence=conf,
                     trial_block=block or 128)
    return g, o


def _check(rep):
    # the line model uses no trigonometry: no tie of any kind is allowed
    G.check_parity(rep, tau=0.1)


def test_frame64(ctx):
    w = synth.WORKLOADS["frame64"]
    f = synth.make_frame(w)
    g, o = _pair(ctx, f.azimuth, f.doppler, f.offsets, H=256, seed=1)
    _check(G.compare(g, o, f.offsets))
    assert (g["status"] == 0).all()


@pytest.mark.parametrize("name,nc,H", [("dense2d", 160, 1024), ("stress2d", 256, 512), ("dense2d", 64, 97)])
def test_small_frames(ctx, name, nc, H):
    w = synth.WORKLOADS[name]
    f = synth.make_frame(w, n_clusters=nc, gen_seed=w.gen_seed + 700)
    g, o = _pair(ctx, f.azimuth, f.doppler, f.offsets, H=H, seed=2)
    _check(G.compare(g, o, f.offsets))


def test_full_frame(ctx):
    """Every cluster of the full dense 2D frame under Alg. 1 as printed."""
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w)
    g = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=w.num_hypotheses, tau=0.1, seed=w.seed, line_model=True)
    o = G.run_oracle_parallel(f.azimuth, f.doppler, f.offsets, H=w.num_hypotheses, tau=0.1, seed=w.seed,
                              line_model=True)
    _check(G.compare(g, o, f.offsets))


def test_adaptive(ctx):
    w = synth.WORKLOADS["stress2d"]
    f = synth.make_frame(w, n_clusters=192, gen_seed=71)
    g, o = _pair(ctx, f.azimuth, f.doppler, f.offsets, H=1024, seed=3, conf=0.99, block=64)
    _check(G.compare(g, o, f.offsets))


def test_edge_cases(ctx):
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w, sizes=np.array([0, 1, 2, 3, 5, 40, 1536, 1537, 2049, 17, 8]), gen_seed=72)
    az, dop, off = f.azimuth.copy(), f.doppler.copy(), f.offsets
    az[off[4]:off[5]] = np.float32(0.25)          # one azimuth: every seed pair shares x
    s = off[9]
    az[s + 1], dop[s + 1] = az[s], dop[s]         # duplicated point
    dop[off[10]:off[11]] = np.float32(3.5)        # one Doppler: MAD 0, only exact hits
    for H in (1, 64, 700):
        g, o = _pair(ctx, az, dop, off, H=H, seed=11)
        _check(G.compare(g, o, off))
    assert g["status"][0] & 1 and g["status"][1] & 1 and g["status"][4] & 2


def test_doppler_scaling_is_exact(ctx):
    w = synth.WORKLOADS["frame64"]
    f = synth.make_frame(w, n_clusters=48, gen_seed=73)
    a = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=256, tau=0.1, seed=5, line_model=True)
    b = G.run_rvh(ctx, f.azimuth, f.doppler * np.float32(4.0), f.offsets, H=256, tau=0.1, seed=5, line_model=True)
    for k in ("inlier_mask", "inlier_count", "best_hypothesis", "status"):
        assert np.array_equal(a[k], b[k]), k
    assert np.allclose(a["vx"] * 4.0, b["vx"], rtol=1e-12, atol=1e-9)


def test_baseline_rejects_line_model(ctx):
    w = synth.WORKLOADS["frame64"]
    f = synth.make_frame(w, n_clusters=4, gen_seed=74)
    with pytest.raises(RuntimeError, match="-1"):
        G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=16, tau=0.1, seed=1, baseline=True, line_model=True)


def test_threshold_output_on_every_entry_point(ctx):
    """The optional per-cluster threshold output: each cluster's MAD threshold
    under Alg. 1 (bit-exact against the oracle's, NaN for clusters of one
    point) and tau under the cosine model, through rvh_estimate with device
    and host buffers, the serving path and the allocation-free call."""
    import ctypes
    import torch
    from paper_2012_12618_gb300 import rvh
    w = synth.WORKLOADS["stress2d"]
    f = synth.make_frame(w, n_clusters=96, gen_seed=w.gen_seed + 900)
    # a cluster of one point at the end: it has no threshold
    az = np.concatenate([f.azimuth, np.float32([0.3])])
    dop = np.concatenate([f.doppler, np.float32([1.5])])
    off = np.concatenate([f.offsets, np.int32([f.offsets[-1] + 1])]).astype(np.int32)
    nc, npts = off.shape[0] - 1, az.shape[0]
    want = G.run_oracle(az, dop, off, H=64, tau=0.1, seed=3, line_model=True)["threshold"]
    assert np.isnan(want[-1]) and np.isfinite(want[:-1]).all()
    dev = torch.device("cuda", 0)
    t = {k: torch.from_numpy(v).to(dev) for k, v in (("az", az), ("dop", dop), ("off", off))}
    frame = rvh.make_frame(t["az"], t["dop"], t["off"])
    line = rvh.make_params(2, 64, 0.1, 3, hypothesis_model=rvh.RVH_MODEL_PAPER_LINE)
    cosine = rvh.make_params(2, 64, 0.1, 3)

    def same(got, ref):
        got = np.asarray(got)
        assert np.array_equal(np.isnan(got), np.isnan(ref)) and np.array_equal(got[~np.isnan(ref)],
                                                                              ref[~np.isnan(ref)])

    for device in ("cuda", "cpu"):  # device buffers, then host buffers (staged)
        outs = rvh.alloc_outputs(nc, npts, device, threshold=True)
        ctx.check(rvh.rvh_estimate(ctx.handle, frame, line, rvh.make_result(outs), None), "estimate")
        torch.cuda.synchronize()
        same(outs["threshold"].cpu().numpy(), want)
        ctx.check(rvh.rvh_estimate(ctx.handle, frame, cosine, rvh.make_result(outs), None), "estimate")
        torch.cuda.synchronize()
        assert (outs["threshold"].cpu().numpy() == 0.1).all()
    # serving path, host outputs
    outs = rvh.alloc_outputs(nc, npts, "cpu", threshold=True)
    tk = ctypes.c_uint64(0)
    ctx.check(rvh.rvh_submit(ctx.handle, frame, line, rvh.make_result(outs), tk), "submit")
    assert rvh.rvh_wait(ctx.handle, tk, 30_000_000) == rvh.RVH_OK, rvh.rvh_last_error(None)
    same(outs["threshold"].numpy(), want)
    # allocation-free call, device outputs
    outs = rvh.alloc_outputs(nc, npts, dev, threshold=True)
    assert rvh.rvh_estimate_noalloc(frame, line, rvh.make_result(outs), None) == rvh.RVH_OK
    torch.cuda.synchronize()
    same(outs["threshold"].cpu().numpy(), want)
