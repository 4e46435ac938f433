"""GPU parity of the local-optimisation rounds (refine_iterations > 0)
against the FP64 oracle, with the same bar as the single-pass path: masks,
counts, winners and status bit-exact, velocities within 1e-6 m/s, headings
within 1e-6 rad.  A round re-thresholds against a least-squares velocity
whose last bits depend on the summation order; the oracle logs decisions
within that reach of tau as fragile, and a disagreement there is a rounding
tie (none expected at these sizes)."""
import dataclasses

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


def _pair(ctx, az, dop, off, *, el=None, H, tau, seed, iters, subset=None):
    g = G.run_rvh(ctx, az, dop, off, el=el, H=H, tau=tau, seed=seed, refine_iterations=iters)
    o = G.run_oracle(az, dop, off, el=el, H=H, tau=tau, seed=seed, subset=subset, refine_iterations=iters)
    return g, o


def _check(rep, tau=0.1):
    G.check_parity(rep, tau=tau)


@pytest.mark.parametrize("iters", [1, 3, 8])
def test_frame64(ctx, iters):
    w = synth.WORKLOADS["frame64"]
    f = synth.make_frame(w)
    g, o = _pair(ctx, f.azimuth, f.doppler, f.offsets, H=w.num_hypotheses, tau=w.tau, seed=w.seed, iters=iters)
    _check(G.compare(g, o, f.offsets))
    base = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=w.num_hypotheses, tau=w.tau, seed=w.seed)
    # the rounds move some points (and never the winner)
    assert (base["inlier_mask"] != g["inlier_mask"]).sum() > 0
    assert np.array_equal(base["best_hypothesis"], g["best_hypothesis"])


@pytest.mark.parametrize("name,nc,iters", [("dense2d", 160, 4), ("stress2d", 256, 2), ("dense3d", 64, 4)])
def test_small_frames(ctx, name, nc, iters):
    w = synth.WORKLOADS[name]
    f = synth.make_frame(w, n_clusters=nc, gen_seed=w.gen_seed + 300)
    g, o = _pair(ctx, f.azimuth, f.doppler, f.offsets, el=f.elevation, H=w.num_hypotheses, tau=w.tau,
                 seed=w.seed, iters=iters)
    _check(G.compare(g, o, f.offsets))


def test_full_frame(ctx):
    """Every cluster of the full dense 2D frame with two rounds."""
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w)
    g = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=w.num_hypotheses, tau=w.tau, seed=w.seed,
                  refine_iterations=2)
    o = G.run_oracle_parallel(f.azimuth, f.doppler, f.offsets, H=w.num_hypotheses, tau=w.tau, seed=w.seed,
                              refine_iterations=2)
    _check(G.compare(g, o, f.offsets))


def test_noise_free_band(ctx):
    """Noise-free inliers: the least-squares velocity is the truth to ~1e-15,
    so the band points placed at tau +- 2e-5 sit in the FP32 error band of
    every round and are decided in FP64."""
    w = dataclasses.replace(synth.WORKLOADS["stress2d"], noise_sigma=0.0)
    f = synth.make_frame(w, n_clusters=256, gen_seed=78)
    g, o = _pair(ctx, f.azimuth, f.doppler, f.offsets, H=256, tau=w.tau, seed=3, iters=3)
    _check(G.compare(g, o, f.offsets))


def test_edge_cases(ctx):
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w, sizes=np.array([0, 1, 2, 3, 5, 40, 1536, 1537, 2049, 17]), gen_seed=18)
    for H, tau in ((1, 0.1), (64, 0.0), (300, 5.0), (700, 0.1)):
        g, o = _pair(ctx, f.azimuth, f.doppler, f.offsets, H=H, tau=tau, seed=5, iters=5)
        _check(G.compare(g, o, f.offsets), tau=tau)
    w3 = synth.WORKLOADS["dense3d"]
    f3 = synth.make_frame(w3, sizes=np.array([0, 2, 3, 4, 9, 1500, 2100, 100]), gen_seed=19)
    g, o = _pair(ctx, f3.azimuth, f3.doppler, f3.offsets, el=f3.elevation, H=300, tau=0.1, seed=2, iters=4)
    _check(G.compare(g, o, f3.offsets))


def test_zero_rounds_is_the_plain_path(ctx):
    w = synth.WORKLOADS["frame64"]
    f = synth.make_frame(w, n_clusters=48, gen_seed=41)
    a = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=256, tau=0.1, seed=7)
    b = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=256, tau=0.1, seed=7, refine_iterations=0)
    for k in G.OUT_KEYS:
        assert np.array_equal(a[k], b[k], equal_nan=True), k


def test_baseline_rejects_rounds(ctx):
    w = synth.WORKLOADS["frame64"]
    f = synth.make_frame(w, n_clusters=4, gen_seed=42)
    with pytest.raises(RuntimeError, match="-1"):
        G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=16, tau=0.1, seed=1, baseline=True, refine_iterations=2)
