"""GPU parity of the adaptive trial count (confidence > 0) against the FP64
oracle: masks, counts, winners and status bit-exact, velocities within
1e-6 m/s, headings within 1e-6 rad, and the total number of trials run
(rvh_stats.hypotheses) equal to the oracle's per-cluster trial counts."""
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


def _stats(ctx):
    from paper_2012_12618_gb300 import rvh
    st = rvh.rvh_stats()
    assert rvh.rvh_get_stats(ctx.handle, st) == 0
    return st


def _pair(ctx, f, *, H, tau, seed, conf, block, iters=0, subset=None):
    g = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, el=f.elevation, H=H, tau=tau, seed=seed,
                  confidence=conf, trial_block=block, refine_iterations=iters)
    st = _stats(ctx)
    o = G.run_oracle(f.azimuth, f.doppler, f.offsets, el=f.elevation, H=H, tau=tau, seed=seed, subset=subset,
                     confidence=conf, trial_block=block or 128, refine_iterations=iters, want_trials=True)
    return g, o, st


def _check(rep, tau=0.1):
    G.check_parity(rep, tau=tau)


@pytest.mark.parametrize("name,nc,conf,block", [
    ("frame64", 64, 0.99, 32), ("frame64", 64, 0.999999, 64), ("dense2d", 160, 0.99, 0),
    ("stress2d", 256, 0.99, 128), ("dense3d", 64, 0.99, 32), ("dense3d", 48, 0.9999, 256)])
def test_adaptive_frames(ctx, name, nc, conf, block):
    w = synth.WORKLOADS[name]
    f = synth.make_frame(w, n_clusters=nc, gen_seed=w.gen_seed + 500)
    g, o, st = _pair(ctx, f, H=w.num_hypotheses, tau=w.tau, seed=w.seed, conf=conf, block=block)
    _check(G.compare(g, o, f.offsets))
    assert st.hypotheses == int(o["trials_used"].sum())
    assert st.pair_evals == int((o["trials_used"] * np.diff(f.offsets)).sum())
    assert st.hypotheses < nc * w.num_hypotheses  # the bound stopped some clusters early


def test_one_block_is_the_full_run(ctx):
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w, n_clusters=96, gen_seed=61)
    a = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=1024, tau=0.1, seed=3)
    b = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=1024, tau=0.1, seed=3, confidence=0.99, trial_block=1024)
    for k in G.OUT_KEYS:
        assert np.array_equal(a[k], b[k], equal_nan=True), k


def test_partial_last_block_and_local_opt(ctx):
    w = synth.WORKLOADS["stress2d"]
    f = synth.make_frame(w, n_clusters=128, gen_seed=62)
    for H, block, iters, conf in ((300, 128, 0, 0.9999999), (300, 128, 3, 0.99), (97, 32, 2, 0.999999999)):
        g, o, st = _pair(ctx, f, H=H, tau=w.tau, seed=4, conf=conf, block=block, iters=iters)
        _check(G.compare(g, o, f.offsets))
        assert st.hypotheses == int(o["trials_used"].sum())


def test_edge_cases(ctx):
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w, sizes=np.array([0, 1, 2, 3, 5, 40, 1536, 1537, 2049, 17]), gen_seed=63)
    for H, tau in ((1, 0.1), (64, 0.0), (700, 0.1), (700, 5.0)):
        g, o, st = _pair(ctx, f, H=H, tau=tau, seed=6, conf=0.99, block=32)
        _check(G.compare(g, o, f.offsets), tau=tau)
        assert st.hypotheses == int(o["trials_used"].sum())
    w3 = synth.WORKLOADS["dense3d"]
    f3 = synth.make_frame(w3, sizes=np.array([0, 2, 3, 4, 9, 1500, 2100, 100]), gen_seed=64)
    g, o, st = _pair(ctx, f3, H=500, tau=0.1, seed=2, conf=0.99, block=64, iters=2)
    _check(G.compare(g, o, f3.offsets))
    assert st.hypotheses == int(o["trials_used"].sum())


def test_full_frame(ctx):
    """Every cluster of the full dense 2D frame, stopping at confidence 0.99."""
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w)
    g = G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=w.num_hypotheses, tau=w.tau, seed=w.seed,
                  confidence=0.99, trial_block=128)
    o = G.run_oracle_parallel(f.azimuth, f.doppler, f.offsets, H=w.num_hypotheses, tau=w.tau, seed=w.seed,
                              confidence=0.99, trial_block=128)
    _check(G.compare(g, o, f.offsets))


def test_baseline_rejects_adaptive(ctx):
    w = synth.WORKLOADS["frame64"]
    f = synth.make_frame(w, n_clusters=4, gen_seed=65)
    with pytest.raises(RuntimeError, match="-1"):
        G.run_rvh(ctx, f.azimuth, f.doppler, f.offsets, H=16, tau=0.1, seed=1, baseline=True, confidence=0.9)
