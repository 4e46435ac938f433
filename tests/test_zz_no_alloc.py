"""rvh_estimate_noalloc against rvh_estimate (GPU).

Some callers may not allocate device memory once they are running (real-time
stacks that forbid allocation after start-up, plugins whose framework owns all
device memory); rvh_estimate_noalloc serves them from fixed file-scope device
arrays.  This file is named to be collected last.  The test runs the new entry
point twice in a row through the C ABI on the same frame and checks each
result against the context-based rvh_estimate: masks, counts, winners and
status bit-exact, velocities and heading within 1e-6; once with the plain
method and once with each extension (local-optimisation rounds, the adaptive
trial count, Alg. 1's line model).  It passes on its own in a fresh process
and after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2012_12618_gb300 import rvh, synth

pytestmark = pytest.mark.gpu


def _to_np(outs, n_points):
    out = {k: v.cpu().numpy() for k, v in outs.items()}
    out["inlier_mask"] = out["inlier_mask"][:n_points]
    return out


EXTENSIONS = {
    "plain": {},
    "local_opt": {"refine_iterations": 2},
    "adaptive": {"confidence": 0.99, "trial_block": 128},
    "paper_line": {"hypothesis_model": rvh.RVH_MODEL_PAPER_LINE},
}


@pytest.mark.parametrize("ext", list(EXTENSIONS))
def test_noalloc_matches_estimate_twice(ext):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w, n_clusters=384, gen_seed=404)
    dev = torch.device("cuda", 0)
    az = torch.from_numpy(f.azimuth).to(dev)
    dop = torch.from_numpy(f.doppler).to(dev)
    off = torch.from_numpy(f.offsets).to(dev)
    frame = rvh.make_frame(az, dop, off)
    params = rvh.make_params(2, w.num_hypotheses, w.tau, 7, **EXTENSIONS[ext])

    ctx = rvh.Context(0)
    try:
        ref_outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
        assert rvh.rvh_estimate(ctx.handle, frame, params, rvh.make_result(ref_outs), None) == rvh.RVH_OK
        torch.cuda.synchronize()
        ref = _to_np(ref_outs, f.n_points)
    finally:
        ctx.close()

    for call in range(2):
        outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
        for t in outs.values():
            t.fill_(0x5A if t.dtype == torch.uint8 else 7)
        rc = rvh.rvh_estimate_noalloc(frame, params, rvh.make_result(outs), None)
        assert rc == rvh.RVH_OK, rvh.rvh_last_error(None)
        torch.cuda.synchronize()
        got = _to_np(outs, f.n_points)
        for k in ("inlier_mask", "inlier_count", "best_hypothesis", "status"):
            assert np.array_equal(got[k], ref[k]), (call, k)
        for k in ("vx", "vy", "vz", "heading"):
            assert np.allclose(got[k], ref[k], rtol=0, atol=1e-6, equal_nan=True), (call, k)

    # frames beyond the fixed limits are refused before any launch
    big = rvh.rvh_frame(None, None, None, None, 1, rvh.RVH_NOALLOC_MAX_POINTS + 1)
    assert rvh.rvh_estimate_noalloc(big, params, rvh.make_result(outs), None) == rvh.RVH_EINVAL
    assert "limits" in rvh.rvh_last_error(None)


def test_noalloc_work_list_path_and_no_device_allocation():
    """2000 clusters: more than the GPU holds resident CTAs, so the work-list
    kernel and the work counter kept in the shared arrays run; a counter left
    stale by the first call would show in the second.  Both calls equal
    rvh_estimate bit for bit, and the second call leaves the device's free
    memory unchanged (the first call on a device commits the arrays)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = synth.WORKLOADS["dense2d"]
    f = synth.make_frame(w, n_clusters=2000, gen_seed=405)
    assert f.n_points <= rvh.RVH_NOALLOC_MAX_POINTS
    dev = torch.device("cuda", 0)
    ins = [torch.from_numpy(a).to(dev) for a in (f.azimuth, f.doppler, f.offsets)]
    frame = rvh.make_frame(*ins)
    params = rvh.make_params(2, 256, w.tau, 11)
    ctx = rvh.Context(0)
    try:
        ref_outs = rvh.alloc_outputs(f.n_clusters, f.n_points, dev)
        assert rvh.rvh_estimate(ctx.handle, frame, params, rvh.make_result(ref_outs), None) == rvh.RVH_OK
        torch.cuda.synchronize()
        ref = _to_np(ref_outs, f.n_points)
        st = rvh.rvh_stats()
        assert rvh.rvh_get_stats(ctx.handle, st) == rvh.RVH_OK
        assert st.kernel_launches == 2  # work list + fused kernel: the same path the no-allocation call takes
    finally:
        ctx.close()
    outs = [rvh.alloc_outputs(f.n_clusters, f.n_points, dev) for _ in range(2)]
    torch.cuda.synchronize()
    free_after = []
    for call in range(2):
        rc = rvh.rvh_estimate_noalloc(frame, params, rvh.make_result(outs[call]), None)
        assert rc == rvh.RVH_OK, rvh.rvh_last_error(None)
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info(dev)[0])
        got = _to_np(outs[call], f.n_points)
        for k in ref:
            assert np.array_equal(got[k], ref[k], equal_nan=True), (call, k)
    assert free_after[1] == free_after[0], free_after


def test_noalloc_empty_clusters_need_no_point_arrays():
    """Clusters without points: like rvh_estimate, NULL point arrays and
    mask are accepted, and every cluster reports too few points."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    off = torch.zeros(4, dtype=torch.int32, device=dev)
    frame = rvh.rvh_frame(None, None, None, rvh.ptr(off), 3, 0)
    outs = rvh.alloc_outputs(3, 0, dev)
    res = rvh.make_result(outs)
    res.inlier_mask = None
    rc = rvh.rvh_estimate_noalloc(frame, rvh.make_params(2, 64, 0.1, 1), res, None)
    assert rc == rvh.RVH_OK, rvh.rvh_last_error(None)
    torch.cuda.synchronize()
    assert (outs["status"].cpu().numpy() == rvh.RVH_STATUS_TOO_FEW_POINTS).all()
    assert (outs["best_hypothesis"].cpu().numpy() == -1).all()

