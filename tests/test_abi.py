"""The C ABI library builds, loads and exports every entry point that
include/rvh.h declares; calls that need no GPU behave as documented."""
import ctypes
import os
import re

import pytest

from paper_2012_12618_gb300 import build, rvh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rvh.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rvh_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("rvh_create", "rvh_destroy", "rvh_estimate", "rvh_submit", "rvh_poll", "rvh_wait",
                 "rvh_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(build.build())
    for name in declared_functions():
        assert hasattr(L, name), name
    # the binding covers the same names
    assert set(declared_functions()) == set(rvh.SIGNATURES)


def test_null_context_is_rejected():
    f = rvh.rvh_frame()
    p = rvh.make_params(2, 8, 0.1, 1)
    r = rvh.rvh_result()
    assert rvh.rvh_estimate(None, f, p, r) == rvh.RVH_EINVAL
    assert "ctx" in rvh.rvh_last_error(None)
    assert rvh.rvh_poll(None, 1) == rvh.RVH_EINVAL
    assert rvh.rvh_set_schedule(None, 1, 4) == rvh.RVH_EINVAL
    assert rvh.rvh_set_pruning(None, 1) == rvh.RVH_EINVAL


def test_create_without_gpu_reports_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = rvh.rvh_create(ctypes.byref(h), 0, 0)
    assert rc == rvh.RVH_ECUDA and not h.value
    assert rvh.rvh_last_error(None)


def test_params_layout_and_refine_range():
    # rvh_params as declared in include/rvh.h
    assert ctypes.sizeof(rvh.rvh_params) == 56
    assert rvh.rvh_params.refine_iterations.offset == 36
    assert rvh.rvh_params.confidence.offset == 40 and rvh.rvh_params.trial_block.offset == 48
    assert rvh.rvh_params.hypothesis_model.offset == 52
    f = rvh.rvh_frame()
    r = rvh.rvh_result()
    for bad in (-1, 65):
        p = rvh.make_params(2, 8, 0.1, 1, refine_iterations=bad)
        assert rvh.rvh_estimate_noalloc(f, p, r, None) == rvh.RVH_EINVAL
        assert "refine_iterations" in rvh.rvh_last_error(None)
    for conf, block in ((1.0, 0), (-0.5, 0), (float("nan"), 0), (0.9, 16), (0.9, 2048), (0.9, 100)):
        p = rvh.make_params(2, 8, 0.1, 1, confidence=conf, trial_block=block)
        assert rvh.rvh_estimate_noalloc(f, p, r, None) == rvh.RVH_EINVAL
        msg = rvh.rvh_last_error(None)
        assert "confidence" in msg or "trial_block" in msg, msg
    # the checks are rvh_estimate's: point arrays are needed once there are points
    p = rvh.make_params(2, 8, 0.1, 1)
    pts = rvh.rvh_frame(None, None, None, None, 1, 5)
    assert rvh.rvh_estimate_noalloc(pts, p, r, None) == rvh.RVH_EINVAL
    assert "azimuth" in rvh.rvh_last_error(None)
    for dim, model, iters in ((2, 2, 0), (2, -1, 0), (3, 1, 0), (2, 1, 2)):
        p = rvh.make_params(dim, 8, 0.1, 1, refine_iterations=iters, hypothesis_model=model)
        assert rvh.rvh_estimate_noalloc(f, p, r, None) == rvh.RVH_EINVAL
        msg = rvh.rvh_last_error(None)
        assert "hypothesis_model" in msg or "model_dim" in msg, msg


def test_result_layout_matches_the_header(tmp_path):
    """rvh_result as the C compiler lays it out (offsetof through gcc) equals
    the binding's ctypes structure, the optional threshold output included."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "rvh.h"\n'
        'int main(void) { printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(rvh_result), offsetof(rvh_result, inlier_mask),'
        ' offsetof(rvh_result, threshold), sizeof(rvh_stats), offsetof(rvh_stats, graph_builds),'
        ' offsetof(rvh_stats, serving_graph_replays)); return 0; }\n')
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    size, mask_off, thr_off, ssize, gb_off, sgr_off = map(int, subprocess.run(
        [str(exe)], check=True, capture_output=True, text=True).stdout.split())
    assert size == ctypes.sizeof(rvh.rvh_result)
    assert mask_off == rvh.rvh_result.inlier_mask.offset and thr_off == rvh.rvh_result.threshold.offset
    # rvh_stats, with the graph and serving counters at its end
    assert ssize == ctypes.sizeof(rvh.rvh_stats)
    assert gb_off == rvh.rvh_stats.graph_builds.offset and sgr_off == rvh.rvh_stats.serving_graph_replays.offset
