"""Device-level checks of the FP32 filter's assumptions (GPU).

Builds tests/cuda/device_checks.cu with the library's compiler flags and runs:
  rows    every float in [-pi, pi]: sincosf within 2^-23 relative of the FP64
          value (the filter's bound assumes 2^-22, twice that), and the
          table-based FP64 sincos within 4 * 2^-53 (absolute) of the library's;
  filter  ~10^8 (trial, point) pairs of ordinary, near-degenerate and
          large-velocity minimal sets, with and without the refinement step:
          no FP32 'certainly in/out' decision disagrees with FP64, and
          |r32 - r64| never exceeds the band.
"""
import os
import re
import subprocess

import pytest

from paper_2012_12618_gb300 import build

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = str(tmp_path_factory.mktemp("dev") / "device_checks")
    cmd = [build.nvcc(), *build.ARCH, *build.FLAGS, os.path.join(HERE, "cuda", "device_checks.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _run(exe, *args):
    r = subprocess.run([exe, *args], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return dict(kv.split("=") for kv in r.stdout.split() if "=" in kv)


def test_row_accuracy_exhaustive(exe):
    d = _run(exe, "rows")
    assert int(d["count"]) > 2_000_000_000
    assert float(d["max_rel_sincosf"]) <= 2.0 ** -23, d
    assert int(d["table_vs_sincos_max_abs_2^-53"]) <= 4, d


def test_filter_soundness(exe):
    d = _run(exe, "filter", str(1 << 19), "128")
    assert int(d["pairs"]) > 10_000_000
    assert int(d["bad_in"]) == 0 and int(d["bad_out"]) == 0 and int(d["bound_exceeded"]) == 0, d
    assert int(d["refined_trials"]) > 1000, d  # the refinement step is exercised
