"""The fused kernel's scoring pass run on its own (GPU).

Builds tests/cuda/scoring_bench.cu, which runs the library's phase_a_tiles
(rvh_scoring.cuh, the hot loop of step a4) on one synthetic cluster per CTA
with the fused kernel's launch shape, and checks every trial's count against
a host evaluation of the same FP32 formula.  The measured rate is printed:
it is the scoring pass alone, without the other stages of the fused kernel.
"""
import os
import subprocess

import pytest

from paper_2012_12618_gb300 import build

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
FP32_PEAK_FLOP_PER_CLK_SM = 128 * 2


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = str(tmp_path_factory.mktemp("sb") / "scoring_bench")
    cmd = [build.nvcc(), *build.ARCH, *build.FLAGS, os.path.join(HERE, "cuda", "scoring_bench.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


@pytest.mark.parametrize("dim,n", [(2, 1536), (2, 257), (3, 1536), (3, 61)])
def test_scoring_pass_counts_and_rate(exe, dim, n):
    r = subprocess.run([exe, str(dim), str(n), "8"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    d = dict(kv.split("=") for kv in r.stdout.split() if "=" in kv)
    assert int(d["mismatches"]) == 0, d
    assert int(d["inliers"]) > 0, d
    # pairs/s -> FP32 fraction at the maximum SM clock (2k flop per pair)
    frac = float(d["pairs_per_s"]) * 2 * dim / (int(d["sms"]) * FP32_PEAK_FLOP_PER_CLK_SM * 2.07e9)
    print(f"scoring pass dim={dim} N={n}: {float(d['pairs_per_s']):.3e} pairs/s, FP32 fraction {frac:.3f}")
    assert frac > 0.05, d


def test_fp64_rate(tmp_path):
    """The FP64 FMA rate the design weighs FP64 work by (tests/cuda/fp64_rate.cu)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = str(tmp_path / "fp64_rate")
    cmd = [build.nvcc(), *build.ARCH, *build.FLAGS, os.path.join(HERE, "cuda", "fp64_rate.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    r = subprocess.run([out, "4096"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    d = dict(kv.split("=") for kv in r.stdout.split() if "=" in kv)
    assert d["check"] == "1", d
    print(f"FP64 FMA rate: {float(d['dfma_per_s']):.3e}/s, {float(d['dfma_per_clk_sm']):.3f} per SM per cycle "
          f"at {d['clock_mhz']} MHz")
    assert float(d["dfma_per_clk_sm"]) > 0.5, d

