"""Python access to the FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

The oracle (rvh_oracle.c) is a plain single-threaded restatement of the
paper's RANSAC + least-squares method.  Only tests/, __graft_entry__.smoke()
and the CPU-baseline leg of bench.py may import this package; the product
path (paper_2012_12618_gb300) never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rvh_oracle.c")
LIB = os.path.join(HERE, "librvh_oracle.so")

TOO_FEW_POINTS = 1
ALL_DEGENERATE = 2
LSQ_FALLBACK = 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc.  -ffp-contract=off keeps every product and
    sum rounded where the source writes it (no implicit fused multiply-add)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "rvh_oracle.h"))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class _Params(ctypes.Structure):
    _fields_ = [("model_dim", ctypes.c_int32), ("num_hypotheses", ctypes.c_int32),
                ("tau", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("cond_eps", ctypes.c_double), ("enumerate", ctypes.c_int32),
                ("refine_iterations", ctypes.c_int32), ("confidence", ctypes.c_double),
                ("trial_block", ctypes.c_int32), ("line_model", ctypes.c_int32),
                ("first_cluster", ctypes.c_int32)]


_lib = None


def load(path: str):
    """Load an oracle shared library (the built one, or a test's variant)."""
    L = ctypes.CDLL(path)
    L.oracle_philox4x32_10.restype = None
    L.oracle_draw.restype = ctypes.c_int
    L.oracle_draw.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                              ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    L.oracle_estimate.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def default_cond_eps(model_dim: int) -> float:
    return 1e-4 if model_dim == 2 else 1e-6


def philox4x32_10(ctr, key, _lib=None) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    (_lib or lib()).oracle_philox4x32_10(c.ctypes.data_as(ctypes.c_void_p), k.ctypes.data_as(ctypes.c_void_p),
                               out.ctypes.data_as(ctypes.c_void_p))
    return out


def draw(seed: int, cluster: int, h: int, n: int, k: int, _lib=None) -> np.ndarray:
    q = np.zeros(3, dtype=np.int32)
    rc = (_lib or lib()).oracle_draw(seed, cluster, h, n, k, q.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError("n < k")
    return q[:k]


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def estimate(azimuth, doppler, offsets, *, elevation=None, num_hypotheses: int, tau: float,
             seed: int, cond_eps: float | None = None, enumerate_subsets: bool = False,
             subset=None, want_counts: bool = False, want_fragile: bool = False,
             refine_iterations: int = 0, confidence: float = 0.0, trial_block: int = 128,
             want_trials: bool = False, line_model: bool = False, first_cluster: int = 0, _lib=None) -> dict:
    """Run the oracle over all clusters (or the listed subset).  Inputs are
    widened to FP64 exactly.  refine_iterations > 0 adds that many local
    optimisation rounds (re-threshold against the least-squares velocity,
    re-fit) after the refine.  confidence in (0, 1) selects the adaptive trial
    count (stopping checks every trial_block trials).  line_model selects
    Alg. 1 as printed (normalised line fits, MAD threshold; 2D; tau unused).
    first_cluster: the frame index of cluster 0 of these arrays (a shard of
    a frame draws the whole frame's minimal sets)."""
    az = np.ascontiguousarray(azimuth, dtype=np.float64)
    dp = np.ascontiguousarray(doppler, dtype=np.float64)
    el = None if elevation is None else np.ascontiguousarray(elevation, dtype=np.float64)
    off = np.ascontiguousarray(offsets, dtype=np.int32)
    nc = off.shape[0] - 1
    k = 2 if el is None else 3
    sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int32)
    n_out = nc if sub is None else sub.shape[0]
    H = int(num_hypotheses)
    p = _Params(k, H, float(tau), int(seed) & 0xFFFFFFFFFFFFFFFF,
                default_cond_eps(k) if cond_eps is None else float(cond_eps), int(enumerate_subsets),
                int(refine_iterations), float(confidence), int(trial_block), int(bool(line_model)),
                int(first_cluster))
    out = {
        "vx": np.full(n_out, np.nan), "vy": np.full(n_out, np.nan), "vz": np.full(n_out, np.nan),
        "heading": np.full(n_out, np.nan),
        "inlier_count": np.zeros(n_out, np.int32), "best_hypothesis": np.zeros(n_out, np.int32),
        "status": np.zeros(n_out, np.int32), "inlier_mask": np.zeros(dp.shape[0], np.uint8),
        "threshold": np.full(n_out, np.nan),
    }
    counts = np.zeros(n_out * H, np.int32) if want_counts else None
    fragile = np.zeros(n_out, np.uint8) if want_fragile else None
    trials = np.zeros(n_out, np.int32) if want_trials else None
    rc = (_lib or lib()).oracle_estimate(
        _p(az), _p(el), _p(dp), _p(off), ctypes.c_int32(nc), _p(sub), ctypes.c_int32(n_out),
        ctypes.byref(p), _p(out["vx"]), _p(out["vy"]), _p(out["vz"]), _p(out["heading"]),
        _p(out["inlier_count"]), _p(out["best_hypothesis"]), _p(out["status"]),
        _p(out["inlier_mask"]), _p(counts), _p(fragile), _p(trials), _p(out["threshold"]))
    if rc != 0:
        raise ValueError("oracle_estimate rejected its arguments")
    if want_counts:
        out["hyp_counts"] = counts.reshape(n_out, H)
    if want_fragile:
        out["fragile"] = fragile.astype(bool)
    if want_trials:
        out["trials_used"] = trials
    return out


def dbscan(features, eps: float, min_pts: int, _lib=None) -> dict:
    """DBSCAN of the rows of `features` ([n, dim], dim 1..4, widened to FP64
    exactly): labels (cluster ids numbered by smallest core index, -1 noise),
    core flags and the cluster count."""
    f = np.ascontiguousarray(features, dtype=np.float64)
    if f.ndim == 1:
        f = f[:, None]
    n, dim = f.shape
    labels = np.zeros(n, np.int32)
    core = np.zeros(n, np.uint8)
    nc = ctypes.c_int32(0)
    L = _lib or lib()
    L.oracle_dbscan.restype = ctypes.c_int
    rc = L.oracle_dbscan(_p(f), ctypes.c_int64(n), ctypes.c_int32(dim), ctypes.c_double(eps),
                         ctypes.c_int32(min_pts), _p(labels), _p(core), ctypes.byref(nc))
    if rc != 0:
        raise ValueError("oracle_dbscan rejected its arguments")
    return {"labels": labels, "core": core.astype(bool), "n_clusters": int(nc.value)}
