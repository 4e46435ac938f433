"""Python binding of the rvh C ABI (include/rvh.h): ctypes marshalling only.

Every function named like the C entry point takes the same arguments and
returns the C return code; all computation happens in librvh.so.  Buffers are
torch tensors (host or CUDA) or numpy arrays, passed by pointer.  There is no
fallback: if the CUDA library is missing or cannot be loaded, the first call
raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

RVH_OK = 0
RVH_MODEL_VELOCITY_PROFILE = 0
RVH_MODEL_PAPER_LINE = 1
RVH_PENDING = 1
RVH_EINVAL = -1
RVH_ENOMEM = -2
RVH_EAGAIN = -3
RVH_ECUDA = -4
RVH_ETIMEDOUT = -5

RVH_STATUS_TOO_FEW_POINTS = 1
RVH_STATUS_ALL_DEGENERATE = 2
RVH_STATUS_LSQ_FALLBACK = 4
RVH_STATUS_BAD_OFFSETS = 8

RVH_NOALLOC_MAX_POINTS = 1048576
RVH_NOALLOC_MAX_CLUSTERS = 65536


class rvh_frame(ctypes.Structure):
    _fields_ = [("azimuth", ctypes.c_void_p), ("elevation", ctypes.c_void_p), ("doppler", ctypes.c_void_p),
                ("cluster_offsets", ctypes.c_void_p), ("n_clusters", ctypes.c_int32),
                ("n_points", ctypes.c_int64)]


class rvh_params(ctypes.Structure):
    _fields_ = [("model_dim", ctypes.c_int32), ("num_hypotheses", ctypes.c_int32),
                ("inlier_threshold", ctypes.c_double), ("seed", ctypes.c_uint64), ("cond_eps", ctypes.c_double),
                ("first_cluster", ctypes.c_int32), ("refine_iterations", ctypes.c_int32),
                ("confidence", ctypes.c_double), ("trial_block", ctypes.c_int32),
                ("hypothesis_model", ctypes.c_int32)]


class rvh_result(ctypes.Structure):
    _fields_ = [("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p), ("vz", ctypes.c_void_p),
                ("heading", ctypes.c_void_p), ("inlier_count", ctypes.c_void_p),
                ("best_hypothesis", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("inlier_mask", ctypes.c_void_p), ("threshold", ctypes.c_void_p)]


class rvh_schedule(ctypes.Structure):
    _fields_ = [("points_per_warp", ctypes.c_int32), ("hyps_per_lane", ctypes.c_int32),
                ("kernel_ms", ctypes.c_float)]


class rvh_stats(ctypes.Structure):
    _fields_ = [("hypotheses", ctypes.c_int64), ("pair_evals", ctypes.c_int64), ("candidates", ctypes.c_int64),
                ("band_points", ctypes.c_int64), ("fp64_hypotheses", ctypes.c_int64),
                ("kernel_ms", ctypes.c_float), ("grid", ctypes.c_int32), ("points_per_warp", ctypes.c_int32),
                ("hyps_per_lane", ctypes.c_int32), ("phase_cycles", ctypes.c_int64 * 6),
                ("refined_hypotheses", ctypes.c_int64), ("graph_replays", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int32), ("graph_builds", ctypes.c_int64),
                ("serving_steps", ctypes.c_int64), ("serving_graph_replays", ctypes.c_int64),
                ("pairs_scored", ctypes.c_int64)]


# exported symbols and their ctypes signatures (restype, argtypes)
_P = ctypes.c_void_p
SIGNATURES = {
    "rvh_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_size_t]),
    "rvh_destroy": (None, [_P]),
    "rvh_estimate": (ctypes.c_int, [_P, ctypes.POINTER(rvh_frame), ctypes.POINTER(rvh_params),
                                    ctypes.POINTER(rvh_result), _P]),
    "rvh_estimate_baseline": (ctypes.c_int, [_P, ctypes.POINTER(rvh_frame), ctypes.POINTER(rvh_params),
                                             ctypes.POINTER(rvh_result), _P]),
    "rvh_estimate_noalloc": (ctypes.c_int, [ctypes.POINTER(rvh_frame), ctypes.POINTER(rvh_params),
                                            ctypes.POINTER(rvh_result), _P]),
    "rvh_submit": (ctypes.c_int, [_P, ctypes.POINTER(rvh_frame), ctypes.POINTER(rvh_params),
                                  ctypes.POINTER(rvh_result), ctypes.POINTER(ctypes.c_uint64)]),
    "rvh_poll": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "rvh_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int64]),
    "rvh_last_error": (ctypes.c_char_p, [_P]),
    "rvh_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(rvh_stats)]),
    "rvh_set_schedule": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "rvh_set_pruning": (ctypes.c_int, [_P, ctypes.c_int32]),
    "rvh_autotune": (ctypes.c_int, [_P, ctypes.POINTER(rvh_frame), ctypes.POINTER(rvh_params),
                                    ctypes.POINTER(rvh_result), ctypes.c_int32, ctypes.POINTER(rvh_schedule)]),
    "rvh_cluster": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                   _P, _P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _P]),
    "rvh_gather": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P]),
}

_lib = None


def load(path: str | None = None, build_if_missing: bool = True):
    """Loads librvh.so (building it in-tree with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    if path is None:
        path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"rvh CUDA library not found at {path}")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    if path == _build.LIB:
        _lib = L
    return L


def rvh_create(out, device: int = 0, mem_budget_bytes: int = 0) -> int:
    return load().rvh_create(out, device, mem_budget_bytes)


def rvh_destroy(ctx) -> None:
    load().rvh_destroy(ctx)


def rvh_estimate(ctx, frame, params, result, stream=None) -> int:
    return load().rvh_estimate(ctx, ctypes.byref(frame), ctypes.byref(params), ctypes.byref(result), stream)


def rvh_estimate_baseline(ctx, frame, params, result, stream=None) -> int:
    return load().rvh_estimate_baseline(ctx, ctypes.byref(frame), ctypes.byref(params), ctypes.byref(result),
                                        stream)


def rvh_estimate_noalloc(frame, params, result, stream=None) -> int:
    return load().rvh_estimate_noalloc(ctypes.byref(frame), ctypes.byref(params), ctypes.byref(result), stream)


def rvh_submit(ctx, frame, params, result, ticket) -> int:
    return load().rvh_submit(ctx, ctypes.byref(frame), ctypes.byref(params), ctypes.byref(result),
                             ctypes.byref(ticket))


def rvh_poll(ctx, ticket: int) -> int:
    return load().rvh_poll(ctx, ticket)


def rvh_wait(ctx, ticket: int, timeout_us: int) -> int:
    return load().rvh_wait(ctx, ticket, timeout_us)


def rvh_last_error(ctx=None) -> str:
    return load().rvh_last_error(ctx).decode()


def rvh_get_stats(ctx, out) -> int:
    return load().rvh_get_stats(ctx, ctypes.byref(out))


def rvh_set_schedule(ctx, points_per_warp: int, hyps_per_lane: int) -> int:
    return load().rvh_set_schedule(ctx, points_per_warp, hyps_per_lane)


def rvh_set_pruning(ctx, enabled: int) -> int:
    return load().rvh_set_pruning(ctx, enabled)


def rvh_autotune(ctx, frame, params, result, reps: int, best) -> int:
    return load().rvh_autotune(ctx, ctypes.byref(frame), ctypes.byref(params), ctypes.byref(result), reps,
                               None if best is None else ctypes.byref(best))


def rvh_cluster(ctx, features, n_points: int, dim: int, eps: float, min_pts: int, labels, perm, offsets,
                max_clusters: int, n_clusters, stream=None) -> int:
    return load().rvh_cluster(ctx, ptr(features), n_points, dim, eps, min_pts, ptr(labels), ptr(perm),
                              ptr(offsets), max_clusters, ctypes.byref(n_clusters), stream)


def rvh_gather(ctx, perm, m: int, src0, dst0, src1=None, dst1=None, src2=None, dst2=None, stream=None) -> int:
    return load().rvh_gather(ctx, ptr(perm), m, ptr(src0), ptr(dst0), ptr(src1), ptr(dst1), ptr(src2),
                             ptr(dst2), stream)


# ---- marshalling helpers ---------------------------------------------------------------

def ptr(buf) -> int | None:
    """Address of a torch tensor or numpy array (None passes through)."""
    if buf is None:
        return None
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("buffers must be contiguous")
        return buf.data_ptr()
    return buf.ctypes.data


def make_frame(azimuth, doppler, offsets, elevation=None) -> rvh_frame:
    n_points = int(azimuth.shape[0])
    return rvh_frame(ptr(azimuth), ptr(elevation), ptr(doppler), ptr(offsets), int(offsets.shape[0]) - 1, n_points)


def make_params(model_dim: int, num_hypotheses: int, inlier_threshold: float, seed: int,
                cond_eps: float = 0.0, first_cluster: int = 0, refine_iterations: int = 0,
                confidence: float = 0.0, trial_block: int = 0, hypothesis_model: int = 0) -> rvh_params:
    return rvh_params(model_dim, num_hypotheses, inlier_threshold, seed & 0xFFFFFFFFFFFFFFFF, cond_eps,
                      first_cluster, refine_iterations, confidence, trial_block, hypothesis_model)


def make_result(out: dict) -> rvh_result:
    return rvh_result(ptr(out["vx"]), ptr(out["vy"]), ptr(out.get("vz")), ptr(out["heading"]),
                      ptr(out["inlier_count"]), ptr(out["best_hypothesis"]), ptr(out["status"]),
                      ptr(out["inlier_mask"]), ptr(out.get("threshold")))


def alloc_outputs(n_clusters: int, n_points: int, device="cuda", threshold: bool = False) -> dict:
    """Result buffers as torch tensors on `device` ("cpu" gives host memory);
    threshold=True adds the optional per-cluster threshold output."""
    import torch
    kw = dict(device=device)
    out = {
        "vx": torch.empty(n_clusters, dtype=torch.float64, **kw),
        "vy": torch.empty(n_clusters, dtype=torch.float64, **kw),
        "vz": torch.empty(n_clusters, dtype=torch.float64, **kw),
        "heading": torch.empty(n_clusters, dtype=torch.float64, **kw),
        "inlier_count": torch.empty(n_clusters, dtype=torch.int32, **kw),
        "best_hypothesis": torch.empty(n_clusters, dtype=torch.int32, **kw),
        "status": torch.empty(n_clusters, dtype=torch.int32, **kw),
        "inlier_mask": torch.empty(max(n_points, 1), dtype=torch.uint8, **kw),
    }
    if threshold:
        out["threshold"] = torch.empty(n_clusters, dtype=torch.float64, **kw)
    return out


class Context:
    """Owns an rvh context; `check` turns return codes into exceptions."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self.handle = ctypes.c_void_p()
        self.check(rvh_create(ctypes.byref(self.handle), device, mem_budget_bytes), "rvh_create")

    def check(self, rc: int, what: str) -> int:
        if rc not in (RVH_OK, RVH_PENDING):
            raise RuntimeError(f"{what} failed ({rc}): {rvh_last_error(None)}")
        return rc

    def close(self):
        if self.handle:
            rvh_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
