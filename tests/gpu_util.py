"""Helpers for the GPU tests: run the library on a frame, compare with the oracle."""
from __future__ import annotations

import ctypes
import math

import numpy as np

import oracle

OUT_KEYS = ("vx", "vy", "vz", "heading", "inlier_count", "best_hypothesis", "status", "inlier_mask")


def torch_mod():
    import torch
    return torch


def alloc_outputs(n_clusters: int, n_points: int, device: str):
    from paper_2012_12618_gb300 import rvh
    return rvh.alloc_outputs(n_clusters, n_points, device)


def run_rvh(ctx, az, dop, off, *, el=None, H: int, tau: float, seed: int, cond_eps: float = 0.0,
            baseline: bool = False, device: str = "cuda", stream=None, refine_iterations: int = 0,
            confidence: float = 0.0, trial_block: int = 0, line_model: bool = False) -> dict:
    """Runs rvh_estimate (or the baseline) through the C ABI and returns numpy outputs."""
    torch = torch_mod()
    from paper_2012_12618_gb300 import rvh

    def t(a, dt):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(device)

    taz, tdop, toff = t(az, torch.float32), t(dop, torch.float32), t(off, torch.int32)
    tel = None if el is None else t(el, torch.float32)
    n_points = int(np.asarray(az).shape[0])
    outs = alloc_outputs(int(np.asarray(off).shape[0]) - 1, n_points, device)
    frame = rvh.make_frame(taz, tdop, toff, tel)
    params = rvh.make_params(3 if el is not None else 2, H, tau, seed, cond_eps,
                             refine_iterations=refine_iterations, confidence=confidence,
                             trial_block=trial_block, hypothesis_model=1 if line_model else 0)
    res = rvh.make_result(outs)
    fn = rvh.rvh_estimate_baseline if baseline else rvh.rvh_estimate
    rc = fn(ctx.handle, frame, params, res, stream)
    if rc != rvh.RVH_OK:
        raise RuntimeError(f"rvh returned {rc}: {rvh.rvh_last_error(None)}")
    if device.startswith("cuda"):
        torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in outs.items()}
    out["inlier_mask"] = out["inlier_mask"][:n_points]
    return out


def run_oracle(az, dop, off, *, el=None, H: int, tau: float, seed: int, cond_eps=None, subset=None,
               refine_iterations: int = 0, confidence: float = 0.0, trial_block: int = 128,
               want_trials: bool = False, line_model: bool = False) -> dict:
    return oracle.estimate(az, dop, off, elevation=el, num_hypotheses=H, tau=tau, seed=seed,
                           cond_eps=cond_eps, subset=subset, want_fragile=True,
                           refine_iterations=refine_iterations, confidence=confidence,
                           trial_block=trial_block, want_trials=want_trials, line_model=line_model)


def compare(gpu: dict, orc: dict, off, *, subset=None, vel_tol: float = 1e-6, head_tol: float = 1e-6) -> dict:
    """Element-wise comparison.  Masks, counts, winners and status are bit-exact;
    velocities within vel_tol m/s; headings (wrapped) within head_tol rad where
    |v| >= 1e-3 m/s.  Disagreements on clusters the oracle flags as fragile (a
    decision within rounding distance of its threshold) are listed as ties."""
    off = np.asarray(off)
    nc = off.shape[0] - 1
    idx = np.arange(nc) if subset is None else np.asarray(subset)
    frag = orc["fragile"]
    report = {"clusters": int(idx.shape[0]), "fragile": int(frag.sum()), "mismatch": [], "ties": []}
    for k_out, ci in enumerate(idx):
        s, e = off[ci], off[ci + 1]
        bad = []
        for key in ("inlier_count", "best_hypothesis", "status"):
            if gpu[key][ci] != orc[key][k_out]:
                bad.append((int(ci), key, int(gpu[key][ci]), int(orc[key][k_out])))
        if not np.array_equal(gpu["inlier_mask"][s:e], orc["inlier_mask"][s:e]):
            bad.append((int(ci), "inlier_mask", None, None))
        for key in ("vx", "vy", "vz"):
            g, o = gpu[key][ci], orc[key][k_out]
            if np.isnan(o) != np.isnan(g) or (not np.isnan(o) and abs(g - o) > vel_tol):
                bad.append((int(ci), key, float(g), float(o)))
        if not np.isnan(orc["vx"][k_out]) and math.hypot(orc["vx"][k_out], orc["vy"][k_out]) >= 1e-3:
            d = (gpu["heading"][ci] - orc["heading"][k_out] + math.pi) % (2 * math.pi) - math.pi
            if abs(d) > head_tol:
                bad.append((int(ci), "heading", float(gpu["heading"][ci]), float(orc["heading"][k_out])))
        # a disagreement on a cluster whose oracle run logged a decision within
        # rounding distance of its threshold is a rounding tie, reported apart
        report["ties" if frag[k_out] else "mismatch"].extend(bad)
    return report
