"""Helpers for the GPU tests: run the library on a frame, compare with the oracle."""
from __future__ import annotations

import ctypes
import math
import os

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


# ---- the oracle over many host cores: spawned processes (never forked: a fork
# after the first CUDA call can hang), each running the unmodified oracle on a
# contiguous, cost-balanced share of the requested clusters
_POOL_FRAME = None


def _pool_init(frame):
    global _POOL_FRAME
    oracle.lib()
    _POOL_FRAME = frame


def _pool_run(args):
    clusters, kw = args
    az, dop, off, el = _POOL_FRAME
    o = oracle.estimate(az, dop, off, elevation=el, subset=clusters, want_fragile=True, **kw)
    pts = np.concatenate([np.arange(off[c], off[c + 1]) for c in clusters]) if len(clusters) else np.zeros(0, int)
    o["inlier_mask"] = o["inlier_mask"][pts]
    return clusters, pts, o


def run_oracle_parallel(az, dop, off, *, el=None, H: int, tau: float, seed: int, subset=None,
                        processes: int | None = None, **kw) -> dict:
    """run_oracle over (a sorted subset of) a frame on all host cores; the
    result has run_oracle's layout (per-cluster arrays in subset order, the
    mask over the whole frame)."""
    import multiprocessing as mp
    off = np.asarray(off)
    nc = off.shape[0] - 1
    idx = np.arange(nc, dtype=np.int32) if subset is None else np.asarray(subset, dtype=np.int32)
    assert np.all(np.diff(idx) > 0), "subset must be sorted and distinct"
    procs = processes or min(len(os.sched_getaffinity(0)), 32)
    cost = (np.diff(off)[idx].astype(np.int64) + 64) * int(H)
    cum = np.cumsum(cost)
    parts = max(1, min(len(idx), 4 * procs))
    cuts = np.searchsorted(cum, cum[-1] * np.arange(1, parts) / parts) if len(idx) else []
    chunks = [c for c in np.split(idx, cuts) if len(c)]
    okw = dict(num_hypotheses=H, tau=tau, seed=seed, **kw)
    frame = (np.ascontiguousarray(az), np.ascontiguousarray(dop), off, None if el is None else np.ascontiguousarray(el))
    with mp.get_context("spawn").Pool(procs, initializer=_pool_init, initargs=(frame,)) as pool:
        parts_out = pool.map(_pool_run, [(c, okw) for c in chunks], chunksize=1)
    out = {"inlier_mask": np.zeros(np.asarray(dop).shape[0], np.uint8)}
    per = {}
    for clusters, pts, o in parts_out:
        out["inlier_mask"][pts] = o["inlier_mask"]
        for k, v in o.items():
            if k != "inlier_mask":
                per.setdefault(k, []).append(v)
    for k, v in per.items():
        out[k] = np.concatenate(v)
    return out


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


# One line per parity comparison of the session: printed in pytest's terminal
# summary (tests/conftest.py), so a GPU log shows how many clusters were
# compared, how many the oracle flagged fragile and how many tied.
PARITY_LOG: list[str] = []


def check_parity(rep: dict, *, tau: float, label: str = "") -> None:
    """The parity bar of every cosine-model comparison: no mismatch at all,
    and with tau > 0 no rounding tie either (every mask entry, count and
    winner bit-exact).  Only tau = 0, where every inlier decision is an
    exact-zero residual test that the last ulp of cos/sin decides, accepts
    ties on clusters the oracle flags as fragile."""
    tie_clusters = sorted({t[0] for t in rep["ties"]})
    if not label:
        label = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    PARITY_LOG.append(f"{label}: tau={tau:g} clusters={rep['clusters']} oracle_fragile={rep['fragile']} "
                      f"mismatches={len(rep['mismatch'])} tie_clusters={len(tie_clusters)}")
    assert not rep["mismatch"], rep["mismatch"][:20]
    if tau > 0:
        assert not rep["ties"], rep["ties"][:20]
