"""Serving load: many radars streaming frames into one context.

Each radar emits frames as a Poisson process (20 frames/s by default); each
frame holds 50..2000 clusters with sizes log-uniform in 8..2048.  Radars
0..31 use the 2D model with 256 hypotheses, 32..63 the 3D model with 2048.
Frames are submitted with rvh_submit as they arrive and completions are seen
with rvh_poll; the frame latency is arrival -> completion observed.

Frame inputs are resident in device memory (a pool of distinct frames per
model, drawn once with the seeded generator and cycled); every submission
gets its own output buffers.
"""
from __future__ import annotations

import ctypes
import dataclasses
import time

import numpy as np

from . import rvh, synth


@dataclasses.dataclass
class ServingResult:
    frames: int
    clusters: int
    duration_s: float
    latencies_ms: np.ndarray
    eagain: int

    def summary(self) -> dict:
        lat = self.latencies_ms
        return {
            "frames": self.frames,
            "clusters_per_s": self.clusters / self.duration_s,
            "frames_per_s": self.frames / self.duration_s,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "max_ms": float(lat.max()) if lat.size else None,
            "eagain_retries": self.eagain,
        }


class FramePool:
    """Device-resident frames of one radar model."""

    def __init__(self, spec: synth.ServingSpec, radar: int, count: int, device):
        import torch
        self.items = []
        for k in range(count):
            f, w = synth.serving_frame(spec, radar, k)
            az = torch.from_numpy(f.azimuth).to(device)
            el = None if f.elevation is None else torch.from_numpy(f.elevation).to(device)
            dop = torch.from_numpy(f.doppler).to(device)
            off = torch.from_numpy(f.offsets).to(device)
            frame = rvh.make_frame(az, dop, off, el)
            params = rvh.make_params(w.model_dim, w.num_hypotheses, w.tau, synth.radar_frame_seed(radar, k))
            self.items.append((f, w, frame, params, (az, el, dop, off)))


def run_load(ctx, spec: synth.ServingSpec, device, *, pool_frames: int = 8, seed: int = 5,
             time_scale: float = 1.0) -> ServingResult:
    """Replays the arrival schedule in real time (time_scale > 1 compresses it)."""
    import torch
    pools = {2: FramePool(spec, 0, pool_frames, device), 3: FramePool(spec, 32, pool_frames, device)}
    events = synth.arrival_schedule(spec, seed)
    outstanding = {}   # ticket -> (t_arrival, measured, n_clusters, outputs)
    lat, clusters, frames, eagain = [], 0, 0, 0
    t0 = time.perf_counter()
    warm_end = spec.warmup_s / time_scale
    i = 0

    def reap():
        nonlocal clusters, frames
        now = time.perf_counter()
        done = []
        for t, (ta, meas, nc, _) in outstanding.items():
            rc = rvh.rvh_poll(ctx.handle, t)
            if rc == rvh.RVH_OK:
                done.append(t)
                if meas:
                    lat.append((now - ta) * 1e3)
                    clusters += nc
                    frames += 1
            elif rc != rvh.RVH_PENDING:
                raise RuntimeError(f"rvh_poll failed ({rc}): {rvh.rvh_last_error(None)}")
        for t in done:
            del outstanding[t]

    while i < len(events) or outstanding:
        now = time.perf_counter() - t0
        if i < len(events) and events[i][0] / time_scale <= now:
            ta_rel, radar, k = events[i]
            pool = pools[2 if radar < 32 else 3]
            f, w, frame, params, _ = pool.items[k % len(pool.items)]
            outs = rvh.alloc_outputs(f.n_clusters, f.n_points, device)
            params = rvh.make_params(w.model_dim, w.num_hypotheses, w.tau, synth.radar_frame_seed(radar, k))
            ticket = ctypes.c_uint64(0)
            while True:
                rc = rvh.rvh_submit(ctx.handle, frame, params, rvh.make_result(outs), ticket)
                if rc == rvh.RVH_OK:
                    break
                if rc != rvh.RVH_EAGAIN:
                    raise RuntimeError(f"rvh_submit failed ({rc}): {rvh.rvh_last_error(None)}")
                eagain += 1
                reap()
            measured = ta_rel / time_scale >= warm_end
            outstanding[ticket.value] = (t0 + ta_rel / time_scale, measured, f.n_clusters, outs)
            i += 1
            continue
        reap()
        if i < len(events):
            wait = events[i][0] / time_scale - (time.perf_counter() - t0)
            if wait > 2e-4 and not outstanding:
                time.sleep(wait - 1e-4)
    dur = (len(events) and (events[-1][0] / time_scale - warm_end)) or 1.0
    torch.cuda.synchronize()
    return ServingResult(frames, clusters, max(dur, 1e-9), np.asarray(lat), eagain)
