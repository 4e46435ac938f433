"""Serving load: many radars streaming frames into one context.

Each radar emits frames as a Poisson process (20 frames/s by default); each
frame holds 50..2000 clusters with sizes log-uniform in 8..2048.  Radars
0..31 use the 2D model with 256 hypotheses, 32..63 the 3D model with 2048.
Frames are submitted with rvh_submit as they arrive and completions are seen
with rvh_poll; the frame latency is arrival -> completion observed.

Frame inputs are resident in device memory (a pool of distinct frames per
model, drawn once with the seeded generator and cycled); every submission
writes its own output buffers, taken from a ring allocated before the load
starts (a slot is reused only once its earlier submission has completed),
so the driving loop allocates nothing while it measures; Python's garbage
collector is paused for the run.
"""
from __future__ import annotations

import ctypes
import dataclasses
import gc
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
    """Device-resident frames of one radar model, each with a ring of output
    buffer sets."""

    def __init__(self, spec: synth.ServingSpec, radar: int, count: int, device, ring: int = 16):
        import torch
        self.items = []
        self.rings = []
        self.next = [0] * count
        for k in range(count):
            f, w = synth.serving_frame(spec, radar, k)
            az = torch.from_numpy(f.azimuth).to(device)
            el = None if f.elevation is None else torch.from_numpy(f.elevation).to(device)
            dop = torch.from_numpy(f.doppler).to(device)
            off = torch.from_numpy(f.offsets).to(device)
            frame = rvh.make_frame(az, dop, off, el)
            params = rvh.make_params(w.model_dim, w.num_hypotheses, w.tau, synth.radar_frame_seed(radar, k))
            self.items.append((f, w, frame, params, (az, el, dop, off)))
            self.rings.append([rvh.alloc_outputs(f.n_clusters, f.n_points, device) for _ in range(ring)])

    def outputs(self, k: int, busy: set):
        """An output set of item k that no outstanding submission uses (a new
        one if the whole ring is in flight)."""
        ring = self.rings[k]
        for _ in range(len(ring)):
            j = self.next[k]
            self.next[k] = (j + 1) % len(ring)
            if id(ring[j]) not in busy:
                return ring[j]
        f = self.items[k][0]
        return rvh.alloc_outputs(f.n_clusters, f.n_points, ring[0]["vx"].device)


def run_load(ctx, spec: synth.ServingSpec, device, *, pool_frames: int = 8, seed: int = 5,
             time_scale: float = 1.0) -> ServingResult:
    """Replays the arrival schedule in real time (time_scale > 1 compresses it)."""
    import torch
    pools = {2: FramePool(spec, 0, pool_frames, device), 3: FramePool(spec, 32, pool_frames, device)}
    events = synth.arrival_schedule(spec, seed)
    outstanding = {}   # ticket -> (t_arrival, measured, n_clusters, outputs)
    busy = set()       # ids of the output sets of outstanding submissions
    lat, clusters, frames, eagain = [], 0, 0, 0
    gc.collect()
    gc.disable()
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
            busy.discard(id(outstanding[t][3]))
            del outstanding[t]

    try:
        while i < len(events) or outstanding:
            now = time.perf_counter() - t0
            if i < len(events) and events[i][0] / time_scale <= now:
                ta_rel, radar, k = events[i]
                pool = pools[2 if radar < 32 else 3]
                f, w, frame, params, _ = pool.items[k % len(pool.items)]
                outs = pool.outputs(k % len(pool.items), busy)
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
                busy.add(id(outs))
                i += 1
                continue
            reap()
            if i < len(events):
                wait = events[i][0] / time_scale - (time.perf_counter() - t0)
                if wait > 2e-4 and not outstanding:
                    time.sleep(wait - 1e-4)
    finally:
        gc.enable()
    dur = (len(events) and (events[-1][0] / time_scale - warm_end)) or 1.0
    torch.cuda.synchronize()
    return ServingResult(frames, clusters, max(dur, 1e-9), np.asarray(lat), eagain)
