"""Throughput of the fused RANSAC + LSQ path on the dense 2D traffic frame.

One step = one rvh_estimate over a whole frame: 4096 clusters with sizes
log-uniform in 8..2048 (1.53 M points), 2D model, 1024 hypotheses per
cluster, tau = 0.1 m/s.  Inputs are resident in device memory; between
timed steps the L2 is flushed (a 256 MiB write), outside the step's events.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead (each step: a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "dense2d"
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM (Blackwell)
SM_MAX_MHZ_FALLBACK = 2070.0
KERNEL_SOURCES = ["rvh_fused.cu", "rvh_scoring.cuh", "rvh_device.cuh", "rvh_kernels.h"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2012_12618_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per fused launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "fused_dense2d_traffic.txt")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("kernel_hash") != kernel_hash():
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """SM clocks and throttle reasons during the timed region.

    NVML (libnvidia-ml, read-only queries) is polled every millisecond from a
    thread, so even a timed region of a few milliseconds gets samples; a
    streaming nvidia-smi process (100 ms) runs beside it, and one nvidia-smi
    query is taken right before and right after the region.  Nothing here
    changes a GPU setting."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # nvmlClocksEventReasons bits
    NVML_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, index: int):
        self.index = index
        self.samples = []        # nvidia-smi rows
        self.nvml = []           # (sm MHz, reason bits)
        self.edges = []          # nvidia-smi rows at entry and exit
        self.nvml_max = None
        self._stop = threading.Event()
        self._t = None
        self._tn = None
        self._p = None

    def _query_once(self):
        try:
            out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
            line = out.stdout.strip().splitlines()[0] if out.stdout.strip() else ""
            if line:
                self.edges.append([x.strip() for x in line.split(",")])
        except (OSError, subprocess.SubprocessError, IndexError):
            pass

    def _run(self):
        for line in self._p.stdout:
            if self._stop.is_set():
                break
            line = line.strip()
            if line:
                self.samples.append([x.strip() for x in line.split(",")])

    def _nvml_open(self):
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0:
                return None
            mx = ctypes.c_uint(0)
            if lib.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
                self.nvml_max = float(mx.value)
            return lib, h
        except (OSError, AttributeError):
            return None

    def _run_nvml(self, lib, h):
        clk, rs = ctypes.c_uint(0), ctypes.c_ulonglong(0)
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        while not self._stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, ctypes.c_int(1), ctypes.byref(clk)) == 0 and \
                    get_reasons(h, ctypes.byref(rs)) == 0:
                self.nvml.append((float(clk.value), int(rs.value)))
            time.sleep(0.001)

    def __enter__(self):
        self._query_once()
        try:
            self._p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                        "--format=csv,noheader,nounits", "-lms", "100"],
                                       stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        except OSError:
            self._p = None
        nv = self._nvml_open()
        if nv:
            self._tn = threading.Thread(target=self._run_nvml, args=nv, daemon=True)
            self._tn.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._tn is not None:
            self._tn.join(timeout=5)
        if self._p is not None:
            self._p.terminate()
            try:
                self._p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._p.kill()
                self._p.wait(timeout=5)
            self._t.join(timeout=10)
        self._query_once()

    def summary(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

        def smi(rows):
            sm = [float(r[0]) for r in rows if r and r[0].replace(".", "").isdigit()]
            mx = [float(r[1]) for r in rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
            rs = {names[i] for r in rows for i in range(4) if len(r) > 4 + i and r[4 + i].lower().startswith("active")}
            return sm, mx, rs

        sm_s, mx_s, rs_s = smi(self.samples)
        sm_e, mx_e, rs_e = smi(self.edges)
        sm_n = [c for c, _ in self.nvml]
        rs_n = {name for _, bits in self.nvml for bit, name in self.NVML_REASONS.items() if bits & bit}
        during = sm_n or sm_s
        sm = during or sm_e
        mx = ([self.nvml_max] if self.nvml_max else []) + mx_s + mx_e
        reasons = sorted(rs_n | rs_s | (rs_e if not during else set()))
        if not sm:
            reasons = ["unsampled"]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.nvml) + len(self.samples),
                "nvml_samples": len(self.nvml), "smi_samples": len(self.samples),
                "sm_mhz_min": min(sm) if sm else None,
                "edge_samples_mhz": sm_e, "source": "nvml 1 ms" if sm_n else ("nvidia-smi 100 ms" if sm_s else "entry/exit")}


# ---- the oracle over all host cores: one spawned process per core, each
# running the unmodified oracle on contiguous cluster ranges of the frame
_ORACLE_FRAME = None


def _oracle_init(frame):
    global _ORACLE_FRAME
    import oracle
    oracle.lib()
    _ORACLE_FRAME = frame


def _oracle_range(c0c1):
    import oracle
    az, dop, off, el, H, tau, seed = _ORACLE_FRAME
    oracle.estimate(az, dop, off, elevation=el, num_hypotheses=H, tau=tau, seed=seed,
                    subset=np.arange(c0c1[0], c0c1[1], dtype=np.int32))
    return c0c1[1] - c0c1[0]


def oracle_all_cores(f, w, wname):
    import multiprocessing as mp
    from paper_2012_12618_gb300 import partition
    cores = len(os.sched_getaffinity(0))
    ranges = [r for r in partition.balanced_ranges(f.offsets, w.num_hypotheses, 8 * cores) if r[1] > r[0]]
    frame = (f.azimuth, f.doppler, f.offsets, f.elevation, w.num_hypotheses, w.tau, w.seed)
    with mp.get_context("spawn").Pool(cores, initializer=_oracle_init, initargs=(frame,)) as pool:
        pool.map(_oracle_range, [(0, 1)] * cores)  # every worker up, oracle loaded
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_range, ranges, chunksize=1))
        dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "clusters/s", "cores": cores, "kind": "oracle",
            "sample": f"the whole {wname} frame ({done} clusters), one process per core over "
                      f"{len(ranges)} cost-balanced contiguous cluster ranges", "seconds": dt}


def measure_workload(ctx, name, dev, stream, sptr, flush, steps, sms, max_mhz):
    """One single-frame workload timed like the headline one: autotuned
    schedule, device-resident inputs, L2 flushed between steps (outside the
    events), CUDA events around each estimate and the library's own events
    around the fused kernel."""
    import torch
    from paper_2012_12618_gb300 import rvh, synth
    w = synth.WORKLOADS[name]
    f = synth.make_frame(w)
    nc, npts, dim = f.n_clusters, f.n_points, w.model_dim
    pairs = int(np.diff(f.offsets).astype(np.int64).sum()) * w.num_hypotheses
    ins = [None if a is None else torch.from_numpy(a).to(dev) for a in (f.azimuth, f.doppler, f.offsets, f.elevation)]
    frame = rvh.make_frame(*ins)
    params = rvh.make_params(dim, w.num_hypotheses, w.tau, w.seed)
    outs = rvh.alloc_outputs(nc, npts, dev)
    res = rvh.make_result(outs)
    tuned = rvh.rvh_schedule()
    ctx.check(rvh.rvh_autotune(ctx.handle, frame, params, res, 5, tuned), "rvh_autotune")
    stats = rvh.rvh_stats()
    for _ in range(3):
        flush.fill_(2)
        ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, res, sptr), "rvh_estimate")
    torch.cuda.synchronize()
    step_ms, kern_ms, phase, band, scored = [], [], np.zeros(6), 0, 0
    with ClockSampler(dev.index or 0) as clk:
        for i in range(steps):
            flush.fill_(np.uint8(i & 0xFF))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, res, sptr), "rvh_estimate")
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            ctx.check(rvh.rvh_get_stats(ctx.handle, stats), "rvh_get_stats")
            kern_ms.append(stats.kernel_ms)
            phase += np.array(list(stats.phase_cycles), dtype=np.float64)
            band += stats.band_points
            scored += stats.pairs_scored
    ck = clk.summary()
    k_s = float(np.mean(kern_ms)) * 1e-3
    t_s = float(np.mean(step_ms)) * 1e-3
    # the roofline counts the (trial, point) pairs the scoring pass evaluated:
    # with exact pruning, fewer than the method's N x H
    scored_per_step = scored / max(steps, 1)
    flops = 2.0 * dim * scored_per_step
    peak = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    ach = flops / k_s / 1e12
    share = float(phase[2] / max(phase.sum(), 1.0))
    at_clk = (sms * FP32_LANES_PER_SM * 2 * ck["sm_mhz"] * 1e6 / 1e12) if ck.get("sm_mhz") else None
    out = {"workload": f"{name}: {nc} clusters, sizes {w.size_law} {w.size_lo}..{w.size_hi}, {npts} points, "
                       f"{dim}D, H={w.num_hypotheses}, tau={w.tau} m/s, outliers {w.outlier_frac:g}, "
                       f"noise {w.noise_sigma:g} m/s",
           "steps": steps, "ms_per_step": t_s * 1e3, "kernel_ms": k_s * 1e3, "clusters_per_s": nc / t_s,
           "pair_evals_per_s": pairs / t_s, "pairs_scored_fraction": scored_per_step / pairs,
           "roofline_achieved_tflops": ach, "roofline_frac": ach / peak,
           "roofline_frac_full_pairs": 2.0 * dim * pairs / k_s / 1e12 / peak,
           "roofline_frac_at_measured_clock": ach / at_clk if at_clk else None,
           "scoring_loop_frac": (flops / (share * k_s) / 1e12) / peak if share > 0 else None,
           "scoring_stage_share": share, "fp64_band_decisions_per_step": band / max(steps, 1),
           "schedule": [tuned.points_per_warp, tuned.hyps_per_lane], "grid": stats.grid, "clocks": ck,
           "stage_share": dict(zip(["rows", "hypotheses", "scoring", "exact_rescoring", "mask_refine", "other"],
                                   [round(float(x), 4) for x in phase / max(phase.sum(), 1.0)]))}
    if nc <= 256:
        out["us_per_frame"] = t_s * 1e6
    return out


def measure_clustering(ctx, dev, stream, sptr, flush, steps):
    """DBSCAN of the unclustered traffic scene, then the pipeline cluster ->
    gather -> estimate (2D, H = 1024, tau = 0.1 m/s), timed with CUDA events
    on the stream: 3 warm-up calls, then `steps` timed ones."""
    import torch
    from paper_2012_12618_gb300 import rvh, synth
    w = synth.WORKLOADS["dense2d"]
    sc = synth.SCENES["scene"]
    scene = synth.make_scene(sc)
    n_s = scene.n_points
    d_feat = torch.from_numpy(scene.features().reshape(-1).copy()).to(dev)
    s_az, s_dop = torch.from_numpy(scene.azimuth).to(dev), torch.from_numpy(scene.doppler).to(dev)
    c_lab = torch.empty(n_s, dtype=torch.int32, device=dev)
    c_perm = torch.empty(n_s, dtype=torch.int32, device=dev)
    c_off = torch.empty(n_s + 1, dtype=torch.int32, device=dev)
    g_az = torch.empty(n_s, dtype=torch.float32, device=dev)
    g_dop = torch.empty(n_s, dtype=torch.float32, device=dev)
    ncl = ctypes.c_int32(0)
    # one call sizes the result buffers, reused by every step (stable addresses)
    ctx.check(rvh.rvh_cluster(ctx.handle, d_feat, n_s, 2, sc.eps, sc.min_pts, c_lab, c_perm, c_off, n_s, ncl,
                              sptr), "rvh_cluster")
    m_s = int(c_off[ncl.value].item())  # clustered points: the same every step (deterministic)
    cl_outs = rvh.alloc_outputs(ncl.value, m_s, dev)
    cl_frame = rvh.make_frame(g_az[:m_s], g_dop[:m_s], c_off[:ncl.value + 1])
    cl_params = rvh.make_params(2, w.num_hypotheses, w.tau, w.seed)
    cl_res = rvh.make_result(cl_outs)
    cl_ms, ga_ms, es_ms, pipe_ms = [], [], [], []
    for i in range(3 + steps):
        flush.fill_(8)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        ctx.check(rvh.rvh_cluster(ctx.handle, d_feat, n_s, 2, sc.eps, sc.min_pts, c_lab, c_perm, c_off, n_s, ncl,
                                  sptr), "rvh_cluster")
        ev[1].record(stream)
        ctx.check(rvh.rvh_gather(ctx.handle, c_perm, m_s, s_az, g_az, s_dop, g_dop, stream=sptr), "rvh_gather")
        ev[2].record(stream)
        ctx.check(rvh.rvh_estimate(ctx.handle, cl_frame, cl_params, cl_res, sptr), "rvh_estimate(scene)")
        ev[3].record(stream)
        ev[3].synchronize()
        if i >= 3:
            cl_ms.append(ev[0].elapsed_time(ev[1]))
            ga_ms.append(ev[1].elapsed_time(ev[2]))
            es_ms.append(ev[2].elapsed_time(ev[3]))
            pipe_ms.append(ev[0].elapsed_time(ev[3]))
    ck, pk = float(np.mean(cl_ms)), float(np.mean(pipe_ms))
    return {"workload": f"scene: {sc.n_objects} objects, {n_s} points (x, y features), eps {sc.eps} m, "
                        f"min_pts {sc.min_pts}; estimate H={w.num_hypotheses}, tau={w.tau}",
            "n_clusters": int(ncl.value), "clustered_points": m_s,
            "dbscan_ms": ck, "dbscan_points_per_s": n_s / (ck * 1e-3),
            "gather_ms": float(np.mean(ga_ms)), "estimate_ms": float(np.mean(es_ms)),
            "pipeline_ms": pk, "pipeline_clusters_per_s": ncl.value / (pk * 1e-3),
            "note": "CUDA events on the stream; rvh_cluster reads its cluster count back (one sync)",
            "steps": steps}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reference_arm(args):
    """The FP64 CPU oracle, as it stands, on the host cores: each step
    estimates a bounded sample of the workload's clusters."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2012_12618_gb300 import synth
    w = synth.WORKLOADS[WORKLOAD]
    f = synth.make_frame(w)
    n_sample = 256
    rng = np.random.default_rng(0)
    times = []
    for step in range(args.warmup + args.steps):
        sub = np.sort(rng.choice(f.n_clusters, n_sample, replace=False))
        t0 = time.perf_counter()
        oracle.estimate(f.azimuth, f.doppler, f.offsets, num_hypotheses=w.num_hypotheses, tau=w.tau,
                        seed=w.seed, subset=sub)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = n_sample * len(times) / total
    line = {
        "impl": "reference", "metric": "clusters/s", "value": value, "unit": "clusters/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: {w.n_clusters} clusters, sizes log-uniform 8..2048, 2D, "
                               f"H={w.num_hypotheses}, tau={w.tau}", "sample_clusters_per_step": n_sample},
        "cpu_baseline": {"value": value, "unit": "clusters/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n_sample} random clusters of the {WORKLOAD} frame per step"},
        "e2e": {"value": value, "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="rvh", choices=["rvh", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=["frame64", "dense2d", "stress2d", "dense3d"],
                    help="dense2d is the headline workload; the others are the precision, 3D and small-frame cases")
    ap.add_argument("--clustering-only", type=int, default=0, metavar="STEPS",
                    help="time only the clustering stage and pipeline on the traffic scene (3 warm-up calls, then "
                         "STEPS timed ones) and print that object")
    ap.add_argument("--strong", action="store_true",
                    help="strong scaling: the ranks split one frame into contiguous cost-balanced cluster ranges "
                         "(partition.rank_shard, first_cluster = range start) instead of one frame each; rank 0 "
                         "checks, after the timed steps, that the merged results equal its own estimate of the "
                         "whole frame")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-gpu-baseline", action="store_true")
    ap.add_argument("--schedule", default="",
                    help="points_per_warp,hyps_per_lane for the scoring pass (default: the library's choice)")
    ap.add_argument("--serving-seconds", type=float, default=10.0,
                    help="measured seconds of the 64-radar serving load, after 1 s of warm-up (0 skips it)")
    ap.add_argument("--workload-steps", type=int, default=100,
                    help="timed steps of each of the other single-frame workloads (frame64, stress2d, dense3d "
                         "beside the headline one; 0 skips them)")
    ap.add_argument("--unpruned-steps", type=int, default=200,
                    help="steps timed again with exact pruning off (roofline.unpruned; 0 skips them)")
    ap.add_argument("--refine-iterations", type=int, default=0,
                    help="local-optimisation rounds in the timed steps (default 0: the single-pass method)")
    ap.add_argument("--local-opt-steps", type=int, default=50,
                    help="steps of each extra measurement on the same frame: 2 local-optimisation rounds, "
                         "the adaptive trial count at confidence 0.99, Alg. 1's line model, and the clustering "
                         "stage with the whole pipeline on a traffic scene (0 skips them)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2012_12618_gb300 import rvh, synth
    if args.clustering_only > 0:
        ctx = rvh.Context(local)
        stream = torch.cuda.Stream(dev)
        torch.cuda.set_stream(stream)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        out = measure_clustering(ctx, dev, stream, ctypes.c_void_p(stream.cuda_stream), flush, args.clustering_only)
        print(json.dumps({"clustering": out}), flush=True)
        ctx.close()
        return 0
    wname = args.workload
    w = synth.WORKLOADS[wname]
    dim = w.model_dim
    first_cluster = 0
    whole = None
    if args.strong:
        # strong scaling: every rank estimates its share of one frame
        import dataclasses
        from paper_2012_12618_gb300 import partition
        whole = synth.make_frame(w)
        sh = partition.rank_shard(whole.azimuth, whole.doppler, whole.offsets, w.num_hypotheses, rank, ws,
                                  whole.elevation)
        f = dataclasses.replace(whole, azimuth=sh.azimuth, doppler=sh.doppler, offsets=sh.offsets,
                                elevation=sh.elevation, truth_v=whole.truth_v[sh.c0:sh.c1],
                                outlier=whole.outlier[sh.p0:sh.p1], band=whole.band[sh.p0:sh.p1])
        first_cluster = sh.c0
    else:
        # weak scaling: every rank estimates its own frame (independent sensors)
        f = synth.make_frame(w, gen_seed=w.gen_seed + 1000 * rank)
    nc, npts = f.n_clusters, f.n_points
    sizes = np.diff(f.offsets).astype(np.int64)
    pairs = int(sizes.sum()) * w.num_hypotheses

    ctx = rvh.Context(local)
    if args.schedule:
        pw, hpl = (int(x) for x in args.schedule.split(","))
        ctx.check(rvh.rvh_set_schedule(ctx.handle, pw, hpl), "rvh_set_schedule")
    d_az = torch.from_numpy(f.azimuth).to(dev)
    d_el = None if f.elevation is None else torch.from_numpy(f.elevation).to(dev)
    d_dop = torch.from_numpy(f.doppler).to(dev)
    d_off = torch.from_numpy(f.offsets).to(dev)
    outs = rvh.alloc_outputs(nc, npts, dev)
    frame = rvh.make_frame(d_az, d_dop, d_off, d_el)
    params = rvh.make_params(dim, w.num_hypotheses, w.tau, w.seed, refine_iterations=args.refine_iterations,
                             first_cluster=first_cluster)
    res = rvh.make_result(outs)
    # a dedicated stream: the library and the timing events share it
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    sptr = ctypes.c_void_p(stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stats = rvh.rvh_stats()

    def step():
        ctx.check(rvh.rvh_estimate(ctx.handle, frame, params, res, sptr), "rvh_estimate")

    # the scoring schedule is picked by the library's autotuner on this workload (untimed)
    tuned = rvh.rvh_schedule()
    if not args.schedule:
        ctx.check(rvh.rvh_autotune(ctx.handle, frame, params, res, 7, tuned), "rvh_autotune")

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()

    step_ms, kern_ms = [], []
    band = cand = fp64h = refined = launches = scored = 0
    phase = np.zeros(6)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(np.uint8(_ & 0xFF))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            ctx.check(rvh.rvh_get_stats(ctx.handle, stats), "rvh_get_stats")
            kern_ms.append(stats.kernel_ms)
            band += stats.band_points
            cand += stats.candidates
            fp64h += stats.fp64_hypotheses
            refined += stats.refined_hypotheses
            launches += stats.kernel_launches
            scored += stats.pairs_scored
            phase += np.array(list(stats.phase_cycles), dtype=np.float64)
        torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    if ws > 1:
        torch.distributed.barrier()
    t_step = float(np.mean(step_ms)) * 1e-3
    t_max = t_step
    if ws > 1:
        tt = torch.tensor([t_step], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_max = float(tt.item())
    value = (whole.n_clusters if args.strong else nc * ws) / t_max
    grid = stats.grid

    # ---- strong scaling: the ranks' shards merged equal one GPU's estimate of the frame
    strong = None
    if args.strong:
        from paper_2012_12618_gb300 import partition
        mine = {k: v.cpu().numpy() for k, v in outs.items()}
        mine["inlier_mask"] = mine["inlier_mask"][:npts]
        parts = [(first_cluster, first_cluster + nc, mine)]
        if ws > 1:
            parts = [None] * ws
            torch.distributed.all_gather_object(parts, (first_cluster, first_cluster + nc, mine))
        if rank == 0:
            w_outs = rvh.alloc_outputs(whole.n_clusters, whole.n_points, dev)
            w_ins = [None if a is None else torch.from_numpy(a).to(dev)
                     for a in (whole.azimuth, whole.doppler, whole.offsets, whole.elevation)]
            ctx.check(rvh.rvh_estimate(ctx.handle, rvh.make_frame(*w_ins),
                                       rvh.make_params(dim, w.num_hypotheses, w.tau, w.seed,
                                                       refine_iterations=args.refine_iterations),
                                       rvh.make_result(w_outs), sptr), "rvh_estimate(whole frame)")
            torch.cuda.synchronize()
            one = {k: v.cpu().numpy() for k, v in w_outs.items()}
            one["inlier_mask"] = one["inlier_mask"][:whole.n_points]
            merged = partition.merge([p[2] for p in parts], [(p[0], p[1]) for p in parts], whole.offsets)
            strong = {"ranks": ws, "shard_clusters": [p[1] - p[0] for p in parts],
                      "merged_equals_one_gpu": all(np.array_equal(merged[k], one[k], equal_nan=True) for k in one)}

    # ---- roofline of the fused kernel (FP32 pipe; k FMA = 2k flop per trial x point pair)
    kern_s = float(np.mean(kern_ms)) * 1e-3
    # the (trial, point) pairs the scoring pass evaluated: the method's N x H
    # less those of trials dropped by exact pruning (they cannot win)
    scored_per_step = scored / max(args.steps, 1)
    flops = 2.0 * dim * scored_per_step
    achieved = flops / kern_s / 1e12
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    clocks = clk.summary()
    max_mhz = float(peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or SM_MAX_MHZ_FALLBACK)
    peak = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": recorded_traffic(),
                "kernel": f"rvh::fused_kernel<{dim}>",
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 FMA lanes x 2 flop x {max_mhz:.0f} MHz",
                "frac_at_measured_clock": (achieved / (sms * FP32_LANES_PER_SM * 2 * clocks["sm_mhz"] * 1e6 / 1e12)
                                           if clocks.get("sm_mhz") else None),
                "algorithmic_flops_per_launch": flops, "kernel_ms": kern_s * 1e3,
                "pairs_basis": "trial x point pairs the scoring pass evaluated (rvh_stats.pairs_scored)",
                "pairs_scored_fraction": scored_per_step / pairs,
                "frac_full_pairs": 2.0 * dim * pairs / kern_s / 1e12 / peak}
    # the scoring pass alone: its share of the per-CTA stage clocks (clock64,
    # summed over CTAs) times the kernel time; co-resident CTAs in other
    # stages share the SM meanwhile, so this is an attribution, not a solo run
    share = float(phase[2] / max(phase.sum(), 1.0))
    if share > 0:
        sc = flops / (share * kern_s) / 1e12
        roofline["scoring_loop_achieved"] = sc
        roofline["scoring_loop_frac"] = sc / peak
        roofline["scoring_loop_stage_share"] = share
        roofline["scoring_loop_frac_at_measured_clock"] = (
            sc / (sms * FP32_LANES_PER_SM * 2 * clocks["sm_mhz"] * 1e6 / 1e12) if clocks.get("sm_mhz") else None)
        roofline["scoring_loop_basis"] = "scoring-pass share of the per-CTA stage clocks x kernel time"
    if clocks.get("sm_mhz") and grid:
        # CTA clocks summed over the persistent grid against grid x kernel time:
        # what is missing is the tail after each CTA's last cluster
        roofline["cta_busy_fraction"] = float(phase.sum()) / (args.steps * grid * kern_s * clocks["sm_mhz"] * 1e6)

    # the same kernel without pruning (every trial over every point), for the
    # kernel-quality fraction on the full pair count
    if rank == 0 and args.unpruned_steps > 0:
        ctx.check(rvh.rvh_set_pruning(ctx.handle, 0), "rvh_set_pruning")
        u_ms = []
        for i in range(3 + args.unpruned_steps):
            flush.fill_(np.uint8(i & 0xFF))
            step()
            ctx.check(rvh.rvh_get_stats(ctx.handle, stats), "rvh_get_stats")
            if i >= 3:
                u_ms.append(stats.kernel_ms)
        ctx.check(rvh.rvh_set_pruning(ctx.handle, 1), "rvh_set_pruning")
        u_s = float(np.mean(u_ms)) * 1e-3
        roofline["unpruned"] = {"kernel_ms": u_s * 1e3, "frac": 2.0 * dim * pairs / u_s / 1e12 / peak,
                                "steps": args.unpruned_steps}

    # ---- the other single-frame workloads, each timed like the headline one
    workloads = {}
    if args.workload_steps > 0 and rank == 0:
        for other in ("frame64", "dense2d", "stress2d", "dense3d"):
            if other != wname:
                workloads[other] = measure_workload(ctx, other, dev, stream, sptr, flush, args.workload_steps,
                                                    sms, max_mhz)

    # ---- serving: 64 radars x 20 frames/s (Poisson), mixed 2D/3D, continuous batching
    # (right after the timed steps, before the other measurements churn the GPU)
    serve = None
    if args.serving_seconds > 0 and rank == 0:
        from paper_2012_12618_gb300 import serving
        spec = synth.ServingSpec(duration_s=args.serving_seconds, warmup_s=1.0)
        sres = serving.run_load(ctx, spec, dev)
        serve = sres.summary()
        ctx.check(rvh.rvh_get_stats(ctx.handle, stats), "rvh_get_stats")
        serve["steps"] = stats.serving_steps
        serve["graph_replays"] = stats.serving_graph_replays
        serve["config"] = (f"{spec.n_radars} radars x {spec.fps:g} frames/s Poisson, clusters "
                           f"{spec.clusters_lo}..{spec.clusters_hi} per frame, sizes log-uniform "
                           f"{spec.size_lo}..{spec.size_hi}; radars 0-31 2D H=256, 32-63 3D H=2048; "
                           f"{spec.duration_s:g} s measured after {spec.warmup_s:g} s")

    # ---- local-optimisation rounds (refine_iterations = 2) on the same frame:
    # kernel time and how many mask entries the rounds change
    local_opt = None
    if args.local_opt_steps > 0 and args.refine_iterations == 0:
        lo_outs = rvh.alloc_outputs(nc, npts, dev)
        lo_res = rvh.make_result(lo_outs)
        lo_params = rvh.make_params(dim, w.num_hypotheses, w.tau, w.seed, refine_iterations=2)
        lo_ms = []
        for i in range(3 + args.local_opt_steps):
            flush.fill_(5)
            ctx.check(rvh.rvh_estimate(ctx.handle, frame, lo_params, lo_res, sptr), "rvh_estimate(local opt)")
            ctx.check(rvh.rvh_get_stats(ctx.handle, stats), "rvh_get_stats")
            if i >= 3:
                lo_ms.append(stats.kernel_ms)
        torch.cuda.synchronize()
        changed = int((lo_outs["inlier_mask"] != outs["inlier_mask"]).sum().item())
        lk = float(np.mean(lo_ms))
        local_opt = {"refine_iterations": 2, "kernel_ms": lk, "clusters_per_s": nc / (lk * 1e-3),
                     "kernel_ms_single_pass": kern_s * 1e3, "mask_changed": changed,
                     "mask_changed_fraction": changed / max(npts, 1),
                     "inliers_single_pass": int(outs["inlier_count"].sum().item()),
                     "inliers_after_rounds": int(lo_outs["inlier_count"].sum().item()),
                     "steps": args.local_opt_steps}

    # ---- adaptive trial count (confidence 0.99, blocks of 128 trials) on the same frame
    adaptive = None
    if args.local_opt_steps > 0 and args.refine_iterations == 0:
        ad_outs = rvh.alloc_outputs(nc, npts, dev)
        ad_res = rvh.make_result(ad_outs)
        ad_params = rvh.make_params(dim, w.num_hypotheses, w.tau, w.seed, confidence=0.99, trial_block=128)
        ad_ms, ad_trials, ad_pairs = [], 0, 0
        for i in range(3 + args.local_opt_steps):
            flush.fill_(6)
            ctx.check(rvh.rvh_estimate(ctx.handle, frame, ad_params, ad_res, sptr), "rvh_estimate(adaptive)")
            ctx.check(rvh.rvh_get_stats(ctx.handle, stats), "rvh_get_stats")
            if i >= 3:
                ad_ms.append(stats.kernel_ms)
                ad_trials, ad_pairs = stats.hypotheses, stats.pair_evals
        torch.cuda.synchronize()
        ak = float(np.mean(ad_ms))
        adaptive = {"confidence": 0.99, "trial_block": 128, "kernel_ms": ak, "clusters_per_s": nc / (ak * 1e-3),
                    "pair_evals_per_s": ad_pairs / (ak * 1e-3), "trials_per_cluster": ad_trials / nc,
                    "pair_fraction_of_full": ad_pairs / pairs,
                    "inliers_full": int(outs["inlier_count"].sum().item()),
                    "inliers_adaptive": int(ad_outs["inlier_count"].sum().item()),
                    "same_winner_fraction": float((ad_outs["best_hypothesis"] == outs["best_hypothesis"])
                                                  .float().mean().item()),
                    "steps": args.local_opt_steps}

    # ---- Alg. 1 as printed (line fits in the normalised plane, MAD threshold) on
    # the same frame: kernel time and velocity error against the synthetic truth
    paper_line = None
    if args.local_opt_steps > 0 and args.refine_iterations == 0 and dim == 2:
        pl_outs = rvh.alloc_outputs(nc, npts, dev)
        pl_res = rvh.make_result(pl_outs)
        pl_params = rvh.make_params(dim, w.num_hypotheses, w.tau, w.seed, hypothesis_model=rvh.RVH_MODEL_PAPER_LINE)
        pl_ms = []
        for i in range(3 + args.local_opt_steps):
            flush.fill_(7)
            ctx.check(rvh.rvh_estimate(ctx.handle, frame, pl_params, pl_res, sptr), "rvh_estimate(paper line)")
            ctx.check(rvh.rvh_get_stats(ctx.handle, stats), "rvh_get_stats")
            if i >= 3:
                pl_ms.append(stats.kernel_ms)
        torch.cuda.synchronize()

        def verr(o):
            return float(np.nanmedian(np.hypot(o["vx"].cpu().numpy() - f.truth_v[:, 0],
                                               o["vy"].cpu().numpy() - f.truth_v[:, 1])))

        pk = float(np.mean(pl_ms))
        paper_line = {"kernel_ms": pk, "clusters_per_s": nc / (pk * 1e-3),
                      "median_velocity_error_m_s": verr(pl_outs),
                      "median_velocity_error_cosine_model_m_s": verr(outs),
                      "inliers": int(pl_outs["inlier_count"].sum().item()), "steps": args.local_opt_steps}

    # ---- the clustering stage (Fig. 1) on an unclustered traffic scene: DBSCAN,
    # then the whole pipeline cluster -> gather -> estimate (H = 1024, 2D)
    clustering = None
    if args.local_opt_steps > 0 and args.refine_iterations == 0 and dim == 2:
        clustering = measure_clustering(ctx, dev, stream, sptr, flush, args.local_opt_steps)

    # ---- end to end through the C ABI from host buffers: every step moves the
    # frame's inputs from host memory to the GPU and its results back, inside
    # the timed region.  Page-locked buffers (the headline): inputs copied in
    # by the call, results written in place by the kernels over the CPU-GPU
    # link; pageable ones: inputs and results staged with copies.
    def e2e_run(pinned: bool):
        def host(a):
            t = torch.from_numpy(a.copy())
            return t.pin_memory() if pinned else t
        h_in = [None if a is None else host(a) for a in (f.azimuth, f.doppler, f.offsets, f.elevation)]
        h_outs = {k: (v.cpu().pin_memory() if pinned else v.cpu().clone()) for k, v in outs.items()}
        h_frame = rvh.make_frame(*h_in)
        h_res = rvh.make_result(h_outs)
        for _ in range(2):
            ctx.check(rvh.rvh_estimate(ctx.handle, h_frame, params, h_res, sptr), "rvh_estimate(host)")
        ts = []
        for _ in range(max(50, args.steps // 2)):
            flush.fill_(3)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.check(rvh.rvh_estimate(ctx.handle, h_frame, params, h_res, sptr), "rvh_estimate(host)")
            ts.append(time.perf_counter() - t0)
        same = all(np.array_equal(h_outs[k].numpy(), outs[k].cpu().numpy(), equal_nan=True) for k in outs)
        return ts, same

    h2d = npts * 4 * dim + (nc + 1) * 4  # azimuth, Doppler (and elevation in 3D), offsets
    d2h = nc * (4 * 8 + 3 * 4) + npts
    e2e_t, e2e_same = e2e_run(True)
    st_t, st_same = e2e_run(False)
    e2e = {"value": nc / float(np.mean(e2e_t)), "unit": "clusters/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * float(np.mean(e2e_t)),
           "ms_per_step_median": 1e3 * float(np.median(e2e_t)), "steps": len(e2e_t),
           "results_equal_device_run": e2e_same,
           "timing": "host clock around rvh_estimate with page-locked host buffers: the inputs' bulk copies in, the "
                     "kernels, which write the results in place in host memory over the CPU-GPU link, and the "
                     "stream synchronisation that completes the call; L2 flushed outside the region",
           "staged": {"value": nc / float(np.mean(st_t)), "ms_per_step": 1e3 * float(np.mean(st_t)),
                      "ms_per_step_median": 1e3 * float(np.median(st_t)), "results_equal_device_run": st_same,
                      "timing": "the same call with pageable host buffers: inputs copied into device scratch and "
                                "results copied back inside the call"}}

    # ---- plain all-FP64 one-launch-per-cluster GPU version (same frame)
    gpu_base = None
    if not args.no_gpu_baseline and args.refine_iterations == 0:
        base_out = rvh.alloc_outputs(nc, npts, dev)
        bres = rvh.make_result(base_out)
        ctx.check(rvh.rvh_estimate_baseline(ctx.handle, frame, params, bres, sptr), "baseline")
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        ctx.check(rvh.rvh_estimate_baseline(ctx.handle, frame, params, bres, sptr), "baseline")
        b1.record(stream)
        b1.synchronize()
        bms = b0.elapsed_time(b1)
        same = bool(torch.equal(base_out["inlier_mask"], outs["inlier_mask"]) and
                    torch.equal(base_out["best_hypothesis"], outs["best_hypothesis"]))
        gpu_base = {"value": nc / (bms * 1e-3), "unit": "clusters/s", "kind": "plain all-FP64 GPU kernel, "
                    "one launch per cluster", "ms_per_step": bms, "fused_speedup": value / ws / (nc / (bms * 1e-3)),
                    "identical_masks_and_winners": same}

    # ---- the FP64 oracle on this host (rank 0, N = 1 only)
    cpu = cpu_all = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        sub = np.sort(np.random.default_rng(1).choice(nc, min(nc, 1024 if dim == 2 else 256), replace=False))
        t0 = time.perf_counter()
        oracle.estimate(f.azimuth, f.doppler, f.offsets, elevation=f.elevation, num_hypotheses=w.num_hypotheses,
                        tau=w.tau, seed=w.seed, subset=sub)
        dt = time.perf_counter() - t0
        cpu = {"value": sub.shape[0] / dt, "unit": "clusters/s", "cores": 1, "kind": "oracle",
               "sample": f"{sub.shape[0]} random clusters of the {wname} frame, single-threaded FP64 C",
               "seconds": dt}
        cpu_all = oracle_all_cores(f, w, wname)

    if rank == 0:
        line = {
            "metric": "clusters/s", "value": value, "unit": "clusters/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": t_max * 1e3, "higher_is_better": True,
            "scaling": "strong" if args.strong else "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"{wname}: {nc} clusters, sizes {w.size_law} {w.size_lo}..{w.size_hi}, "
                                   f"{npts} points, {dim}D, H={w.num_hypotheses}, tau={w.tau} m/s, "
                                   f"outliers {w.outlier_frac:g}, noise {w.noise_sigma:g} m/s, seed={w.seed}, "
                                   f"refine_iterations={args.refine_iterations}",
                       "l2": "flushed between timed steps (256 MiB write outside the step events)",
                       "per_rank": ("a contiguous cost-balanced cluster range of one frame (first_cluster = "
                                    "range start)" if args.strong else "one independent frame per rank")},
            "strong_scaling_check": strong,
            "pair_evals_per_s": pairs * ws / t_max,
            "roofline": roofline,
            "workloads": workloads,
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
            "gpu_baseline": gpu_base,
            "serving": serve,
            "local_opt": local_opt,
            "adaptive": adaptive,
            "paper_line": paper_line,
            "clustering": clustering,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": launches,
            "band": {"fp64_band_decisions_per_step": band / args.steps, "candidates_per_step": cand / args.steps,
                     "fp64_trials_per_step": fp64h / args.steps,
                     "refined_trials_per_step": refined / args.steps,
                     "band_rate_per_pair": band / args.steps / pairs},
            "schedule": {"grid": grid, "points_per_warp": stats.points_per_warp,
                         "hyps_per_lane": stats.hyps_per_lane, "autotuned": not args.schedule,
                         "cuda_graph_replays": stats.graph_replays, "cuda_graph_builds": stats.graph_builds},
            "stage_share": dict(zip(["rows", "hypotheses", "scoring", "exact_rescoring", "mask_refine", "other"],
                                    [round(float(x), 4) for x in phase / max(phase.sum(), 1.0)])),
            "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
