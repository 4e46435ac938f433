"""Seeded synthetic radar frames shaped like traffic scenes.

This module only draws inputs.  It holds none of the estimator's arithmetic
(no minimal-set solve, residual test, argmax or least squares): it evaluates
the forward model of Eq. (LSQ_eq), v_d = vx cos(t) + vy sin(t) (plus
vz sin(e) with an elevation e, the 3D extension), to synthesise Doppler
values, then adds noise and micro-Doppler outliers.  The paper measures on
captured 78.6 GHz traffic data that is not public; these frames stand in for
it with the cluster-size mix, angle spread, noise and outlier model of the
workloads measured here:

  dense2d    4096 clusters, sizes log-uniform in 8..2048, 2D, 20% outliers
  frame64    64 clusters, sizes uniform in 16..128, 2D, 20% outliers
  stress2d   16384 clusters, sizes 32..512, 40% outliers, sigma 0.08,
             5% of inliers placed within +-2e-5 m/s of the 0.1 m/s threshold
  dense3d    8192 clusters, sizes 24..1024, elevation +-15 deg, 25% outliers

Values are generated in FP64 and stored as FP32 (unless float64 is asked
for, which the exact-recovery tests use).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DEG = math.pi / 180.0


@dataclasses.dataclass
class Frame:
    azimuth: np.ndarray            # [n_points] rad
    elevation: np.ndarray | None   # [n_points] rad, None for 2D
    doppler: np.ndarray            # [n_points] m/s
    offsets: np.ndarray            # [n_clusters + 1] int32 CSR offsets
    truth_v: np.ndarray            # [n_clusters, 3] true (vx, vy, vz)
    outlier: np.ndarray            # [n_points] bool, planted outliers
    band: np.ndarray               # [n_points] bool, points placed near the threshold

    @property
    def n_clusters(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_points(self) -> int:
        return int(self.offsets[-1])

    @property
    def model_dim(self) -> int:
        return 2 if self.elevation is None else 3


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named workload: how frames are drawn and the estimator settings."""
    name: str
    n_clusters: int
    size_law: str            # "uniform" or "loguniform"
    size_lo: int
    size_hi: int
    model_dim: int
    num_hypotheses: int
    outlier_frac: float
    noise_sigma: float
    band_frac: float = 0.0
    tau: float = 0.1
    gen_seed: int = 1
    seed: int = 1            # RANSAC (Philox) seed
    az_deg: float = 60.0
    el_deg: float = 15.0
    vz_max: float = 5.0
    speed_max: float = 40.0


WORKLOADS = {
    "frame64": Workload("frame64", 64, "uniform", 16, 128, 2, 256, 0.20, 0.05, gen_seed=1),
    "dense2d": Workload("dense2d", 4096, "loguniform", 8, 2048, 2, 1024, 0.20, 0.05, gen_seed=2),
    "stress2d": Workload("stress2d", 16384, "uniform", 32, 512, 2, 1024, 0.40, 0.08,
                         band_frac=0.05, gen_seed=3),
    "dense3d": Workload("dense3d", 8192, "uniform", 24, 1024, 3, 2048, 0.25, 0.05, gen_seed=4),
}


def draw_sizes(rng: np.random.Generator, n: int, law: str, lo: int, hi: int) -> np.ndarray:
    if law == "uniform":
        return rng.integers(lo, hi + 1, size=n).astype(np.int64)
    if law == "loguniform":
        # floor(exp(U[ln lo, ln (hi + 1)))) lies in lo..hi
        s = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi + 1), size=n))).astype(np.int64)
        return np.clip(s, lo, hi)
    raise ValueError(law)


def _rank_within(cluster_id: np.ndarray, key: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """Rank of each point's key among the points of its cluster (0-based)."""
    order = np.lexsort((key, cluster_id))
    rank = np.empty_like(order)
    starts = offsets[:-1][cluster_id[order]]
    rank[order] = np.arange(order.shape[0]) - starts
    return rank


def make_frame(w: Workload, *, n_clusters: int | None = None, gen_seed: int | None = None,
               sizes: np.ndarray | None = None, dtype=np.float32) -> Frame:
    rng = np.random.default_rng(w.gen_seed if gen_seed is None else gen_seed)
    nc = w.n_clusters if n_clusters is None else n_clusters
    if sizes is None:
        sizes = draw_sizes(rng, nc, w.size_law, w.size_lo, w.size_hi)
    sizes = np.asarray(sizes, dtype=np.int64)
    nc = sizes.shape[0]
    offsets = np.zeros(nc + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    npts = int(offsets[-1])
    cid = np.repeat(np.arange(nc), sizes)

    # per-cluster rigid-body velocity: |v_h| ~ U(0, vmax), heading ~ U[0, 2 pi)
    speed_h = rng.uniform(0.0, w.speed_max, size=nc)
    head = rng.uniform(0.0, 2.0 * math.pi, size=nc)
    vx = speed_h * np.cos(head)
    vy = speed_h * np.sin(head)
    vz = rng.uniform(-w.vz_max, w.vz_max, size=nc) if w.model_dim == 3 else np.zeros(nc)
    speed = np.sqrt(vx * vx + vy * vy + vz * vz)

    theta = rng.uniform(-w.az_deg * DEG, w.az_deg * DEG, size=npts).astype(dtype).astype(np.float64)
    if w.model_dim == 3:
        elev = rng.uniform(-w.el_deg * DEG, w.el_deg * DEG, size=npts).astype(dtype).astype(np.float64)
        model = (vx[cid] * np.cos(theta) * np.cos(elev) + vy[cid] * np.sin(theta) * np.cos(elev)
                 + vz[cid] * np.sin(elev))
    else:
        elev = None
        model = vx[cid] * np.cos(theta) + vy[cid] * np.sin(theta)
    dop = model + rng.normal(0.0, w.noise_sigma, size=npts) if w.noise_sigma > 0 else model.copy()

    # exactly round(f * N) outliers per cluster, chosen uniformly
    n_out = np.rint(w.outlier_frac * sizes).astype(np.int64)
    rank = _rank_within(cid, rng.random(npts), offsets)
    outlier = rank < n_out[cid]
    dop[outlier] = rng.uniform(0.0, 1.0, size=int(outlier.sum())) * 2.0 * speed[cid[outlier]]

    # band points: round(band_frac * n_inliers) inliers moved to tau +- 2e-5 of the model
    band = np.zeros(npts, dtype=bool)
    if w.band_frac > 0:
        n_band = np.rint(w.band_frac * (sizes - n_out)).astype(np.int64)
        key = rng.random(npts) + outlier.astype(np.float64) * 2.0  # outliers rank last
        rank2 = _rank_within(cid, key, offsets)
        band = (rank2 < n_band[cid]) & ~outlier
        nb = int(band.sum())
        sign = np.where(rng.random(nb) < 0.5, -1.0, 1.0)
        dop[band] = model[band] + sign * (w.tau + rng.uniform(-2e-5, 2e-5, size=nb))

    return Frame(
        azimuth=theta.astype(dtype),
        elevation=None if elev is None else elev.astype(dtype),
        doppler=dop.astype(dtype),
        offsets=offsets.astype(np.int32),
        truth_v=np.stack([vx, vy, vz], axis=1),
        outlier=outlier,
        band=band,
    )


# ---- serving stream: many radars, Poisson frame arrivals ---------------------------------

@dataclasses.dataclass(frozen=True)
class ServingSpec:
    n_radars: int = 64
    fps: float = 20.0
    clusters_lo: int = 50
    clusters_hi: int = 2000
    size_lo: int = 8
    size_hi: int = 2048
    duration_s: float = 10.0
    warmup_s: float = 1.0


def radar_workload(radar: int) -> Workload:
    """Radars 0..31 run the 2D model (256 hypotheses), 32..63 the 3D one (2048)."""
    if radar % 64 < 32:
        return dataclasses.replace(WORKLOADS["frame64"], name=f"radar{radar}", num_hypotheses=256,
                                   size_law="loguniform", size_lo=8, size_hi=2048)
    return dataclasses.replace(WORKLOADS["dense3d"], name=f"radar{radar}", num_hypotheses=2048,
                               size_law="loguniform", size_lo=8, size_hi=2048)


def radar_frame_seed(radar: int, frame_no: int) -> int:
    ss = np.random.SeedSequence([5, radar, frame_no])
    return int(ss.generate_state(1, dtype=np.uint64)[0])


def arrival_schedule(spec: ServingSpec, seed: int = 5) -> list[tuple[float, int, int]]:
    """(arrival time s, radar, frame number) sorted by time: per radar a Poisson process."""
    rng = np.random.default_rng(seed)
    events = []
    for r in range(spec.n_radars):
        t = rng.uniform(0.0, 1.0 / spec.fps)
        k = 0
        while t < spec.duration_s + spec.warmup_s:
            events.append((t, r, k))
            t += rng.exponential(1.0 / spec.fps)
            k += 1
    events.sort()
    return events


def serving_frame(spec: ServingSpec, radar: int, frame_no: int) -> tuple[Frame, Workload]:
    w = radar_workload(radar)
    fseed = radar_frame_seed(radar, frame_no)
    rng = np.random.default_rng(fseed)
    nc = int(rng.integers(spec.clusters_lo, spec.clusters_hi + 1))
    sizes = draw_sizes(rng, nc, "loguniform", spec.size_lo, spec.size_hi)
    return make_frame(w, sizes=sizes, gen_seed=fseed + 1), w


# ---- raw scenes for the clustering stage (Fig. 1: point cloud -> clusters) -----------------

@dataclasses.dataclass
class Scene:
    """An unclustered radar point cloud: objects plus clutter, in random order."""
    x: np.ndarray            # [n] m, FP32 (longitudinal)
    y: np.ndarray            # [n] m, FP32 (lateral)
    azimuth: np.ndarray      # [n] rad, FP32, atan2(y, x)
    doppler: np.ndarray      # [n] m/s, FP32
    object_id: np.ndarray    # [n] int, the object a point came from, -1 for clutter
    truth_v: np.ndarray      # [n_objects, 2] true (vx, vy)

    @property
    def n_points(self) -> int:
        return int(self.x.shape[0])

    def features(self) -> np.ndarray:
        """[n, 2] FP32 feature vectors (x, y) for DBSCAN."""
        return np.stack([self.x, self.y], axis=1)


@dataclasses.dataclass(frozen=True)
class SceneSpec:
    name: str
    n_objects: int
    size_lo: int = 8
    size_hi: int = 1024
    range_lo: float = 5.0      # m
    range_hi: float = 300.0   # field of view: centres on 10 m cells within range_lo + 10 .. range_hi
    spread_lo: float = 0.3     # per-object position spread (sigma, m)
    spread_hi: float = 1.2
    clutter_frac: float = 0.03
    outlier_frac: float = 0.20
    noise_sigma: float = 0.05
    speed_max: float = 40.0
    eps: float = 1.0           # DBSCAN radius (m) the scene is drawn for
    min_pts: int = 4
    gen_seed: int = 9


SCENES = {
    "scene_small": SceneSpec("scene_small", 48, size_hi=128, range_hi=120.0, gen_seed=9),
    "scene": SceneSpec("scene", 512, range_hi=400.0, gen_seed=10),
}


def make_scene(s: SceneSpec, *, n_objects: int | None = None, gen_seed: int | None = None) -> Scene:
    """Objects at separated positions in the field of view (azimuth +-60 deg,
    centres on a jittered 10 m grid), each a Gaussian blob of points whose Doppler follows
    the velocity profile of Eq. (LSQ_eq) with noise and micro-Doppler
    outliers, plus uniformly scattered clutter; points shuffled."""
    rng = np.random.default_rng(s.gen_seed if gen_seed is None else gen_seed)
    n_obj = s.n_objects if n_objects is None else n_objects
    # centres on a jittered grid of cells inside the +-60 deg wedge, so that
    # blobs (3 sigma <= 3.6 m) stay more than eps apart
    cell = 10.0
    gx, gy = np.meshgrid(np.arange(0.0, s.range_hi, cell) + cell / 2,
                         np.arange(-s.range_hi, s.range_hi, cell) + cell / 2, indexing="ij")
    gr, ga = np.hypot(gx, gy), np.arctan2(gy, gx)
    ok = (gr >= s.range_lo + cell) & (gr <= s.range_hi) & (np.abs(ga) <= 60.0 * DEG)
    gx, gy = gx[ok], gy[ok]
    if gx.shape[0] < n_obj:
        raise ValueError("field of view too small for the number of objects")
    pick = rng.choice(gx.shape[0], size=n_obj, replace=False)
    cx = gx[pick] + rng.uniform(-0.1, 0.1, size=n_obj) * cell
    cy = gy[pick] + rng.uniform(-0.1, 0.1, size=n_obj) * cell
    sizes = draw_sizes(rng, n_obj, "loguniform", s.size_lo, s.size_hi)
    oid = np.repeat(np.arange(n_obj), sizes)
    spread = rng.uniform(s.spread_lo, s.spread_hi, size=n_obj)
    px = cx[oid] + rng.normal(0.0, 1.0, size=oid.shape[0]) * spread[oid]
    py = cy[oid] + rng.normal(0.0, 1.0, size=oid.shape[0]) * spread[oid]
    speed = rng.uniform(0.0, s.speed_max, size=n_obj)
    head = rng.uniform(0.0, 2.0 * math.pi, size=n_obj)
    vx, vy = speed * np.cos(head), speed * np.sin(head)
    theta = np.arctan2(py, px)
    dop = vx[oid] * np.cos(theta) + vy[oid] * np.sin(theta) + rng.normal(0.0, s.noise_sigma, size=oid.shape[0])
    out = rng.random(oid.shape[0]) < s.outlier_frac
    dop[out] = rng.uniform(0.0, 2.0, size=int(out.sum())) * speed[oid[out]]
    # clutter over the field of view
    nclut = int(round(s.clutter_frac * oid.shape[0]))
    r = np.exp(rng.uniform(math.log(s.range_lo), math.log(s.range_hi), size=nclut))
    a = rng.uniform(-60.0 * DEG, 60.0 * DEG, size=nclut)
    px = np.concatenate([px, r * np.cos(a)])
    py = np.concatenate([py, r * np.sin(a)])
    dop = np.concatenate([dop, rng.uniform(-s.speed_max, s.speed_max, size=nclut)])
    oid = np.concatenate([oid, np.full(nclut, -1)])
    perm = rng.permutation(oid.shape[0])
    px32, py32 = px[perm].astype(np.float32), py[perm].astype(np.float32)
    return Scene(x=px32, y=py32,
                 azimuth=np.arctan2(py32.astype(np.float64), px32.astype(np.float64)).astype(np.float32),
                 doppler=dop[perm].astype(np.float32), object_id=oid[perm],
                 truth_v=np.stack([vx, vy], axis=1))
