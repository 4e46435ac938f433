"""Sharding a frame across GPUs (or processes) by contiguous cluster ranges.

Clusters are independent (the paper parallelises across them, Eq. 4), so a
frame splits into contiguous cluster ranges of near-equal cost with no
exchange during the estimate; each shard is estimated with
`first_cluster` = the index of its first cluster, which keeps every trial's
random minimal set that of the whole frame, so the merged result equals the
single-device result exactly.  Results are concatenated on the host.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# per-cluster cost in point-evaluations of fixed work (load, hypothesis
# generation, reductions), added to N * H when balancing
CLUSTER_OVERHEAD = 4096


def balanced_ranges(offsets, num_hypotheses: int, parts: int) -> list[tuple[int, int]]:
    """Contiguous [c0, c1) cluster ranges, one per part, with near-equal
    sum over clusters of (N_i * H + overhead).  Ranges may be empty."""
    off = np.asarray(offsets, dtype=np.int64)
    nc = off.shape[0] - 1
    if parts < 1:
        raise ValueError("parts must be >= 1")
    cost = np.diff(off) * int(num_hypotheses) + CLUSTER_OVERHEAD
    cum = np.concatenate([[0], np.cumsum(cost)])
    total = cum[-1]
    cuts = [0]
    for p in range(1, parts):
        cuts.append(int(np.searchsorted(cum, total * p / parts, side="left")))
    cuts.append(nc)
    cuts = np.maximum.accumulate(np.clip(cuts, 0, nc))
    return [(int(cuts[i]), int(cuts[i + 1])) for i in range(parts)]


def shard(azimuth, doppler, offsets, c0: int, c1: int, elevation=None):
    """The points and rebased CSR offsets of clusters [c0, c1)."""
    off = np.asarray(offsets, dtype=np.int64)
    p0, p1 = int(off[c0]), int(off[c1])
    sub_off = (off[c0:c1 + 1] - p0).astype(np.int32)
    el = None if elevation is None else elevation[p0:p1]
    return azimuth[p0:p1], doppler[p0:p1], sub_off, el, (p0, p1)


def merge(parts: list[dict], ranges: list[tuple[int, int]], offsets) -> dict:
    """Concatenates per-shard results (numpy dicts in shard order)."""
    off = np.asarray(offsets, dtype=np.int64)
    out = {}
    for key in parts[0]:
        out[key] = np.concatenate([p[key] for p in parts])
    assert out["inlier_mask"].shape[0] == int(off[ranges[-1][1]] - off[ranges[0][0]])
    return out


@dataclasses.dataclass
class Shard:
    """One rank's part of a frame: clusters [c0, c1) (points [p0, p1)) with
    their offsets rebased to 0; estimate it with first_cluster = c0."""
    azimuth: np.ndarray
    doppler: np.ndarray
    offsets: np.ndarray
    elevation: np.ndarray | None
    c0: int
    c1: int
    p0: int
    p1: int

    @property
    def n_clusters(self) -> int:
        return self.c1 - self.c0

    @property
    def n_points(self) -> int:
        return self.p1 - self.p0


def rank_shard(azimuth, doppler, offsets, num_hypotheses: int, rank: int, world: int, elevation=None) -> Shard:
    """The shard of `rank` out of `world` ranks: its range of
    balanced_ranges and the points of that range."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    c0, c1 = balanced_ranges(offsets, num_hypotheses, world)[rank]
    az, dop, off, el, (p0, p1) = shard(azimuth, doppler, offsets, c0, c1, elevation)
    return Shard(az, dop, off, el, c0, c1, p0, p1)

