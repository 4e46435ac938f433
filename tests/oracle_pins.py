"""Checks that pin the FP64 oracle to facts other than itself.

Each check takes an oracle library handle (the built oracle, or a variant with
a planted mistake, see test_oracle_mutants.py) and raises AssertionError on a
violation.  What pins what:

  philox      published known-answer vectors of Philox4x32-10 (SC'11)
  draws       distinct, in-range and chi-square uniform minimal sets
  recovery    closed form: noise-free clusters give back the true velocity
              (Eq. LSQ_eq, Eq. eq:LSQPerCluster) and heading atan2(vy, vx)
  brute       exhaustive all-pairs / all-triples RANSAC written with numpy
              (np.linalg.solve per minimal set) on tiny clusters
  symmetry    exact: azimuth -> -azimuth negates vy and the heading, keeps
              the masks; Doppler and tau times 2^m scale the velocity by 2^m
  rotation    azimuth -> azimuth + alpha rotates the velocity by alpha
  lstsq       the refine equals numpy.linalg.lstsq on the inlier rows (the
              least-squares comparator of the paper's Table II)
  status      too-few-points, all-degenerate and least-squares fallback cases
  adaptive    the adaptive trial count: the winner is the first maximum of the
              full run's counts over the trials run; the stopping rule
              (1 - eps^k)^m <= 1 - p, evaluated with Python's float power,
              holds where the count stopped and at no earlier block end;
              all-inlier clusters stop after one block
  paper_line  Alg. 1 as printed (line fits in the normalised plane, MAD
              threshold): exhaustive all-pairs counts against numpy (min/max
              normalisation, np.median, the distance from the cross product
              of the seed difference, an independent formula); the refine
              is numpy.linalg.lstsq of the inliers; 2^m Doppler scaling is
              exact; affine (azimuth, Doppler) data is all inliers
  dbscan      the clustering stage: core points, noise and the partition of
              core points equal scikit-learn's DBSCAN; border points join
              their lowest-index core neighbour (numpy distance matrix);
              cluster ids follow the smallest core index; min_pts = 1 gives
              the connected components of the eps-graph (scipy); permuting
              the input permutes the result
  fragile     the oracle's log of decisions within rounding distance of a
              threshold (the only place a last-ulp difference of cos/sin
              could flip a decision): an extra point planted within a few
              ulps of tau, or a minimal set whose |det| is within a few ulps
              of cond_eps, is flagged; the same planted 1e-9 m/s (or a
              relative 1e-6) away is not; no cluster of the full frame64 and
              dense2d frames is flagged
  first_cluster  a shard of a frame (clusters [c0, c1), offsets rebased)
              estimated with first_cluster = c0 gives the whole frame's
              results for those clusters, and differs from the same
              arrays estimated as a frame of their own
  local_opt   the re-threshold + re-fit rounds: one round's inlier set is
              numpy's re-threshold of the refined velocity, every result is
              numpy.linalg.lstsq of its own inlier set, a converged result is
              a fixed point of threshold-then-fit, the exact symmetries hold
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np

import oracle
from paper_2012_12618_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _est(L, az, dop, off, **kw):
    return oracle.estimate(az, dop, off, _lib=L, **kw)


def check_philox(L):
    path = os.path.join(GOLDEN, "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        words = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(words[0:4], words[4:6], _lib=L)
        assert [int(x) for x in out] == words[6:10], (r, [hex(x) for x in out])


def check_draws(L):
    seed = 0x1234_5678_9ABC_DEF0
    # the draw is the documented map of the Philox words: floor(w * n / 2^32) with skips
    for h in range(50):
        w = oracle.philox4x32_10([h, 7, 0, 0], [seed & 0xFFFFFFFF, seed >> 32], _lib=L)
        n = 1000
        q0 = (int(w[0]) * n) >> 32
        q1 = (int(w[1]) * (n - 1)) >> 32
        q1 += q1 >= q0
        assert list(oracle.draw(seed, 7, h, n, 2, _lib=L)) == [q0, q1]
    for n in (2, 3, 5, 17, 1000):
        for h in range(300):
            q = oracle.draw(seed, 3, h, n, 2, _lib=L)
            assert q[0] != q[1] and 0 <= q.min() and q.max() < n
            if n >= 3:
                q = oracle.draw(seed, 3, h, n, 3, _lib=L)
                assert len(set(q.tolist())) == 3 and 0 <= q.min() and q.max() < n
    # chi-square uniformity of unordered pairs (n=5: 10 cells) and triples (n=6: 20 cells)
    from scipy.stats import chisquare
    for n, k, cells in ((5, 2, 10), (6, 3, 20)):
        idx = {c: i for i, c in enumerate(itertools.combinations(range(n), k))}
        counts = np.zeros(cells)
        ordered = np.zeros((n, n))
        for h in range(20000):
            q = oracle.draw(99, 11, h, n, k, _lib=L)
            counts[idx[tuple(sorted(q.tolist()))]] += 1
            ordered[q[0], q[1]] += 1
        assert chisquare(counts).pvalue > 1e-4, counts
        # ordered first/second index: uniform over the n(n-1) ordered pairs
        off = ordered[~np.eye(n, dtype=bool)]
        assert chisquare(off).pvalue > 1e-4, ordered


def _noise_free(rng, n, dim, v):
    th = rng.uniform(-1.0, 1.0, n)
    if dim == 2:
        dop = v[0] * np.cos(th) + v[1] * np.sin(th)
        return th, None, dop
    el = rng.uniform(-0.26, 0.26, n)
    dop = v[0] * np.cos(th) * np.cos(el) + v[1] * np.sin(th) * np.cos(el) + v[2] * np.sin(el)
    return th, el, dop


def check_recovery(L):
    rng = np.random.default_rng(5)
    for dim in (2, 3):
        for trial in range(20):
            v = rng.uniform(-30, 30, 3)
            n = int(rng.integers(dim, 60))
            th, el, dop = _noise_free(rng, n, dim, v)
            o = _est(L, th, dop, [0, n], elevation=el, num_hypotheses=16, tau=0.1, seed=trial)
            assert o["status"][0] == 0 or (n == dim and o["status"][0] == 0), o["status"]
            assert o["inlier_count"][0] == n
            assert abs(o["vx"][0] - v[0]) < 1e-10 and abs(o["vy"][0] - v[1]) < 1e-10
            if dim == 3:
                assert abs(o["vz"][0] - v[2]) < 1e-10
            assert abs(o["heading"][0] - math.atan2(v[1], v[0])) < 1e-10


def _brute(th, el, dop, tau, eps):
    """All k-subsets in lexicographic order, each solved with np.linalg.solve."""
    n = th.shape[0]
    if el is None:
        A = np.stack([np.cos(th), np.sin(th)], 1)
    else:
        A = np.stack([np.cos(th) * np.cos(el), np.sin(th) * np.cos(el), np.sin(el)], 1)
    k = A.shape[1]
    counts, vels, margin = [], [], np.inf
    for q in itertools.combinations(range(n), k):
        M = A[list(q)]
        d = np.linalg.det(M)
        margin = min(margin, abs(abs(d) - eps))
        if not abs(d) >= eps:
            counts.append(-1)
            vels.append(None)
            continue
        v = np.linalg.solve(M, dop[list(q)])
        r = np.abs(dop - A @ v)
        margin = min(margin, np.min(np.abs(r - tau)))
        counts.append(int((r <= tau).sum()))
        vels.append(v)
    return A, np.array(counts), vels, margin


def check_brute(L):
    rng = np.random.default_rng(11)
    done = 0
    while done < 24:
        dim = 2 if done % 2 == 0 else 3
        n = int(rng.integers(dim + 2, 11 if dim == 2 else 9))
        v = rng.uniform(-20, 20, 3)
        th, el, dop = _noise_free(rng, n, dim, v)
        dop = dop + rng.normal(0, 0.05, n)
        bad = rng.random(n) < 0.3
        dop[bad] = rng.uniform(-40, 40, int(bad.sum()))
        tau, eps = 0.1, (1e-4 if dim == 2 else 1e-6)
        A, counts, vels, margin = _brute(th, el, dop, tau, eps)
        if margin < 1e-9:
            continue  # a decision too close to call across rounding orders
        H = counts.shape[0]
        o = _est(L, th, dop, [0, n], elevation=el, num_hypotheses=H, tau=tau, seed=1,
                 cond_eps=eps, enumerate_subsets=True, want_counts=True)
        assert np.array_equal(o["hyp_counts"][0], counts), (o["hyp_counts"][0], counts)
        best = int(np.argmax(counts))          # first maximum
        assert o["best_hypothesis"][0] == best
        r = np.abs(dop - A @ vels[best])
        assert np.array_equal(o["inlier_mask"].astype(bool), r <= tau)
        # random draws can never beat the exhaustive search
        o2 = _est(L, th, dop, [0, n], elevation=el, num_hypotheses=64, tau=tau, seed=done,
                  cond_eps=eps, want_counts=True)
        assert o2["hyp_counts"].max() <= counts.max()
        assert o2["inlier_count"][0] == o2["hyp_counts"][0].max()
        done += 1


def _frame(name, n_clusters):
    w = synth.WORKLOADS[name]
    return w, synth.make_frame(w, n_clusters=n_clusters)


def check_symmetry(L):
    for name, nc in (("frame64", 48), ("dense3d", 12)):
        w, f = _frame(name, nc)
        kw = dict(num_hypotheses=w.num_hypotheses if name == "frame64" else 256, tau=w.tau, seed=3)
        base = _est(L, f.azimuth, f.doppler, f.offsets, elevation=f.elevation, want_counts=True, **kw)
        neg = _est(L, -f.azimuth.astype(np.float64), f.doppler, f.offsets, elevation=f.elevation,
                   want_counts=True, **kw)
        assert np.array_equal(base["hyp_counts"], neg["hyp_counts"])
        assert np.array_equal(base["inlier_mask"], neg["inlier_mask"])
        assert np.array_equal(base["best_hypothesis"], neg["best_hypothesis"])
        assert np.array_equal(base["vx"], neg["vx"])
        assert np.array_equal(base["vy"], -neg["vy"])
        assert np.array_equal(base["vz"], neg["vz"])
        assert np.array_equal(base["heading"], -neg["heading"])
        for m in (-3, 5):
            s = 2.0 ** m
            sc = _est(L, f.azimuth, f.doppler.astype(np.float64) * s, f.offsets, elevation=f.elevation,
                      want_counts=True, **dict(kw, tau=w.tau * s))
            assert np.array_equal(base["hyp_counts"], sc["hyp_counts"])
            assert np.array_equal(base["inlier_mask"], sc["inlier_mask"])
            assert np.array_equal(base["vx"] * s, sc["vx"])
            assert np.array_equal(base["vy"] * s, sc["vy"])
            assert np.array_equal(base["vz"] * s, sc["vz"])
            assert np.array_equal(base["heading"], sc["heading"])


def check_rotation(L):
    rng = np.random.default_rng(21)
    for trial in range(20):
        v = rng.uniform(-30, 30, 3)
        n = 40
        th, _, dop = _noise_free(rng, n, 2, v)
        a = rng.uniform(-0.5, 0.5)
        o = _est(L, th + a, dop, [0, n], num_hypotheses=8, tau=0.1, seed=trial)
        ex = v[0] * math.cos(a) - v[1] * math.sin(a)
        ey = v[0] * math.sin(a) + v[1] * math.cos(a)
        assert abs(o["vx"][0] - ex) < 1e-10 and abs(o["vy"][0] - ey) < 1e-10
        dh = (o["heading"][0] - (math.atan2(v[1], v[0]) + a) + math.pi) % (2 * math.pi) - math.pi
        assert abs(dh) < 1e-10


def check_lstsq(L):
    for name, nc, H in (("frame64", 64, 256), ("dense3d", 16, 256)):
        w, f = _frame(name, nc)
        o = _est(L, f.azimuth, f.doppler, f.offsets, elevation=f.elevation, num_hypotheses=H,
                 tau=w.tau, seed=1)
        th = f.azimuth.astype(np.float64)
        dop = f.doppler.astype(np.float64)
        if f.elevation is None:
            A = np.stack([np.cos(th), np.sin(th)], 1)
        else:
            el = f.elevation.astype(np.float64)
            A = np.stack([np.cos(th) * np.cos(el), np.sin(th) * np.cos(el), np.sin(el)], 1)
        checked = 0
        for c in range(nc):
            if o["status"][c] != 0:
                continue
            s, e = f.offsets[c], f.offsets[c + 1]
            m = o["inlier_mask"][s:e].astype(bool)
            assert m.sum() == o["inlier_count"][c]
            ref = np.linalg.lstsq(A[s:e][m], dop[s:e][m], rcond=None)[0]
            got = np.array([o["vx"][c], o["vy"][c], o["vz"][c]])[:A.shape[1]]
            assert np.allclose(got, ref, rtol=1e-9, atol=1e-9), (c, got, ref)
            assert abs(o["heading"][c] - math.atan2(ref[1], ref[0])) < 1e-9
            checked += 1
        assert checked >= nc // 2
    # exactly k rows: the least-squares answer is the minimal solve
    th = np.array([0.2, -0.7])
    dop = np.array([3.0, -11.0])
    o = _est(L, th, dop, [0, 2], num_hypotheses=4, tau=0.1, seed=9)
    ref = np.linalg.solve(np.stack([np.cos(th), np.sin(th)], 1), dop)
    assert o["status"][0] == 0 and o["inlier_count"][0] == 2
    assert np.allclose([o["vx"][0], o["vy"][0]], ref, rtol=1e-12, atol=1e-12)


def check_status(L):
    # clusters of 0 and 1 points (2D), 2 points (3D): too few
    th = np.array([0.1, 0.2, 0.3])
    dop = np.array([1.0, 2.0, 3.0])
    o = _est(L, th, dop, [0, 0, 1, 3], num_hypotheses=8, tau=0.1, seed=1)
    assert list(o["status"][:2]) == [oracle.TOO_FEW_POINTS] * 2
    assert o["status"][2] == 0
    assert np.isnan(o["vx"][:2]).all() and list(o["best_hypothesis"][:2]) == [-1, -1]
    o = _est(L, th[:2], dop[:2], [0, 2], elevation=np.zeros(2), num_hypotheses=8, tau=0.1, seed=1)
    assert o["status"][0] == oracle.TOO_FEW_POINTS
    # every point at one azimuth: every minimal set is singular
    o = _est(L, np.full(6, 0.4), np.arange(6.0), [0, 6], num_hypotheses=32, tau=0.1, seed=1)
    assert o["status"][0] == oracle.ALL_DEGENERATE and o["best_hypothesis"][0] == -1
    assert o["inlier_mask"].sum() == 0 and np.isnan(o["heading"][0])
    # tau = 0: winners with fewer than k inliers keep their minimal-set velocity
    rng = np.random.default_rng(2)
    seen = 0
    for trial in range(40):
        n = 12
        th = rng.uniform(-1, 1, n)
        dop = rng.uniform(-20, 20, n)
        o = _est(L, th, dop, [0, n], num_hypotheses=8, tau=0.0, seed=trial, want_counts=True)
        b = o["best_hypothesis"][0]
        assert o["hyp_counts"][0][b] == o["hyp_counts"][0].max() == o["inlier_count"][0]
        if o["inlier_count"][0] < 2:
            assert o["status"][0] == oracle.LSQ_FALLBACK
            q = oracle.draw(trial, 0, int(b), n, 2, _lib=L)
            M = np.stack([np.cos(th[q]), np.sin(th[q])], 1)
            ref = np.linalg.solve(M, dop[q])
            assert np.allclose([o["vx"][0], o["vy"][0]], ref, rtol=1e-12, atol=1e-12)
            seen += 1
    assert seen > 0


def check_planted(L):
    w, f = _frame("frame64", 64)
    o = _est(L, f.azimuth, f.doppler, f.offsets, num_hypotheses=w.num_hypotheses, tau=w.tau, seed=1)
    m = o["inlier_mask"].astype(bool)
    assert m[~f.outlier].mean() > 0.9 and m[f.outlier].mean() < 0.05
    err = np.hypot(o["vx"] - f.truth_v[:, 0], o["vy"] - f.truth_v[:, 1])
    assert np.median(err) < 0.05


def _rows(f):
    th = f.azimuth.astype(np.float64)
    if f.elevation is None:
        return np.stack([np.cos(th), np.sin(th)], 1)
    el = f.elevation.astype(np.float64)
    return np.stack([np.cos(th) * np.cos(el), np.sin(th) * np.cos(el), np.sin(el)], 1)


def check_local_opt(L):
    for name, nc, H in (("stress2d", 96, 256), ("dense3d", 12, 256)):
        w, f = _frame(name, nc)
        A, dop, off = _rows(f), f.doppler.astype(np.float64), f.offsets
        k = A.shape[1]
        kw = dict(elevation=f.elevation, num_hypotheses=H, tau=w.tau, seed=1)
        base = _est(L, f.azimuth, f.doppler, off, **kw)
        zero = _est(L, f.azimuth, f.doppler, off, refine_iterations=0, **kw)
        for key in ("vx", "vy", "vz", "inlier_mask", "inlier_count", "status"):
            assert np.array_equal(base[key], zero[key], equal_nan=True), key
        one = _est(L, f.azimuth, f.doppler, off, refine_iterations=1, **kw)
        many = _est(L, f.azimuth, f.doppler, off, refine_iterations=12, **kw)
        more = _est(L, f.azimuth, f.doppler, off, refine_iterations=13, **kw)
        moved = fixed = 0
        for c in range(nc):
            if base["status"][c] != 0:
                continue
            s, e = off[c], off[c + 1]
            Ac, wc = A[s:e], dop[s:e]
            vb = np.array([base["vx"][c], base["vy"][c], base["vz"][c]])[:k]
            # one round: the inlier set is the re-threshold of the refined velocity
            r = np.abs(wc - Ac @ vb)
            clear = np.abs(r - w.tau) > 1e-9
            m1 = one["inlier_mask"][s:e].astype(bool)
            re = r <= w.tau
            if re.sum() >= k and not np.array_equal(re, base["inlier_mask"][s:e].astype(bool)):
                assert np.array_equal(m1[clear], re[clear]), c
                moved += 1
            for o in (one, many):
                m = o["inlier_mask"][s:e].astype(bool)
                assert m.sum() == o["inlier_count"][c]
                ref = np.linalg.lstsq(Ac[m], wc[m], rcond=None)[0]
                got = np.array([o["vx"][c], o["vy"][c], o["vz"][c]])[:k]
                assert np.allclose(got, ref, rtol=1e-9, atol=1e-9), (name, c, got, ref)
                assert abs(o["heading"][c] - math.atan2(got[1], got[0])) < 1e-12
            # converged (one more round changes nothing): threshold-then-fit fixed point
            if np.array_equal(many["inlier_mask"][s:e], more["inlier_mask"][s:e]):
                vm = np.array([many["vx"][c], many["vy"][c], many["vz"][c]])[:k]
                rm = np.abs(wc - Ac @ vm)
                cl = np.abs(rm - w.tau) > 1e-9
                assert np.array_equal(many["inlier_mask"][s:e].astype(bool)[cl], (rm <= w.tau)[cl]), c
                fixed += 1
        assert moved >= 5 and fixed >= nc // 2, (name, moved, fixed)
        # exact symmetries survive the rounds
        neg = _est(L, -f.azimuth.astype(np.float64), f.doppler, off, refine_iterations=12, **kw)
        assert np.array_equal(many["inlier_mask"], neg["inlier_mask"])
        assert np.array_equal(many["vy"], -neg["vy"]) and np.array_equal(many["vx"], neg["vx"])
        sc = _est(L, f.azimuth, f.doppler.astype(np.float64) * 8.0, off, refine_iterations=12,
                  **dict(kw, tau=w.tau * 8.0))
        assert np.array_equal(many["inlier_mask"], sc["inlier_mask"])
        assert np.array_equal(many["vx"] * 8.0, sc["vx"]) and np.array_equal(many["vy"] * 8.0, sc["vy"])


def _bound_holds(best, n, k, m, p):
    """(1 - (best/n)^k)^m <= 1 - p by Python's float power, or None when the
    two sides are too close to call against another evaluation order."""
    if best < 0:
        return False
    lhs = (1.0 - (best / n) ** k) ** m
    rhs = 1.0 - p
    if abs(lhs - rhs) <= 1e-9 * max(rhs, 1e-300):
        return None
    return lhs <= rhs


def check_adaptive(L):
    for name, nc, H, p, B in (("stress2d", 128, 512, 0.99, 32), ("frame64", 64, 256, 0.999, 64),
                              ("dense3d", 16, 512, 0.99, 32), ("stress2d", 64, 512, 0.9999999, 32)):
        w, f = _frame(name, nc)
        k = 2 if f.elevation is None else 3
        kw = dict(elevation=f.elevation, num_hypotheses=H, tau=w.tau, seed=2)
        full = _est(L, f.azimuth, f.doppler, f.offsets, want_counts=True, want_trials=True, **kw)
        assert (full["trials_used"][np.diff(f.offsets) >= k] == H).all()
        ad = _est(L, f.azimuth, f.doppler, f.offsets, confidence=p, trial_block=B, want_counts=True,
                  want_trials=True, **kw)
        n = np.diff(f.offsets)
        early = 0
        for c in range(nc):
            if n[c] < k:
                continue
            m = int(ad["trials_used"][c])
            assert m == H or m % B == 0, (c, m)
            cnt = full["hyp_counts"][c]
            assert np.array_equal(ad["hyp_counts"][c][:m], cnt[:m]) and (ad["hyp_counts"][c][m:] == -1).all()
            best = int(cnt[:m].max())
            assert ad["best_hypothesis"][c] == (int(np.argmax(cnt[:m])) if best >= 0 else -1)
            if best >= 0:
                assert ad["inlier_count"][c] == best or ad["status"][c] != 0
            if m < H:
                early += 1
                assert _bound_holds(best, int(n[c]), k, m, p) in (True, None), (c, m)
            for m2 in range(B, m, B):
                assert _bound_holds(int(cnt[:m2].max()), int(n[c]), k, m2, p) in (False, None), (c, m2)
            if ad["best_hypothesis"][c] == full["best_hypothesis"][c]:
                s_, e_ = f.offsets[c], f.offsets[c + 1]
                assert np.array_equal(ad["inlier_mask"][s_:e_], full["inlier_mask"][s_:e_])
                assert ad["vx"][c] == full["vx"][c] and ad["vy"][c] == full["vy"][c]
        assert early >= nc // 2, (name, early)
    # all-inlier (noise-free) clusters: eps = 1 stops after the first block
    rng = np.random.default_rng(8)
    th, _, dop = _noise_free(rng, 50, 2, np.array([12.0, -5.0, 0.0]))
    o = _est(L, th, dop, [0, 50], num_hypotheses=512, tau=0.1, seed=4, confidence=0.99, trial_block=32,
             want_trials=True)
    assert o["trials_used"][0] == 32 and o["inlier_count"][0] == 50


def _mad_threshold(th, dop):
    """Alg. 1's threshold with numpy: min-max normalised Doppler, then the
    median of its absolute deviations from its median."""
    dop = np.asarray(dop, np.float64)
    y = (dop - dop.min()) * (1.0 / (dop.max() - dop.min())) if dop.max() > dop.min() else np.zeros_like(dop)
    return np.median(np.abs(y - np.median(y)))


def _line_brute(th, dop):
    """Alg. 1 by exhaustion with numpy: counts of every seed pair (lexicographic),
    the MAD threshold, and the smallest decision margin."""
    x = (th - th.min()) * (1.0 / (th.max() - th.min())) if th.max() > th.min() else np.zeros_like(th)
    y = (dop - dop.min()) * (1.0 / (dop.max() - dop.min())) if dop.max() > dop.min() else np.zeros_like(dop)
    T = _mad_threshold(th, dop)
    counts, margin = [], np.inf
    for a, b in itertools.combinations(range(th.shape[0]), 2):
        dx, dy = x[b] - x[a], y[b] - y[a]
        if dx == 0.0:
            counts.append(-1)
            continue
        d = np.abs(dx * (y[a] - y) - (x[a] - x) * dy) / math.hypot(dx, dy)
        margin = min(margin, np.min(np.abs(d - T)))
        counts.append(int((d <= T).sum()))
    return np.array(counts), T, margin


def check_paper_line(L):
    rng = np.random.default_rng(31)
    done = 0
    while done < 20:
        n = int(rng.integers(4, 12))
        v = rng.uniform(-20, 20, 3)
        th, _, dop = _noise_free(rng, n, 2, v)
        dop = dop + rng.normal(0, 0.3, n)
        bad = rng.random(n) < 0.3
        dop[bad] = rng.uniform(-40, 40, int(bad.sum()))
        th = th.astype(np.float32).astype(np.float64)
        dop = dop.astype(np.float32).astype(np.float64)
        counts, T, margin = _line_brute(th, dop)
        if margin < 1e-9 or T == 0.0:
            continue
        o = _est(L, th, dop, [0, n], num_hypotheses=counts.shape[0], tau=0.1, seed=1, enumerate_subsets=True,
                 want_counts=True, line_model=True)
        assert np.array_equal(o["hyp_counts"][0], counts), (o["hyp_counts"][0], counts)
        assert o["best_hypothesis"][0] == int(np.argmax(counts))
        assert o["threshold"][0] == T  # the MAD threshold, numpy's median of |y - median y|
        done += 1
    # frames: refine = lstsq of the inliers; Doppler x 2^m exact; shapes of the outputs
    w, f = _frame("stress2d", 64)
    kw = dict(num_hypotheses=256, tau=w.tau, seed=5, line_model=True)
    o = _est(L, f.azimuth, f.doppler, f.offsets, want_counts=True, **kw)
    A = _rows(f)
    dop = f.doppler.astype(np.float64)
    checked = 0
    for c in range(64):
        s_, e_ = f.offsets[c], f.offsets[c + 1]
        m = o["inlier_mask"][s_:e_].astype(bool)
        assert m.sum() == o["inlier_count"][c] == o["hyp_counts"][c].max()
        if o["status"][c] == 0:
            ref = np.linalg.lstsq(A[s_:e_][m], dop[s_:e_][m], rcond=None)[0]
            assert np.allclose([o["vx"][c], o["vy"][c]], ref, rtol=1e-9, atol=1e-9), c
            checked += 1
    assert checked >= 60
    for c in range(64):  # each cluster's MAD threshold, as numpy forms it
        s_, e_ = f.offsets[c], f.offsets[c + 1]
        assert o["threshold"][c] == _mad_threshold(f.azimuth[s_:e_], dop[s_:e_]), c
    # the cosine model reports tau for every cluster
    cos_o = _est(L, f.azimuth, f.doppler, f.offsets, num_hypotheses=8, tau=w.tau, seed=5)
    assert np.all(cos_o["threshold"] == w.tau)
    sc = _est(L, f.azimuth, dop * 4.0, f.offsets, want_counts=True, **kw)
    assert np.array_equal(o["hyp_counts"], sc["hyp_counts"]) and np.array_equal(o["inlier_mask"], sc["inlier_mask"])
    assert np.array_equal(o["vx"] * 4.0, sc["vx"]) and np.array_equal(o["vy"] * 4.0, sc["vy"])
    # affine (azimuth, Doppler): every point lies on the seeds' line
    th = np.linspace(-0.9, 0.8, 33)
    lin = _est(L, th, 3.0 * th + 1.0, [0, 33], num_hypotheses=16, tau=0.1, seed=2, want_counts=True, line_model=True)
    assert (lin["hyp_counts"][0] == 33).all() and lin["inlier_count"][0] == 33
    # one azimuth for every point: every seed pair shares x
    deg = _est(L, np.full(6, 0.3), np.arange(6.0), [0, 6], num_hypotheses=8, tau=0.1, seed=1, line_model=True)
    assert deg["status"][0] == oracle.ALL_DEGENERATE
    # NaN Dopplers (the reading of Alg. 1's normalize() and median for them):
    # the extremes are taken over the numbers, the medians sort NaN after
    # every number, and a NaN point is never an inlier
    rng2 = np.random.default_rng(37)
    for trial in range(6):
        n = int(rng2.integers(9, 15))
        th = np.sort(rng2.uniform(-1.0, 1.0, n))
        dop = 5.0 * np.cos(th) + rng2.normal(0, 0.2, n)
        nan_at = rng2.choice(n, size=int(rng2.integers(1, 3)), replace=False)
        dop[nan_at] = np.nan

        def med_nan_last(a):
            s_ = np.sort(a)  # numpy sorts NaN after every number
            k = s_.shape[0]
            return s_[k // 2] if k % 2 else 0.5 * (s_[k // 2 - 1] + s_[k // 2])

        lo, hi = np.nanmin(dop), np.nanmax(dop)
        y = (dop - lo) * (1.0 / (hi - lo))
        T = med_nan_last(np.abs(y - med_nan_last(np.abs(y))))
        o = _est(L, th, dop, [0, n], num_hypotheses=64, tau=0.1, seed=trial, line_model=True)
        assert np.isfinite(T) and o["threshold"][0] == T, (o["threshold"][0], T)
        assert not o["inlier_mask"][nan_at].any()


def _canonical(labels):
    """Partition as a set of frozensets of point indices (noise dropped)."""
    out = {}
    for i, l in enumerate(labels.tolist()):
        if l >= 0:
            out.setdefault(l, []).append(i)
    return {frozenset(v) for v in out.values()}


def check_dbscan(L):
    pytest_sklearn = __import__("importlib").util.find_spec("sklearn") is not None
    rng = np.random.default_rng(17)
    cases = [(rng.uniform(0, 20, (400, 2)), 0.9, 4), (rng.normal(0, 3, (300, 3)), 1.1, 5),
             (rng.uniform(0, 10, (250, 1)), 0.08, 3), (rng.uniform(0, 6, (200, 4)), 1.6, 6)]
    w = synth.make_scene(synth.SCENES["scene_small"])
    cases.append((w.features().astype(np.float64), 1.0, 4))
    for f, eps, mp in cases:
        f = f.astype(np.float32).astype(np.float64)
        D = np.sqrt(((f[:, None, :] - f[None, :, :]) ** 2).sum(-1))
        if np.min(np.abs(D - eps)) < 1e-9 * eps:
            continue
        o = oracle.dbscan(f, eps, mp, _lib=L)
        lab, core = o["labels"], o["core"]
        nb = D <= eps
        assert np.array_equal(core, nb.sum(1) >= mp)
        # numbering: cluster ids in the order of their smallest core index
        firsts = [int(np.flatnonzero(core & (lab == c))[0]) for c in range(o["n_clusters"])]
        assert firsts == sorted(firsts)
        # border points: the lowest-index core neighbour's cluster; noise: no core neighbour
        for p in np.flatnonzero(~core):
            cn = np.flatnonzero(nb[p] & core)
            assert lab[p] == (lab[cn[0]] if cn.size else -1), p
        if pytest_sklearn:
            from sklearn.cluster import DBSCAN
            sk = DBSCAN(eps=eps, min_samples=mp).fit(f)
            skcore = np.zeros(f.shape[0], bool)
            skcore[sk.core_sample_indices_] = True
            assert np.array_equal(core, skcore)
            assert np.array_equal(lab == -1, sk.labels_ == -1)
            assert _canonical(np.where(core, lab, -1)) == _canonical(np.where(core, sk.labels_, -1))
        # permuting the points permutes the partition of the core points
        perm = rng.permutation(f.shape[0])
        op = oracle.dbscan(f[perm], eps, mp, _lib=L)
        back = np.empty_like(perm)
        back[perm] = np.arange(perm.shape[0])
        assert np.array_equal(op["core"][back], core)
        assert _canonical(np.where(core, op["labels"][back], -1)) == _canonical(np.where(core, lab, -1))
    # min_pts = 1: every point is core; clusters = connected components of the eps-graph
    from scipy.sparse.csgraph import connected_components
    f = rng.uniform(0, 12, (300, 2)).astype(np.float32).astype(np.float64)
    D = np.sqrt(((f[:, None, :] - f[None, :, :]) ** 2).sum(-1))
    o = oracle.dbscan(f, 0.7, 1, _lib=L)
    ncc, cc = connected_components(D <= 0.7, directed=False)
    assert o["core"].all() and o["n_clusters"] == ncc
    assert _canonical(o["labels"]) == _canonical(cc)
    # eps = 0: only coincident points are neighbours
    g = np.repeat(np.arange(5.0)[:, None], 3, axis=0)
    o = oracle.dbscan(g, 0.0, 3, _lib=L)
    assert o["n_clusters"] == 5 and o["core"].all()


def check_fragile(L):
    v = np.array([12.5, -3.25])
    th = np.linspace(-1.0, 1.0, 30)               # minimal sets far from singular
    dop = v[0] * np.cos(th) + v[1] * np.sin(th)  # noise-free inliers
    t_x = 0.3125
    base = v[0] * math.cos(t_x) + v[1] * math.sin(t_x)
    tau = 0.1

    def flagged(w_extra, t_extra=t_x):
        az = np.append(th, t_extra)
        dp = np.append(dop, w_extra)
        o = _est(L, az, dp, [0, az.shape[0]], num_hypotheses=64, tau=tau, seed=3, want_fragile=True)
        assert o["inlier_count"][0] in (30, 31) and o["status"][0] == 0
        return bool(o["fragile"][0])

    # at the threshold to within a few ulps, on either side: flagged
    for sign in (1.0, -1.0):
        w0 = base + sign * tau
        for k in range(-2, 3):
            w = w0
            for _ in range(abs(k)):
                w = np.nextafter(w, math.inf if k > 0 else -math.inf)
            assert flagged(w), (sign, k)
    # clear of it by 1e-9 m/s: not flagged
    for w in (base + tau + 1e-9, base + tau - 1e-9, base - tau + 1e-9, base - tau - 1e-9, base, base + 1.0):
        assert not flagged(w), w
    # a minimal set whose determinant sits on cond_eps (two points, one trial)
    a0, a1 = 0.2, 0.9
    det = math.cos(a0) * math.sin(a1) - math.sin(a0) * math.cos(a1)  # = sin(a1 - a0) to ~1e-16
    for eps, want in ((abs(det), True), (abs(det) * (1 + 1e-6), False), (abs(det) * (1 - 1e-6), False)):
        o = _est(L, np.array([a0, a1]), np.array([1.0, 2.0]), [0, 2], num_hypotheses=1, tau=tau, seed=1,
                 cond_eps=eps, want_fragile=True)
        assert bool(o["fragile"][0]) == want, (eps, det)
    # realistic frames: nothing within rounding distance of a decision
    for name in ("frame64", "dense2d"):
        w = synth.WORKLOADS[name]
        f = synth.make_frame(w)
        sub = None if name == "frame64" else np.sort(np.random.default_rng(2).choice(f.n_clusters, 384, replace=False))
        o = _est(L, f.azimuth, f.doppler, f.offsets, num_hypotheses=w.num_hypotheses, tau=w.tau, seed=w.seed,
                 subset=sub, want_fragile=True)
        assert not o["fragile"].any(), (name, np.flatnonzero(o["fragile"]))


def check_first_cluster(L):
    w = synth.WORKLOADS["frame64"]
    f = synth.make_frame(w, n_clusters=24, gen_seed=29)
    c0, c1 = 9, 17
    p0, p1 = int(f.offsets[c0]), int(f.offsets[c1])
    off = (f.offsets[c0:c1 + 1] - p0).astype(np.int32)
    part = _est(L, f.azimuth[p0:p1], f.doppler[p0:p1], off, num_hypotheses=64, tau=w.tau, seed=5, first_cluster=c0)
    whole = _est(L, f.azimuth, f.doppler, f.offsets, num_hypotheses=64, tau=w.tau, seed=5,
                 subset=np.arange(c0, c1, dtype=np.int32))
    for k in ("best_hypothesis", "inlier_count", "status", "vx", "vy"):
        assert np.array_equal(part[k], whole[k], equal_nan=True), k
    assert np.array_equal(part["inlier_mask"], whole["inlier_mask"][p0:p1])
    # and not the draws of a frame whose clusters start at 0
    plain = _est(L, f.azimuth[p0:p1], f.doppler[p0:p1], off, num_hypotheses=64, tau=w.tau, seed=5)
    assert not np.array_equal(plain["best_hypothesis"], part["best_hypothesis"])


ALL_CHECKS = [check_philox, check_draws, check_recovery, check_brute, check_symmetry,
              check_rotation, check_lstsq, check_status, check_planted, check_local_opt, check_adaptive,
              check_paper_line, check_dbscan, check_fragile, check_first_cluster]
