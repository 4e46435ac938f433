/*
 * rvh oracle -- TEST INFRASTRUCTURE ONLY (see rvh_oracle.h).
 *
 * Plain single-threaded FP64 C, built with -ffp-contract=off so that every
 * multiply and add below rounds exactly where it is written; fused
 * multiply-adds appear only as explicit fma() calls.
 *
 * Parity pins: the not-gpu tests check this file against closed forms
 * (noise-free recovery), brute force on tiny clusters, exact symmetries and
 * numpy's least squares; see tests/test_oracle.py.
 */
#include "rvh_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  Stands in for the "random numbers spanning
 * indices for every cluster" that Alg. 1 takes as input.
 * ------------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;  /* round multipliers */
  const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;  /* key schedule increments */
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += weyl0;
      k1 += weyl1;
    }
    uint64_t p0 = (uint64_t)mult0 * x0;
    uint64_t p1 = (uint64_t)mult1 * x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* floor(w * n / 2^32): a 32-bit random word scaled to [0, n). */
static uint32_t scale_to_range(uint32_t w, uint32_t n) {
  return (uint32_t)(((uint64_t)w * (uint64_t)n) >> 32);
}

int oracle_draw(uint64_t seed, int32_t cluster, int32_t h, int32_t n, int32_t k, int32_t* q) {
  if (n < k || (k != 2 && k != 3)) return -1;
  uint32_t ctr[4] = {(uint32_t)h, (uint32_t)cluster, 0u, 0u};
  uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
  uint32_t w[4];
  oracle_philox4x32_10(ctr, key, w);
  /* first index uniform on [0, n); second uniform on the n-1 others */
  uint32_t q0 = scale_to_range(w[0], (uint32_t)n);
  uint32_t q1 = scale_to_range(w[1], (uint32_t)n - 1u);
  if (q1 >= q0) q1 += 1u;
  q[0] = (int32_t)q0;
  q[1] = (int32_t)q1;
  if (k == 3) {
    /* third index uniform on the n-2 indices not yet taken */
    uint32_t lo = q0 < q1 ? q0 : q1;
    uint32_t hi = q0 < q1 ? q1 : q0;
    uint32_t q2 = scale_to_range(w[2], (uint32_t)n - 2u);
    if (q2 >= lo) q2 += 1u;
    if (q2 >= hi) q2 += 1u;
    q[2] = (int32_t)q2;
  }
  return 0;
}

/* The h-th k-subset (k = 2 or 3) of {0..n-1} in lexicographic order; returns
 * -1 when h is past the last one.  Used by the brute-force tests. */
static int enumerate_subset(int64_t h, int32_t n, int32_t k, int32_t* q) {
  if (h < 0) return -1;
  if (k == 2) {
    for (int32_t a = 0; a < n - 1; ++a) {
      int64_t span = n - 1 - a;
      if (h < span) { q[0] = a; q[1] = a + 1 + (int32_t)h; return 0; }
      h -= span;
    }
    return -1;
  }
  for (int32_t a = 0; a < n - 2; ++a) {
    for (int32_t b = a + 1; b < n - 1; ++b) {
      int64_t span = n - 1 - b;
      if (h < span) { q[0] = a; q[1] = b; q[2] = b + 1 + (int32_t)h; return 0; }
      h -= span;
    }
  }
  return -1;
}

/* 2x2 determinant |x y; z w| = x*w - y*z, one rounding for the product y*z
 * and one for the fused x*w - (y*z). */
static double det2(double x, double y, double z, double w) {
  return fma(x, w, -(y * z));
}

/* 3x3 determinant by cofactor expansion along row 0 (rows m0, m1, m2). */
static double det3(const double* m0, const double* m1, const double* m2) {
  double k0 = det2(m1[1], m1[2], m2[1], m2[2]);
  double k1 = det2(m1[0], m1[2], m2[0], m2[2]);
  double k2 = det2(m1[0], m1[1], m2[0], m2[1]);
  return fma(m0[2], k2, fma(-m0[1], k1, m0[0] * k0));
}

/* Solve the k x k system with rows a[0..k-1] (a[i] has k entries) and right
 * side w by Cramer's rule.  Returns the determinant; v is written only when
 * |det| >= eps (the conditioning test).  NaN determinants are rejected. */
static double cramer_solve(int k, const double* a0, const double* a1, const double* a2,
                           const double* w, double eps, double* v, int* ok) {
  if (k == 2) {
    double det = det2(a0[0], a0[1], a1[0], a1[1]);
    *ok = fabs(det) >= eps;
    if (*ok) {
      v[0] = det2(w[0], a0[1], w[1], a1[1]) / det;
      v[1] = det2(a0[0], w[0], a1[0], w[1]) / det;
      v[2] = 0.0;
    }
    return det;
  }
  double det = det3(a0, a1, a2);
  *ok = fabs(det) >= eps;
  if (*ok) {
    for (int col = 0; col < 3; ++col) {
      double r0[3] = {a0[0], a0[1], a0[2]};
      double r1[3] = {a1[0], a1[1], a1[2]};
      double r2[3] = {a2[0], a2[1], a2[2]};
      r0[col] = w[0];
      r1[col] = w[1];
      r2[col] = w[2];
      v[col] = det3(r0, r1, r2) / det;
    }
  }
  return det;
}

/* Doppler residual of point row a (k entries) with Doppler w under velocity v:
 * the deviation from Eq. (LSQ_eq), r = w - a.v. */
static double residual(int k, const double* a, double w, const double* v) {
  if (k == 2) return w - fma(v[0], a[0], v[1] * a[1]);
  return w - fma(v[0], a[0], fma(v[1], a[1], v[2] * a[2]));
}

/* x^n by binary exponentiation (squarings from the lowest bit up), one
 * rounding per multiplication in this order. */
static double pow_uint(double x, int32_t n) {
  double r = 1.0, b = x;
  while (n > 0) {
    if (n & 1) r = r * b;
    b = b * b;
    n >>= 1;
  }
  return r;
}

/* Adaptive trial count: after m trials with best count `best` of n points,
 * stop once (1 - eps^k)^m <= 1 - p with eps = best / n. */
static int adaptive_stop(int32_t best, int32_t n, int k, int32_t m, double p) {
  if (best < 0) return 0;
  double eps = (double)best / (double)n;
  double ek = k == 2 ? eps * eps : (eps * eps) * eps;
  return pow_uint(1.0 - ek, m) <= 1.0 - p;
}

/* Ascending order with NaN after every number. */
static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  if (isnan(x) || isnan(y)) return isnan(x) - isnan(y);
  return (x > y) - (x < y);
}

/* Median of v[0..n-1] (n >= 1); v is reordered.  Even n: the mean of the two
 * middle values, 0.5 * (lo + hi). */
static double median(double* v, int32_t n) {
  qsort(v, (size_t)n, sizeof(double), cmp_double);
  if (n & 1) return v[n / 2];
  return 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

/* Alg. 1 point-to-line test: perpendicular distance of (x, y) to
 * y = m x + c, with aa = -m, bb = 1, cc = -c, evaluated as printed:
 * distn = aa x + bb y + cc, distd = sqrt(aa^2 + bb^2), dist = |distn / distd|. */
static int line_inlier(double m, double c, double distd, double x, double y, double thresh) {
  double distn = (-m) * x + 1.0 * y + (-c);
  return fabs(distn / distd) <= thresh;
}

static void write_invalid(int32_t out, double* vx, double* vy, double* vz, double* heading,
                          int32_t* inlier_count, int32_t* best, int32_t* status, int32_t bits) {
  vx[out] = NAN;
  vy[out] = NAN;
  if (vz) vz[out] = NAN;
  heading[out] = NAN;
  inlier_count[out] = 0;
  best[out] = -1;
  status[out] = bits;
}

int oracle_estimate(const double* azimuth, const double* elevation, const double* doppler,
                    const int32_t* offsets, int32_t n_clusters,
                    const int32_t* subset, int32_t n_subset, const orc_params* p,
                    double* vx, double* vy, double* vz, double* heading,
                    int32_t* inlier_count, int32_t* best_hypothesis, int32_t* status,
                    uint8_t* mask, int32_t* hyp_counts, uint8_t* fragile, int32_t* trials_used,
                    double* threshold) {
  if (!p || !offsets || !azimuth || !doppler || n_clusters < 0) return -1;
  const int k = p->model_dim;
  if (k != 2 && k != 3) return -1;
  if ((k == 3) != (elevation != NULL)) return -1;
  if (p->num_hypotheses < 1 || !(p->tau >= 0.0)) return -1;
  if (!(p->confidence >= 0.0 && p->confidence < 1.0)) return -1;
  if (p->confidence > 0.0 && p->trial_block < 1) return -1;
  if (p->line_model && (k != 2 || p->refine_iterations != 0)) return -1;
  if (p->first_cluster < 0 || (int64_t)p->first_cluster + n_clusters > 0x7fffffffLL) return -1;
  const int32_t H = p->num_hypotheses;
  const double tau = p->tau;
  const int32_t n_out = subset ? n_subset : n_clusters;

  for (int32_t oi = 0; oi < n_out; ++oi) {
    const int32_t ci = subset ? subset[oi] : oi;
    if (ci < 0 || ci >= n_clusters) return -1;
    const int64_t o = offsets[ci];
    const int32_t n = (int32_t)(offsets[ci + 1] - offsets[ci]);
    if (fragile) fragile[oi] = 0;
    if (trials_used) trials_used[oi] = 0;
    if (threshold) threshold[oi] = p->line_model ? NAN : tau;
    for (int32_t q = 0; q < n; ++q) mask[o + q] = 0;
    if (hyp_counts)
      for (int32_t h = 0; h < H; ++h) hyp_counts[(int64_t)oi * H + h] = -1;

    if (n < k) {
      write_invalid(oi, vx, vy, vz, heading, inlier_count, best_hypothesis, status,
                    ORC_TOO_FEW_POINTS);
      continue;
    }

    /* Rows of A_i (Eq. eq:LSQPerCluster): (cos t, sin t) in 2D; with an
     * elevation e, (cos t cos e, sin t cos e, sin e). */
    double* a = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    int32_t* counts = (int32_t*)malloc(sizeof(int32_t) * (size_t)H);
    double* hyp_v = (double*)malloc(sizeof(double) * 3 * (size_t)H);
    double* hyp_det = (double*)malloc(sizeof(double) * (size_t)H);
    for (int32_t q = 0; q < n; ++q) {
      double t = azimuth[o + q];
      double c = cos(t), s = sin(t);
      if (k == 2) {
        a[3 * q + 0] = c;
        a[3 * q + 1] = s;
        a[3 * q + 2] = 0.0;
      } else {
        double e = elevation[o + q];
        double ce = cos(e), se = sin(e);
        a[3 * q + 0] = c * ce;
        a[3 * q + 1] = s * ce;
        a[3 * q + 2] = se;
      }
      w[q] = doppler[o + q];
    }

    /* Alg. 1 as printed (line_model): normalised (azimuth, Doppler) points
     * and the cluster's MAD threshold (Eq. eq:MAD, read as med |y - med y|). */
    double* xn = NULL;
    double* yn = NULL;
    double thresh = 0.0;
    if (p->line_model) {
      xn = (double*)malloc(sizeof(double) * (size_t)n);
      yn = (double*)malloc(sizeof(double) * (size_t)n);
      /* extremes over the numbers (NaN ignored) */
      double tmin = INFINITY, tmax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
      for (int32_t q = 0; q < n; ++q) {
        tmin = fmin(tmin, azimuth[o + q]);
        tmax = fmax(tmax, azimuth[o + q]);
        vmin = fmin(vmin, w[q]);
        vmax = fmax(vmax, w[q]);
      }
      double rt = tmax > tmin ? 1.0 / (tmax - tmin) : 0.0;
      double rv = vmax > vmin ? 1.0 / (vmax - vmin) : 0.0;
      for (int32_t q = 0; q < n; ++q) {
        xn[q] = (azimuth[o + q] - tmin) * rt;
        yn[q] = (w[q] - vmin) * rv;
      }
      double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
      for (int32_t q = 0; q < n; ++q) tmp[q] = fabs(yn[q]);  /* y >= 0; fabs makes NaN positive */
      double med = median(tmp, n);
      for (int32_t q = 0; q < n; ++q) tmp[q] = fabs(yn[q] - med);
      thresh = median(tmp, n);
      free(tmp);
      if (threshold) threshold[oi] = thresh;
    }

    /* Alg. 1 for every trial h: draw the minimal set, solve it, count the
     * points within tau.  The winner is the first trial with the largest
     * count (Sec. III-A). */
    int32_t best = -1, best_count = -1;
    double min_det_margin = INFINITY;
    int32_t trials = 0;
    for (int32_t h = 0; h < H; ++h) {
      counts[h] = -1;
      hyp_det[h] = INFINITY;
    }
    for (int32_t h = 0; h < H; ++h) {
      trials = h + 1;
      do {
        int32_t qs[3] = {0, 0, 0};
        int drawn = p->enumerate ? enumerate_subset(h, n, k, qs)
                                 : oracle_draw(p->seed, p->first_cluster + ci, h, n, k, qs);
        if (drawn != 0) break;
        if (p->line_model) {
          /* Alg. 1: slope and intercept through the two normalised seeds */
          double dx = xn[qs[1]] - xn[qs[0]];
          if (dx == 0.0) break;
          double m = (yn[qs[1]] - yn[qs[0]]) / dx;
          double c = yn[qs[0]] - m * xn[qs[0]];
          double distd = sqrt(m * m + 1.0);
          int32_t count = 0;
          for (int32_t q = 0; q < n; ++q) count += line_inlier(m, c, distd, xn[q], yn[q], thresh);
          counts[h] = count;
          hyp_v[3 * h + 0] = m;
          hyp_v[3 * h + 1] = c;
          hyp_v[3 * h + 2] = distd;
          if (count > best_count) {
            best_count = count;
            best = h;
          }
          break;
        }
        double rhs[3] = {w[qs[0]], w[qs[1]], k == 3 ? w[qs[2]] : 0.0};
        double v[3] = {0.0, 0.0, 0.0};
        int ok = 0;
        double det = cramer_solve(k, &a[3 * qs[0]], &a[3 * qs[1]], k == 3 ? &a[3 * qs[2]] : NULL,
                                  rhs, p->cond_eps, v, &ok);
        double dm = fabs(fabs(det) - p->cond_eps);
        if (dm < min_det_margin) min_det_margin = dm;
        hyp_det[h] = det;
        if (!ok) break;
        int32_t count = 0;
        for (int32_t q = 0; q < n; ++q)
          if (fabs(residual(k, &a[3 * q], w[q], v)) <= tau) ++count;
        counts[h] = count;
        hyp_v[3 * h + 0] = v[0];
        hyp_v[3 * h + 1] = v[1];
        hyp_v[3 * h + 2] = v[2];
        if (count > best_count) {
          best_count = count;
          best = h;
        }
      } while (0);
      /* adaptive trial count: check the bound after every block of trials */
      if (p->confidence > 0.0 && trials % p->trial_block == 0 && trials < H &&
          adaptive_stop(best_count, n, k, trials, p->confidence))
        break;
    }
    if (trials_used) trials_used[oi] = trials;
    if (hyp_counts)
      for (int32_t h = 0; h < H; ++h) hyp_counts[(int64_t)oi * H + h] = counts[h];

    int frag = min_det_margin < 1e-13;
    if (best < 0) {
      write_invalid(oi, vx, vy, vz, heading, inlier_count, best_hypothesis, status,
                    ORC_ALL_DEGENERATE);
      if (fragile) fragile[oi] = (uint8_t)frag;
      free(a); free(w); free(counts); free(hyp_v); free(hyp_det); free(xn); free(yn);
      continue;
    }

    /* Fragility log: a residual test of a trial within one of the winning
     * count whose margin |(|r| - tau)| is below what a few-ulp change of the
     * row values (another libm's cos/sin) can move it: the trial's velocity
     * moves by ~ulp * |v| / |det| and the residual by that times |a| <= 1. */
    if (fragile && !p->line_model) {
      for (int32_t h = 0; h < trials && !frag; ++h) {
        if (counts[h] < 0 || counts[h] < best_count - 1) continue;
        const double* v = &hyp_v[3 * h];
        double scale = fabs(v[0]) + fabs(v[1]) + fabs(v[2]);
        double amp = 1e-14 * (1.0 + 1.0 / fabs(hyp_det[h]));
        for (int32_t q = 0; q < n; ++q) {
          double r = residual(k, &a[3 * q], w[q], v);
          if (fabs(fabs(r) - tau) <= amp * (scale + fabs(w[q]) + tau)) { frag = 1; break; }
        }
      }
    }

    /* Inlier mask of the winner (the per-cluster mask; the frame mask of
     * Sec. III-A is their union over clusters) and the refine sums over the
     * inliers in index order: G = sum a a^T, g = sum a w. */
    const double* vb = &hyp_v[3 * best];
    int32_t n_in = 0;
    double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double g[3] = {0, 0, 0};
    for (int32_t q = 0; q < n; ++q) {
      const double* aq = &a[3 * q];
      int in = p->line_model ? line_inlier(vb[0], vb[1], vb[2], xn[q], yn[q], thresh)
                             : fabs(residual(k, aq, w[q], vb)) <= tau;
      if (!in) continue;
      mask[o + q] = 1;
      ++n_in;
      for (int r = 0; r < k; ++r) {
        for (int c = r; c < k; ++c) G[r][c] = fma(aq[r], aq[c], G[r][c]);
        g[r] = fma(aq[r], w[q], g[r]);
      }
    }
    for (int r = 0; r < k; ++r)
      for (int c = 0; c < r; ++c) G[r][c] = G[c][r];

    /* Eq. (eq:LSQPerCluster): v = A^+ v_r = (A^T A)^-1 A^T v_r on the
     * inliers, solved by Cramer's rule; singular or short systems fall back
     * to the winning minimal-set velocity. */
    double trace = 0.0;
    for (int r = 0; r < k; ++r) trace += G[r][r];
    double limit = 1e-12 * (k == 2 ? trace * trace : trace * trace * trace);
    double vout[3] = {vb[0], vb[1], vb[2]};
    int32_t st = 0;
    double detG = k == 2 ? det2(G[0][0], G[0][1], G[1][0], G[1][1])
                         : det3(G[0], G[1], G[2]);
    if (fabs(fabs(detG) - limit) <= 1e-13 * (k == 2 ? trace * trace : trace * trace * trace))
      frag = 1;
    int solved = 0;
    double cnd = 0.0; /* trace^k / |det G|: bounds the condition number of G */
    if (n_in >= k && fabs(detG) > limit) {
      double vs[3];
      int ok = 0;
      cramer_solve(k, G[0], G[1], G[2], g, 0.0, vs, &ok);
      vout[0] = vs[0];
      vout[1] = vs[1];
      vout[2] = k == 3 ? vs[2] : 0.0;
      solved = 1;
      cnd = (k == 2 ? trace * trace : trace * trace * trace) / fabs(detG);
    } else {
      st |= ORC_LSQ_FALLBACK;
      if (p->line_model) vout[0] = vout[1] = vout[2] = NAN;
    }

    /* Local optimisation rounds: re-threshold all points against the current
     * least-squares velocity (the same residual test as Alg. 1) and solve the
     * normal equations of the new inlier set.  A round that changes nothing
     * ends the loop; so does a new set whose system is short or singular,
     * in which case the previous velocity and inlier set stand.  After a
     * fallback the current velocity is the winner's, whose re-threshold
     * reproduces the current set, so nothing changes. */
    if (solved && p->refine_iterations > 0) {
      uint8_t* m2 = (uint8_t*)malloc((size_t)n);
      for (int32_t it = 0; it < p->refine_iterations; ++it) {
        int32_t n2 = 0, changed = 0;
        double G2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        double g2[3] = {0, 0, 0};
        /* another order of the same sums moves the solved velocity by about
         * n u cond(G) |v|: decisions that close to tau are rounding ties */
        double amp = 1e-12 * (1.0 + cnd);
        double vs1 = fabs(vout[0]) + fabs(vout[1]) + fabs(vout[2]);
        for (int32_t q = 0; q < n; ++q) {
          const double* aq = &a[3 * q];
          double r = residual(k, aq, w[q], vout);
          uint8_t in = fabs(r) <= tau;
          if (fabs(fabs(r) - tau) <= amp * (vs1 + fabs(w[q]) + tau)) frag = 1;
          m2[q] = in;
          if (in != mask[o + q]) changed = 1;
          if (!in) continue;
          ++n2;
          for (int rr = 0; rr < k; ++rr) {
            for (int cc = rr; cc < k; ++cc) G2[rr][cc] = fma(aq[rr], aq[cc], G2[rr][cc]);
            g2[rr] = fma(aq[rr], w[q], g2[rr]);
          }
        }
        if (!changed) break;
        for (int rr = 0; rr < k; ++rr)
          for (int cc = 0; cc < rr; ++cc) G2[rr][cc] = G2[cc][rr];
        double tr2 = 0.0;
        for (int rr = 0; rr < k; ++rr) tr2 += G2[rr][rr];
        double trk = k == 2 ? tr2 * tr2 : tr2 * tr2 * tr2;
        double det2G = k == 2 ? det2(G2[0][0], G2[0][1], G2[1][0], G2[1][1]) : det3(G2[0], G2[1], G2[2]);
        if (fabs(fabs(det2G) - 1e-12 * trk) <= 1e-13 * trk) frag = 1;
        if (!(n2 >= k && fabs(det2G) > 1e-12 * trk)) break;
        double vs[3];
        int ok = 0;
        cramer_solve(k, G2[0], G2[1], G2[2], g2, 0.0, vs, &ok);
        vout[0] = vs[0];
        vout[1] = vs[1];
        vout[2] = k == 3 ? vs[2] : 0.0;
        cnd = trk / fabs(det2G);
        n_in = n2;
        for (int32_t q = 0; q < n; ++q) mask[o + q] = m2[q];
      }
      free(m2);
    }

    vx[oi] = vout[0];
    vy[oi] = vout[1];
    if (vz) vz[oi] = k == 3 ? vout[2] : 0.0;
    heading[oi] = atan2(vout[1], vout[0]); /* Alg. 2 heading, quadrant-aware */
    inlier_count[oi] = n_in;
    best_hypothesis[oi] = best;
    status[oi] = st;
    if (fragile) fragile[oi] = (uint8_t)frag;
    free(a); free(w); free(counts); free(hyp_v); free(hyp_det); free(xn); free(yn);
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * DBSCAN (Ester, Kriegel, Sander, Xu, KDD'96), the clustering that precedes
 * the estimator in Fig. 1.  Brute force over all pairs: plain and O(n^2).
 * ------------------------------------------------------------------------- */

/* Squared Euclidean distance, accumulated in FP64 over the components in order. */
static double feat_dist2(const double* a, const double* b, int32_t dim) {
  double s = 0.0;
  for (int32_t k = 0; k < dim; ++k) {
    double d = a[k] - b[k];
    s = s + d * d;
  }
  return s;
}

int oracle_dbscan(const double* feat, int64_t n, int32_t dim, double eps, int32_t min_pts,
                  int32_t* labels, uint8_t* core, int32_t* n_clusters) {
  if (n < 0 || dim < 1 || dim > 4 || !(eps >= 0.0) || min_pts < 1 || !labels || !n_clusters) return -1;
  if (n > 0 && !feat) return -1;
  const double eps2 = eps * eps;
  uint8_t* is_core = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  /* core points: at least min_pts neighbours, the point itself included */
  for (int64_t p = 0; p < n; ++p) {
    int64_t count = 0;
    for (int64_t q = 0; q < n && count < min_pts; ++q)
      if (feat_dist2(&feat[p * dim], &feat[q * dim], dim) <= eps2) ++count;
    is_core[p] = count >= min_pts;
    labels[p] = -1;
  }
  /* clusters: grow each from its lowest-index unlabelled core point over the
   * core-to-core neighbour relation */
  int32_t c = 0;
  for (int64_t p = 0; p < n; ++p) {
    if (!is_core[p] || labels[p] != -1) continue;
    int64_t top = 0;
    labels[p] = c;
    stack[top++] = p;
    while (top > 0) {
      int64_t u = stack[--top];
      for (int64_t q = 0; q < n; ++q) {
        if (!is_core[q] || labels[q] != -1) continue;
        if (feat_dist2(&feat[u * dim], &feat[q * dim], dim) <= eps2) {
          labels[q] = c;
          stack[top++] = q;
        }
      }
    }
    ++c;
  }
  /* border points: the cluster of the lowest-index core neighbour */
  for (int64_t p = 0; p < n; ++p) {
    if (is_core[p]) continue;
    for (int64_t q = 0; q < n; ++q) {
      if (is_core[q] && feat_dist2(&feat[p * dim], &feat[q * dim], dim) <= eps2) {
        labels[p] = labels[q];
        break;
      }
    }
  }
  if (core)
    for (int64_t p = 0; p < n; ++p) core[p] = is_core[p];
  *n_clusters = c;
  free(is_core);
  free(stack);
  return 0;
}
