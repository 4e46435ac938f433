// Device building blocks shared by the rvh kernels: the counter-based draw of
// minimal sets, FP32 point rows, the FP32 minimal-set solve with its rigorous
// error bound, and the FP64 solve whose rounding sequence defines the exact
// inlier decisions.
//
// The whole library is compiled with -fmad=false: every fused multiply-add is
// an explicit fmaf()/fma() call, so the FP32 error bounds below describe the
// operations that actually run.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rvh.h"
#include "rvh_kernels.h"

namespace rvh {

// ---- counter-based random minimal sets (stand-in for Alg. 1's host-side index arrays) --

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint2 key) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round) {
      key.x += 0x9E3779B9u;
      key.y += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * x.x, p1 = (uint64_t)0xCD9E8D57u * x.z;  // one wide multiply each
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    x = make_uint4(hi1 ^ x.y ^ key.x, lo1, hi0 ^ x.w ^ key.y, lo0);
  }
  return x;
}

// Minimal set of hypothesis h of cluster `cluster` (frame-local index) with n >= k points.
template <int DIM>
__device__ __forceinline__ void draw_minimal_set(uint2 key, int cluster, int h, int n, int q[3]) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)h, (uint32_t)cluster, 0u, 0u), key);
  uint32_t q0 = __umulhi(w.x, (uint32_t)n);
  uint32_t q1 = __umulhi(w.y, (uint32_t)(n - 1));
  q1 += (q1 >= q0);
  q[0] = (int)q0;
  q[1] = (int)q1;
  if (DIM == 3) {
    const uint32_t lo = min(q0, q1), hi = max(q0, q1);
    uint32_t q2 = __umulhi(w.z, (uint32_t)(n - 2));
    q2 += (q2 >= lo);
    q2 += (q2 >= hi);
    q[2] = (int)q2;
  } else {
    q[2] = 0;
  }
}

// ---- FP64 arithmetic that fixes every decision --------------------------------------
// Each formula is evaluated in this exact order: x*w - y*z as fma(x, w, -(y*z)),
// the 3x3 determinant by cofactors along row 0, Cramer's rule for the solve.

__device__ __forceinline__ double det2_f64(double x, double y, double z, double w) {
  return fma(x, w, -(y * z));
}

__device__ __forceinline__ double det3_f64(const double* m0, const double* m1, const double* m2) {
  const double k0 = det2_f64(m1[1], m1[2], m2[1], m2[2]);
  const double k1 = det2_f64(m1[0], m1[2], m2[0], m2[2]);
  const double k2 = det2_f64(m1[0], m1[1], m2[0], m2[1]);
  return fma(m0[2], k2, fma(-m0[1], k1, m0[0] * k0));
}

// FP64 cos/sin of an FP32 angle by angle addition: t = k/128 + x with
// |x| <= 1/256 exactly (FP32 arithmetic), (cos, sin)(k/128) from a table of
// correctly rounded values built on the host, and cos x - 1, sin x from their
// Taylor series (truncation below 5e-18 absolute).  Absolute error within a
// few 2^-53 (tests bound it against the library sincos over every float in
// [-pi, pi]), at a third of the library's FP64 instruction count; near the
// zeros of cos and sin the relative error grows, which no formula here
// depends on.  Angles beyond the table fall back to the library sincos.
__device__ __forceinline__ void sincos_f64(const double2* __restrict__ trig, float t, double* s, double* c) {
  const float kf = rintf(t * 128.0f);
  if (!(fabsf(kf) <= (float)kTrigHalf)) {
    sincos((double)t, s, c);
    return;
  }
  const float xf = fmaf(kf, -0.0078125f, t);  // exact
  const double x = (double)xf;
  const double x2 = x * x;
  const double cm1 = x2 * fma(x2, 1.0 / 24.0, -0.5);
  const double sx = fma(x * x2, fma(x2, 1.0 / 120.0, -1.0 / 6.0), x);
  const double2 cs = __ldg(&trig[(int)kf + kTrigHalf]);  // (cos, sin)(k/128)
  *c = fma(cs.x, cm1, fma(-cs.y, sx, cs.x));
  *s = fma(cs.y, cm1, fma(cs.x, sx, cs.y));
}

// Rows of A_i (Eq. eq:LSQPerCluster) in FP64: (cos t, sin t) or
// (cos t cos e, sin t cos e, sin e).
template <int DIM>
__device__ __forceinline__ void row_f64(const double2* __restrict__ trig, float az, float el, double a[3]) {
  double s, c;
  sincos_f64(trig, az, &s, &c);
  if (DIM == 2) {
    a[0] = c;
    a[1] = s;
    a[2] = 0.0;
  } else {
    double se, ce;
    sincos_f64(trig, el, &se, &ce);
    a[0] = c * ce;
    a[1] = s * ce;
    a[2] = se;
  }
}

// Solves the k x k system (rows a0, a1[, a2], right side w) by Cramer's rule.
// Returns false (and leaves v) when !(|det| >= eps).
template <int DIM>
__device__ __forceinline__ bool solve_f64(const double* a0, const double* a1, const double* a2,
                                          const double* w, double eps, double v[3], double* det_out) {
  if (DIM == 2) {
    const double det = det2_f64(a0[0], a0[1], a1[0], a1[1]);
    if (det_out) *det_out = det;
    if (!(fabs(det) >= eps)) return false;
    v[0] = det2_f64(w[0], a0[1], w[1], a1[1]) / det;
    v[1] = det2_f64(a0[0], w[0], a1[0], w[1]) / det;
    v[2] = 0.0;
    return true;
  } else {
    const double det = det3_f64(a0, a1, a2);
    if (det_out) *det_out = det;
    if (!(fabs(det) >= eps)) return false;
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      double r0[3] = {a0[0], a0[1], a0[2]};
      double r1[3] = {a1[0], a1[1], a1[2]};
      double r2[3] = {a2[0], a2[1], a2[2]};
      r0[col] = w[0];
      r1[col] = w[1];
      r2[col] = w[2];
      v[col] = det3_f64(r0, r1, r2) / det;
    }
    return true;
  }
}

// Doppler residual r = w - a.v of Eq. LSQ_eq in FP64.
template <int DIM>
__device__ __forceinline__ double residual_f64(const double* a, double w, const double* v) {
  if (DIM == 2) return w - fma(v[0], a[0], v[1] * a[1]);
  return w - fma(v[0], a[0], fma(v[1], a[1], v[2] * a[2]));
}

// ---- FP32 rows and FP32 hypotheses with rigorous error bounds ------------------------

// Relative accuracy assumed for sincosf on |t| <= pi: |c32 - c64| <= rho |c64|.
// Tests check every float in that range against twice this margin; outside it
// the row is the FP64 one rounded to nearest.
constexpr float kRowRel = 0x1p-22f;
constexpr float kU = 0x1p-24f;                                 // FP32 unit roundoff
constexpr float kRowRel3 = 2.0f * 0x1p-22f + 2.0f * 0x1p-24f;  // products cos t * cos e
constexpr float kSafety = 1.0f + 0x1p-14f;   // covers second-order terms and bound roundings
constexpr float kTiny = 0x1p-120f;           // absolute slack for underflow
constexpr float kBandFloor = 1e-5f;          // minimum half-width of the FP64 band (m/s)
// |det32 - det64| over unit rows: (2 rho + 2u)(1 + 1e-4) for 2D,
// sqrt(3)(3 rho3 + 5u) for 3D, rounded up, plus the FP64 rounding of det64.
constexpr float kDetErr2 = 5.98e-7f;
constexpr float kDetErr3 = 3.65e-6f;
// Trials (of callers that allow refinement) whose band would be wider than
// this get one refinement step; 3D minimal sets are ill-conditioned in the
// vertical direction, so most 3D trials do.
constexpr float kRefineBand = 1e-4f;

// FP32 row of a point plus its Doppler: (c, s, w, t) or (a0, a1, a2, w); the
// 2D row keeps the FP32 azimuth t, from which the FP64 row is computed.
template <int DIM>
__device__ __forceinline__ float4 row_f32(float az, float el, float w) {
  float s, c;
  if (fabsf(az) <= 3.1415925f) {
    sincosf(az, &s, &c);
  } else {
    double sd, cd;
    sincos((double)az, &sd, &cd);
    s = __double2float_rn(sd);
    c = __double2float_rn(cd);
  }
  if (DIM == 2) return make_float4(c, s, w, az);
  float se, ce;
  if (fabsf(el) <= 3.1415925f) {
    sincosf(el, &se, &ce);
  } else {
    double sd, cd;
    sincos((double)el, &sd, &cd);
    se = __double2float_rn(sd);
    ce = __double2float_rn(cd);
  }
  return make_float4(c * ce, s * ce, se, w);
}

// Hypothesis record used by the scoring loops: negated velocity (so the
// residual is fmaf(nx, c, fmaf(ny, s, w))), thresholds and a kind.
enum HypKind : int { kHypNormal = 0, kHypRejected = 1, kHypExactOnly = 2, kHypUndecided = 3 };

struct Hyp32 {
  float nx, ny, nz;   // -X, -Y, -Z
  float thi;          // |r32| >  thi  => certainly an outlier
  float tlo;          // |r32| <= tlo  => certainly an inlier
  int kind;
  int refined;
};

// Reciprocal by rcp.approx.f32 (one instruction; at most one ulp from 1/x,
// i.e. relative error below 2^-23, for normal x).  Used instead of IEEE
// division in the FP32 solve: the error bounds below account for it.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// |rcp_approx(x)| * kRcpUp, rounded to nearest, is >= 1/|x| even after one
// more rounding of x itself: (1 - 2^-23)(1 - 2^-24)^2 (1 + 2^-19) > 1.
constexpr float kRcpUp = 1.0f + 0x1p-19f;

// >= 1 / (|d| - eD) for |d| > eD.
__device__ __forceinline__ float inv_minus(float d, float eD) { return rcp_approx(fabsf(d) - eD) * kRcpUp; }

// Reciprocals of a trial's FP32 determinant d: rd = rcp(d) (|rd - 1/d| <=
// 2^-23 |1/d|), inv >= 1/|d| and slack >= eD / (|d| - eD) (meaningful while
// |d| > eD; callers treat |d| <= 2 eD as unusable).
struct DetRcp {
  float rd, inv, slack;
};
__device__ __forceinline__ DetRcp det_rcp(float d, float eD) {
  DetRcp r;
  r.rd = rcp_approx(d);
  r.inv = fabsf(r.rd) * kRcpUp;
  r.slack = eD * inv_minus(d, eD) * kRcpUp;
  return r;
}

// FP32 Cramer solve of the rows p, q[, r] with right side b (exact floats),
// determinant d already formed (reciprocals in R).  X receives the solution,
// e a bound on |X - A64^-1 b| per component, where A64 holds the FP64 rows:
// the bound covers the FP32 rows' error (rho per entry), every FP32
// rounding, the error of d (eD, through slack), and the quotient n * rd,
// whose relative error is below 2^-23 + 2^-24 + 2^-47 < 4u.
template <int DIM>
__device__ __forceinline__ void cramer_f32(float4 p, float4 q, float4 r, const float* b, const DetRcp& R,
                                           float* X, float* e) {
  const float inv = R.inv;
  const float slack = R.slack;
  if (DIM == 2) {
    const float n0 = fmaf(b[0], q.y, -(b[1] * p.y));
    const float n1 = fmaf(p.x, b[1], -(b[0] * q.x));
    X[0] = n0 * R.rd;
    X[1] = n1 * R.rd;
    X[2] = 0.0f;
    const float A = (kRowRel + kU) * 1.0001f * (fabsf(b[0]) + fabsf(b[1]));
    const float e0 = A + kU * fabsf(n0), e1 = A + kU * fabsf(n1);
    e[0] = (e0 + (fabsf(n0) + e0) * slack) * inv + 4.0f * kU * fabsf(X[0]);
    e[1] = (e1 + (fabsf(n1) + e1) * slack) * inv + 4.0f * kU * fabsf(X[1]);
    e[2] = 0.0f;
  } else {
    float n[3];
    {  // column 0 replaced by b
      const float c0 = fmaf(q.y, r.z, -(q.z * r.y));
      const float c1 = fmaf(b[1], r.z, -(q.z * b[2]));
      const float c2 = fmaf(b[1], r.y, -(q.y * b[2]));
      n[0] = fmaf(p.z, c2, fmaf(-p.y, c1, b[0] * c0));
    }
    {  // column 1 replaced by b
      const float c0 = fmaf(b[1], r.z, -(q.z * b[2]));
      const float c1 = fmaf(q.x, r.z, -(q.z * r.x));
      const float c2 = fmaf(q.x, b[2], -(b[1] * r.x));
      n[1] = fmaf(p.z, c2, fmaf(-b[0], c1, p.x * c0));
    }
    {  // column 2 replaced by b
      const float c0 = fmaf(q.y, b[2], -(b[1] * r.y));
      const float c1 = fmaf(q.x, b[2], -(b[1] * r.x));
      const float c2 = fmaf(q.x, r.y, -(q.y * r.x));
      n[2] = fmaf(b[0], c2, fmaf(-p.y, c1, p.x * c0));
    }
    const float A = (4.0f * kRowRel3 + 8.0f * kU) * 1.0001f * (fabsf(b[0]) + fabsf(b[1]) + fabsf(b[2]));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      X[k] = n[k] * R.rd;
      const float ek = A + kU * fabsf(n[k]);
      e[k] = (ek + (fabsf(n[k]) + ek) * slack) * inv + 4.0f * kU * fabsf(X[k]);
    }
  }
}

// Half-width of the band around tau outside of which the FP32 residual of any
// point decides like the FP64 residual, for a trial X with |X - X64| <= e.
template <int DIM>
__device__ __forceinline__ float band_f32(float wmax, const float* X, const float* e) {
  float b;
  if (DIM == 2) {
    b = (2.0f * kU + 0x1p-52f) * wmax + (kU + kRowRel + 0x1p-52f) * fabsf(X[0]) +
        (2.0f * kU + kRowRel + 0x1p-52f) * fabsf(X[1]) + e[0] + e[1];
  } else {
    b = (3.0f * kU + 0x1p-52f) * wmax + (kU + kRowRel3 + 0x1p-52f) * fabsf(X[0]) +
        (2.0f * kU + kRowRel3 + 0x1p-52f) * fabsf(X[1]) + (3.0f * kU + kRowRel + 0x1p-52f) * fabsf(X[2]) +
        e[0] + e[1] + e[2];
  }
  return b * kSafety + kTiny;
}

// The trial's FP32 hypothesis and band.  p, q[, r]: FP32 rows (with Doppler);
// seed64(i) returns the FP64 row (a0, a1, a2, w) of seed point i, called only
// by the refinement step, which runs when the band exceeds refine_band
// (+inf disables it).  wmax = max |w| over
// the cluster.  Conditioning: |det32| >= acc => FP64 accepts; |det32| < rej =>
// FP64 rejects; otherwise kHypUndecided (the caller decides in FP64).
//
// Refinement (when the band would exceed refine_band): the seed residuals
// r = w - A64 X are formed in FP64, the correction A^-1 r is solved in FP32
// and added.  Since X64 - X = A64^-1 (w - A64 X) exactly, the corrected
// error is the correction's own error (tiny: r is tiny) plus
// ||A64^-1||_inf (|fl(r) - r| + FP64 rounding) plus the FP32 rounding of X+dX.
template <int DIM, typename Seed64>
__device__ __forceinline__ Hyp32 hyp_f32(float4 p, float4 q, float4 r, const Seed64& seed64, float refine_band,
                                         float wmax, float acc, float rej, TauPair tau) {
  Hyp32 h;
  h.nx = h.ny = h.nz = 0.0f;
  h.thi = __int_as_float(0x7fc00000);  // NaN: never counted
  h.tlo = -1.0f;
  h.refined = 0;
  float d;
  if (DIM == 2) {
    d = fmaf(p.x, q.y, -(p.y * q.x));
  } else {
    const float k0 = fmaf(q.y, r.z, -(q.z * r.y));
    const float k1 = fmaf(q.x, r.z, -(q.z * r.x));
    const float k2 = fmaf(q.x, r.y, -(q.y * r.x));
    d = fmaf(p.z, k2, fmaf(-p.y, k1, p.x * k0));
  }
  const float ad = fabsf(d);
  if (!(ad >= acc)) {
    h.kind = (ad < rej) ? kHypRejected : kHypUndecided;
    return h;
  }
  const float eD = DIM == 2 ? kDetErr2 : kDetErr3;
  const float w[3] = {DIM == 2 ? p.z : p.w, DIM == 2 ? q.z : q.w, DIM == 2 ? 0.0f : r.w};
  const DetRcp R = det_rcp(d, eD);
  float X[3], e[3];
  cramer_f32<DIM>(p, q, r, w, R, X, e);
  // error of the FP64 solve (the oracle's X64) against the exact solution with FP64 rows
  const float sw = fabsf(w[0]) + fabsf(w[1]) + fabsf(w[2]);
  const float sx = fabsf(X[0]) + fabsf(X[1]) + fabsf(X[2]);
  const float e64 = (DIM == 2 ? 0x1p-50f : 0x1p-48f) * (2.0f * sw + 2.0f * sx) * R.inv;
#pragma unroll
  for (int k = 0; k < DIM; ++k) e[k] += e64;
  float b = band_f32<DIM>(wmax, X, e);
  if (b > refine_band && ad > 2.0f * eD && b < 1e30f) {
    float rf[3] = {0.0f, 0.0f, 0.0f};
    float rerr = 0.0f;
    const double X0 = X[0], X1 = X[1], X2 = X[2];
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      const double4_32a a = seed64(i);
      const double ri = DIM == 2 ? a.w - fma(X0, a.x, X1 * a.y) : a.w - fma(X0, a.x, fma(X1, a.y, X2 * a.z));
      rf[i] = __double2float_rn(ri);
      // |fl32(r) - r| + FP64 rounding of r
      rerr = fmaxf(rerr, kU * fabsf(rf[i]) + 0x1p-51f * (fabsf(w[i]) + sx));
    }
    float dX[3], de[3];
    cramer_f32<DIM>(p, q, r, rf, R, dX, de);
    const float inv_norm = (float)DIM * inv_minus(d, eD) * kRcpUp;  // >= ||A64^-1||_inf (adjugate entries <= 1)
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      X[k] = X[k] + dX[k];
      e[k] = de[k] + inv_norm * rerr + kU * fabsf(X[k]) + e64;
    }
    b = band_f32<DIM>(wmax, X, e);
    h.refined = 1;
  }
  h.nx = -X[0];
  h.ny = -X[1];
  h.nz = -X[2];
  if (!(b < 1e30f) || !(fabsf(X[0]) < 1e30f) || !(fabsf(X[1]) < 1e30f) || !(fabsf(X[2]) < 1e30f) ||
      !(ad > 2.0f * eD)) {
    h.kind = kHypExactOnly;
    h.thi = __int_as_float(0x7f800000);  // +inf: nothing certainly out
    h.tlo = -1.0f;                        // nothing certainly in
    return h;
  }
  b = fmaxf(b, kBandFloor);
  h.thi = __fadd_ru(tau.hi, b);
  h.tlo = __fsub_rd(tau.lo, b);
  h.kind = kHypNormal;
  return h;
}

// FP32 residual of a row under a hypothesis (negated velocity).
template <int DIM>
__device__ __forceinline__ float resid_f32(float4 row, float nx, float ny, float nz) {
  if (DIM == 2) return fmaf(nx, row.x, fmaf(ny, row.y, row.z));
  return fmaf(nx, row.x, fmaf(ny, row.y, fmaf(nz, row.z, row.w)));
}

}  // namespace rvh
