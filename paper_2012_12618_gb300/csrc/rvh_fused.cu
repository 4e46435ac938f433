// Fused persistent kernel: per cluster, FP32 and FP64 rows -> counter-RNG
// minimal sets -> FP32 solve with error bound (refined in FP64 residuals when
// ill-conditioned) -> FP32 scoring pass (upper-bound counts) -> exact counts,
// in index order, of the trials that can still win (FP64 only inside the
// error band) -> lowest-index argmax -> FP64 inlier mask and normal-equation
// refine -> heading.  Sec. III-A (Alg. 1, Eq. 4) and Sec. III-B (Eq. LSQ_eq,
// Eq. eq:LSQPerCluster, Alg. 2) of arXiv 2012.12618.
//
// Parallel mapping (GB300-first, not the paper's thread-per-trial): clusters
// are work items taken by persistent CTAs from an LPT-ordered list; inside a
// cluster, trials map to warps/lanes and points to lanes, with the cluster's
// FP32 rows staged in shared memory and its FP64 rows in L1/L2-resident
// global scratch.
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "rvh_device.cuh"
#include "rvh_kernels.h"
#include "rvh_scoring.cuh"

namespace rvh {

__device__ __forceinline__ unsigned long long best_key(int count, int h) {
  return ((unsigned long long)(uint32_t)(count + 1) << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)h);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int block_max_int(int v, int* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int r = red[0];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) r = max(r, red[w]);
  return r;
}

__device__ __forceinline__ int block_min_int(int v, int* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int r = red[0];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) r = min(r, red[w]);
  return r;
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  unsigned long long r = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) r += red[w];
  return r;
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  unsigned long long r = red[0];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) r = max(r, red[w]);
  return r;
}

__device__ __forceinline__ float block_max_float(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float r = red[0];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) r = fmaxf(r, red[w]);
  return r;
}

// ---- a4: upper-bound counts U_h = #{|r32| <= thi_h} (the hot loop) -----------------
// Lane l handles trial sub-group l / PW and points l % PW, l % PW + PW, ...;
// each lane keeps HPL trials in registers.  PW = 32 is warp-per-trial-group
// with lanes over points; PW = 1 is lanes over trials with broadcast rows.
template <int DIM, int PW, int HPL>
__device__ __forceinline__ void phase_a(const float4* __restrict__ rows, int N, const Smem& S, int nh) {  // global rows
  constexpr int NHL = 32 / PW;
  constexpr int G = NHL * HPL;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int hl = lane / PW, pl = lane % PW;
  const int ngroups = (nh + G - 1) / G;
  for (int g = warp; g < ngroups; g += kWarps) {
    const int base = g * G + hl * HPL;
    float nx[HPL], ny[HPL], nz[HPL], th[HPL], cnt[HPL];
#pragma unroll
    for (int m = 0; m < HPL; ++m) {
      const int h = base + m;
      float4 v = (h < nh) ? S.hyp[h] : make_float4(0.f, 0.f, 0.f, __int_as_float(0x7fc00000));
      nx[m] = v.x;
      ny[m] = v.y;
      nz[m] = v.z;
      th[m] = v.w;
      cnt[m] = 0.0f;
    }
    for (int j = pl; j < N; j += PW) {
      const float4 p = rows[j];
#pragma unroll
      for (int m = 0; m < HPL; ++m) {
        const float r = resid_f32<DIM>(p, nx[m], ny[m], nz[m]);
        cnt[m] += (fabsf(r) <= th[m]) ? 1.0f : 0.0f;
      }
    }
#pragma unroll
    for (int m = 0; m < HPL; ++m) {
#pragma unroll
      for (int o = PW / 2; o > 0; o >>= 1) cnt[m] += __shfl_xor_sync(0xffffffffu, cnt[m], o);
    }
    if (pl == 0) {
#pragma unroll
      for (int m = 0; m < HPL; ++m) {
        const int h = base + m;
        if (h < nh && S.kind[h] == kHypNormal) S.U[h] = (int)cnt[m];
      }
    }
  }
}

// The tiled pass keeps four trials per lane whatever hpl asks: eight packed
// trials (pairs of registers per coordinate) do not fit in the 64 registers a
// thread has at four CTAs per SM.
template <int DIM>
__device__ void phase_a_dispatch(int pw, int hpl, const TileRowsOf<DIM> rows, int N, const Smem& S, int nh) {
  (void)hpl;
  if (pw == 1) {
    phase_a_tiles<DIM, 1, 4>(rows, N, S, nh);
  } else if (pw == 8) {
    phase_a_tiles<DIM, 8, 4>(rows, N, S, nh);
  } else {
    phase_a_tiles<DIM, 32, 4>(rows, N, S, nh);
  }
}

template <int DIM>
__device__ void phase_a_dispatch(int pw, int hpl, const AosRows rows, int N, const Smem& S, int nh) {
  if (pw == 1) {
    if (hpl == 8) phase_a<DIM, 1, 8>(rows.p, N, S, nh); else phase_a<DIM, 1, 4>(rows.p, N, S, nh);
  } else if (pw == 8) {
    if (hpl == 8) phase_a<DIM, 8, 8>(rows.p, N, S, nh); else phase_a<DIM, 8, 4>(rows.p, N, S, nh);
  } else {
    if (hpl == 8) phase_a<DIM, 32, 8>(rows.p, N, S, nh); else phase_a<DIM, 32, 4>(rows.p, N, S, nh);
  }
}

// FP64 rows (a0, a1, a2, w) of a cluster's points.  The 3D model keeps them
// in global scratch, written once when the cluster is loaded (every 3D trial
// refines its solve with them); the 2D model computes them when asked (only
// the winner's inliers, band points and rare refinements need them).
template <int DIM>
struct Rows64 {
  const FrameDesc* a;
  int64_t o;
  double4_32a* pre;
  __device__ __forceinline__ double4_32a at(int j) const {
    if (DIM == 3) return pre[j];
    double t[3];
    row_f64<2>(a->trig, a->az[o + j], 0.0f, t);
    return make_double4_32a(t[0], t[1], 0.0, (double)a->dop[o + j]);
  }
  // The same row when the point's FP32 cosine-model row is at hand: in 2D it
  // carries the Doppler (row_f32), so only the azimuth is read.
  __device__ __forceinline__ double4_32a at(int j, float4 row) const {
    if (DIM == 3) return pre[j];
    double t[3];
    row_f64<2>(a->trig, a->az[o + j], 0.0f, t);
    return make_double4_32a(t[0], t[1], 0.0, (double)row.z);
  }
};

// FP64 rows computed from the frame's inputs in both models: the source of
// the finishing pass, which runs after the CTA's row slot has moved on to
// later clusters.
template <int DIM>
struct Rows64Inputs {
  const FrameDesc* a;
  int64_t o;
  __device__ __forceinline__ double4_32a at(int j) const {
    double t[3];
    row_f64<DIM>(a->trig, a->az[o + j], DIM == 3 ? a->el[o + j] : 0.0f, t);
    return make_double4_32a(t[0], t[1], t[2], (double)a->dop[o + j]);
  }
};

// FP64 velocity of trial h in the oracle's exact rounding sequence.  Returns
// false if rejected.
template <int DIM, typename RS>
__device__ bool hyp_f64(const FrameDesc& a, const RS& R, int ci, int h, int N, double v[3]) {
  int q[3];
  draw_minimal_set<DIM>(a.key, a.cluster_base + ci, h, N, q);
  const double4_32a s0 = R.at(q[0]), s1 = R.at(q[1]), s2 = R.at(DIM == 3 ? q[2] : q[0]);
  const double r0[3] = {s0.x, s0.y, s0.z}, r1[3] = {s1.x, s1.y, s1.z}, r2[3] = {s2.x, s2.y, s2.z};
  const double w[3] = {s0.w, s1.w, DIM == 3 ? s2.w : 0.0};
  return solve_f64<DIM>(r0, r1, r2, w, a.eps, v, nullptr);
}

struct ClusterShared {
  unsigned long long best;
  float wmax;
  float4 win;      // winner's FP32 record
  float win_tlo;
  int red_i[kWarps];
  float red_f[kWarps];
  double red_t[9];            // the normal-equation sums of the winner's inliers
  unsigned long long ctr[4];  // exact counts, band points, fp64 trials, refined trials
  unsigned long long clk[6];  // cycles per stage (thread 0's view of the CTA)
  unsigned long long red_u[kWarps];
  double cv64[3];             // FP64 velocity of the trial being counted (when it has band points)
  double win_v64[3];          // FP64 velocity of the current winner (valid if win_has_v64)
  int win_has_v64;
  int red_c[kWarps];          // changed mask entries (local-optimisation rounds)
  double lo_v[3];             // least-squares velocity of the current inlier set
  float4 lo_hy;               // its FP32 record (-X, -Y, -Z, thi) and lower threshold
  float lo_tlo;
  int lo_ok;
  int stop;                   // adaptive trial count: enough trials have run
  double ln_T;                // line model (Alg. 1): the cluster's MAD threshold
  int sel_digit, sel_k;       // radix select: digit and rank inside it
  float red4[4][kWarps];      // line model: min / max of azimuth and Doppler
  unsigned long long runs[2];  // trials run, pairs scored
  unsigned long long scored;   // (trial, point) pairs the scoring pass evaluated
  int nref;                   // 2D trials queued for refinement in the current chunk
};

// Adaptive trial count: with `best` the best (count + 1, -index) key so far,
// n points, k = DIM and m trials run, true once (1 - eps^k)^m <= 1 - p for
// eps = count / n: the standard RANSAC bound on the chance that every trial
// so far drew an outlier.  The power is taken by binary exponentiation in
// the same order as the oracle's, one IEEE rounding per operation, so both
// decide alike.  One thread; kept out of line.
__device__ __noinline__ int adaptive_stop(unsigned long long best, int n, int k, int m, double p) {
  const int count = (int)(best >> 32) - 1;
  if (count < 0) return 0;
  const double eps = (double)count / (double)n;
  const double ek = k == 2 ? eps * eps : (eps * eps) * eps;
  double r = 1.0, b = 1.0 - ek;
  for (int e = m; e > 0; e >>= 1) {
    if (e & 1) r = r * b;
    b = b * b;
  }
  return r <= 1.0 - p ? 1 : 0;
}

// FP32 record of an FP64 velocity v for the re-threshold of a local
// optimisation round: X = fl32(v), e >= |X - v|, the band of band_f32 around
// tau outside which FP32 residuals decide like FP64 ones.
template <int DIM>
__device__ __forceinline__ void velocity_record(const double v[3], float wmax, TauPair tau, float4* hy, float* tlo) {
  float X[3], e[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    X[k] = __double2float_rn(v[k]);
    e[k] = __double2float_ru(fabs((double)X[k] - v[k]));
  }
  float b = band_f32<DIM>(wmax, X, e);
  if (!(b < 1e30f) || !(fabsf(X[0]) < 1e30f) || !(fabsf(X[1]) < 1e30f) || !(fabsf(X[2]) < 1e30f)) {
    *hy = make_float4(-X[0], -X[1], -X[2], __int_as_float(0x7f800000));  // every point decided in FP64
    *tlo = -1.0f;
    return;
  }
  b = fmaxf(b, kBandFloor);
  *hy = make_float4(-X[0], -X[1], -X[2], __fadd_ru(tau.hi, b));
  *tlo = __fsub_rd(tau.lo, b);
}

// ---- Alg. 1 as printed (line model, 2D): normalised (azimuth, Doppler) points,
// line fits through two seed points, perpendicular-distance test against the
// cluster's median absolute deviation.  The FP64 values of each point are
// kept in its FP64 row slot (x, y, |y - med y|, -), which the 2D cosine
// model does not use.

// Alg. 1 point-to-line test in FP64, evaluated as printed: aa = -m, bb = 1,
// cc = -c, distn = aa x + bb y + cc, distd = sqrt(aa^2 + bb^2) (passed in),
// dist = |distn / distd| <= thresh.
__device__ __forceinline__ bool line_in64(double m, double c, double distd, double x, double y, double thresh) {
  const double distn = (-m) * x + y + (-c);
  return fabs(distn / distd) <= thresh;
}

// FP64 line (m, c, distd) of trial h through its two normalised seed points;
// false when they share x (no slope).
__device__ __forceinline__ bool line_hyp64(const FrameDesc& a, const double4_32a* pre, int ci, int h, int N, double v[3]) {
  int q[3];
  draw_minimal_set<2>(a.key, a.cluster_base + ci, h, N, q);
  const double4_32a p0 = pre[q[0]], p1 = pre[q[1]];
  const double dx = p1.x - p0.x;
  if (dx == 0.0) return false;
  const double m = (p1.y - p0.y) / dx;
  v[0] = m;
  v[1] = p0.y - m * p0.x;
  v[2] = sqrt(m * m + 1.0);
  return true;
}

// FP32 scoring record of an FP64 line: (-m32, -c32, 0, thi) and tlo, such
// that with rows (x32, 1, y32) the FP32 residual r32 = fmaf(-m32, x32,
// fmaf(-c32, 1, y32)) satisfies |r32| <= tlo => inlier and |r32| > thi =>
// outlier under line_in64.  With |x|, |y| <= 1 (normalised), rounding the
// inputs and the arithmetic to FP32 moves the residual by at most
// u (2.01 (1 + |c| + |m|) + 1.0001 |r|), the FP64 residual carries
// 3 * 2^-53 (1 + |c| + |m|), and the FP64 quotient test is certain outside
// T distd (1 -+ 2^-50); b below covers both sides with margin.
__device__ __forceinline__ Hyp32 line_record(const double v[3], double T) {
  Hyp32 h;
  h.refined = 0;
  h.nx = -__double2float_rn(v[0]);
  h.ny = -__double2float_rn(v[1]);
  h.nz = 0.0f;
  const double td = T * v[2];
  const double am = fabs(v[0]), ac = fabs(v[1]);
  const double b = (0x1p-22 * (1.0 + ac + am + td) + 0x1p-50 * (1.0 + ac + am)) * (1.0 + 0x1p-20);
  const double hi = td * (1.0 + 0x1p-50) + b, lo = td * (1.0 - 0x1p-50) - b;
  if (!(hi < 1e30) || !(am < 1e30) || !(ac < 1e30)) {
    h.kind = kHypExactOnly;
    h.thi = __int_as_float(0x7f800000);
    h.tlo = -1.0f;
    return h;
  }
  h.thi = __double2float_ru(hi);
  h.tlo = lo >= 0.0 ? __double2float_rd(lo) : -1.0f;
  h.kind = kHypNormal;
  return h;
}

// k-th smallest (0-based, k < N) of the keys |field| of the FP64 point slots
// (field 1: y, field 2: |y - med y|) as 64-bit patterns of non-negative
// doubles (monotone as integers; NaN sorts last), by radix digits of 8 bits
// from the top.  hist: 256 ints of shared memory.  Exact: returns the key.
template <int FIELD>
__device__ unsigned long long block_select(const double4_32a* pre, int N, int k, int* hist, ClusterShared& cs) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long prefix = 0ull, hmask = 0ull;
  for (int shift = 56; shift >= 0; shift -= 8) {
    hist[tid] = 0;  // kThreads == 256 bins
    __syncthreads();
    for (int j = tid; j < N; j += kThreads) {
      const double4_32a p = pre[j];
      const unsigned long long kb = (unsigned long long)__double_as_longlong(fabs(FIELD == 1 ? p.y : p.z));
      if ((kb & hmask) == prefix) atomicAdd(&hist[(int)((kb >> shift) & 255ull)], 1);
    }
    __syncthreads();
    if (warp == 0) {
      int c[8], tot = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        c[i] = hist[8 * lane + i];
        tot += c[i];
      }
      int incl = tot;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
      }
      const int excl = incl - tot;
      if (excl <= k && k < incl) {
        int kk = k - excl, d = 0;
        while (d < 7 && kk >= c[d]) kk -= c[d++];
        cs.sel_digit = 8 * lane + d;
        cs.sel_k = kk;
      }
    }
    __syncthreads();
    prefix |= (unsigned long long)cs.sel_digit << shift;
    hmask |= 0xFFull << shift;
    k = cs.sel_k;
  }
  return prefix;
}

// Median of the keys (even N: 0.5 * (lower + upper middle)).
template <int FIELD>
__device__ double block_median(const double4_32a* pre, int N, int* hist, ClusterShared& cs) {
  const double hi = __longlong_as_double((long long)block_select<FIELD>(pre, N, N / 2, hist, cs));
  if (N & 1) return hi;
  const double lo = __longlong_as_double((long long)block_select<FIELD>(pre, N, N / 2 - 1, hist, cs));
  return 0.5 * (lo + hi);
}

// The line model's rows stage: min / max of azimuth and Doppler, normalised
// FP64 points into the FP64 slots and FP32 rows (x, 1, y) into the scoring
// rows, then the MAD threshold into cs.ln_T.  Normalisation (the paper's
// normalize(), undefined there): min-max scaling, x = (t - t_min) *
// (1 / (t_max - t_min)), 0 when the range is empty.  Out of line: runs once
// per cluster.
template <typename RV>
__device__ __noinline__ void line_rows_and_threshold(const FrameDesc& a, const RV rows, double4_32a* pre, int64_t o,
                                                     int N, int* hist, ClusterShared& cs) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float inf = __int_as_float(0x7f800000);
  float m4[4] = {inf, inf, inf, inf};  // min t, -max t, min v, -max v
  for (int j = tid; j < N; j += kThreads) {
    const float t = a.az[o + j], v = a.dop[o + j];
    m4[0] = fminf(m4[0], t);
    m4[1] = fminf(m4[1], -t);
    m4[2] = fminf(m4[2], v);
    m4[3] = fminf(m4[3], -v);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) m4[i] = fminf(m4[i], __shfl_xor_sync(0xffffffffu, m4[i], d));
    if (lane == 0) cs.red4[i][warp] = m4[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float r = cs.red4[i][0];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) r = fminf(r, cs.red4[i][w]);
    m4[i] = r;
  }
  const double tmin = (double)m4[0], tmax = -(double)m4[1], vmin = (double)m4[2], vmax = -(double)m4[3];
  const double rt = tmax > tmin ? 1.0 / (tmax - tmin) : 0.0;
  const double rv = vmax > vmin ? 1.0 / (vmax - vmin) : 0.0;
  for (int j = tid; j < N; j += kThreads) {
    const double x = ((double)a.az[o + j] - tmin) * rt;
    const double y = ((double)a.dop[o + j] - vmin) * rv;
    pre[j] = make_double4_32a(x, y, 0.0, 0.0);
    const float y32 = __double2float_rn(y);
    rows.put(j, make_float4(__double2float_rn(x), 1.0f, y32, a.az[o + j]));
  }
  __syncthreads();
  // Eq. eq:MAD read as the median absolute deviation of the normalised Doppler
  const double med = block_median<1>(pre, N, hist, cs);
  for (int j = tid; j < N; j += kThreads) pre[j].z = fabs(pre[j].y - med);
  __syncthreads();
  const double T = block_median<2>(pre, N, hist, cs);
  if (tid == 0) cs.ln_T = T;
  __syncthreads();
}

// Exact count of one trial by the whole CTA: FP32 certainties, then an FP64
// re-decision of the points inside the trial's error band.  When there are
// band points the trial's FP64 velocity is left in cs.cv64 and *band > 0.
template <int DIM, typename RV, bool EXT>
__device__ int exact_count_block(const FrameDesc& a, const RV rows, const Rows64<DIM>& R,
                                 int ci, int h, int N, float4 hy, float tlo, ClusterShared& cs, int* band) {
  const int tid = threadIdx.x;
  unsigned long long lb = 0;  // L in the low word, B in the high word
  for (int j = tid; j < N; j += kThreads) {
    const float r = fabsf(resid_f32<DIM>(rows.at(j), hy.x, hy.y, hy.z));
    if (r <= tlo) lb += 1ull;
    else if (!(r > hy.w)) lb += 1ull << 32;
  }
  lb = block_sum_u64(lb, cs.red_u);
  const int L = (int)(lb & 0xFFFFFFFFull), B = (int)(lb >> 32);
  *band = B;
  if (B == 0) return L;
  __syncthreads();
  if (tid == 0) {
    double v[3] = {0.0, 0.0, 0.0};
    if constexpr (EXT && DIM == 2) {
      if (a.line_model) line_hyp64(a, R.pre, ci, h, N, v);
      else hyp_f64<DIM>(a, R, ci, h, N, v);
    } else {
      hyp_f64<DIM>(a, R, ci, h, N, v);
    }
    cs.cv64[0] = v[0];
    cs.cv64[1] = v[1];
    cs.cv64[2] = v[2];
    cs.ctr[1] += (unsigned long long)B;
  }
  __syncthreads();
  const double v[3] = {cs.cv64[0], cs.cv64[1], cs.cv64[2]};
  unsigned long long lbin = 0;
  auto cosine_band = [&]() {
    for (int j = tid; j < N; j += kThreads) {
      const float4 row = rows.at(j);
      const float r = fabsf(resid_f32<DIM>(row, hy.x, hy.y, hy.z));
      if (!(r <= tlo) && !(r > hy.w)) {
        const double4_32a s = R.at(j, row);
        const double a64[3] = {s.x, s.y, s.z};
        if (fabs(residual_f64<DIM>(a64, s.w, v)) <= a.tau) ++lbin;
      }
    }
  };
  if constexpr (EXT && DIM == 2) {
    if (a.line_model) {
      for (int j = tid; j < N; j += kThreads) {
        const float r = fabsf(resid_f32<DIM>(rows.at(j), hy.x, hy.y, hy.z));
        if (!(r <= tlo) && !(r > hy.w)) {
          const double4_32a p = R.pre[j];
          if (line_in64(v[0], v[1], v[2], p.x, p.y, cs.ln_T)) ++lbin;
        }
      }
    } else {
      cosine_band();
    }
  } else {
    cosine_band();
  }
  lbin = block_sum_u64(lbin, cs.red_u);
  return L + (int)lbin;
}

template <int DIM>
__device__ void write_invalid(const FrameDesc& a, int ci, int st) {
  a.vx[ci] = __longlong_as_double(0x7ff8000000000000LL);
  a.vy[ci] = __longlong_as_double(0x7ff8000000000000LL);
  if (a.vz) a.vz[ci] = __longlong_as_double(0x7ff8000000000000LL);
  a.heading[ci] = __longlong_as_double(0x7ff8000000000000LL);
  a.inlier_count[ci] = 0;
  a.best[ci] = -1;
  a.status[ci] = st;
}

// a8: normal equations G v = g over the inliers (sums t: 2D Scc, Scs, Sss,
// Scv, Ssv; 3D the six entries of G then g), solved by Cramer's rule when
// there are at least k inliers and |det G| > 1e-12 trace^k.  Returns false
// (v untouched) otherwise.  The local-optimisation rounds and the final
// solve both use this, so a set accepted by a round solves identically.
template <int DIM>
__device__ __forceinline__ bool solve_normal(const double* t, int n_in, double v[3]) {
  if (DIM == 2) {
    const double tr = t[0] + t[2];
    const double limit = 1e-12 * (tr * tr);
    const double det = det2_f64(t[0], t[1], t[1], t[2]);
    if (!(n_in >= 2 && fabs(det) > limit)) return false;
    const double G0[3] = {t[0], t[1], 0.0}, G1[3] = {t[1], t[2], 0.0}, g[3] = {t[3], t[4], 0.0};
    double vs[3];
    solve_f64<2>(G0, G1, nullptr, g, 0.0, vs, nullptr);
    v[0] = vs[0];
    v[1] = vs[1];
    v[2] = 0.0;
    return true;
  } else {
    const double tr = t[0] + t[3] + t[5];
    const double limit = 1e-12 * (tr * tr * tr);
    const double G0[3] = {t[0], t[1], t[2]}, G1[3] = {t[1], t[3], t[4]}, G2[3] = {t[2], t[4], t[5]};
    const double det = det3_f64(G0, G1, G2);
    if (!(n_in >= 3 && fabs(det) > limit)) return false;
    const double g[3] = {t[6], t[7], t[8]};
    double vs[3];
    solve_f64<3>(G0, G1, G2, g, 0.0, vs, nullptr);
    v[0] = vs[0];
    v[1] = vs[1];
    v[2] = vs[2];
    return true;
  }
}

// Final solve and heading of a cluster: the normal equations, with a
// fallback to the winning minimal-set velocity, heading atan2(vy, vx).
// One thread.
template <int DIM, bool EXT>
__device__ __noinline__ void finish_cluster(const FrameDesc& a, const Rows64Inputs<DIM>& R, int ci, int N, int hstar, int n_in,
                               const double* t, const double* v64, bool has_v64) {
  double vout[3] = {v64[0], v64[1], v64[2]};
  int st = 0;
  const bool ok = solve_normal<DIM>(t, n_in, vout);
  if (!ok) {
    st |= RVH_STATUS_LSQ_FALLBACK;
    if constexpr (EXT && DIM == 2) {
      if (a.line_model) {  // a line has no velocity to fall back to
        vout[0] = vout[1] = vout[2] = __longlong_as_double(0x7ff8000000000000LL);
      } else if (!has_v64) {
        hyp_f64<DIM>(a, R, ci, hstar, N, vout);
      }
    } else {
      if (!has_v64) hyp_f64<DIM>(a, R, ci, hstar, N, vout);
    }
  }
  a.vx[ci] = vout[0];
  a.vy[ci] = vout[1];
  if (a.vz) a.vz[ci] = DIM == 3 ? vout[2] : 0.0;
  a.heading[ci] = atan2(vout[1], vout[0]);
  a.inlier_count[ci] = n_in;
  a.best[ci] = hstar;
  a.status[ci] = st;
}

// A cluster waiting for its final solve and heading (finish_cluster): the
// CTA queues up to kFinishBatch of them in shared memory and finishes them
// together, one lane each.  Serial FP64 on one lane costs as much pipe time
// per instruction as a full warp, so a lone thread finishing each cluster
// kept the other 255 threads at the next barrier for microseconds.
constexpr int kFinishBatch = 16;
struct FinishRec {
  double t[9];
  double v64[3];
  int64_t o;
  int n_in, hstar, ci, frame, N, has_v64;
};

// Accumulates the normal-equation sums of one inlier row (a0, a1, a2, w).
template <int DIM>
__device__ __forceinline__ void accumulate_row(double* sums, const double4_32a& s) {
  if (DIM == 2) {
    sums[0] = fma(s.x, s.x, sums[0]);
    sums[1] = fma(s.x, s.y, sums[1]);
    sums[2] = fma(s.y, s.y, sums[2]);
    sums[3] = fma(s.x, s.w, sums[3]);
    sums[4] = fma(s.y, s.w, sums[4]);
  } else {
    sums[0] = fma(s.x, s.x, sums[0]);
    sums[1] = fma(s.x, s.y, sums[1]);
    sums[2] = fma(s.x, s.z, sums[2]);
    sums[3] = fma(s.y, s.y, sums[3]);
    sums[4] = fma(s.y, s.z, sums[4]);
    sums[5] = fma(s.z, s.z, sums[5]);
    sums[6] = fma(s.x, s.w, sums[6]);
    sums[7] = fma(s.y, s.w, sums[7]);
    sums[8] = fma(s.z, s.w, sums[8]);
  }
}

// a7 + a8: decides every point of the cluster against one velocity (FP32
// certainties from the record hy / tlo, FP64 re-decisions with v64 inside
// the band), writes the mask, and reduces the normal-equation sums of the
// inliers into cs.red_t.  Returns the inlier count; with count_changes,
// *changed receives the number of mask entries that differ from what the
// mask held before.  The trial area of shared memory is free at this point
// and holds the reduction.
template <int DIM, typename RV, bool EXT>
__device__ __forceinline__ int mask_and_sums(const FrameDesc& a, const RV rows, const Rows64<DIM>& R, int64_t o, int N,
                                             float4 hy, float tlo, const double v64[3], const Smem& S,
                                             ClusterShared& cs, bool count_changes, int* changed) {
  const int tid = threadIdx.x;
  constexpr int NS = DIM == 2 ? 5 : 9;
  double sums[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) sums[i] = 0.0;
  int nin = 0, nch = 0;
  auto cosine_pass = [&]() {
    for (int j = tid; j < N; j += kThreads) {
      const float4 row = rows.at(j);
      const float r = fabsf(resid_f32<DIM>(row, hy.x, hy.y, hy.z));
      bool in = r <= tlo;
      const bool band = !in && !(r > hy.w);
      if (in || band) {
        const double4_32a s = R.at(j, row);
        if (band) {
          const double a64[3] = {s.x, s.y, s.z};
          in = fabs(residual_f64<DIM>(a64, s.w, v64)) <= a.tau;
        }
        if (in) {
          ++nin;
          accumulate_row<DIM>(sums, s);
        }
      }
      if (count_changes) nch += (a.mask[o + j] != (in ? 1 : 0));
      a.mask[o + j] = in ? 1 : 0;
    }
  };
  if constexpr (EXT && DIM == 2) {
    if (a.line_model) {
      // the line model decides its band points by Alg. 1's distance test
      for (int j = tid; j < N; j += kThreads) {
        const float r = fabsf(resid_f32<DIM>(rows.at(j), hy.x, hy.y, hy.z));
        bool in = r <= tlo;
        if (!in && !(r > hy.w)) {
          const double4_32a p = R.pre[j];
          in = line_in64(v64[0], v64[1], v64[2], p.x, p.y, cs.ln_T);
        }
        if (in) {
          ++nin;
          accumulate_row<DIM>(sums, R.at(j));
        }
        if (count_changes) nch += (a.mask[o + j] != (in ? 1 : 0));
        a.mask[o + j] = in ? 1 : 0;
      }
    } else {
      cosine_pass();
    }
  } else {
    cosine_pass();
  }
  // Reduce the per-thread sums through shared memory: warp i sums sum i,
  // each lane a strided share of the threads that held points, then a
  // shuffle tree; 12 dependent FP64 adds per sum.
  const int warp = tid >> 5, lane = tid & 31;
  nin = warp_sum(nin);
  if (count_changes) nch = warp_sum(nch);
  const int nact = min(N, kThreads);
  double* red = reinterpret_cast<double*>(S.hyp);  // NS x kThreads
  if (tid < nact) {
#pragma unroll
    for (int i = 0; i < NS; ++i) red[i * kThreads + tid] = sums[i];
  }
  if (lane == 0) {
    cs.red_i[warp] = nin;
    cs.red_c[warp] = nch;
  }
  __syncthreads();
  for (int i = warp; i < NS; i += kWarps) {
    double acc = 0.0;
    for (int k = lane; k < nact; k += 32) acc += red[i * kThreads + k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) cs.red_t[i] = acc;
  }
  int n_in = 0, n_ch = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    n_in += cs.red_i[w];
    n_ch += cs.red_c[w];
  }
  __syncthreads();
  if (changed) *changed = n_ch;
  return n_in;
}

// Local-optimisation rounds (refine_iterations > 0): solve the current set,
// re-threshold every point against that velocity, keep the new set if its
// normal equations are solvable (else restore the previous set by
// re-deciding with the record and velocity that produced it), stop when
// nothing changes.  Starts from the winner's set (its sums in cs.red_t) and
// returns the final set's inlier count, its sums left in cs.red_t.  Kept out
// of line so that the default path's register allocation does not carry it.
template <int DIM, typename RV>
__device__ __noinline__ int local_opt_rounds(const FrameDesc& a, const RV rows, const Rows64<DIM>& R, int64_t o, int N,
                                             float4 gen_hy, float gen_tlo, const double* v64, float wmax, int n_in,
                                             const Smem& S, ClusterShared& cs) {
  const int tid = threadIdx.x;
  double gen_v[3] = {v64[0], v64[1], v64[2]};  // the FP64 velocity that produced the current set
  for (int it = 0; it < a.lo_iters; ++it) {
    if (tid == 0) {
      double v[3] = {0.0, 0.0, 0.0};
      cs.lo_ok = solve_normal<DIM>(cs.red_t, n_in, v) ? 1 : 0;
      if (cs.lo_ok) {
        cs.lo_v[0] = v[0];
        cs.lo_v[1] = v[1];
        cs.lo_v[2] = v[2];
        velocity_record<DIM>(v, wmax, a.tau32, &cs.lo_hy, &cs.lo_tlo);
      }
    }
    __syncthreads();
    if (!cs.lo_ok) break;
    const float4 nhy = cs.lo_hy;
    const float ntlo = cs.lo_tlo;
    const double nv[3] = {cs.lo_v[0], cs.lo_v[1], cs.lo_v[2]};
    int changed = 0;
    const int n2 = mask_and_sums<DIM, RV, true>(a, rows, R, o, N, nhy, ntlo, nv, S, cs, true, &changed);
    if (changed == 0) break;  // same set, same sums
    if (tid == 0) {
      double vt[3];
      cs.lo_ok = solve_normal<DIM>(cs.red_t, n2, vt) ? 1 : 0;
    }
    __syncthreads();
    if (!cs.lo_ok) {
      n_in = mask_and_sums<DIM, RV, true>(a, rows, R, o, N, gen_hy, gen_tlo, gen_v, S, cs, false, nullptr);
      break;
    }
    gen_hy = nhy;
    gen_tlo = ntlo;
    gen_v[0] = nv[0];
    gen_v[1] = nv[1];
    gen_v[2] = nv[2];
    n_in = n2;
  }
  return n_in;
}

// Keeps, in order, the entries of S.list[0 .. n) (from_list) or the trials
// 0 .. n - 1 for which keep(h) holds, writing them to S.list[0 ..); returns
// how many.  Entries are read before any is written (compaction in place).
// red: kWarps ints of shared memory.
template <typename Keep>
__device__ __forceinline__ int compact_list(const Smem& S, int n, bool from_list, Keep keep, int* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int out = 0;
  for (int r0 = 0; r0 < n; r0 += 4 * kThreads) {
    int hv[4], c = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = r0 + 4 * tid + k;
      int h = -1;
      if (i < n) {
        h = from_list ? (int)S.list[i] : i;
        if (h == (int)kDropped || !keep(h)) h = -1;
      }
      hv[k] = h;
      c += h >= 0 ? 1 : 0;
    }
    int incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    if (lane == 31) red[warp] = incl;
    __syncthreads();
    int pos = out + incl - c, tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const int v = red[w];
      tot += v;
      pos += w < warp ? v : 0;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (hv[k] >= 0) S.list[pos++] = (uint16_t)hv[k];
    out += tot;
    __syncthreads();
  }
  return out;
}

// Drops the entries of S.list[0 .. n) (n <= 4 kThreads) for which keep(h)
// fails: marked kDropped in place, and the list compacted (in order) only
// when its groups of 128 would be fewer.  Returns the new list length
// (marked entries included when it was not compacted).  red: kWarps ints.
template <typename Keep>
__device__ __forceinline__ int prune_list(const Smem& S, int n, Keep keep, int* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int hv[4], c = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = 4 * tid + k;
    int h = i < n ? (int)S.list[i] : (int)kDropped;
    if (h != (int)kDropped && !keep(h)) {
      S.list[i] = kDropped;
      h = (int)kDropped;
    }
    hv[k] = h;
    c += h != (int)kDropped ? 1 : 0;
  }
  int incl = c;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) red[warp] = incl;
  __syncthreads();
  int pos = incl - c, tot = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const int v = red[w];
    tot += v;
    pos += w < warp ? v : 0;
  }
  if (((tot + 127) >> 7) == ((n + 127) >> 7)) return n;  // as many groups: keep the marks
  // every entry was read before the barrier above: compact in place
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (hv[k] != (int)kDropped) S.list[pos++] = (uint16_t)hv[k];
  __syncthreads();
  return tot;
}

// Staged scoring pass: the first stage covers kStageQuads quads (4 points
// each), every later one half as many again as the one before; clusters
// of fewer than kStageMinPoints points are scored in one pass (measured:
// below that the stages cost more than pruning saves).
constexpr int kStageQuads = 32;
constexpr int kStageMinPoints = 512;

// a2 + a3 for trials hc0 .. hc0 + nh - 1 of cluster ci under the cosine
// model: draw, FP32 solve (refined when ill-conditioned), bound, records
// into S.  Trials with a wide band refine their velocity.  3D minimal sets
// are often ill-conditioned and refine on the spot above kRefineBand.  2D
// ones have |det| = |sin(t1 - t0)| and mostly narrow bands, whose few band
// points cost less than refining; those above tau / 32 are queued, and when
// they are at least an eighth of the chunk (a cluster of narrow azimuth
// extent, such as a far object, where nearly every seed pair is
// ill-conditioned) a second pass refines them, one per lane.  Elsewhere the
// pass's latency would cost more than the band points it saves; either way
// the decisions are exact.
template <int DIM, typename RV>
__device__ __forceinline__ void cosine_trial_chunk(const FrameDesc& a, const RV rows, const Rows64<DIM>& R,
                                                     const Smem& S, ClusterShared& cs, int ci, int N, int hc0,
                                                     int nh, float wmax, unsigned long long* fp64_count,
                                                     unsigned long long* refined_count) {
  const int tid = threadIdx.x;
  const float refine_band = DIM == 3 ? kRefineBand : a.tau32.hi * 0x1p-5f;
  unsigned long long n_fp64 = 0, n_ref = 0;
  for (int hl = tid; hl < nh; hl += kThreads) {
    int q[3];
    draw_minimal_set<DIM>(a.key, a.cluster_base + ci, hc0 + hl, N, q);
    const int q2 = DIM == 3 ? q[2] : q[0];
    const float4 p0 = rows.at(q[0]), p1 = rows.at(q[1]), p2 = rows.at(q2);
    const int qs[3] = {q[0], q[1], q2};
    auto seed64 = [&](int i) { return R.at(qs[i]); };
    const float rb = DIM == 3 ? refine_band : __int_as_float(0x7f800000);
    Hyp32 hy = hyp_f32<DIM>(p0, p1, p2, seed64, rb, wmax, a.acc, a.rej, a.tau32);
    if (hy.kind == kHypUndecided) {
      ++n_fp64;
      double v[3];
      if (hyp_f64<DIM>(a, R, ci, hc0 + hl, N, v)) {
        hy = hyp_f32<DIM>(p0, p1, p2, seed64, rb, wmax, 0.0f, 0.0f, a.tau32);
        if (hy.kind != kHypNormal) {
          hy.kind = kHypExactOnly;
          hy.thi = __int_as_float(0x7f800000);
          hy.tlo = -1.0f;
        }
      } else {
        hy.kind = kHypRejected;
      }
    }
    if (hy.kind == kHypExactOnly) ++n_fp64;
    n_ref += hy.refined;
    S.hyp[hl] = make_float4(hy.nx, hy.ny, hy.nz, hy.kind == kHypRejected ? __int_as_float(0x7fc00000) : hy.thi);
    S.tlo[hl] = hy.tlo;
    S.kind[hl] = (int8_t)hy.kind;
    if constexpr (DIM == 2) {
      // the queue lives in U until the second pass has read it
      if (hy.kind == kHypNormal && hy.thi - a.tau32.hi > refine_band) S.U[atomicAdd(&cs.nref, 1)] = hl;
    } else {
      S.U[hl] = hy.kind == kHypRejected ? -1 : (hy.kind == kHypExactOnly ? N : 0);
    }
  }
  if constexpr (DIM == 2) {
    __syncthreads();
    const int nr = 8 * cs.nref >= nh ? cs.nref : 0;
    for (int i = tid; i < nr; i += kThreads) {
      const int hl = S.U[i];
      int q[3];
      draw_minimal_set<DIM>(a.key, a.cluster_base + ci, hc0 + hl, N, q);
      const int qs[3] = {q[0], q[1], q[0]};
      // seed rows from the frame's arrays: keeping the loaded FP32 rows
      // alive across the solve instead measured slower on trials that refine
      auto seed64 = [&](int k) { return R.at(qs[k]); };
      // the trial was accepted in the first pass: no conditioning test
      Hyp32 hy = hyp_f32<DIM>(rows.at(q[0]), rows.at(q[1]), rows.at(q[0]), seed64, refine_band, wmax, 0.0f,
                              0.0f, a.tau32);
      if (hy.kind != kHypNormal) {
        hy.kind = kHypExactOnly;
        hy.thi = __int_as_float(0x7f800000);
        hy.tlo = -1.0f;
        ++n_fp64;
      }
      n_ref += hy.refined;
      S.hyp[hl] = make_float4(hy.nx, hy.ny, hy.nz, hy.thi);
      S.tlo[hl] = hy.tlo;
      S.kind[hl] = (int8_t)hy.kind;
    }
    __syncthreads();
    for (int hl = tid; hl < nh; hl += kThreads) {
      const int k = S.kind[hl];
      S.U[hl] = k == kHypRejected ? -1 : (k == kHypExactOnly ? N : 0);
    }
    if (tid == 0) cs.nref = 0;
  }
  *fp64_count += n_fp64;
  *refined_count += n_ref;
}

template <int DIM, bool SMEM_ROWS, bool EXT>
__device__ void process_cluster(const FrameDesc& a, const Smem& S, ClusterShared& cs, int ci, int hchunk,
                                int pw, int hpl, int prune, int frame, FinishRec* fq, int* fq_n,
                                double4_32a* cta_pre) {
  const int tid = threadIdx.x;
  const int64_t o = a.offsets[ci];
  const int64_t e = a.offsets[ci + 1];
  if (o < 0 || e < o || e > a.n_points || (e - o) > 0x7fffffff) {
    if (tid == 0) write_invalid<DIM>(a, ci, RVH_STATUS_BAD_OFFSETS);
    return;
  }
  const int N = (int)(e - o);
  if (N < DIM) {
    for (int j = tid; j < N; j += kThreads) a.mask[o + j] = 0;
    if (tid == 0) write_invalid<DIM>(a, ci, RVH_STATUS_TOO_FEW_POINTS);
    return;
  }
  using RV = typename std::conditional<SMEM_ROWS, TileRowsOf<DIM>, AosRows>::type;
  RV rows;
  if constexpr (SMEM_ROWS) {
    rows.f = S.rows;
  } else {
    rows.p = a.rows_g + o;
  }
  // FP64 rows: the CTA's own slot when the cluster fits it (the slot is
  // reused cluster after cluster and stays in L2), else the frame's
  // per-point scratch
  const Rows64<DIM> R = {&a, o, (SMEM_ROWS && cta_pre) ? cta_pre : a.rows64_g + o};
  long long t_stage = clock64();
  auto stage_done = [&](int k) {
    if (tid == 0) {
      const long long t = clock64();
      cs.clk[k] += (unsigned long long)(t - t_stage);
      t_stage = t;
    }
  };

  // a1: FP32 rows in shared memory (sincosf), FP64 rows in global scratch;
  // the line model of Alg. 1 normalises its points and computes its MAD
  // threshold instead
  float wm = 0.0f;
  auto cosine_rows = [&]() {
    for (int j = tid; j < N; j += kThreads) {
      const float w = a.dop[o + j];
      const float az = a.az[o + j];
      const float el = DIM == 3 ? a.el[o + j] : 0.0f;
      rows.put(j, row_f32<DIM>(az, el, w));
      if (DIM == 3) {
        double a64[3];
        row_f64<DIM>(a.trig, az, el, a64);
        R.pre[j] = make_double4_32a(a64[0], a64[1], a64[2], (double)w);
      }
      wm = fmaxf(wm, fabsf(w));
    }
  };
  if constexpr (EXT && DIM == 2) {
    if (a.line_model) {
      line_rows_and_threshold<RV>(a, rows, R.pre, o, N, S.U, cs);
      if (tid == 0 && a.threshold) a.threshold[ci] = cs.ln_T;  // the API wrote NaN before
    } else {
      cosine_rows();
    }
  } else {
    cosine_rows();
  }
  if constexpr (SMEM_ROWS) {
    // pad the last quad of the scoring pass: NaN Dopplers never count
    if (tid < ((N + 3) & ~3) - N) {
      const float nan = __int_as_float(0x7fc00000);
      rows.put(N + tid, make_float4(0.0f, 0.0f, nan, nan));
    }
  }
  wm = block_max_float(wm, cs.red_f);  // includes a __syncthreads after the row writes
  if (tid == 0) {
    cs.best = 0ull;
    cs.wmax = wm;
    cs.nref = 0;
  }
  __syncthreads();
  const float wmax = cs.wmax;
  unsigned long long n_fp64 = 0, n_cand = 0, n_ref = 0, n_scored = 0;
  stage_done(0);

  // trials run in chunks of hchunk, or in the adaptive blocks of trial_block
  const int chunk = (EXT && a.trial_block > 0) ? a.trial_block : hchunk;
  [[maybe_unused]] int trials_run = a.H;  // all of them, unless the adaptive count stops early
  for (int hc0 = 0; hc0 < a.H; hc0 += chunk) {
    const int nh = min(chunk, a.H - hc0);
    // a2 + a3: draw, FP32 solve (refined when ill-conditioned), bound
    auto cosine_trials = [&]() {
      cosine_trial_chunk<DIM, RV>(a, rows, R, S, cs, ci, N, hc0, nh, wmax, &n_fp64, &n_ref);
    };
    if constexpr (EXT && DIM == 2) {
      if (a.line_model) {
        for (int hl = tid; hl < nh; hl += kThreads) {
          // Alg. 1: the line through the two normalised seed points, in FP64
          double v[3];
          Hyp32 hy;
          if (line_hyp64(a, R.pre, ci, hc0 + hl, N, v)) {
            hy = line_record(v, cs.ln_T);
          } else {
            hy.kind = kHypRejected;
            hy.nx = hy.ny = hy.nz = 0.0f;
            hy.tlo = -1.0f;
            hy.thi = 0.0f;
          }
          if (hy.kind == kHypExactOnly) ++n_fp64;
          S.hyp[hl] = make_float4(hy.nx, hy.ny, hy.nz, hy.kind == kHypRejected ? __int_as_float(0x7fc00000) : hy.thi);
          S.tlo[hl] = hy.tlo;
          S.kind[hl] = (int8_t)hy.kind;
          S.U[hl] = hy.kind == kHypRejected ? -1 : (hy.kind == kHypExactOnly ? N : 0);
        }
      } else {
        cosine_trials();
      }
    } else {
      cosine_trials();
    }
    __syncthreads();
    stage_done(1);

    // a5 + a6 (used by the staged pass and by the best-first counts below):
    // exact count of trial hc0 + c, which leaves the pool (U = -1) and
    // becomes the lead if its key beats it
    auto count_trial = [&](int c) {
      const float4 hy = S.hyp[c];
      const float htlo = S.tlo[c];
      int B = 0;
      const int C = exact_count_block<DIM, RV, EXT>(a, rows, R, ci, hc0 + c, N, hy, htlo, cs, &B);
      ++n_cand;
      if (tid == 0) {
        S.U[c] = -1;
        const unsigned long long k = best_key(C, hc0 + c);
        if (k > cs.best) {
          cs.best = k;
          cs.win = hy;
          cs.win_tlo = htlo;
          cs.win_has_v64 = B > 0;
          cs.win_v64[0] = cs.cv64[0];
          cs.win_v64[1] = cs.cv64[1];
          cs.win_v64[2] = cs.cv64[2];
        }
      }
      __syncthreads();
    };

    // a4: scoring pass (the hot loop)
    bool staged = false;
    if constexpr (SMEM_ROWS) staged = prune && pw == 1 && N >= kStageMinPoints;
    if (!staged) {
      phase_a_dispatch<DIM>(pw, hpl, rows, N, S, nh);
      if (tid == 0) n_scored += (unsigned long long)nh * (unsigned long long)N;
    } else if constexpr (SMEM_ROWS) {
      // Staged, with exact pruning: the trials still in the list are scored
      // in stages (kStageQuads quads, then each stage half as long again);
      // after the first stage the trial with the highest partial count is
      // counted exactly (it leads from then on), and after every stage a
      // trial whose partial count plus the points still to come cannot beat
      // the lead's key leaves the list (U = -1; marked kDropped, or
      // compacted away).  Each remaining point adds at most one to a count and
      // C_h <= U_h, so a trial dropped this way cannot win: the winner is
      // the one scoring every trial over every point gives, found by the
      // best-first counts below among the trials that stayed.
      const int nq = (N + 3) >> 2;
      int A = compact_list(S, nh, false, [&](int h) { return S.kind[h] == kHypNormal; }, cs.red_i);
      bool led = false;
      unsigned long long scored = 0;
      int sq = kStageQuads;
      for (int q0 = 0; q0 < nq && A > 0;) {
        int q1 = min(nq, q0 + sq);
        if (nq - q1 < sq / 2) q1 = nq;  // no short last stage
        sq = (sq * 3) >> 1;
        // (trial group, quad) units split evenly over the warps
        const int span = q1 - q0, total = ((A + 127) >> 7) * span;
        const int per = (total + kWarps - 1) / kWarps;
        for (int u = (tid >> 5) * per, e = min(total, u + per); u < e;) {
          const int g = u / span, qa = q0 + u % span, qb = min(q0 + span, qa + (e - u));
          scored += (unsigned long long)score_segment<DIM>(rows, N, S, A, g, qa, qb);
          u += qb - qa;
        }
        __syncthreads();
        q0 = q1;
        if (q0 >= nq) break;
        const int rem = N - 4 * q0;
        if (!led) {
          led = true;
          unsigned long long km = 0;
          for (int i = tid; i < A; i += kThreads) {
            const int h = S.list[i];
            if (h != (int)kDropped) km = max(km, best_key(S.U[h], hc0 + h));
          }
          km = block_max_u64(km, cs.red_u);
          const int c = (int)(0xFFFFFFFFu - (uint32_t)(km & 0xFFFFFFFFull)) - hc0;
          if (km != 0ull && best_key(S.U[c] + rem, hc0 + c) > cs.best) count_trial(c);
        }
        const unsigned long long lead = cs.best;
        auto alive = [&](int h) {
          const int u = S.U[h];
          const bool keep = u >= 0 && best_key(u + rem, hc0 + h) > lead;
          if (!keep) S.U[h] = -1;
          return keep;
        };
        A = A <= 4 * kThreads ? prune_list(S, A, alive, cs.red_i) : compact_list(S, A, true, alive, cs.red_i);
      }
      if ((tid & 31) == 0) n_scored += scored;
    }
    __syncthreads();
    stage_done(2);

    // a5 + a6: exact counts of the trials whose upper bound can still win,
    // best first: the trial with the highest key (U, then lowest index) is
    // counted next, until no remaining key beats the lead.  C_h <= U_h, so a
    // trial whose key (U_h, h) does not beat the lead cannot win with its
    // exact count either, and the winner -- the highest exact count, the
    // lowest index among equals -- is the one counting every trial would
    // give.  Trials of earlier chunks have lower indices; the lead's key
    // already ranks them.  A counted trial leaves the pool (U = -1).
    for (;;) {
      unsigned long long km = 0;
      for (int hl = tid; hl < nh; hl += kThreads) {
        const int u = S.U[hl];
        if (u >= 0) km = max(km, best_key(u, hc0 + hl));
      }
      km = block_max_u64(km, cs.red_u);
      if (km <= cs.best) break;  // also km == 0: no trial left
      count_trial((int)(0xFFFFFFFFu - (uint32_t)(km & 0xFFFFFFFFull)) - hc0);
    }
    __syncthreads();
    stage_done(3);
    if constexpr (EXT) {
      // adaptive trial count: stop once the bound says enough trials have run
      if (a.confidence > 0.0 && hc0 + nh < a.H) {
        if (tid == 0) cs.stop = adaptive_stop(cs.best, N, DIM, hc0 + nh, a.confidence);
        __syncthreads();
        if (cs.stop) {
          trials_run = hc0 + nh;
          break;
        }
      }
    }
  }

  if (tid == 0) cs.ctr[0] += n_cand;
  if (n_scored) atomicAdd(&cs.scored, n_scored);
  if constexpr (EXT) {
    if (tid == 0) {
      cs.runs[0] += (unsigned long long)trials_run;
      cs.runs[1] += (unsigned long long)trials_run * (unsigned long long)N;
    }
  }
  if (n_fp64) atomicAdd(&cs.ctr[2], n_fp64);
  if (n_ref) atomicAdd(&cs.ctr[3], n_ref);

  const unsigned long long key = cs.best;
  if (key == 0ull) {
    for (int j = tid; j < N; j += kThreads) a.mask[o + j] = 0;
    if (tid == 0) write_invalid<DIM>(a, ci, RVH_STATUS_ALL_DEGENERATE);
    __syncthreads();
    return;
  }
  const int hstar = (int)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));

  // a7 + a8: the winner's mask (FP32 certainties; FP64 for its band points,
  // whose FP64 velocity was computed when it was counted) and the normal
  // equations over its inliers.
  const float4 win = cs.win;
  const float wtlo = cs.win_tlo;
  const double v64[3] = {cs.win_v64[0], cs.win_v64[1], cs.win_v64[2]};
  constexpr int NS = DIM == 2 ? 5 : 9;
  int n_in = mask_and_sums<DIM, RV, EXT>(a, rows, R, o, N, win, wtlo, v64, S, cs, false, nullptr);

  if constexpr (EXT) {
    if (a.lo_iters > 0) n_in = local_opt_rounds<DIM, RV>(a, rows, R, o, N, win, wtlo, v64, wmax, n_in, S, cs);
  }
  if (tid == 0) {
    FinishRec& q = fq[*fq_n];
#pragma unroll
    for (int i = 0; i < NS; ++i) q.t[i] = cs.red_t[i];
    q.v64[0] = v64[0];
    q.v64[1] = v64[1];
    q.v64[2] = v64[2];
    q.o = o;
    q.n_in = n_in;
    q.hstar = hstar;
    q.ci = ci;
    q.frame = frame;
    q.N = N;
    q.has_v64 = cs.win_has_v64;
    *fq_n += 1;
  }
  __syncthreads();
  stage_done(4);
}

// EXT = true: the instantiation with the extensions of the method (the
// local-optimisation rounds and the adaptive trial count), launched only for
// batches that ask for one of them; the default instantiation carries no
// trace of them.
template <int DIM, bool EXT>
__global__ void __launch_bounds__(kThreads, RVH_MIN_BLOCKS) fused_kernel(const __grid_constant__ FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ClusterShared cs;
  __shared__ int s_item;
  __shared__ FinishRec fq[kFinishBatch];
  __shared__ int fq_n;
  Smem S;
  unsigned char* p = smem_raw;
  S.rows = reinterpret_cast<float*>(p);
  p += (size_t)((a.nmax_smem + 31) & ~31) * sizeof(float4);
  S.hyp = reinterpret_cast<float4*>(p);
  p += (size_t)a.hchunk * sizeof(float4);
  S.tlo = reinterpret_cast<float*>(p);
  p += (size_t)a.hchunk * sizeof(float);
  S.U = reinterpret_cast<int*>(p);
  p += (size_t)a.hchunk * sizeof(int);
  S.kind = reinterpret_cast<int8_t*>(p);
  p += ((size_t)a.hchunk * sizeof(int8_t) + 15) & ~(size_t)15;
  S.list = reinterpret_cast<uint16_t*>(p);

  if (threadIdx.x < 4) cs.ctr[threadIdx.x] = 0ull;
  if constexpr (EXT) {
    if (threadIdx.x < 2) cs.runs[threadIdx.x] = 0ull;
  }
  if (threadIdx.x < 6) cs.clk[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) {
    fq_n = 0;
    cs.scored = 0ull;
  }
  // the queued clusters' solves and headings, one lane each
  auto flush = [&]() {
    const int n = fq_n;
    if (threadIdx.x < n) {
      const FinishRec& q = fq[threadIdx.x];
      const FrameDesc& F = a.f[q.frame];
      // the CTA's row slot has moved on to later clusters: rows are
      // recomputed for the (rare) fallback solve
      const Rows64Inputs<DIM> R = {&F, q.o};
      finish_cluster<DIM, EXT>(F, R, q.ci, q.N, q.hstar, q.n_in, q.t, q.v64, q.has_v64 != 0);
    }
    __syncthreads();
    if (threadIdx.x == 0) fq_n = 0;
    __syncthreads();
  };
  const long long t_kernel = clock64();
  for (int round = 0;; ++round) {
    __syncthreads();
    if (threadIdx.x == 0)
      s_item = a.direct ? (round == 0 ? (int)blockIdx.x : a.n_items) : atomicAdd(a.work_counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= a.n_items) break;
    int2 fc;
    if (a.direct) {
      // as many CTAs as items: frame-major order needs no work list
      int f = 0, rem = item;
      while (rem >= a.f[f].n_clusters) rem -= a.f[f++].n_clusters;
      fc = make_int2(f, rem);
    } else {
      fc = a.worklist[item];
    }
    const FrameDesc& F = a.f[fc.x];
    const int ci = fc.y;
    const int64_t o = F.offsets[ci], e = F.offsets[ci + 1];
    double4_32a* cta_pre =
        a.cta_rows64 ? a.cta_rows64 + (size_t)blockIdx.x * cta_slot_stride(DIM, a.nmax_smem) : nullptr;
    if (e - o <= (int64_t)smem_row_capacity(DIM, a.nmax_smem) || e < o) {
      process_cluster<DIM, true, EXT>(F, S, cs, ci, a.hchunk, a.pw, a.hpl, a.prune, fc.x, fq, &fq_n, cta_pre);
    } else {
      process_cluster<DIM, false, EXT>(F, S, cs, ci, a.hchunk, a.pw, a.hpl, a.prune, fc.x, fq, &fq_n, cta_pre);
    }
    __syncthreads();
    if (fq_n == kFinishBatch) flush();
  }
  __syncthreads();
  flush();
  if (threadIdx.x == 0) {
    unsigned long long staged = 0;
    for (int k = 0; k < 5; ++k) staged += cs.clk[k];
    const unsigned long long total = (unsigned long long)(clock64() - t_kernel);
    cs.clk[5] = total > staged ? total - staged : 0ull;
  }
  __syncthreads();
  if (threadIdx.x < 4 && a.stats) {
    unsigned long long v = cs.ctr[threadIdx.x];
    if (v) atomicAdd(&a.stats[threadIdx.x], v);
  }
  if (threadIdx.x < 6 && a.stats) atomicAdd(&a.stats[4 + threadIdx.x], cs.clk[threadIdx.x]);
  if (threadIdx.x == 0 && a.stats) atomicAdd(&a.stats[12], cs.scored);
  if constexpr (EXT) {
    if (threadIdx.x < 2 && a.stats) atomicAdd(&a.stats[10 + threadIdx.x], cs.runs[threadIdx.x]);
  }
}

// Orders the batch's (frame, cluster) items by decreasing cost N * H (H: the
// trial_block of adaptive frames, which mostly stop after one block),
// longest-processing-time first, in buckets of an eighth of an octave (the
// floor of log2 of the cost and its next three bits), and resets the work
// counter.  One CTA.
constexpr int kCostBuckets = 512;
__device__ __forceinline__ int item_bucket(const FrameDesc& F, int ci) {
  const int64_t n = (int64_t)F.offsets[ci + 1] - F.offsets[ci];
  const int64_t cost = n > 0 ? n * (int64_t)(F.trial_block > 0 ? min(F.trial_block, F.H) : F.H) : 1;
  const int lg = 63 - __clzll(cost);
  const int sub = (int)((lg >= 3 ? cost >> (lg - 3) : cost << (3 - lg)) & 7);
  return kCostBuckets - 1 - min((lg << 3) | sub, kCostBuckets - 1);  // 0 = most expensive
}

// Items are numbered frame-major; each thread keeps the buckets of its first
// kItemsKept items in registers between the two passes.  Also zeroes the
// launch's stats counters (the fused kernel adds to them).
constexpr int kItemsKept = 8;
__global__ void worklist_kernel(const __grid_constant__ FusedArgs a) {
  __shared__ int hist[kCostBuckets];
  for (int b = threadIdx.x; b < kCostBuckets; b += blockDim.x) hist[b] = 0;
  if (a.stats && threadIdx.x < kStatsWords) a.stats[threadIdx.x] = 0ull;
  __syncthreads();
  int kept[kItemsKept];
  {
    int f = 0, base = 0, k = 0;
    for (int it = threadIdx.x; it < a.n_items; it += blockDim.x, ++k) {
      while (it - base >= a.f[f].n_clusters) base += a.f[f++].n_clusters;
      const int b = item_bucket(a.f[f], it - base);
      if (k < kItemsKept) kept[k] = b;
      atomicAdd(&hist[b], 1);
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive scan of the histogram, 16 buckets per lane
    constexpr int kPer = kCostBuckets / 32;
    const int lane = threadIdx.x;
    int c[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      c[k] = hist[lane * kPer + k];
      sum += c[k];
    }
    int incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    int run = incl - sum;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      hist[lane * kPer + k] = run;
      run += c[k];
    }
    if (lane == 0) *a.work_counter = 0;
  }
  __syncthreads();
  {
    int f = 0, base = 0, k = 0;
    for (int it = threadIdx.x; it < a.n_items; it += blockDim.x, ++k) {
      while (it - base >= a.f[f].n_clusters) base += a.f[f++].n_clusters;
      const int b = k < kItemsKept ? kept[k] : item_bucket(a.f[f], it - base);
      a.worklist[atomicAdd(&hist[b], 1)] = make_int2(f, it - base);
    }
  }
}

size_t fused_smem_bytes(int nmax_smem, int hchunk) {
  // the trial area also holds the final reduction (up to 9 sums per thread)
  const size_t trials = (size_t)hchunk * (sizeof(float4) + sizeof(float) + sizeof(int) + sizeof(uint16_t)) +
                        (((size_t)hchunk + 15) & ~(size_t)15);
  const size_t reduction = (size_t)9 * kThreads * sizeof(double);
  return (size_t)((nmax_smem + 31) & ~31) * sizeof(float4) + (trials > reduction ? trials : reduction);
}

cudaError_t launch_worklist(const FusedArgs& a, cudaStream_t s) {
  worklist_kernel<<<1, kWorklistThreads, 0, s>>>(a);
  return cudaGetLastError();
}

bool fused_ext(const FusedArgs& a) {
  bool ext = false;
  for (int f = 0; f < a.n_frames; ++f)
    ext = ext || a.f[f].lo_iters > 0 || a.f[f].confidence > 0.0 || a.f[f].line_model != 0;
  return ext;
}

const void* fused_kernel_fn(int dim, bool ext) {
  if (dim == 2) return ext ? (const void*)fused_kernel<2, true> : (const void*)fused_kernel<2, false>;
  return ext ? (const void*)fused_kernel<3, true> : (const void*)fused_kernel<3, false>;
}

const void* worklist_kernel_fn() { return (const void*)worklist_kernel; }

int fused_threads() { return kThreads; }

cudaError_t fused_configure_max(int dim, int device) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  for (int ext = 0; ext < 2 && e == cudaSuccess; ++ext) {
    const void* fn = fused_kernel_fn(dim, ext != 0);
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  }
  return e;
}

cudaError_t fused_occupancy(int dim, size_t smem, int* blocks_per_sm) {
  if (dim == 2)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fused_kernel<2, false>, kThreads, smem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fused_kernel<3, false>, kThreads, smem);
}

cudaError_t launch_fused(int dim, const FusedArgs& a, int grid, size_t smem, cudaStream_t s) {
  const bool ext = fused_ext(a);
  if (dim == 2) {
    if (ext) fused_kernel<2, true><<<grid, kThreads, smem, s>>>(a);
    else fused_kernel<2, false><<<grid, kThreads, smem, s>>>(a);
  } else {
    if (ext) fused_kernel<3, true><<<grid, kThreads, smem, s>>>(a);
    else fused_kernel<3, false><<<grid, kThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace rvh
