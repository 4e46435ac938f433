// The scoring pass of the fused kernel (step a4, the hot loop): upper-bound
// inlier counts of a chunk of trials over a cluster's FP32 rows staged in
// shared memory as 32-point tiles, two points per packed FP32 instruction.
// Sec. III-A, Alg. 1 (the loop over a cluster's points for every trial).
//
// Kept in its own header so that the standalone scoring benchmark
// (tests/cuda/scoring_bench.cu) runs exactly this device code.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rvh_device.cuh"

namespace rvh {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
#ifndef RVH_MIN_BLOCKS
#define RVH_MIN_BLOCKS 4
#endif

struct Smem {
  float* rows;        // [roundup32(nmax_smem) * 4] floats of row tiles (TileRows)
  float4* hyp;        // [hchunk] (-X, -Y, -Z, thi)
  float* tlo;         // [hchunk]
  int* U;             // [hchunk] upper bounds of the exact counts (-1 = rejected)
  int8_t* kind;       // [hchunk]
  uint16_t* list;     // [hchunk] trials still scored by the staged pass
};

// ---- FP32 rows of the cluster being processed ---------------------------------------
// Shared memory holds them as tiles of 32 points, component-major inside a
// tile (32 c | 32 s | 32 w in 2D; 32 a0 | 32 a1 | 32 a2 | 32 w in 3D): a
// warp reading consecutive points touches 32 banks per component, and four
// consecutive points of one component are one aligned float4, which the
// scoring pass consumes as two packed pairs.  NC = 3 (2D) or 4 (3D)
// components; at() of a 2D row leaves .w zero.  Clusters larger than the
// shared memory area keep plain float4 rows in global scratch.
template <int NC>
struct TileRows {
  float* f;
  __device__ __forceinline__ float4 at(int j) const {
    const float* b = f + (j >> 5) * (32 * NC) + (j & 31);
    return make_float4(b[0], b[32], b[64], NC == 4 ? b[96] : 0.0f);
  }
  __device__ __forceinline__ void put(int j, float4 v) const {
    float* b = f + (j >> 5) * (32 * NC) + (j & 31);
    b[0] = v.x;
    b[32] = v.y;
    b[64] = v.z;
    if (NC == 4) b[96] = v.w;
  }
  // component k of points 4q .. 4q + 3
  __device__ __forceinline__ float4 quad(int q, int k) const {
    return *reinterpret_cast<const float4*>(f + (q >> 3) * (32 * NC) + (k << 5) + ((q & 7) << 2));
  }
};
template <int DIM>
using TileRowsOf = TileRows<DIM == 2 ? 3 : 4>;

struct AosRows {
  float4* p;
  __device__ __forceinline__ float4 at(int j) const { return p[j]; }
  __device__ __forceinline__ void put(int j, float4 v) const { p[j] = v; }
};

// Packed FP32 pairs (fma.rn.f32x2 rounds each half like the scalar
// instruction, so results are those of fmaf per element).
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// Sign masks of two floats in one word: 0x0000FFFF if lo < 0 (sign bit set),
// plus 0xFFFF0000 if hi < 0 -- one byte permute (prmt, msb-replicating
// selectors) on the integer pipe.  Summed as 32-bit integers over many
// points, the words give A = 0xFFFF (S_lo + 2^16 S_hi) mod 2^32, with S_lo
// and S_hi the numbers of negative lo and hi values; sign_count recovers
// S_lo + S_hi while both stay below 2^16.
__device__ __forceinline__ uint32_t sign_pair(float lo, float hi) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, 0xFFBB;" : "=r"(d) : "r"(__float_as_uint(lo)), "r"(__float_as_uint(hi)));
  return d;
}
// 0xFFFEFFFF is the inverse of 0xFFFF modulo 2^32: (2^16 - 1)(2^32 - 2^16 - 1)
// = 2^48 - 2^33 + 1.
__device__ __forceinline__ int sign_count(uint32_t acc) {
  const uint32_t x = acc * 0xFFFEFFFFu;  // S_lo + 2^16 S_hi
  return (int)(x & 0xFFFFu) + (int)(x >> 16);
}

// -C with C the smallest float above thi^2 rounded up: C > thi^2, so
// r^2 < C for every |r| <= thi, and r^2 < C holds beyond thi only for r^2
// within two ulps of thi^2.
__device__ __forceinline__ float neg_count_bound(float thi) {
  return -__uint_as_float(__float_as_uint(__fmul_ru(thi, thi)) + 1u);
}

// HPL trial records of one lane in packed registers: (-X, -X), (-Y, -Y),
// (-Z, -Z), (-C, -C) and the sign-mask accumulator of each.
template <int HPL>
struct LaneTrials {
  unsigned long long nx[HPL], ny[HPL], nz[HPL], nc[HPL];
  uint32_t acc[HPL];
  // record (-X, -Y, -Z, thi) into slot m; a NaN thi never counts
  __device__ __forceinline__ void load(int m, float4 v) {
    nx[m] = pack2(v.x, v.x);
    ny[m] = pack2(v.y, v.y);
    nz[m] = pack2(v.z, v.z);
    const float c = neg_count_bound(v.w);
    nc[m] = pack2(c, c);
    acc[m] = 0u;
  }
};

// Scores points 4q .. 4q + 3 against the lane's trials: the residuals of two
// points per instruction, per element resid_f32's arithmetic (w + nz z +
// ny y + nx x by fmaf); the test e = r r - C (one packed FMA for two points,
// exact until its final rounding, which keeps the sign): e < 0 exactly when
// r^2 < C, and C exceeds thi^2 (neg_count_bound), so a count is an upper
// bound of #{|r32| <= thi} that exceeds it only by points within two ulps
// of thi^2.  NaN residuals (NaN Dopplers, the padding) give the canonical
// NaN, whose sign bit is clear, so they do not count (a NaN that did would
// only loosen the bound).  The count leaves the FP32 pipe: two byte permutes
// turn the four sign bits into 16-bit masks and one three-input integer add
// accumulates them (sign_pair / sign_count: the even and the odd points of a
// lane stay below 2^16 each, since a cluster in shared memory has at most
// 227 KB / 12 B points).
template <int DIM, int HPL>
__device__ __forceinline__ void score_quad(const TileRowsOf<DIM>& rows, int q, LaneTrials<HPL>& T) {
  const float4 c = rows.quad(q, 0), sn = rows.quad(q, 1), w = rows.quad(q, DIM == 2 ? 2 : 3);
  const unsigned long long c01 = pack2(c.x, c.y), c23 = pack2(c.z, c.w);
  const unsigned long long s01 = pack2(sn.x, sn.y), s23 = pack2(sn.z, sn.w);
  const unsigned long long w01 = pack2(w.x, w.y), w23 = pack2(w.z, w.w);
  unsigned long long z01 = 0ull, z23 = 0ull;
  if (DIM == 3) {
    const float4 z = rows.quad(q, 2);
    z01 = pack2(z.x, z.y);
    z23 = pack2(z.z, z.w);
  }
#pragma unroll
  for (int m = 0; m < HPL; ++m) {
    unsigned long long r01, r23;
    if (DIM == 2) {
      r01 = fma2(T.nx[m], c01, fma2(T.ny[m], s01, w01));
      r23 = fma2(T.nx[m], c23, fma2(T.ny[m], s23, w23));
    } else {
      r01 = fma2(T.nx[m], c01, fma2(T.ny[m], s01, fma2(T.nz[m], z01, w01)));
      r23 = fma2(T.nx[m], c23, fma2(T.ny[m], s23, fma2(T.nz[m], z23, w23)));
    }
    float e0, e1, e2, e3;
    unpack2(fma2(r01, r01, T.nc[m]), e0, e1);
    unpack2(fma2(r23, r23, T.nc[m]), e2, e3);
    T.acc[m] += sign_pair(e0, e1) + sign_pair(e2, e3);
  }
}

// Quads q0, q0 + step, ... below q1, unrolled by the measured factor.
template <int DIM, int HPL>
__device__ __forceinline__ void score_quads(const TileRowsOf<DIM>& rows, int q0, int q1, int step,
                                            LaneTrials<HPL>& T) {
  constexpr int UN = DIM == 2 ? 8 : 4;  // quads per loop iteration (measured)
  int q = q0;
  for (; q + (UN - 1) * step < q1; q += UN * step) {
#pragma unroll
    for (int u = 0; u < UN; ++u) score_quad<DIM, HPL>(rows, q + u * step, T);
  }
  for (; q < q1; q += step) score_quad<DIM, HPL>(rows, q, T);
}

// a4 over tiled rows, every trial of the chunk over every point.  Lane l
// handles trial sub-group l / PW and point quads l % PW, l % PW + PW, ...;
// the rows stage pads the last quad with NaN Dopplers, which never count.
template <int DIM, int PW, int HPL>
__device__ __forceinline__ void phase_a_tiles(const TileRowsOf<DIM> rows, int N, const Smem& S, int nh) {
  constexpr int NHL = 32 / PW;
  constexpr int G = NHL * HPL;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int hl = lane / PW, pl = lane % PW;
  const int ngroups = (nh + G - 1) / G;
  const int nq = (N + 3) >> 2;
  for (int g = warp; g < ngroups; g += kWarps) {
    const int base = g * G + hl * HPL;
    LaneTrials<HPL> T;
#pragma unroll
    for (int m = 0; m < HPL; ++m) {
      const int h = base + m;
      T.load(m, (h < nh) ? S.hyp[h] : make_float4(0.f, 0.f, 0.f, __int_as_float(0x7fc00000)));
    }
    score_quads<DIM, HPL>(rows, pl, nq, PW, T);
    int cnt[HPL];
#pragma unroll
    for (int m = 0; m < HPL; ++m) {
      cnt[m] = sign_count(T.acc[m]);
#pragma unroll
      for (int o = PW / 2; o > 0; o >>= 1) cnt[m] += __shfl_xor_sync(0xffffffffu, cnt[m], o);
    }
    if (pl == 0) {
#pragma unroll
      for (int m = 0; m < HPL; ++m) {
        const int h = base + m;
        if (h < nh && S.kind[h] == kHypNormal) S.U[h] = cnt[m];
      }
    }
  }
}

// A list entry of a trial dropped in place (the list is compacted only when
// that saves a group of 128).
constexpr uint16_t kDropped = 0xFFFF;
__device__ __forceinline__ int list_trial(const Smem& S, int A, int i) {
  const int e = i < A ? (int)S.list[i] : (int)kDropped;
  return e == (int)kDropped ? -1 : e;
}

// One piece of the staged scoring pass: the 128 trials of group g of the
// list S.list[0 .. A) (four per lane, lane-major) over quads [qa, qb),
// their counts added to S.U (several warps may share a group, each over
// its own quads).  Returns the (trial, point) pairs this warp scored.
template <int DIM>
__device__ __forceinline__ long long score_segment(const TileRowsOf<DIM> rows, int N, const Smem& S, int A, int g,
                                                   int qa, int qb) {
  const int lane = threadIdx.x & 31;
  LaneTrials<4> T;
  int hs[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    hs[m] = list_trial(S, A, g * 128 + lane * 4 + m);
    T.load(m, hs[m] >= 0 ? S.hyp[hs[m]] : make_float4(0.f, 0.f, 0.f, __int_as_float(0x7fc00000)));
  }
  score_quads<DIM, 4>(rows, qa, qb, 1, T);
  int trials = 0;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    if (hs[m] >= 0) atomicAdd(&S.U[hs[m]], sign_count(T.acc[m]));
    trials += __popc(__ballot_sync(0xffffffffu, hs[m] >= 0));
  }
  return (long long)trials * (min(4 * qb, N) - 4 * qa);
}

}  // namespace rvh
