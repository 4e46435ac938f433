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
  float* rows;        // [roundup32(nmax_smem) * 4] row tiles (TileRows)
  float4* hyp;        // [hchunk] (-X, -Y, -Z, thi)
  float* tlo;         // [hchunk]
  int* U;             // [hchunk] upper bounds of the exact counts (-1 = rejected)
  int8_t* kind;       // [hchunk]
};

// ---- FP32 rows of the cluster being processed ---------------------------------------
// Shared memory holds them as tiles of 32 points, component-major inside a
// tile (32 c | 32 s | 32 w | 32 t in 2D; 32 a0 | 32 a1 | 32 a2 | 32 w in
// 3D): a warp reading consecutive points touches 32 banks per component, and
// four consecutive points of one component are one aligned float4, which the
// scoring pass consumes as two packed pairs.  Clusters larger than the shared
// memory area keep plain float4 rows in global scratch.
struct TileRows {
  float* f;
  __device__ __forceinline__ float4 at(int j) const {
    const float* b = f + ((j >> 5) << 7) + (j & 31);
    return make_float4(b[0], b[32], b[64], b[96]);
  }
  __device__ __forceinline__ void put(int j, float4 v) const {
    float* b = f + ((j >> 5) << 7) + (j & 31);
    b[0] = v.x;
    b[32] = v.y;
    b[64] = v.z;
    b[96] = v.w;
  }
  // component k of points 4q .. 4q + 3
  __device__ __forceinline__ float4 quad(int q, int k) const {
    return *reinterpret_cast<const float4*>(f + ((q >> 3) << 7) + (k << 5) + ((q & 7) << 2));
  }
};

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
// Appends the sign bit of e to a 32-bit history of sign bits: the high word
// of (acc:e) << 1, i.e. (acc << 1) | (e >> 31), one funnel shift on the
// integer pipe.
__device__ __forceinline__ uint32_t push_sign(uint32_t acc, float e) {
  uint32_t d;
  asm("shf.l.clamp.b32 %0, %1, %2, 1;" : "=r"(d) : "r"(__float_as_uint(e)), "r"(acc));
  return d;
}

// -C with C the smallest float above thi^2 rounded up: C > thi^2, so
// r^2 < C for every |r| <= thi, and r^2 < C holds beyond thi only for r^2
// within two ulps of thi^2.
__device__ __forceinline__ float neg_count_bound(float thi) {
  return -__uint_as_float(__float_as_uint(__fmul_ru(thi, thi)) + 1u);
}

// a4 over tiled rows: the residuals of two points per instruction.  Lane l
// handles trial sub-group l / PW and point quads l % PW, l % PW + PW, ...;
// the rows stage pads the last quad with NaN Dopplers, which never count.
// Per element the arithmetic is resid_f32's: w + nz z + ny y + nx x by fmaf.
// The test is e = r r - C (one packed FMA for two points, exact until its
// final rounding, which keeps the sign): e < 0 exactly when r^2 < C, and C
// exceeds thi^2 (neg_count_bound), so the count U_h is an upper bound of
// #{|r32| <= thi} that exceeds it only by points within two ulps of thi^2.
// NaN residuals (NaN Dopplers, the padding) give the canonical NaN, whose
// sign bit is clear, so they do not count (a NaN that did would only loosen
// the bound).  The
// count leaves the FP32 pipe: sign bits are shifted into a 32-bit history
// (push_sign, integer pipe) and popcounted every block of quads (8 quads = 32
// points fill the history exactly; 2D uses blocks of 4 with a reset, which
// measured faster for its shorter loop body).
template <int DIM, int PW, int HPL>
__device__ __forceinline__ void phase_a_tiles(const TileRows rows, int N, const Smem& S, int nh) {
  constexpr int NHL = 32 / PW;
  constexpr int G = NHL * HPL;
  constexpr int BLOCK = DIM == 2 ? 4 : 8;  // quads per popcount
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int hl = lane / PW, pl = lane % PW;
  const int ngroups = (nh + G - 1) / G;
  const int nq = (N + 3) >> 2;
  for (int g = warp; g < ngroups; g += kWarps) {
    const int base = g * G + hl * HPL;
    unsigned long long nx[HPL], ny[HPL], nz[HPL], nc[HPL];
    uint32_t bits[HPL];
    int cnt[HPL];
#pragma unroll
    for (int m = 0; m < HPL; ++m) {
      const int h = base + m;
      const float4 v = (h < nh) ? S.hyp[h] : make_float4(0.f, 0.f, 0.f, __int_as_float(0x7fc00000));
      nx[m] = pack2(v.x, v.x);
      ny[m] = pack2(v.y, v.y);
      nz[m] = pack2(v.z, v.z);
      const float c = neg_count_bound(v.w);
      nc[m] = pack2(c, c);
      bits[m] = 0u;
      cnt[m] = 0;
    }
    auto quad = [&](int q) {
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
          r01 = fma2(nx[m], c01, fma2(ny[m], s01, w01));
          r23 = fma2(nx[m], c23, fma2(ny[m], s23, w23));
        } else {
          r01 = fma2(nx[m], c01, fma2(ny[m], s01, fma2(nz[m], z01, w01)));
          r23 = fma2(nx[m], c23, fma2(ny[m], s23, fma2(nz[m], z23, w23)));
        }
        float e0, e1, e2, e3;
        unpack2(fma2(r01, r01, nc[m]), e0, e1);
        unpack2(fma2(r23, r23, nc[m]), e2, e3);
        bits[m] = push_sign(push_sign(push_sign(push_sign(bits[m], e0), e1), e2), e3);
      }
    };
    int q = pl;
    for (; q + (BLOCK - 1) * PW < nq; q += BLOCK * PW) {
#pragma unroll
      for (int u = 0; u < BLOCK; ++u) quad(q + u * PW);
#pragma unroll
      for (int m = 0; m < HPL; ++m) {
        cnt[m] += __popc(bits[m]);
        if (BLOCK < 8) bits[m] = 0u;  // a block of 8 quads shifts all 32 bits out
      }
    }
#pragma unroll
    for (int m = 0; m < HPL; ++m) bits[m] = 0u;
    for (; q < nq; q += PW) quad(q);  // fewer than BLOCK quads
#pragma unroll
    for (int m = 0; m < HPL; ++m) {
      cnt[m] += __popc(bits[m]);
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

}  // namespace rvh
