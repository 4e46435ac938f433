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
// tile (32 c | 32 s | 32 w | 32 unused in 2D; 32 a0 | 32 a1 | 32 a2 | 32 w in
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

// Packed FP32 pairs (fma.rn.f32x2 / add.rn.f32x2 round each half like the
// scalar instruction, so results are those of fmaf / FP32 add per element).
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
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// min(1, max(0, C - r^2)) in one saturated FMA (NaN gives 0).  With
// C >= t^2 + 1 it is 1 whenever |r| <= t, and 0 once r^2 >= C; in between a
// fraction, so sums of it bound the count of |r| <= t from above.
__device__ __forceinline__ float sat_square(float r, float C) {
  float e;
  asm("{.reg .f32 n; neg.f32 n, %1; fma.rn.sat.f32 %0, n, %1, %2;}" : "=f"(e) : "f"(r), "f"(C));
  return e;
}
// 1.0f if |r| <= t else 0.0f (false for NaN)
__device__ __forceinline__ float in_band(float r, float t) {
  float e;
  asm("{.reg .f32 a; abs.f32 a, %1; set.le.f32.f32 %0, a, %2;}" : "=f"(e) : "f"(r), "f"(t));
  return e;
}

// a4 over tiled rows: the residuals of two points per instruction.  Lane l
// handles trial sub-group l / PW and point quads l % PW, l % PW + PW, ...;
// the rows stage pads the last quad with NaN Dopplers, which never count.
// Per element the arithmetic is resid_f32's: w + nz z + ny y + nx x by fmaf.
// 2D evaluates it 2^20 times larger (the rows' fourth slot holds 2^20 w, the
// velocity is scaled likewise, both exactly) and counts with the saturated
// square test against C = 2^40 thi^2 + 1 rounded up, which keeps the count
// on the FP32 pipe: U_h >= #{|r32| <= thi}, exceeding it only by points
// whose squared residual lies within 2^-40 of thi^2.  3D counts with FSET.
template <int DIM, int PW, int HPL>
__device__ __forceinline__ void phase_a_tiles(const TileRows rows, int N, const Smem& S, int nh) {
  constexpr int NHL = 32 / PW;
  constexpr int G = NHL * HPL;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int hl = lane / PW, pl = lane % PW;
  const int ngroups = (nh + G - 1) / G;
  const int nq = (N + 3) >> 2;
  for (int g = warp; g < ngroups; g += kWarps) {
    const int base = g * G + hl * HPL;
    unsigned long long nx[HPL], ny[HPL], nz[HPL], acc[HPL];
    float th[HPL];
#pragma unroll
    for (int m = 0; m < HPL; ++m) {
      const int h = base + m;
      const float4 v = (h < nh) ? S.hyp[h] : make_float4(0.f, 0.f, 0.f, __int_as_float(0x7fc00000));
      if (DIM == 2) {
        const float sx = v.x * kScoreScale, sy = v.y * kScoreScale, st = v.w * kScoreScale;
        nx[m] = pack2(sx, sx);
        ny[m] = pack2(sy, sy);
        th[m] = __fadd_ru(__fmul_ru(st, st), 1.0f);  // C = (2^20 thi)^2 + 1, rounded up
      } else {
        nx[m] = pack2(v.x, v.x);
        ny[m] = pack2(v.y, v.y);
        th[m] = v.w;
      }
      nz[m] = pack2(v.z, v.z);
      acc[m] = 0ull;
    }
    for (int q = pl; q < nq; q += PW) {
      const float4 c = rows.quad(q, 0), sn = rows.quad(q, 1), z = rows.quad(q, DIM == 2 ? 3 : 2);
      const unsigned long long c01 = pack2(c.x, c.y), c23 = pack2(c.z, c.w);
      const unsigned long long s01 = pack2(sn.x, sn.y), s23 = pack2(sn.z, sn.w);
      unsigned long long w01, w23, z01 = 0ull, z23 = 0ull;
      if (DIM == 2) {  // 2^20 w
        w01 = pack2(z.x, z.y);
        w23 = pack2(z.z, z.w);
      } else {
        const float4 w = rows.quad(q, 3);
        z01 = pack2(z.x, z.y);
        z23 = pack2(z.z, z.w);
        w01 = pack2(w.x, w.y);
        w23 = pack2(w.z, w.w);
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
        float a0, a1, a2, a3;
        unpack2(r01, a0, a1);
        unpack2(r23, a2, a3);
        if (DIM == 2) {
          acc[m] = add2(acc[m], pack2(sat_square(a0, th[m]), sat_square(a1, th[m])));
          acc[m] = add2(acc[m], pack2(sat_square(a2, th[m]), sat_square(a3, th[m])));
        } else {
          acc[m] = add2(acc[m], pack2(in_band(a0, th[m]), in_band(a1, th[m])));
          acc[m] = add2(acc[m], pack2(in_band(a2, th[m]), in_band(a3, th[m])));
        }
      }
    }
    float cnt[HPL];
#pragma unroll
    for (int m = 0; m < HPL; ++m) {
      float lo, hi;
      unpack2(acc[m], lo, hi);
      cnt[m] = lo + hi;  // integers below 2^24 (3D); 2D: at least the count (rounding is monotone)
#pragma unroll
      for (int o = PW / 2; o > 0; o >>= 1) cnt[m] += __shfl_xor_sync(0xffffffffu, cnt[m], o);
    }
    if (pl == 0) {
#pragma unroll
      for (int m = 0; m < HPL; ++m) {
        const int h = base + m;
        if (h < nh && S.kind[h] == kHypNormal) S.U[h] = (int)cnt[m];  // floor
      }
    }
  }
}

}  // namespace rvh
