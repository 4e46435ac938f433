// Plain all-FP64 GPU version of the same method, one launch per cluster: the
// baseline that the fused kernel is measured against.  Every trial is solved
// and scored in FP64 by one thread (the paper's thread-per-trial mapping of
// Alg. 1 and Eq. 4), the argmax is a block reduction, and the mask and normal
// equations of the winner follow (Alg. 2).
#include <cstdint>
#include <cuda_runtime.h>

#include "rvh_device.cuh"
#include "rvh_kernels.h"

namespace rvh {

constexpr int kBaseThreads = 256;

template <int DIM>
__global__ void __launch_bounds__(kBaseThreads) baseline_kernel(BaselineArgs a, int ci) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long s_best;
  __shared__ double s_v[3];
  __shared__ double s_red[kBaseThreads / 32][10];
  __shared__ int s_redi[kBaseThreads / 32];
  const int tid = threadIdx.x;
  const int64_t o = a.offsets[ci], e = a.offsets[ci + 1];
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  if (o < 0 || e < o || e > a.n_points || (e - o) > 0x7fffffff) {
    if (tid == 0) {
      a.vx[ci] = a.vy[ci] = a.heading[ci] = nan;
      if (a.vz) a.vz[ci] = nan;
      a.inlier_count[ci] = 0;
      a.best[ci] = -1;
      a.status[ci] = RVH_STATUS_BAD_OFFSETS;
    }
    return;
  }
  const int N = (int)(e - o);
  if (N < DIM) {
    for (int j = tid; j < N; j += kBaseThreads) a.mask[o + j] = 0;
    if (tid == 0) {
      a.vx[ci] = a.vy[ci] = a.heading[ci] = nan;
      if (a.vz) a.vz[ci] = nan;
      a.inlier_count[ci] = 0;
      a.best[ci] = -1;
      a.status[ci] = RVH_STATUS_TOO_FEW_POINTS;
    }
    return;
  }
  // FP64 rows (a0, a1, a2, w) of every point
  double* rows = N <= a.nmax_smem ? reinterpret_cast<double*>(smem_raw) : a.rows64_g + 4 * o;
  for (int j = tid; j < N; j += kBaseThreads) {
    double r[3];
    row_f64<DIM>(a.trig, a.az[o + j], DIM == 3 ? a.el[o + j] : 0.0f, r);
    rows[4 * j + 0] = r[0];
    rows[4 * j + 1] = r[1];
    rows[4 * j + 2] = r[2];
    rows[4 * j + 3] = (double)a.dop[o + j];
  }
  if (tid == 0) s_best = 0ull;
  __syncthreads();
  unsigned long long mine = 0ull;
  for (int h = tid; h < a.H; h += kBaseThreads) {
    int q[3];
    draw_minimal_set<DIM>(a.key, a.cluster_base + ci, h, N, q);
    const double* r0 = rows + 4 * q[0];
    const double* r1 = rows + 4 * q[1];
    const double* r2 = rows + 4 * q[DIM == 3 ? 2 : 0];
    const double w[3] = {r0[3], r1[3], DIM == 3 ? r2[3] : 0.0};
    double v[3];
    if (!solve_f64<DIM>(r0, r1, r2, w, a.eps, v, nullptr)) continue;
    int c = 0;
    for (int j = 0; j < N; ++j)
      if (fabs(residual_f64<DIM>(rows + 4 * j, rows[4 * j + 3], v)) <= a.tau) ++c;
    const unsigned long long key =
        ((unsigned long long)(uint32_t)(c + 1) << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)h);
    if (key > mine) mine = key;
  }
  atomicMax(&s_best, mine);
  __syncthreads();
  const unsigned long long key = s_best;
  if (key == 0ull) {
    for (int j = tid; j < N; j += kBaseThreads) a.mask[o + j] = 0;
    if (tid == 0) {
      a.vx[ci] = a.vy[ci] = a.heading[ci] = nan;
      if (a.vz) a.vz[ci] = nan;
      a.inlier_count[ci] = 0;
      a.best[ci] = -1;
      a.status[ci] = RVH_STATUS_ALL_DEGENERATE;
    }
    return;
  }
  const int hstar = (int)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
  if (tid == 0) {
    int q[3];
    draw_minimal_set<DIM>(a.key, a.cluster_base + ci, hstar, N, q);
    const double* r0 = rows + 4 * q[0];
    const double* r1 = rows + 4 * q[1];
    const double* r2 = rows + 4 * q[DIM == 3 ? 2 : 0];
    const double w[3] = {r0[3], r1[3], DIM == 3 ? r2[3] : 0.0};
    double v[3] = {0.0, 0.0, 0.0};
    solve_f64<DIM>(r0, r1, r2, w, a.eps, v, nullptr);
    s_v[0] = v[0];
    s_v[1] = v[1];
    s_v[2] = v[2];
  }
  __syncthreads();
  const double v[3] = {s_v[0], s_v[1], s_v[2]};
  constexpr int NS = DIM == 2 ? 5 : 9;
  double sums[NS];
  for (int i = 0; i < NS; ++i) sums[i] = 0.0;
  int nin = 0;
  for (int j = tid; j < N; j += kBaseThreads) {
    const double* r = rows + 4 * j;
    const bool in = fabs(residual_f64<DIM>(r, r[3], v)) <= a.tau;
    a.mask[o + j] = in ? 1 : 0;
    if (!in) continue;
    ++nin;
    if (DIM == 2) {
      sums[0] = fma(r[0], r[0], sums[0]);
      sums[1] = fma(r[0], r[1], sums[1]);
      sums[2] = fma(r[1], r[1], sums[2]);
      sums[3] = fma(r[0], r[3], sums[3]);
      sums[4] = fma(r[1], r[3], sums[4]);
    } else {
      sums[0] = fma(r[0], r[0], sums[0]);
      sums[1] = fma(r[0], r[1], sums[1]);
      sums[2] = fma(r[0], r[2], sums[2]);
      sums[3] = fma(r[1], r[1], sums[3]);
      sums[4] = fma(r[1], r[2], sums[4]);
      sums[5] = fma(r[2], r[2], sums[5]);
      sums[6] = fma(r[0], r[3], sums[6]);
      sums[7] = fma(r[1], r[3], sums[7]);
      sums[8] = fma(r[2], r[3], sums[8]);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    nin += __shfl_xor_sync(0xffffffffu, nin, off);
    for (int i = 0; i < NS; ++i) sums[i] += __shfl_xor_sync(0xffffffffu, sums[i], off);
  }
  if ((tid & 31) == 0) {
    s_redi[tid >> 5] = nin;
    for (int i = 0; i < NS; ++i) s_red[tid >> 5][i] = sums[i];
  }
  __syncthreads();
  if (tid != 0) return;
  int n_in = 0;
  double t[NS];
  for (int i = 0; i < NS; ++i) t[i] = 0.0;
  for (int w = 0; w < kBaseThreads / 32; ++w) {
    n_in += s_redi[w];
    for (int i = 0; i < NS; ++i) t[i] += s_red[w][i];
  }
  double vout[3] = {v[0], v[1], v[2]};
  int st = 0;
  if (DIM == 2) {
    const double tr = t[0] + t[2];
    const double det = det2_f64(t[0], t[1], t[1], t[2]);
    if (n_in >= 2 && fabs(det) > 1e-12 * (tr * tr)) {
      const double G0[3] = {t[0], t[1], 0.0}, G1[3] = {t[1], t[2], 0.0}, g[3] = {t[3], t[4], 0.0};
      solve_f64<2>(G0, G1, nullptr, g, 0.0, vout, nullptr);
    } else {
      st |= RVH_STATUS_LSQ_FALLBACK;
    }
  } else {
    const double tr = t[0] + t[3] + t[5];
    const double G0[3] = {t[0], t[1], t[2]}, G1[3] = {t[1], t[3], t[4]}, G2[3] = {t[2], t[4], t[5]};
    const double det = det3_f64(G0, G1, G2);
    if (n_in >= 3 && fabs(det) > 1e-12 * (tr * tr * tr)) {
      const double g[3] = {t[6], t[7], t[8]};
      solve_f64<3>(G0, G1, G2, g, 0.0, vout, nullptr);
    } else {
      st |= RVH_STATUS_LSQ_FALLBACK;
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

size_t baseline_smem_bytes(int nmax_smem) { return (size_t)nmax_smem * 4 * sizeof(double); }

cudaError_t baseline_configure(int dim, size_t smem) {
  if (dim == 2)
    return cudaFuncSetAttribute(baseline_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaFuncSetAttribute(baseline_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_baseline_cluster(int dim, const BaselineArgs& a, int cluster, size_t smem, cudaStream_t s) {
  if (dim == 2) baseline_kernel<2><<<1, kBaseThreads, smem, s>>>(a, cluster);
  else baseline_kernel<3><<<1, kBaseThreads, smem, s>>>(a, cluster);
  return cudaGetLastError();
}

}  // namespace rvh
