// Standalone run of the fused kernel's scoring pass (step a4: upper-bound
// inlier counts of every trial over a cluster's FP32 rows in shared memory),
// built and run by tests/test_scoring_bench.py with the library's own flags.
//
// Every CTA stages one synthetic cluster of N points (2D or 3D rows, 20%
// outliers) as 32-point tiles, fills H trial records, and runs the library's
// phase_a_tiles<DIM, 1, 4> (the schedule the library picks for H >= 1024)
// `reps` times.  The grid is 4 CTAs of 256 threads per SM, as in the fused
// kernel.  The counts of the last pass are checked against a host
// evaluation of the same FP32 formula (fmaf chain): each count must be an
// upper bound of #{|r| <= thi} that exceeds it only by points whose |r|
// exceeds thi by at most 1e-6 (the pass counts r^2 < C with C two ulps
// above thi^2).
//
//   scoring_bench <dim 2|3> <N <= 1536> <reps>
// Output: "key=value ..." (ms, pairs, pairs_per_s, sms, ctas_per_sm, mismatches).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "rvh_scoring.cuh"

using namespace rvh;

#define CK(x)                                                           \
  do {                                                                  \
    cudaError_t e = (x);                                                \
    if (e != cudaSuccess) {                                             \
      printf("cuda error %s at %d\n", cudaGetErrorString(e), __LINE__); \
      return 2;                                                         \
    }                                                                   \
  } while (0)

constexpr int kH = 1024;
constexpr int kNmax = 1536;

template <int DIM>
__global__ void __launch_bounds__(kThreads, RVH_MIN_BLOCKS)
    scoring_kernel(const float4* __restrict__ pts, int N, const float4* __restrict__ hyp, int reps, int* __restrict__ U_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem S;
  unsigned char* p = smem_raw;
  S.rows = reinterpret_cast<float*>(p);
  p += (size_t)((N + 31) & ~31) * sizeof(float4);
  S.hyp = reinterpret_cast<float4*>(p);
  p += (size_t)kH * sizeof(float4);
  S.tlo = reinterpret_cast<float*>(p);
  p += (size_t)kH * sizeof(float);
  S.U = reinterpret_cast<int*>(p);
  p += (size_t)kH * sizeof(int);
  S.kind = reinterpret_cast<int8_t*>(p);
  const TileRowsOf<DIM> rows{S.rows};
  for (int j = threadIdx.x; j < N; j += kThreads) rows.put(j, pts[j]);
  if (threadIdx.x < ((N + 3) & ~3) - N) {
    const float nan = __int_as_float(0x7fc00000);
    rows.put(N + threadIdx.x, make_float4(0.0f, 0.0f, nan, nan));
  }
  for (int h = threadIdx.x; h < kH; h += kThreads) {
    S.hyp[h] = hyp[h];
    S.tlo[h] = 0.0f;
    S.kind[h] = (int8_t)kHypNormal;
    S.U[h] = 0;
  }
  __syncthreads();
  for (int r = 0; r < reps; ++r) {
    phase_a_tiles<DIM, 1, 4>(rows, N, S, kH);
    __syncthreads();
  }
  if (blockIdx.x == 0)
    for (int h = threadIdx.x; h < kH; h += kThreads) U_out[h] = S.U[h];
}

template <int DIM>
int run(int N, int reps) {
  std::mt19937_64 g(12345);
  std::uniform_real_distribution<double> U01(0.0, 1.0);
  const double kPi = 3.14159265358979323846;
  // one cluster: azimuth U(+-60 deg), elevation U(+-15 deg) in 3D, |v| 0..40,
  // Doppler = model + N(0, 0.05), 20% outliers U(0, 2|v|)
  const double sp = 40.0 * U01(g), hd = 2.0 * kPi * U01(g), vz = DIM == 3 ? 10.0 * U01(g) - 5.0 : 0.0;
  const double vx = sp * cos(hd), vy = sp * sin(hd);
  std::normal_distribution<double> noise(0.0, 0.05);
  std::vector<float4> pts(N);
  for (int j = 0; j < N; ++j) {
    const double t = (U01(g) * 2.0 - 1.0) * kPi / 3.0;
    const double e = DIM == 3 ? (U01(g) * 2.0 - 1.0) * kPi / 12.0 : 0.0;
    const double a0 = cos(t) * cos(e), a1 = sin(t) * cos(e), a2 = sin(e);
    double w = vx * a0 + vy * a1 + vz * a2 + noise(g);
    if (j % 5 == 4) w = U01(g) * 2.0 * sqrt(sp * sp + vz * vz);
    pts[j] = DIM == 2 ? make_float4((float)a0, (float)a1, (float)w, 0.0f)
                      : make_float4((float)a0, (float)a1, (float)a2, (float)w);
  }
  // trial records (-X, -Y, -Z, thi) scattered around the true velocity
  std::vector<float4> hyp(kH);
  for (int h = 0; h < kH; ++h) {
    const double s = (h % 3 == 0) ? 0.02 : 2.0;
    hyp[h] = make_float4((float)-(vx + s * (U01(g) - 0.5)), (float)-(vy + s * (U01(g) - 0.5)),
                         (float)-(vz + (DIM == 3 ? s * (U01(g) - 0.5) : 0.0)), 0.1f + 1e-5f);
  }
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  const int grid = sms * RVH_MIN_BLOCKS;
  float4 *d_pts = nullptr, *d_hyp = nullptr;
  int* d_U = nullptr;
  CK(cudaMalloc(&d_pts, N * sizeof(float4)));
  CK(cudaMalloc(&d_hyp, kH * sizeof(float4)));
  CK(cudaMalloc(&d_U, kH * sizeof(int)));
  CK(cudaMemcpy(d_pts, pts.data(), N * sizeof(float4), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_hyp, hyp.data(), kH * sizeof(float4), cudaMemcpyHostToDevice));
  const size_t smem = (size_t)((N + 31) & ~31) * sizeof(float4) + (size_t)kH * (sizeof(float4) + sizeof(float) + sizeof(int) + 1);
  CK(cudaFuncSetAttribute(scoring_kernel<DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int resident = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, scoring_kernel<DIM>, kThreads, smem));
  scoring_kernel<DIM><<<grid, kThreads, smem>>>(d_pts, N, d_hyp, 1, d_U);  // warm-up
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0));
  scoring_kernel<DIM><<<grid, kThreads, smem>>>(d_pts, N, d_hyp, reps, d_U);
  CK(cudaEventRecord(e1));
  CK(cudaEventSynchronize(e1));
  CK(cudaGetLastError());
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  std::vector<int> Ug(kH);
  CK(cudaMemcpy(Ug.data(), d_U, kH * sizeof(int), cudaMemcpyDeviceToHost));
  // host evaluation of the same FP32 formula
  long long mism = 0, total_in = 0;
  for (int h = 0; h < kH; ++h) {
    int c = 0, c_wide = 0;
    for (int j = 0; j < N; ++j) {
      const float4 q = pts[j], v = hyp[h];
      const float r = DIM == 2 ? std::fmaf(v.x, q.x, std::fmaf(v.y, q.y, q.z))
                               : std::fmaf(v.x, q.x, std::fmaf(v.y, q.y, std::fmaf(v.z, q.z, q.w)));
      c += (std::fabs(r) <= v.w) ? 1 : 0;
      c_wide += (std::fabs(r) <= v.w + 1e-6f) ? 1 : 0;
    }
    mism += (Ug[h] < c || Ug[h] > c_wide);
    total_in += c;
  }
  const double pairs = (double)grid * reps * (double)kH * N;
  printf("dim=%d N=%d H=%d grid=%d ctas_per_sm=%d reps=%d ms=%.4f pairs=%.6e pairs_per_s=%.6e sms=%d mismatches=%lld "
         "inliers=%lld\n",
         DIM, N, kH, grid, resident, reps, ms, pairs, pairs / (ms * 1e-3), sms, mism, total_in);
  cudaFree(d_pts);
  cudaFree(d_hyp);
  cudaFree(d_U);
  return mism == 0 ? 0 : 1;
}

int main(int argc, char** argv) {
  if (argc < 4) {
    printf("usage: scoring_bench <dim 2|3> <N <= %d> <reps>\n", kNmax);
    return 2;
  }
  const int dim = atoi(argv[1]), N = atoi(argv[2]), reps = atoi(argv[3]);
  if ((dim != 2 && dim != 3) || N < 4 || N > kNmax || reps < 1) {
    printf("bad arguments\n");
    return 2;
  }
  return dim == 2 ? run<2>(N, reps) : run<3>(N, reps);
}
