// FP64 FMA throughput of the GPU: every thread runs 8 independent chains of
// dependent fma() on doubles, 4 CTAs of 256 threads per SM.  The rate (FP64
// FMAs per second, and per SM per cycle at the device's maximum SM clock) is
// what the design weighs FP64 work by.  Built and run by
// tests/test_scoring_bench.py.
//
//   fp64_rate <iterations>
// Output: "key=value ..." (ms, dfma, dfma_per_s, dfma_per_clk_sm, sms, clock_mhz, check).
#include <cstdio>
#include <cstdlib>

#include <cuda_runtime.h>

#define CK(x)                                                           \
  do {                                                                  \
    cudaError_t e = (x);                                                \
    if (e != cudaSuccess) {                                             \
      printf("cuda error %s at %d\n", cudaGetErrorString(e), __LINE__); \
      return 2;                                                         \
    }                                                                   \
  } while (0)

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fma_chains(int iters, double a, double* out) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, 1e-9);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main(int argc, char** argv) {
  const int iters = argc > 1 ? atoi(argv[1]) : 4096;
  int sms = 0, khz = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, 0));
  const int grid = sms * 4, block = 256;
  double* d = nullptr;
  CK(cudaMalloc(&d, sizeof(double) * grid * block));
  fma_chains<<<grid, block>>>(16, 0.999999, d);  // warm-up
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    CK(cudaEventRecord(e0));
    fma_chains<<<grid, block>>>(iters, 0.999999, d);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaGetLastError());
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) best = ms;
  }
  double h0 = 0.0;
  CK(cudaMemcpy(&h0, d, sizeof(double), cudaMemcpyDeviceToHost));
  const double dfma = (double)grid * block * iters * kChains;
  const double rate = dfma / (best * 1e-3);
  printf("ms=%.4f dfma=%.6e dfma_per_s=%.6e dfma_per_clk_sm=%.4f sms=%d clock_mhz=%.0f check=%d\n", best, dfma, rate,
         rate / sms / (khz * 1e3), sms, khz / 1e3, h0 > 0.0 && h0 < 1e9 ? 1 : 0);
  cudaFree(d);
  return 0;
}
