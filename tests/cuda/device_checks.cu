// Device-level checks of the assumptions behind the FP32 filter, built and run
// by tests/test_device_checks.py with the library's own flags (-fmad=false).
//
//   rows     every float t in [-pi, pi]: |sincosf - sincos(double)| relative
//            error (the filter assumes <= 2^-22; this reports the maximum);
//            the table-based FP64 sincos against the library sincos (absolute
//            difference in units of 2^-53).
//   filter   random and adversarial minimal sets and points: wherever the FP32
//            residual classifies a point as certainly in (|r32| <= tlo) or
//            certainly out (|r32| > thi), the FP64 residual must agree, and
//            |r32 - r64| must stay within the band half-width.
//
// Output: one line "key=value ..." per mode; violations must be 0.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "rvh_device.cuh"

using namespace rvh;

#define CK(x)                                                                 \
  do {                                                                        \
    cudaError_t e = (x);                                                      \
    if (e != cudaSuccess) {                                                   \
      printf("cuda error %s at %d\n", cudaGetErrorString(e), __LINE__);       \
      return 2;                                                               \
    }                                                                         \
  } while (0)

__device__ unsigned long long g_max_rel_bits;   // float bits of the max relative error (monotone for >= 0)
__device__ unsigned long long g_max_ulp;
__device__ unsigned long long g_count;
__device__ unsigned long long g_viol[4];

// float bit patterns of [-pi, pi] enumerated as signed magnitudes
__global__ void k_rows(const double2* trig, unsigned int n_pos) {
  const unsigned int stride = gridDim.x * blockDim.x;
  float worst = 0.0f;
  unsigned long long worst_ulp = 0, cnt = 0;
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pos; i += stride) {
    for (int sgn = 0; sgn < 2; ++sgn) {
      const float t = __uint_as_float(i | (sgn ? 0x80000000u : 0u));
      float sf, cf;
      sincosf(t, &sf, &cf);
      double sd, cd;
      sincos((double)t, &sd, &cd);
      const float es = (sd != 0.0) ? (float)(fabs((double)sf - sd) / fabs(sd)) : (float)fabs((double)sf);
      const float ec = (float)(fabs((double)cf - cd) / fabs(cd));
      worst = fmaxf(worst, fmaxf(es, ec));
      double st, ct;
      sincos_f64(trig, t, &st, &ct);
      // absolute difference in units of 2^-53 (half an ulp of 1): rows enter
      // every formula multiplied by velocities, so absolute accuracy is what counts
      const double da = fmax(fabs(st - sd), fabs(ct - cd)) * 0x1p53;
      worst_ulp = max(worst_ulp, (unsigned long long)ceil(da));
      ++cnt;
    }
  }
  atomicMax(&g_max_rel_bits, (unsigned long long)__float_as_uint(worst));
  atomicMax(&g_max_ulp, worst_ulp);
  atomicAdd(&g_count, cnt);
}

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}
__device__ __forceinline__ float urand(uint32_t& s, float lo, float hi) {
  s = hash32(s + 0x9E3779B9u);
  return lo + (hi - lo) * ((s >> 8) * (1.0f / 16777216.0f));
}

template <int DIM>
__global__ void k_filter(const double2* trig, int n_hyp, int pts_per_hyp, unsigned seed) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= n_hyp) return;
  uint32_t s = hash32(seed * 2654435761u + gid);
  // scenario mix: ordinary traffic values, near-degenerate sets, large velocities
  const int scen = gid % 4;
  const float vscale = scen == 2 ? 400.0f : 40.0f;
  const float spread = scen == 1 ? 2e-3f : 1.05f;
  const float c0 = urand(s, -1.05f, 1.05f);
  float az[3], el[3], w[3];
  for (int k = 0; k < DIM; ++k) {
    az[k] = c0 + urand(s, -spread, spread);
    el[k] = DIM == 3 ? urand(s, -0.26f, 0.26f) : 0.0f;
    w[k] = urand(s, -vscale, vscale);
  }
  float wmax = 0.0f;
  for (int k = 0; k < DIM; ++k) wmax = fmaxf(wmax, fabsf(w[k]));
  // points: ordinary, plus a wide Doppler spread
  const float pw = scen == 3 ? 2000.0f : 2.0f * vscale;
  wmax = fmaxf(wmax, pw);
  float4 r[3];
  for (int k = 0; k < DIM; ++k) r[k] = row_f32<DIM>(az[k], el[k], w[k]);
  const TauPair tau = {0.1f, 0.1f};
  double a0[3], a1[3], a2[3] = {0, 0, 0};
  row_f64<DIM>(trig, az[0], el[0], a0);
  row_f64<DIM>(trig, az[1], el[1], a1);
  if (DIM == 3) row_f64<DIM>(trig, az[2], el[2], a2);
  // the FP64 rows the library keeps per point: (a0, a1, a2, w)
  const double4_32a s64[3] = {make_double4_32a(a0[0], a0[1], a0[2], (double)w[0]),
                              make_double4_32a(a1[0], a1[1], a1[2], (double)w[1]),
                              make_double4_32a(a2[0], a2[1], a2[2], DIM == 3 ? (double)w[2] : 0.0)};
  // odd trials run without the refinement step, even ones with it when it applies
  const float refine_band = (gid & 1) == 0 ? kRefineBand : __int_as_float(0x7f800000);
  auto seed64 = [&](int i) { return s64[i]; };
  Hyp32 hy = hyp_f32<DIM>(r[0], r[1], DIM == 3 ? r[2] : r[0], seed64, refine_band, wmax, 0.0f, 0.0f, tau);
  if (hy.kind != kHypNormal) return;
  if (hy.refined) atomicAdd(&g_viol[3], 1ull);
  const double wd[3] = {w[0], w[1], DIM == 3 ? (double)w[2] : 0.0};
  double v[3];
  if (!solve_f64<DIM>(a0, a1, a2, wd, 0.0, v, nullptr)) return;
  const float b = hy.thi - 0.1f;  // band half-width (>= the bound)
  unsigned long long bad_in = 0, bad_out = 0, bad_bound = 0, n = 0;
  for (int p = 0; p < pts_per_hyp; ++p) {
    const float paz = c0 + urand(s, -1.05f, 1.05f);
    const float pel = DIM == 3 ? urand(s, -0.26f, 0.26f) : 0.0f;
    // Doppler near the hypothesis' prediction half the time (residuals near tau)
    double ap[3];
    row_f64<DIM>(trig, paz, pel, ap);
    const double pred = v[0] * ap[0] + v[1] * ap[1] + v[2] * ap[2];
    float pwv = (p & 1) ? (float)(pred + urand(s, -0.2f, 0.2f)) : urand(s, -pw, pw);
    if (!(fabsf(pwv) <= pw)) pwv = urand(s, -pw, pw);
    const float4 row = row_f32<DIM>(paz, pel, pwv);
    const float r32 = resid_f32<DIM>(row, hy.nx, hy.ny, hy.nz);
    const double r64 = residual_f64<DIM>(ap, (double)pwv, v);
    if (fabs((double)r32 - r64) > (double)b) ++bad_bound;
    // thresholds placed around this pair's FP64 residual so decisions are close
    const double offs[6] = {-2.0, -1.001, -0.999, 0.999, 1.001, 2.0};
    for (int k = 0; k < 6; ++k) {
      const double tau64 = fabs(r64) + offs[k] * (double)b;
      if (!(tau64 >= 0.0)) continue;
      const float tlo = __fsub_rd(__double2float_rd(tau64), b);
      const float thi = __fadd_ru(__double2float_ru(tau64), b);
      const bool in64 = fabs(r64) <= tau64;
      if (fabsf(r32) <= tlo && !in64) ++bad_in;
      if (fabsf(r32) > thi && in64) ++bad_out;
    }
    ++n;
  }
  atomicAdd(&g_viol[0], bad_in);
  atomicAdd(&g_viol[1], bad_out);
  atomicAdd(&g_viol[2], bad_bound);
  atomicAdd(&g_count, n);
}

int main(int argc, char** argv) {
  const char* mode = argc > 1 ? argv[1] : "rows";
  std::vector<double2> tab(kTrigSize);
  for (int k = -kTrigHalf; k <= kTrigHalf; ++k)
    tab[k + kTrigHalf] = make_double2(std::cos(k / 128.0), std::sin(k / 128.0));
  double2* trig = nullptr;
  CK(cudaMalloc(&trig, sizeof(double2) * kTrigSize));
  CK(cudaMemcpy(trig, tab.data(), sizeof(double2) * kTrigSize, cudaMemcpyHostToDevice));
  unsigned long long zero = 0, z4[4] = {0, 0, 0, 0};
  CK(cudaMemcpyToSymbol(g_count, &zero, 8));
  CK(cudaMemcpyToSymbol(g_max_rel_bits, &zero, 8));
  CK(cudaMemcpyToSymbol(g_max_ulp, &zero, 8));
  CK(cudaMemcpyToSymbol(g_viol, z4, 32));
  if (!strcmp(mode, "rows")) {
    float pi_below;
    {
      float p = (float)M_PI;
      pi_below = ((double)p > M_PI) ? std::nextafter(p, 0.0f) : p;
    }
    unsigned int n_pos;
    memcpy(&n_pos, &pi_below, 4);
    n_pos += 1;  // bit patterns 0 .. pi_below inclusive
    k_rows<<<152 * 8, 256>>>(trig, n_pos);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    unsigned long long rel_bits, ulp, cnt;
    CK(cudaMemcpyFromSymbol(&rel_bits, g_max_rel_bits, 8));
    CK(cudaMemcpyFromSymbol(&ulp, g_max_ulp, 8));
    CK(cudaMemcpyFromSymbol(&cnt, g_count, 8));
    unsigned int rb = (unsigned int)rel_bits;
    float rel;
    memcpy(&rel, &rb, 4);
    printf("mode=rows count=%llu max_rel_sincosf=%.6e max_rel_over_2^-22=%.4f table_vs_sincos_max_abs_2^-53=%llu\n",
           cnt, rel, rel / std::ldexp(1.0, -22), ulp);
  } else {
    const int n_hyp = argc > 2 ? atoi(argv[2]) : (1 << 20);
    const int pts = argc > 3 ? atoi(argv[3]) : 256;
    k_filter<2><<<(n_hyp + 255) / 256, 256>>>(trig, n_hyp, pts, 1u);
    k_filter<3><<<(n_hyp + 255) / 256, 256>>>(trig, n_hyp, pts, 2u);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    unsigned long long cnt, v[4];
    CK(cudaMemcpyFromSymbol(&cnt, g_count, 8));
    CK(cudaMemcpyFromSymbol(v, g_viol, 32));
    printf("mode=filter pairs=%llu bad_in=%llu bad_out=%llu bound_exceeded=%llu refined_trials=%llu\n", cnt, v[0],
           v[1], v[2], v[3]);
  }
  CK(cudaFree(trig));
  return 0;
}
