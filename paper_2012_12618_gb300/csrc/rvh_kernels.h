// Launch interfaces of the rvh kernels (host side of the library).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace rvh {

// Table of (cos, sin)(k/128) for the FP64 rows: k = -kTrigHalf..kTrigHalf
// covers |t| <= 3.28 rad (beyond pi).
constexpr int kTrigHalf = 420;
constexpr int kTrigSize = 2 * kTrigHalf + 1;

// tau rounded outward to FP32: lo = largest float <= tau, hi = smallest float >= tau.
struct TauPair {
  float lo, hi;
};

// One frame of a batch: inputs, per-frame estimator settings, outputs.
struct FrameDesc {
  const float* az;
  const float* el;
  const float* dop;
  const int32_t* offsets;
  int32_t n_clusters;
  int32_t H;
  int64_t n_points;
  float4* rows_g;            // [n_points] FP32 rows of clusters beyond the shared-memory row capacity
  double4_32a* rows64_g;         // [n_points] FP64 rows (a0, a1, a2, w) of every point
  const double2* trig;       // (cos, sin)(k/128), k = -420..420
  double tau;
  double eps;
  TauPair tau32;
  float acc, rej;            // FP32 conditioning thresholds (certain accept / certain reject)
  uint2 key;                 // Philox key = seed
  int32_t cluster_base;      // Philox cluster counter = cluster_base + cluster index
  int32_t lo_iters;          // local-optimisation rounds after the refine (0 = none)
  double confidence;         // adaptive trial count: p in (0, 1), 0 = all H trials
  int32_t trial_block;       // adaptive: trials per block between checks (0 = not adaptive)
  int32_t line_model;        // 1: Alg. 1 as printed (normalised line fits, MAD threshold), 2D
  double* vx;
  double* vy;
  double* vz;
  double* heading;
  int32_t* inlier_count;
  int32_t* best;
  int32_t* status;
  uint8_t* mask;
  double* threshold;         // optional per-cluster threshold output (line model: the MAD threshold)
};

constexpr int kMaxBatchFrames = 32;
constexpr int kStatsWords = 13;

// A batch of frames of one model dimension, processed by one persistent launch.
struct FusedArgs {
  FrameDesc f[kMaxBatchFrames];
  int n_frames;
  int n_items;               // sum of n_clusters over the frames
  int2* worklist;            // [n_items] (frame, cluster), written by the worklist kernel
  int* work_counter;
  unsigned long long* stats;  // [kStatsWords]: exact counts, band points, fp64 trials, refined trials,
                              // 6 stage cycles, trials run, pairs of the trials run (extensions),
                              // pairs the scoring pass evaluated
  int nmax_smem;
  int hchunk;
  int pw, hpl;
  int direct;                // 1: one item per CTA, item = blockIdx.x (no work list)
  int prune;                 // 1: staged scoring pass with exact pruning of trials that cannot win
  // [grid * cta_slot_stride(dim, nmax_smem)] FP64 rows, one slot per CTA,
  // used for clusters whose rows fit shared memory (a working set that
  // stays in L2); NULL: every cluster uses its frame's per-point rows64_g
  double4_32a* cta_rows64;
};

// Points of a cluster whose FP32 rows fit the shared-memory row area of a
// fused launch, roundup32(nmax_smem) rows of 16 bytes: 3D rows (a0, a1, a2,
// w) take 16 bytes, 2D rows (c, s, w) 12, so 2D fits four thirds as many.
// The CTAs' FP64 row slots hold the 2D capacity, the larger one.
__host__ __device__ inline int smem_row_capacity(int dim, int nmax_smem) {
  return dim == 2 ? ((((nmax_smem + 31) & ~31) * 4 / 3) & ~31) : nmax_smem;
}
// Entries between consecutive CTAs' FP64 row slots for the model dimension
// dim: its shared-memory capacity, padded in 2D, whose capacity is a power of
// two (2048 entries, 64 KB) -- slots at power-of-two strides fall on the
// same L2 sets and were written back; the API allocates the larger stride.
__host__ __device__ inline int cta_slot_stride(int dim, int nmax_smem) {
  return dim == 2 ? smem_row_capacity(2, nmax_smem) + 64 : nmax_smem;
}

size_t fused_smem_bytes(int nmax_smem, int hchunk);
// Opts both instantiations of the fused kernel of this model dimension in to
// the largest dynamic shared memory a block can have on `device` (the
// opt-in maximum less the kernel's static shared memory).  Every caller
// uses this one setting, so no caller lowers a limit another relies on.
cudaError_t fused_configure_max(int dim, int device);
cudaError_t fused_occupancy(int dim, size_t smem, int* blocks_per_sm);
cudaError_t launch_worklist(const FusedArgs& a, cudaStream_t s);
cudaError_t launch_fused(int dim, const FusedArgs& a, int grid, size_t smem, cudaStream_t s);
// The instantiation a batch needs: with the extensions (local optimisation,
// adaptive trial count, line model) when any frame uses one.
bool fused_ext(const FusedArgs& a);
// Kernel entry points and launch shapes, for graph nodes built by the host
// (rvh_graph.cu): the fused kernel takes kThreads threads per CTA, the
// work-list kernel one CTA of kWorklistThreads.
const void* fused_kernel_fn(int dim, bool ext);
const void* worklist_kernel_fn();
int fused_threads();
constexpr int kWorklistThreads = 1024;

struct BaselineArgs {
  const float* az;
  const float* el;
  const float* dop;
  const int32_t* offsets;
  int64_t n_points;
  double* rows64_g;          // [n_points * 4] FP64 rows of clusters larger than nmax_smem
  const double2* trig;
  int32_t cluster_base;
  int H;
  double tau;
  double eps;
  uint2 key;
  double* vx;
  double* vy;
  double* vz;
  double* heading;
  int32_t* inlier_count;
  int32_t* best;
  int32_t* status;
  uint8_t* mask;
  int nmax_smem;
};

size_t baseline_smem_bytes(int nmax_smem);
cudaError_t baseline_configure(int dim, size_t smem);
cudaError_t launch_baseline_cluster(int dim, const BaselineArgs& a, int cluster, size_t smem, cudaStream_t s);

}  // namespace rvh
