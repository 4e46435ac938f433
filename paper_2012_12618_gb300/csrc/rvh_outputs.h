// The per-call outputs of rvh_result as a table, shared by the entry points
// that stage them (rvh_estimate, the serving loop, the allocation-free call):
// one slot per array, its element size, and which slot is per point.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "rvh.h"

namespace rvh {

constexpr int kOutputs = 9;
constexpr int kMaskOutput = 7;  // inlier_mask: n_points entries; the others n_clusters
constexpr size_t kOutputSize[kOutputs] = {8, 8, 8, 8, 4, 4, 4, 1, 8};

inline void result_ptrs(const rvh_result& r, void* p[kOutputs]) {
  p[0] = r.vx;
  p[1] = r.vy;
  p[2] = r.vz;
  p[3] = r.heading;
  p[4] = r.inlier_count;
  p[5] = r.best_hypothesis;
  p[6] = r.status;
  p[7] = r.inlier_mask;
  p[8] = r.threshold;
}

inline rvh_result result_from(void* const p[kOutputs]) {
  rvh_result r;
  r.vx = (double*)p[0];
  r.vy = (double*)p[1];
  r.vz = (double*)p[2];
  r.heading = (double*)p[3];
  r.inlier_count = (int32_t*)p[4];
  r.best_hypothesis = (int32_t*)p[5];
  r.status = (int32_t*)p[6];
  r.inlier_mask = (uint8_t*)p[7];
  r.threshold = (double*)p[8];
  return r;
}

// Fills a frame's optional threshold output before its launch: tau for the
// cosine model; NaN for the line model, whose kernel then writes each
// cluster's MAD threshold (clusters too small to have one keep NaN).
// Nothing is launched when the output is NULL.
cudaError_t launch_threshold_fill(double* threshold, int32_t n_clusters, bool line_model, double tau,
                                  cudaStream_t s);

}  // namespace rvh
