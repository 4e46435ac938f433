// rvh_estimate_noalloc: the fused estimate for callers that must not allocate
// device memory while running (for example real-time perception stacks that
// forbid allocation after start-up, or plugins whose host framework owns all
// device memory).  It runs the same worklist and fused kernels as
// rvh_estimate, with their scratch (work list, work counter, FP32 rows of
// large clusters, FP64 rows) and the FP64 row table in file-scope device arrays of fixed
// size instead of context memory.  It calls no cudaMalloc, cudaFree or other
// allocating routine.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "rvh.h"
#include "rvh_kernels.h"
#include "rvh_outputs.h"
#include "rvh_runtime.h"

namespace {

constexpr int64_t kMaxPoints = RVH_NOALLOC_MAX_POINTS;
constexpr int32_t kMaxClusters = RVH_NOALLOC_MAX_CLUSTERS;
constexpr size_t kWorklistBytes = sizeof(int2) * (size_t)kMaxClusters;
constexpr size_t kCounterBytes = 256;
constexpr size_t kRowsBytes = sizeof(float4) * (size_t)kMaxPoints;
constexpr size_t kRows64Bytes = sizeof(double4_32a) * (size_t)kMaxPoints;
constexpr size_t kScratchBytes = kWorklistBytes + kCounterBytes + kRowsBytes + kRows64Bytes;
constexpr int kNmaxSmem = 1536;
constexpr int kHchunk = 1024;

// Shared by every call on a device; held by each device that loads the
// library until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) double2 g_trig[rvh::kTrigSize];

struct DeviceSetup {
  bool done = false;
  unsigned char* scratch = nullptr;  // device address of g_scratch on this device
  double2* trig = nullptr;           // device address of g_trig on this device
  int sms = 0;
  int occ[4] = {0, 0, 0, 0};
};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
DeviceSetup g_setup[kMaxDevices];

// Once per device, with that device current: device addresses of the arrays
// (host code only sees host-side stand-ins for them), the row table, and the
// kernels' shared-memory opt-in.
int setup_device(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceSetup& d = g_setup[dev];
  if (!d.done) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return rvh::set_error(RVH_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    d.scratch = (unsigned char*)p;
    e = cudaGetSymbolAddress(&p, g_trig);
    if (e != cudaSuccess) return rvh::set_error(RVH_ECUDA, std::string("cudaGetSymbolAddress(trig): ") + cudaGetErrorString(e));
    d.trig = (double2*)p;
    double2 tab[rvh::kTrigSize];
    for (int k = -rvh::kTrigHalf; k <= rvh::kTrigHalf; ++k)
      tab[k + rvh::kTrigHalf] = make_double2(std::cos(k / 128.0), std::sin(k / 128.0));
    e = cudaMemcpyToSymbol(g_trig, tab, sizeof(tab));
    if (e != cudaSuccess) return rvh::set_error(RVH_ECUDA, std::string("trig table upload: ") + cudaGetErrorString(e));
    e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return rvh::set_error(RVH_ECUDA, cudaGetErrorString(e));
    const size_t smem = rvh::fused_smem_bytes(kNmaxSmem, kHchunk);
    for (int dim = 2; dim <= 3; ++dim) {
      // the same opt-in as context launches use: neither lowers the other's limit
      e = rvh::fused_configure_max(dim, dev);
      if (e == cudaSuccess) e = rvh::fused_occupancy(dim, smem, &d.occ[dim]);
      if (e != cudaSuccess) return rvh::set_error(RVH_ECUDA, std::string("kernel set-up: ") + cudaGetErrorString(e));
      if (d.occ[dim] < 1) d.occ[dim] = 1;
    }
    d.done = true;
  }
  *out = &d;
  return RVH_OK;
}

}  // namespace

extern "C" int rvh_estimate_noalloc(const rvh_frame* f, const rvh_params* p, rvh_result* r, void* stream) {
  if (f && (f->n_clusters > kMaxClusters || f->n_points > kMaxPoints))
    return rvh::set_error(RVH_EINVAL, "frame exceeds the no-allocation limits (" + std::to_string(kMaxClusters) +
                                          " clusters, " + std::to_string(kMaxPoints) + " points)");
  int rc = rvh::check_args(f, p, r);  // the checks of rvh_estimate
  if (rc) return rc;
  if (f->n_clusters == 0) return RVH_OK;
  // what the launch reads or writes must be device memory: per-point arrays
  // when there are points, per-cluster arrays always
  const bool pts = f->n_points > 0;
  const void* offs = f->cluster_offsets;
  const void* need[10] = {offs, r->vx, r->vy, r->heading, r->inlier_count, r->best_hypothesis, r->status,
                          pts ? (const void*)f->azimuth : offs, pts ? (const void*)f->doppler : offs,
                          pts ? (const void*)r->inlier_mask : offs};
  for (const void* q : need)
    if (!rvh::device_ptr(q)) return rvh::set_error(RVH_EINVAL, "every input and output must be device memory");
  if (pts && p->model_dim == 3 && !rvh::device_ptr(f->elevation))
    return rvh::set_error(RVH_EINVAL, "every input and output must be device memory");
  if (r->vz && !rvh::device_ptr(r->vz)) return rvh::set_error(RVH_EINVAL, "vz must be device memory or NULL");
  if (r->threshold && !rvh::device_ptr(r->threshold))
    return rvh::set_error(RVH_EINVAL, "threshold must be device memory or NULL");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return rvh::set_error(RVH_ECUDA, "no current device");
  DeviceSetup* d = nullptr;
  rc = setup_device(dev, &d);
  if (rc) return rc;

  const int dim = p->model_dim;
  rvh::FusedArgs a;
  memset(&a, 0, sizeof(a));  // cta_rows64 = NULL: FP64 rows in the per-point array below
  rvh::FrameDesc& fd = a.f[0];
  rvh::fill_desc(d->trig, fd, *f, *p, f->azimuth, f->elevation, f->doppler, f->cluster_offsets,
                 (float4*)(d->scratch + kWorklistBytes + kCounterBytes),
                 (double4_32a*)(d->scratch + kWorklistBytes + kCounterBytes + kRowsBytes), *r);
  a.n_frames = 1;
  a.n_items = f->n_clusters;
  a.worklist = (int2*)d->scratch;
  a.work_counter = (int*)(d->scratch + kWorklistBytes);  // zeroed by the worklist kernel each call
  a.stats = nullptr;
  a.prune = 1;
  a.nmax_smem = kNmaxSmem;
  a.hchunk = kHchunk;
  // the scoring schedule follows the trials scored together (the adaptive block, or all)
  if ((fd.trial_block > 0 ? std::min(fd.trial_block, p->num_hypotheses) : p->num_hypotheses) >= 1024) {
    a.pw = 1;
    a.hpl = 4;
  } else {
    a.pw = 8;
    a.hpl = 4;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int resident = d->sms * d->occ[dim];
  a.direct = a.n_items <= resident ? 1 : 0;
  e = rvh::launch_threshold_fill(r->threshold, f->n_clusters, fd.line_model != 0, p->inlier_threshold, s);
  if (e == cudaSuccess && !a.direct) e = rvh::launch_worklist(a, s);
  if (e == cudaSuccess) {
    const int grid = std::max(1, std::min(resident, a.n_items));
    e = rvh::launch_fused(dim, a, grid, rvh::fused_smem_bytes(kNmaxSmem, kHchunk), s);
  }
  if (e != cudaSuccess) return rvh::set_error(RVH_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return RVH_OK;
}
