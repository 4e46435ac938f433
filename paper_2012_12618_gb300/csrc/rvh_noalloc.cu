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
    // opt the kernels in to (nearly) the device's per-block maximum, so this
    // never lowers a limit that context-based launches rely on
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return rvh::set_error(RVH_ECUDA, cudaGetErrorString(e));
    const size_t allow = std::max(smem, (size_t)optin > 8192 ? (size_t)optin - 8192 : smem);
    for (int dim = 2; dim <= 3; ++dim) {
      e = rvh::fused_configure(dim, allow);
      if (e == cudaSuccess) e = rvh::fused_occupancy(dim, smem, &d.occ[dim]);
      if (e != cudaSuccess) return rvh::set_error(RVH_ECUDA, std::string("kernel set-up: ") + cudaGetErrorString(e));
      if (d.occ[dim] < 1) d.occ[dim] = 1;
    }
    d.done = true;
  }
  *out = &d;
  return RVH_OK;
}

float round_up_f(double x) {
  float f = (float)x;
  return ((double)f < x) ? std::nextafter(f, INFINITY) : f;
}
float round_down_f(double x) {
  float f = (float)x;
  return ((double)f > x) ? std::nextafter(f, -INFINITY) : f;
}

}  // namespace

extern "C" int rvh_estimate_noalloc(const rvh_frame* f, const rvh_params* p, rvh_result* r, void* stream) {
  if (!f || !p || !r) return rvh::set_error(RVH_EINVAL, "frame, params and result must be non-NULL");
  if (f->n_clusters < 0 || f->n_points < 0) return rvh::set_error(RVH_EINVAL, "negative size");
  if (f->n_clusters > kMaxClusters || f->n_points > kMaxPoints)
    return rvh::set_error(RVH_EINVAL, "frame exceeds the no-allocation limits (" + std::to_string(kMaxClusters) +
                                          " clusters, " + std::to_string(kMaxPoints) + " points)");
  if (p->model_dim != 2 && p->model_dim != 3) return rvh::set_error(RVH_EINVAL, "model_dim must be 2 or 3");
  if ((p->model_dim == 3) != (f->elevation != nullptr))
    return rvh::set_error(RVH_EINVAL, "model_dim 3 needs elevation, model_dim 2 needs elevation == NULL");
  if (p->num_hypotheses < 1) return rvh::set_error(RVH_EINVAL, "num_hypotheses must be >= 1");
  if (std::isnan(p->inlier_threshold) || p->inlier_threshold < 0 || std::isnan(p->cond_eps))
    return rvh::set_error(RVH_EINVAL, "inlier_threshold must be >= 0 and cond_eps not NaN");
  if (p->first_cluster < 0 || (int64_t)p->first_cluster + f->n_clusters > 0x7fffffffLL)
    return rvh::set_error(RVH_EINVAL, "first_cluster out of range");
  if (p->refine_iterations < 0 || p->refine_iterations > RVH_MAX_REFINE_ITERATIONS)
    return rvh::set_error(RVH_EINVAL, "refine_iterations out of range [0, RVH_MAX_REFINE_ITERATIONS]");
  if (!(p->confidence >= 0.0 && p->confidence < 1.0)) return rvh::set_error(RVH_EINVAL, "confidence must be in [0, 1)");
  if (p->confidence > 0.0 && p->trial_block != 0 &&
      (p->trial_block < 32 || p->trial_block > 1024 || p->trial_block % 32 != 0))
    return rvh::set_error(RVH_EINVAL, "trial_block must be 0 or a multiple of 32 in [32, 1024]");
  if (p->hypothesis_model != RVH_MODEL_VELOCITY_PROFILE && p->hypothesis_model != RVH_MODEL_PAPER_LINE)
    return rvh::set_error(RVH_EINVAL, "hypothesis_model must be RVH_MODEL_VELOCITY_PROFILE or RVH_MODEL_PAPER_LINE");
  if (p->hypothesis_model == RVH_MODEL_PAPER_LINE && (p->model_dim != 2 || p->refine_iterations != 0))
    return rvh::set_error(RVH_EINVAL, "hypothesis_model RVH_MODEL_PAPER_LINE needs model_dim 2 and refine_iterations 0");
  if (f->n_clusters == 0) return f->n_points == 0 ? RVH_OK : rvh::set_error(RVH_EINVAL, "points without clusters");
  const void* ptrs[11] = {f->azimuth, f->doppler, f->cluster_offsets, r->vx, r->vy, r->heading, r->inlier_count,
                          r->best_hypothesis, r->status, r->inlier_mask, p->model_dim == 3 ? f->elevation : f->azimuth};
  for (const void* q : ptrs)
    if (!q || !rvh::device_ptr(q)) return rvh::set_error(RVH_EINVAL, "every input and output must be device memory");
  if (r->vz && !rvh::device_ptr(r->vz)) return rvh::set_error(RVH_EINVAL, "vz must be device memory or NULL");
  if (r->threshold && !rvh::device_ptr(r->threshold))
    return rvh::set_error(RVH_EINVAL, "threshold must be device memory or NULL");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return rvh::set_error(RVH_ECUDA, "no current device");
  DeviceSetup* d = nullptr;
  int rc = setup_device(dev, &d);
  if (rc) return rc;

  const int dim = p->model_dim;
  rvh::FusedArgs a;
  memset(&a, 0, sizeof(a));
  rvh::FrameDesc& fd = a.f[0];
  const double eps = p->cond_eps > 0 ? p->cond_eps : (dim == 2 ? 1e-4 : 1e-6);
  const double eD = (dim == 2 ? 5.98e-7 : 3.65e-6) + 0x1p-50;
  fd.az = f->azimuth;
  fd.el = f->elevation;
  fd.dop = f->doppler;
  fd.offsets = f->cluster_offsets;
  fd.n_clusters = f->n_clusters;
  fd.H = p->num_hypotheses;
  fd.n_points = f->n_points;
  fd.rows_g = (float4*)(d->scratch + kWorklistBytes + kCounterBytes);
  fd.rows64_g = (double4_32a*)(d->scratch + kWorklistBytes + kCounterBytes + kRowsBytes);
  fd.trig = d->trig;
  fd.tau = p->inlier_threshold;
  fd.eps = eps;
  fd.tau32.lo = round_down_f(p->inlier_threshold);
  fd.tau32.hi = round_up_f(p->inlier_threshold);
  fd.acc = round_up_f(eps + eD);
  fd.rej = (eps - eD > 0) ? round_down_f(eps - eD) : -1.0f;
  fd.key = make_uint2((uint32_t)(p->seed & 0xFFFFFFFFu), (uint32_t)(p->seed >> 32));
  fd.cluster_base = p->first_cluster;
  fd.lo_iters = p->refine_iterations;
  fd.confidence = p->confidence;
  fd.trial_block = p->confidence > 0.0 ? (p->trial_block ? p->trial_block : RVH_DEFAULT_TRIAL_BLOCK) : 0;
  fd.line_model = p->hypothesis_model == RVH_MODEL_PAPER_LINE ? 1 : 0;
  fd.vx = r->vx;
  fd.vy = r->vy;
  fd.vz = r->vz;
  fd.heading = r->heading;
  fd.inlier_count = r->inlier_count;
  fd.best = r->best_hypothesis;
  fd.status = r->status;
  fd.mask = r->inlier_mask;
  fd.threshold = r->threshold;
  a.n_frames = 1;
  a.n_items = f->n_clusters;
  a.worklist = (int2*)d->scratch;
  a.work_counter = (int*)(d->scratch + kWorklistBytes);  // zeroed by the worklist kernel each call
  a.stats = nullptr;
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
