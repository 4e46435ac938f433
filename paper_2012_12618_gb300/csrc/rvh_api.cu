// C ABI of the rvh library (include/rvh.h): contexts, validation, the
// estimate and baseline launch paths, statistics, and the serving loop.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "rvh.h"
#include "rvh_kernels.h"
#include "rvh_cluster.h"
#include "rvh_outputs.h"
#include "rvh_runtime.h"

namespace rvh {

__global__ void k_fill_f64(double* p, int32_t n, double v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

cudaError_t launch_threshold_fill(double* threshold, int32_t n_clusters, bool line_model, double tau,
                                  cudaStream_t s) {
  if (!threshold || n_clusters <= 0) return cudaSuccess;
  const double v = line_model ? __builtin_nan("") : tau;
  k_fill_f64<<<(unsigned)((n_clusters + 255) / 256), 256, 0, s>>>(threshold, n_clusters, v);
  return cudaGetLastError();
}

}  // namespace rvh

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define RVH_CUDA(x)                                                                           \
  do {                                                                                        \
    cudaError_t e_ = (x);                                                                     \
    if (e_ != cudaSuccess) return fail(RVH_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Where a buffer lives, for the kernels: device memory (used as is), page-
// locked host memory the GPU maps (outputs there are written in place
// through its device address, over the CPU-GPU link), or pageable host
// memory (staged through the context's scratch).
enum class Mem { kNone, kDevice, kPinned, kPageable };

Mem mem_kind(const void* p, void** dev) {
  *dev = nullptr;
  if (!p) return Mem::kNone;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return Mem::kPageable;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    *dev = const_cast<void*>(p);
    return Mem::kDevice;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    *dev = at.devicePointer;
    return Mem::kPinned;
  }
  return Mem::kPageable;
}

// Host-side argument checks shared by every entry point.
int check_args_impl(const rvh_frame* f, const rvh_params* p, const rvh_result* r) {
  if (!f || !p || !r) return fail(RVH_EINVAL, "frame, params and result must be non-NULL");
  if (f->n_clusters < 0) return fail(RVH_EINVAL, "n_clusters < 0");
  if (f->n_points < 0 || f->n_points > 0x7fffffffLL) return fail(RVH_EINVAL, "n_points out of range [0, 2^31)");
  if (p->model_dim != 2 && p->model_dim != 3) return fail(RVH_EINVAL, "model_dim must be 2 or 3");
  if ((p->model_dim == 3) != (f->elevation != nullptr))
    return fail(RVH_EINVAL, "model_dim 3 needs elevation, model_dim 2 needs elevation == NULL");
  if (p->num_hypotheses < 1) return fail(RVH_EINVAL, "num_hypotheses must be >= 1");
  if (std::isnan(p->inlier_threshold) || p->inlier_threshold < 0)
    return fail(RVH_EINVAL, "inlier_threshold must be >= 0");
  if (std::isnan(p->cond_eps)) return fail(RVH_EINVAL, "cond_eps is NaN");
  if (p->first_cluster < 0 || (int64_t)p->first_cluster + f->n_clusters > 0x7fffffffLL)
    return fail(RVH_EINVAL, "first_cluster out of range");
  if (p->refine_iterations < 0 || p->refine_iterations > RVH_MAX_REFINE_ITERATIONS)
    return fail(RVH_EINVAL, "refine_iterations out of range [0, RVH_MAX_REFINE_ITERATIONS]");
  if (!(p->confidence >= 0.0 && p->confidence < 1.0)) return fail(RVH_EINVAL, "confidence must be in [0, 1)");
  if (p->confidence > 0.0 && p->trial_block != 0 &&
      (p->trial_block < 32 || p->trial_block > 1024 || p->trial_block % 32 != 0))
    return fail(RVH_EINVAL, "trial_block must be 0 or a multiple of 32 in [32, 1024]");
  if (p->hypothesis_model != RVH_MODEL_VELOCITY_PROFILE && p->hypothesis_model != RVH_MODEL_PAPER_LINE)
    return fail(RVH_EINVAL, "hypothesis_model must be RVH_MODEL_VELOCITY_PROFILE or RVH_MODEL_PAPER_LINE");
  if (p->hypothesis_model == RVH_MODEL_PAPER_LINE && (p->model_dim != 2 || p->refine_iterations != 0))
    return fail(RVH_EINVAL, "hypothesis_model RVH_MODEL_PAPER_LINE needs model_dim 2 and refine_iterations 0");
  if (f->n_points > 0 && (!f->azimuth || !f->doppler)) return fail(RVH_EINVAL, "azimuth/doppler NULL");
  if (f->n_clusters > 0 && !f->cluster_offsets) return fail(RVH_EINVAL, "cluster_offsets NULL");
  if (f->n_clusters > 0 && (!r->vx || !r->vy || !r->heading || !r->inlier_count || !r->best_hypothesis || !r->status))
    return fail(RVH_EINVAL, "result arrays NULL");
  if (f->n_points > 0 && !r->inlier_mask) return fail(RVH_EINVAL, "inlier_mask NULL");
  if (f->n_clusters == 0 && f->n_points != 0) return fail(RVH_EINVAL, "points without clusters");
  return RVH_OK;
}

int check_host_offsets(const int32_t* off, int32_t n, int64_t n_points) {
  if (off[0] != 0) return fail(RVH_EINVAL, "cluster_offsets[0] != 0");
  for (int32_t i = 0; i < n; ++i)
    if (off[i + 1] < off[i]) return fail(RVH_EINVAL, "cluster_offsets not non-decreasing at " + std::to_string(i));
  if ((int64_t)off[n] != n_points) return fail(RVH_EINVAL, "cluster_offsets[n_clusters] != n_points");
  return RVH_OK;
}

double default_eps(int dim) { return dim == 2 ? 1e-4 : 1e-6; }

// Trials the fused kernel scores together in one chunk: the adaptive block,
// or all of them (the scoring schedule is chosen and tuned for this size).
int trials_per_chunk(const rvh_params& p) {
  if (p.confidence > 0.0) return std::min(p.num_hypotheses, p.trial_block ? p.trial_block : RVH_DEFAULT_TRIAL_BLOCK);
  return p.num_hypotheses;
}

rvh::TauPair tau_pair(double tau) {
  float f = (float)tau;
  rvh::TauPair t;
  t.lo = ((double)f > tau) ? std::nextafter(f, -INFINITY) : f;
  t.hi = ((double)f < tau) ? std::nextafter(f, INFINITY) : f;
  return t;
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

// ---------------------------------------------------------------------------------------
struct ServeReq;

struct rvh_ctx {
  int device = 0;
  size_t budget = 0;
  size_t used = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  // scratch of rvh_estimate / rvh_estimate_baseline
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  void* cl_scratch = nullptr;  // scratch of rvh_cluster
  size_t cl_scratch_bytes = 0;
  cudaEvent_t last_done = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  unsigned long long* stats_d = nullptr;
  bool have_launch = false;
  rvh_stats last{};
  int pw_fixed = 0, hpl_fixed = 0;
  int nmax_smem = 1536;
  int hchunk = 1024;
  int occ[4] = {0, 0, 0, 0};
  std::mutex mu;  // serialises rvh_estimate calls on this context
  rvh::Server* server = nullptr;
  double2* trig = nullptr;  // device table of (cos, sin)(k/128)
  std::map<int, std::pair<int, int>> tuned;  // (dim << 8 | log2 H) -> (pw, hpl)
  // CUDA graphs of the fused launch, one per kernel instantiation (model
  // dimension x extensions), replayed with each call's arguments
  bool graphs = true;
  rvh::LaunchGraph graph[2][2];
  bool cta_rows = true;  // per-CTA FP64 row slots for clusters that fit shared memory
  bool prune = true;     // staged scoring pass with exact pruning (rvh_set_pruning)
  std::string tune_prefix;                    // "<gpu name>|<sms>|"
  bool last_counts_trials = false;  // the last launch counted its trials on the device (extensions)
};

namespace rvh {

int ctx_alloc(rvh_ctx* ctx, void** p, size_t bytes) {
  if (ctx->used + bytes > ctx->budget)
    return fail(RVH_ENOMEM, "memory budget exceeded (" + std::to_string(ctx->used + bytes) + " > " +
                                std::to_string(ctx->budget) + " bytes)");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(RVH_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  ctx->used += bytes;
  return RVH_OK;
}

void ctx_free(rvh_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  ctx->used -= bytes;
}

int ctx_device(rvh_ctx* ctx) { return ctx->device; }
bool ctx_graphs(rvh_ctx* ctx) { return ctx->graphs; }
const double2* ctx_trig(rvh_ctx* ctx) { return ctx->trig; }
int ctx_sms(rvh_ctx* ctx) { return ctx->sms; }

int tune_key(int dim, int H) {
  int b = 0;
  while ((H >> (b + 1)) > 0) ++b;
  return dim << 8 | b;
}

void choose_schedule(rvh_ctx* ctx, int dim, int H, int* pw, int* hpl) {
  if (ctx->pw_fixed) {
    *pw = ctx->pw_fixed;
    *hpl = ctx->hpl_fixed ? ctx->hpl_fixed : 4;
    return;
  }
  auto it = ctx->tuned.find(tune_key(dim, H));
  if (it != ctx->tuned.end()) {
    *pw = it->second.first;
    *hpl = it->second.second;
    return;
  }
  if (H >= 1024) {
    *pw = 1;
    *hpl = 4;
  } else {
    *pw = 8;
    *hpl = 4;
  }
}

// Fills the per-frame descriptor; the pointers must already be device pointers.
void fill_desc(const double2* trig, FrameDesc& d, const rvh_frame& f, const rvh_params& p, const float* az,
               const float* el, const float* dop, const int32_t* off, float4* rows_g, double4_32a* rows64_g,
               const rvh_result& out) {
  d.trig = trig;
  d.rows64_g = rows64_g;
  const int dim = p.model_dim;
  const double eps = p.cond_eps > 0 ? p.cond_eps : default_eps(dim);
  const double eD = (dim == 2 ? 5.98e-7 : 3.65e-6) + 0x1p-50;
  d.az = az;
  d.el = el;
  d.dop = dop;
  d.offsets = off;
  d.n_clusters = f.n_clusters;
  d.H = p.num_hypotheses;
  d.n_points = f.n_points;
  d.rows_g = rows_g;
  d.tau = p.inlier_threshold;
  d.eps = eps;
  d.tau32 = tau_pair(p.inlier_threshold);
  d.acc = round_up_f(eps + eD);
  d.rej = (eps - eD > 0) ? round_down_f(eps - eD) : -1.0f;
  d.key = make_uint2((uint32_t)(p.seed & 0xFFFFFFFFu), (uint32_t)(p.seed >> 32));
  d.cluster_base = p.first_cluster;
  d.lo_iters = p.refine_iterations;
  d.confidence = p.confidence;
  d.trial_block = p.confidence > 0.0 ? (p.trial_block ? p.trial_block : RVH_DEFAULT_TRIAL_BLOCK) : 0;
  d.line_model = p.hypothesis_model == RVH_MODEL_PAPER_LINE ? 1 : 0;
  d.vx = out.vx;
  d.vy = out.vy;
  d.vz = out.vz;
  d.heading = out.heading;
  d.inlier_count = out.inlier_count;
  d.best = out.best_hypothesis;
  d.status = out.status;
  d.mask = out.inlier_mask;
  d.threshold = out.threshold;
}

int configure_dim(rvh_ctx* ctx, int dim) {
  const size_t smem = fused_smem_bytes(ctx->nmax_smem, ctx->hchunk);
  if (ctx->occ[dim] == 0) {
    RVH_CUDA(fused_configure_max(dim, ctx->device));
    int b = 0;
    RVH_CUDA(fused_occupancy(dim, smem, &b));
    ctx->occ[dim] = std::max(1, b);
  }
  return RVH_OK;
}

// Grid, shared memory and item mapping of a batch launch.
int prepare_launch(rvh_ctx* ctx, FusedArgs& a, int dim, int* grid, size_t* smem) {
  int rc = configure_dim(ctx, dim);
  if (rc) return rc;
  *smem = fused_smem_bytes(ctx->nmax_smem, ctx->hchunk);
  a.nmax_smem = ctx->nmax_smem;
  a.hchunk = ctx->hchunk;
  const int resident = ctx->sms * ctx->occ[dim];
  *grid = std::max(1, std::min(resident, a.n_items));
  // when every item gets its own resident CTA the order cannot matter: skip
  // the work-list kernel
  a.direct = a.n_items <= resident ? 1 : 0;
  a.prune = ctx->prune ? 1 : 0;
  return RVH_OK;
}

// Launches worklist + fused kernel for a prepared batch.
int launch_batch(rvh_ctx* ctx, FusedArgs& a, int dim, cudaStream_t s, cudaEvent_t t0, cudaEvent_t t1) {
  int grid = 1;
  size_t smem = 0;
  int rc = prepare_launch(ctx, a, dim, &grid, &smem);
  if (rc) return rc;
  if (!a.direct) RVH_CUDA(launch_worklist(a, s));
  if (t0) RVH_CUDA(cudaEventRecord(t0, s));
  RVH_CUDA(launch_fused(dim, a, grid, smem, s));
  if (t1) RVH_CUDA(cudaEventRecord(t1, s));
  ctx->last.grid = grid;
  ctx->last.kernel_launches = a.direct ? 1 : 2;
  return RVH_OK;
}

// Launches the fused kernel through the context's CUDA graph of its kernel
// instantiation, the call's arguments written into the graph's kernel node
// (rvh_graph.cu).  The stats reset, the work-list kernel and the timing
// events stay outside the graph, so the events time the fused kernel.
int launch_graph(rvh_ctx* ctx, FusedArgs& a, int dim, cudaStream_t s) {
  int grid = 1;
  size_t smem = 0;
  int rc = prepare_launch(ctx, a, dim, &grid, &smem);
  if (rc) return rc;
  // the work-list kernel zeroes the stats; a direct launch has none before it
  if (a.direct) RVH_CUDA(cudaMemsetAsync(a.stats, 0, sizeof(unsigned long long) * kStatsWords, s));
  else RVH_CUDA(launch_worklist(a, s));
  RVH_CUDA(cudaEventRecord(ctx->ev0, s));
  const cudaError_t e = ctx->graph[dim == 3][fused_ext(a) ? 1 : 0].launch(a, dim, grid, smem, false, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(RVH_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  }
  RVH_CUDA(cudaEventRecord(ctx->ev1, s));
  ctx->last.grid = grid;
  ctx->last.kernel_launches = a.direct ? 1 : 2;
  return RVH_OK;
}

// Tune cache: one line per choice, "<gpu>|<sms>|<dim>|<log2 H> <pw> <hpl> <ms>".
void load_tune_cache(rvh_ctx* ctx) {
  const char* path = getenv("RVH_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[512];
  while (fgets(line, sizeof(line), f)) {
    std::string l(line);
    if (l.compare(0, ctx->tune_prefix.size(), ctx->tune_prefix) != 0) continue;
    int dim = 0, b = 0, pw = 0, hpl = 0;
    float ms = 0.f;
    if (sscanf(l.c_str() + ctx->tune_prefix.size(), "%d|%d %d %d %f", &dim, &b, &pw, &hpl, &ms) == 5 &&
        (pw == 1 || pw == 8 || pw == 32) && (hpl == 4 || hpl == 8))
      ctx->tuned[dim << 8 | b] = std::make_pair(pw, hpl);
  }
  fclose(f);
}

void save_tune_cache(rvh_ctx* ctx, int key, int pw, int hpl, float ms) {
  const char* path = getenv("RVH_TUNE_CACHE");
  if (!path || !*path) return;
  std::vector<std::string> keep;
  const std::string mine = ctx->tune_prefix + std::to_string(key >> 8) + "|" + std::to_string(key & 255) + " ";
  if (FILE* f = fopen(path, "r")) {
    char line[512];
    while (fgets(line, sizeof(line), f)) {
      std::string l(line);
      if (l.compare(0, mine.size(), mine) != 0) keep.push_back(l);
    }
    fclose(f);
  }
  if (FILE* f = fopen(path, "w")) {
    for (auto& l : keep) fputs(l.c_str(), f);
    fprintf(f, "%s%d %d %.6f\n", mine.c_str(), pw, hpl, ms);
    fclose(f);
  }
}

}  // namespace rvh

using namespace rvh;

extern "C" {

int rvh_create(rvh_ctx** out, int device, size_t mem_budget_bytes) {
  if (!out) return fail(RVH_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    return fail(RVH_ECUDA, std::string("no CUDA device: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "count 0"));
  }
  if (device < 0 || device >= n) return fail(RVH_EINVAL, "device index out of range");
  RVH_CUDA(cudaSetDevice(device));
  rvh_ctx* c = new rvh_ctx();
  c->device = device;
  c->budget = mem_budget_bytes ? mem_budget_bytes : ((size_t)4 << 30);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  // tuning knobs for experiments: shared-memory row capacity and trial chunk
  if (const char* e = getenv("RVH_NMAX_SMEM")) c->nmax_smem = std::max(64, atoi(e));
  if (const char* e = getenv("RVH_HCHUNK")) c->hchunk = std::max(64, atoi(e));
  if (const char* e = getenv("RVH_GRAPHS")) c->graphs = atoi(e) != 0;
  if (const char* e = getenv("RVH_CTA_ROWS")) c->cta_rows = atoi(e) != 0;
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->last_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return fail(RVH_ECUDA, "stream/event creation failed");
  }
  {
    // (cos, sin)(k/128), k = -420..420, from the host's libm
    std::vector<double2> tab(kTrigSize);
    for (int k = -kTrigHalf; k <= kTrigHalf; ++k) {
      const double t = k / 128.0;
      tab[k + kTrigHalf] = make_double2(std::cos(t), std::sin(t));
    }
    void* p = nullptr;
    int rc = ctx_alloc(c, &p, sizeof(double2) * kTrigSize);
    if (rc == RVH_OK && cudaMemcpy(p, tab.data(), sizeof(double2) * kTrigSize, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = fail(RVH_ECUDA, "trig table upload failed");
    if (rc != RVH_OK) {
      cudaGetLastError();
      rvh_destroy(c);
      return rc;
    }
    c->trig = (double2*)p;
  }
  {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess)
      c->tune_prefix = std::string(prop.name) + "|" + std::to_string(c->sms) + "|";
    else
      cudaGetLastError();
    load_tune_cache(c);
  }
  *out = c;
  return RVH_OK;
}

void rvh_destroy(rvh_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->server) server_destroy(ctx->server);
  cudaStreamSynchronize(ctx->stream);
  for (auto& row : ctx->graph)
    for (auto& g : row) g.reset();
  if (ctx->scratch) ctx_free(ctx, ctx->scratch, ctx->scratch_bytes);
  if (ctx->cl_scratch) ctx_free(ctx, ctx->cl_scratch, ctx->cl_scratch_bytes);
  if (ctx->trig) ctx_free(ctx, ctx->trig, sizeof(double2) * kTrigSize);
  cudaEventDestroy(ctx->last_done);
  cudaEventDestroy(ctx->ev0);
  cudaEventDestroy(ctx->ev1);
  cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* rvh_last_error(rvh_ctx*) { return g_err.c_str(); }

int rvh_cluster(rvh_ctx* ctx, const float* features, int64_t n_points, int32_t dim, double eps, int32_t min_pts,
                int32_t* labels, int32_t* perm, int32_t* offsets, int32_t max_clusters, int32_t* n_clusters,
                void* stream) {
  if (!ctx) return fail(RVH_EINVAL, "ctx is NULL");
  if (!n_clusters) return fail(RVH_EINVAL, "n_clusters is NULL");
  if (dim < 1 || dim > 4) return fail(RVH_EINVAL, "dim must be 1..4");
  if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(RVH_EINVAL, "eps must be finite and >= 0");
  if (min_pts < 1) return fail(RVH_EINVAL, "min_pts must be >= 1");
  if (n_points < 0 || n_points > cluster_max_points())
    return fail(RVH_EINVAL, "n_points out of range [0, " + std::to_string(cluster_max_points()) + "]");
  if (max_clusters < 0) return fail(RVH_EINVAL, "max_clusters < 0");
  *n_clusters = 0;
  if (n_points == 0) return RVH_OK;
  if (!is_device_ptr(features) || !is_device_ptr(labels) || !is_device_ptr(perm) || !is_device_ptr(offsets))
    return fail(RVH_EINVAL, "features, labels, perm and offsets must be device memory");
  std::lock_guard<std::mutex> lk(ctx->mu);
  RVH_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
  RVH_CUDA(cudaStreamWaitEvent(s, ctx->last_done, 0));
  const size_t need = cluster_scratch_bytes(n_points);
  if (need > ctx->cl_scratch_bytes) {
    RVH_CUDA(cudaEventSynchronize(ctx->last_done));
    if (ctx->cl_scratch) ctx_free(ctx, ctx->cl_scratch, ctx->cl_scratch_bytes);
    ctx->cl_scratch = nullptr;
    ctx->cl_scratch_bytes = 0;
    int rc = ctx_alloc(ctx, &ctx->cl_scratch, need);
    if (rc) return rc;
    ctx->cl_scratch_bytes = need;
  }
  int nc = 0, err = 0;
  RVH_CUDA(launch_cluster(features, n_points, dim, eps, min_pts, ctx->cl_scratch, labels, perm, offsets,
                          max_clusters, &nc, &err, s));
  RVH_CUDA(cudaEventRecord(ctx->last_done, s));
  *n_clusters = nc;
  if (err) return fail(RVH_ECUDA, "rvh_cluster: a union did not settle within its retry limit");
  if (nc > max_clusters)
    return fail(RVH_EINVAL, "rvh_cluster: " + std::to_string(nc) + " clusters exceed max_clusters " +
                                std::to_string(max_clusters) + " (labels written, perm and offsets not)");
  return RVH_OK;
}

int rvh_gather(rvh_ctx* ctx, const int32_t* perm, int64_t m, const float* src0, float* dst0, const float* src1,
               float* dst1, const float* src2, float* dst2, void* stream) {
  if (!ctx) return fail(RVH_EINVAL, "ctx is NULL");
  if (m < 0 || m > 0x7fffffffLL) return fail(RVH_EINVAL, "m out of range");
  if (m == 0) return RVH_OK;
  if (!is_device_ptr(perm)) return fail(RVH_EINVAL, "perm must be device memory");
  const float* srcs[3] = {src0, src1, src2};
  float* dsts[3] = {dst0, dst1, dst2};
  for (int k = 0; k < 3; ++k)
    if (srcs[k] && (!is_device_ptr(srcs[k]) || !dsts[k] || !is_device_ptr(dsts[k])))
      return fail(RVH_EINVAL, "each gathered array and its destination must be device memory");
  RVH_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
  RVH_CUDA(launch_gather(perm, m, src0, dst0, src1, dst1, src2, dst2, s));
  return RVH_OK;
}

int rvh_set_schedule(rvh_ctx* ctx, int32_t pw, int32_t hpl) {
  if (!ctx) return fail(RVH_EINVAL, "ctx is NULL");
  if (pw != 0 && pw != 1 && pw != 8 && pw != 32) return fail(RVH_EINVAL, "points_per_warp must be 0, 1, 8 or 32");
  if (hpl != 0 && hpl != 4 && hpl != 8) return fail(RVH_EINVAL, "hyps_per_lane must be 0, 4 or 8");
  ctx->pw_fixed = pw;
  ctx->hpl_fixed = hpl;
  return RVH_OK;
}

int rvh_set_pruning(rvh_ctx* ctx, int32_t enabled) {
  if (!ctx) return fail(RVH_EINVAL, "ctx is NULL");
  if (enabled != 0 && enabled != 1) return fail(RVH_EINVAL, "enabled must be 0 or 1");
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->prune = enabled != 0;
  return RVH_OK;
}

int rvh_get_stats(rvh_ctx* ctx, rvh_stats* out) {
  if (!ctx || !out) return fail(RVH_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  RVH_CUDA(cudaSetDevice(ctx->device));
  if (ctx->have_launch) {
    RVH_CUDA(cudaEventSynchronize(ctx->last_done));
    unsigned long long h[kStatsWords] = {};
    RVH_CUDA(cudaMemcpy(h, ctx->stats_d, sizeof(h), cudaMemcpyDeviceToHost));
    if (ctx->last_counts_trials) {  // the kernel counted the trials it ran
      ctx->last.hypotheses = (int64_t)h[10];
      ctx->last.pair_evals = (int64_t)h[11];
    }
    for (int k = 0; k < 6; ++k) ctx->last.phase_cycles[k] = (int64_t)h[4 + k];
    ctx->last.refined_hypotheses = (int64_t)h[3];
    ctx->last.candidates = (int64_t)h[0];
    ctx->last.band_points = (int64_t)h[1];
    ctx->last.fp64_hypotheses = (int64_t)h[2];
    ctx->last.pairs_scored = (int64_t)h[12];
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1) == cudaSuccess) ctx->last.kernel_ms = ms;
    else cudaGetLastError();
  }
  ctx->last.graph_replays = ctx->last.graph_builds = 0;
  for (auto& row : ctx->graph)
    for (auto& g : row) {
      ctx->last.graph_replays += g.replays;
      ctx->last.graph_builds += g.builds;
    }
  if (ctx->server) server_counts(ctx->server, &ctx->last.serving_steps, &ctx->last.serving_graph_replays);
  *out = ctx->last;
  return RVH_OK;
}

// Shared front half of rvh_estimate / rvh_estimate_baseline: validation, pointer
// kinds, scratch layout, host->device staging.  fused = false selects the
// baseline's scratch (FP64 rows).
struct Staged {
  const float *az, *el, *dop;
  const int32_t* off;
  rvh_result dev_out;       // device pointers the kernel writes
  bool host_out[rvh::kOutputs];  // staged through scratch (pageable host memory)
  bool sync_out;                 // some output is host memory: the call returns once it is written
  char* base;
  int2* worklist;
  int* counter;
  unsigned long long* stats;
  void* rows;               // float4[n_points] (fused) or double[4 n_points] (baseline)
  double4_32a* rows64;      // double4_32a[n_points] (fused)
  double4_32a* cta_rows64;  // double4_32a[resident CTAs * max over dims of cta_slot_stride] (fused)
};

static int stage(rvh_ctx* ctx, const rvh_frame* f, const rvh_params* p, rvh_result* r, cudaStream_t s,
                 bool fused, Staged& st) {
  const int64_t np = f->n_points;
  const int32_t nc = f->n_clusters;
  const bool dim3 = p->model_dim == 3;
  // inputs in device memory are read where they are; host inputs (pinned or
  // not) are copied in with one bulk copy each: reading them across the
  // CPU-GPU link from the kernels puts the link's latency on every
  // cluster's load and measured slower than the copy
  void* v_az = nullptr;
  void* v_dop = nullptr;
  void* v_el = nullptr;
  void* v_off = nullptr;
  const Mem k_az = mem_kind(f->azimuth, &v_az), k_dop = mem_kind(f->doppler, &v_dop);
  const Mem k_el = dim3 ? mem_kind(f->elevation, &v_el) : Mem::kNone;
  const Mem k_off = mem_kind(f->cluster_offsets, &v_off);
  const bool d_az = k_az == Mem::kDevice;
  const bool d_dop = k_dop == Mem::kDevice;
  const bool d_el = !dim3 || k_el == Mem::kDevice;
  const bool d_off = k_off == Mem::kDevice;
  if (k_off != Mem::kDevice) {  // host offsets are checked here
    int rc = check_host_offsets(f->cluster_offsets, nc, np);
    if (rc) return rc;
  }
  void* outs[rvh::kOutputs];
  void* v_out[rvh::kOutputs];
  rvh::result_ptrs(*r, outs);
  st.sync_out = false;
  for (int i = 0; i < rvh::kOutputs; ++i) {
    const Mem k = mem_kind(outs[i], &v_out[i]);
    st.host_out[i] = k == Mem::kPageable;                     // staged, copied back
    st.sync_out = st.sync_out || k == Mem::kPinned || k == Mem::kPageable;  // host results complete on return
  }
  // layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align_up(bytes);
    return o;
  };
  const size_t o_work = take(sizeof(int2) * (size_t)std::max(nc, 1));
  const size_t o_ctr = take(64);
  const size_t o_stats = take(128);
  const size_t o_rows = take((fused ? sizeof(float4) : 4 * sizeof(double)) * (size_t)std::max<int64_t>(np, 1));
  const size_t o_rows64 = fused ? take(sizeof(double4_32a) * (size_t)std::max<int64_t>(np, 1)) : 0;
  size_t o_cta64 = 0;
  if (fused) {
    const int rc = configure_dim(ctx, p->model_dim);
    if (rc) return rc;
    o_cta64 = take(sizeof(double4_32a) *
                   (size_t)std::max(rvh::cta_slot_stride(2, ctx->nmax_smem), rvh::cta_slot_stride(3, ctx->nmax_smem)) *
                   (size_t)(ctx->sms * ctx->occ[p->model_dim]));
  }
  const size_t o_az = d_az ? 0 : take(4 * (size_t)np);
  const size_t o_el = d_el ? 0 : take(4 * (size_t)np);
  const size_t o_dop = d_dop ? 0 : take(4 * (size_t)np);
  const size_t o_off = d_off ? 0 : take(4 * (size_t)(nc + 1));
  size_t o_out[rvh::kOutputs];
  for (int i = 0; i < rvh::kOutputs; ++i) {
    const size_t n = (i == rvh::kMaskOutput) ? (size_t)np : (size_t)nc;
    o_out[i] = st.host_out[i] ? take(rvh::kOutputSize[i] * std::max<size_t>(n, 1)) : 0;
  }
  if (off > ctx->scratch_bytes) {
    // wait for earlier work that may still use the old scratch
    RVH_CUDA(cudaEventSynchronize(ctx->last_done));
    if (ctx->scratch) ctx_free(ctx, ctx->scratch, ctx->scratch_bytes);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    const size_t want = off + off / 4;
    int rc = ctx_alloc(ctx, &ctx->scratch, want);
    if (rc) return rc;
    ctx->scratch_bytes = want;
  }
  char* b = (char*)ctx->scratch;
  st.base = b;
  st.worklist = (int2*)(b + o_work);
  st.counter = (int*)(b + o_ctr);
  st.stats = (unsigned long long*)(b + o_stats);
  st.rows = b + o_rows;
  st.rows64 = fused ? (double4_32a*)(b + o_rows64) : nullptr;
  st.cta_rows64 = fused ? (double4_32a*)(b + o_cta64) : nullptr;
  st.az = d_az ? (const float*)v_az : (const float*)(b + o_az);
  st.el = dim3 ? (d_el ? (const float*)v_el : (const float*)(b + o_el)) : nullptr;
  st.dop = d_dop ? (const float*)v_dop : (const float*)(b + o_dop);
  st.off = d_off ? (const int32_t*)v_off : (const int32_t*)(b + o_off);
  if (np > 0) {
    if (!d_az) RVH_CUDA(cudaMemcpyAsync((void*)st.az, f->azimuth, 4 * np, cudaMemcpyHostToDevice, s));
    if (dim3 && !d_el) RVH_CUDA(cudaMemcpyAsync((void*)st.el, f->elevation, 4 * np, cudaMemcpyHostToDevice, s));
    if (!d_dop) RVH_CUDA(cudaMemcpyAsync((void*)st.dop, f->doppler, 4 * np, cudaMemcpyHostToDevice, s));
  }
  if (!d_off) RVH_CUDA(cudaMemcpyAsync((void*)st.off, f->cluster_offsets, 4 * (size_t)(nc + 1), cudaMemcpyHostToDevice, s));
  void* dev[rvh::kOutputs];
  for (int i = 0; i < rvh::kOutputs; ++i) dev[i] = st.host_out[i] ? (void*)(b + o_out[i]) : v_out[i];
  st.dev_out = rvh::result_from(dev);
  RVH_CUDA(rvh::launch_threshold_fill(st.dev_out.threshold, nc, p->hypothesis_model == RVH_MODEL_PAPER_LINE,
                                      p->inlier_threshold, s));
  return RVH_OK;
}

static int unstage(const rvh_frame* f, rvh_result* r, const Staged& st, cudaStream_t s) {
  void* outs[rvh::kOutputs];
  void* dev[rvh::kOutputs];
  rvh::result_ptrs(*r, outs);
  rvh::result_ptrs(st.dev_out, dev);
  for (int i = 0; i < rvh::kOutputs; ++i) {
    if (!st.host_out[i]) continue;
    const size_t n = (i == rvh::kMaskOutput) ? (size_t)f->n_points : (size_t)f->n_clusters;
    if (n) RVH_CUDA(cudaMemcpyAsync(outs[i], dev[i], rvh::kOutputSize[i] * n, cudaMemcpyDeviceToHost, s));
  }
  if (st.sync_out) RVH_CUDA(cudaStreamSynchronize(s));
  return RVH_OK;
}

int rvh_estimate(rvh_ctx* ctx, const rvh_frame* frame, const rvh_params* params, rvh_result* result,
                 void* stream) {
  if (!ctx) return fail(RVH_EINVAL, "ctx is NULL");
  int rc = check_args_impl(frame, params, result);
  if (rc) return rc;
  if (frame->n_clusters == 0) return RVH_OK;
  std::lock_guard<std::mutex> lk(ctx->mu);
  RVH_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
  RVH_CUDA(cudaStreamWaitEvent(s, ctx->last_done, 0));
  Staged st{};
  rc = stage(ctx, frame, params, result, s, true, st);
  if (rc) return rc;
  ctx->stats_d = st.stats;
  FusedArgs a;
  memset(&a, 0, sizeof(a));
  fill_desc(ctx->trig, a.f[0], *frame, *params, st.az, st.el, st.dop, st.off, (float4*)st.rows, st.rows64,
            st.dev_out);
  a.n_frames = 1;
  a.n_items = frame->n_clusters;
  a.worklist = st.worklist;
  a.work_counter = st.counter;
  a.stats = st.stats;
  a.cta_rows64 = ctx->cta_rows ? st.cta_rows64 : nullptr;
  choose_schedule(ctx, params->model_dim, trials_per_chunk(*params), &a.pw, &a.hpl);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  RVH_CUDA(cudaStreamIsCapturing(s, &cap));
  if (ctx->graphs && s != nullptr && cap == cudaStreamCaptureStatusNone) {
    rc = launch_graph(ctx, a, params->model_dim, s);
  } else {
    RVH_CUDA(cudaMemsetAsync(st.stats, 0, sizeof(unsigned long long) * kStatsWords, s));
    rc = launch_batch(ctx, a, params->model_dim, s, ctx->ev0, ctx->ev1);
  }
  if (rc) return rc;
  // plain launches run every trial of every cluster; launches with an
  // extension (adaptive count, local optimisation, line model) count on the device
  ctx->last.hypotheses = (int64_t)frame->n_clusters * params->num_hypotheses;
  ctx->last.pair_evals = frame->n_points * (int64_t)params->num_hypotheses;
  ctx->last_counts_trials = params->confidence > 0.0 || params->refine_iterations > 0 || params->hypothesis_model != 0;
  ctx->last.points_per_warp = a.pw;
  ctx->last.hyps_per_lane = a.hpl;
  ctx->have_launch = true;
  rc = unstage(frame, result, st, s);
  RVH_CUDA(cudaEventRecord(ctx->last_done, s));
  return rc;
}

int rvh_estimate_baseline(rvh_ctx* ctx, const rvh_frame* frame, const rvh_params* params, rvh_result* result,
                          void* stream) {
  if (!ctx) return fail(RVH_EINVAL, "ctx is NULL");
  int rc = check_args_impl(frame, params, result);
  if (rc) return rc;
  if (params->refine_iterations != 0 || params->confidence != 0.0 || params->hypothesis_model != 0)
    return fail(RVH_EINVAL,
                "rvh_estimate_baseline runs the plain method (refine_iterations 0, confidence 0, hypothesis_model 0)");
  if (frame->n_clusters == 0) return RVH_OK;
  std::lock_guard<std::mutex> lk(ctx->mu);
  RVH_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
  RVH_CUDA(cudaStreamWaitEvent(s, ctx->last_done, 0));
  Staged st{};
  rc = stage(ctx, frame, params, result, s, false, st);
  if (rc) return rc;
  const int dim = params->model_dim;
  const int nmax = 2048;
  const size_t smem = baseline_smem_bytes(nmax);
  RVH_CUDA(baseline_configure(dim, smem));
  BaselineArgs b;
  memset(&b, 0, sizeof(b));
  FrameDesc d;
  fill_desc(ctx->trig, d, *frame, *params, st.az, st.el, st.dop, st.off, nullptr, nullptr, st.dev_out);
  b.az = d.az;
  b.el = d.el;
  b.dop = d.dop;
  b.offsets = st.off;
  b.n_points = frame->n_points;
  b.rows64_g = (double*)st.rows;
  b.H = d.H;
  b.tau = d.tau;
  b.eps = d.eps;
  b.key = d.key;
  b.cluster_base = d.cluster_base;
  b.vx = d.vx;
  b.vy = d.vy;
  b.vz = d.vz;
  b.heading = d.heading;
  b.inlier_count = d.inlier_count;
  b.best = d.best;
  b.status = d.status;
  b.mask = d.mask;
  b.nmax_smem = nmax;
  b.trig = ctx->trig;
  RVH_CUDA(cudaEventRecord(ctx->ev0, s));
  for (int i = 0; i < frame->n_clusters; ++i) RVH_CUDA(launch_baseline_cluster(dim, b, i, smem, s));
  RVH_CUDA(cudaEventRecord(ctx->ev1, s));
  ctx->have_launch = false;
  rc = unstage(frame, result, st, s);
  RVH_CUDA(cudaEventRecord(ctx->last_done, s));
  return rc;
}

int rvh_autotune(rvh_ctx* ctx, const rvh_frame* frame, const rvh_params* params, rvh_result* result,
                 int32_t reps, rvh_schedule* best) {
  if (!ctx) return fail(RVH_EINVAL, "ctx is NULL");
  if (reps < 1) return fail(RVH_EINVAL, "reps must be >= 1");
  int rc = check_args_impl(frame, params, result);
  if (rc) return rc;
  if (frame->n_clusters == 0) return fail(RVH_EINVAL, "empty frame");
  static const int kCand[6][2] = {{1, 4}, {1, 8}, {8, 4}, {8, 8}, {32, 4}, {32, 8}};
  const int save_pw = ctx->pw_fixed, save_hpl = ctx->hpl_fixed;
  int bpw = 1, bhpl = 4;
  float bms = 1e30f;
  // candidates take turns (round-robin over the repetitions, the first
  // round untimed) so that drifting clocks or caches favour none of them;
  // each is ranked by its median time
  std::vector<std::vector<float>> times(6);
  for (int r = 0; r <= reps && rc == RVH_OK; ++r) {
    for (int ic = 0; ic < 6 && rc == RVH_OK; ++ic) {
      ctx->pw_fixed = kCand[ic][0];
      ctx->hpl_fixed = kCand[ic][1];
      rc = rvh_estimate(ctx, frame, params, result, nullptr);
      if (rc) break;
      rvh_stats st;
      rc = rvh_get_stats(ctx, &st);
      if (r > 0) times[ic].push_back(st.kernel_ms);
    }
  }
  for (int ic = 0; ic < 6 && rc == RVH_OK; ++ic) {
    std::vector<float>& t = times[ic];
    std::sort(t.begin(), t.end());
    const float ms = t.size() % 2 ? t[t.size() / 2] : 0.5f * (t[t.size() / 2 - 1] + t[t.size() / 2]);
    if (ms < bms) {
      bms = ms;
      bpw = kCand[ic][0];
      bhpl = kCand[ic][1];
    }
  }
  ctx->pw_fixed = save_pw;
  ctx->hpl_fixed = save_hpl;
  if (rc) return rc;
  const int key = tune_key(params->model_dim, trials_per_chunk(*params));
  ctx->tuned[key] = std::make_pair(bpw, bhpl);
  save_tune_cache(ctx, key, bpw, bhpl, bms);
  if (best) {
    best->points_per_warp = bpw;
    best->hyps_per_lane = bhpl;
    best->kernel_ms = bms;
  }
  return RVH_OK;
}

int rvh_submit(rvh_ctx* ctx, const rvh_frame* frame, const rvh_params* params, rvh_result* result,
               uint64_t* ticket) {
  if (!ctx || !ticket) return fail(RVH_EINVAL, "NULL argument");
  int rc = check_args_impl(frame, params, result);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->server) {
      rc = server_create(ctx, &ctx->server);
      if (rc) return rc;
    }
  }
  return server_submit(ctx->server, frame, params, result, ticket);
}

int rvh_poll(rvh_ctx* ctx, uint64_t ticket) {
  if (!ctx || !ctx->server) return fail(RVH_EINVAL, "unknown ticket");
  return server_poll(ctx->server, ticket);
}

int rvh_wait(rvh_ctx* ctx, uint64_t ticket, int64_t timeout_us) {
  if (!ctx || !ctx->server) return fail(RVH_EINVAL, "unknown ticket");
  return server_wait(ctx->server, ticket, timeout_us);
}

}  // extern "C"

namespace rvh {
int check_args(const rvh_frame* f, const rvh_params* p, const rvh_result* r) { return check_args_impl(f, p, r); }
int set_error(int code, const std::string& msg) { return fail(code, msg); }
bool device_ptr(const void* p) { return is_device_ptr(p); }
int validate_host_offsets(const int32_t* off, int32_t n, int64_t np) { return check_host_offsets(off, n, np); }
}  // namespace rvh
