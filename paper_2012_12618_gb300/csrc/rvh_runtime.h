// Internal runtime interfaces shared by the C ABI (rvh_api.cu) and the serving
// loop (rvh_server.cu).
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "rvh.h"
#include "rvh_kernels.h"

namespace rvh {

struct Server;

// The batch launch as an instantiated CUDA graph (rvh_graph.cu): the fused
// kernel, after the work-list kernel when with_work is set.  Later launches
// of the same kernel instantiation and node list replay it with the new
// arguments written into its kernel nodes, so new frame addresses and sizes
// need no new graph.  Launches of one executable graph run in order, so a
// stream that overlaps with others keeps a LaunchGraph of its own.  Not
// thread-safe: callers serialise their use of one.
struct LaunchGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t work = nullptr, fused = nullptr;
  int dim_ = 0;
  bool ext_ = false, with_work_ = false;
  FusedArgs last;
  int last_grid = 0;
  size_t last_smem = 0;
  bool have_last = false;
  int64_t builds = 0, replays = 0;
  cudaError_t launch(const FusedArgs& a, int dim, int grid, size_t smem, bool with_work, cudaStream_t s);
  void reset();
  ~LaunchGraph() { reset(); }
};

// context helpers (rvh_api.cu)
int ctx_alloc(rvh_ctx* ctx, void** p, size_t bytes);
void ctx_free(rvh_ctx* ctx, void* p, size_t bytes);
int ctx_device(rvh_ctx* ctx);
int ctx_sms(rvh_ctx* ctx);
bool ctx_graphs(rvh_ctx* ctx);  // CUDA graphs enabled (RVH_GRAPHS unset or non-zero)
const double2* ctx_trig(rvh_ctx* ctx);  // the context's device table of (cos, sin)(k/128)
int set_error(int code, const std::string& msg);
bool device_ptr(const void* p);
int validate_host_offsets(const int32_t* off, int32_t n, int64_t n_points);
void choose_schedule(rvh_ctx* ctx, int dim, int H, int* pw, int* hpl);
void load_tune_cache(rvh_ctx* ctx);
// Host-side argument checks of every estimate entry point (RVH_EINVAL with a
// message, or RVH_OK).
int check_args(const rvh_frame* f, const rvh_params* p, const rvh_result* r);
// The per-frame descriptor of a launch: trig is the device table of
// (cos, sin)(k/128); the pointers must already be device pointers.
void fill_desc(const double2* trig, FrameDesc& d, const rvh_frame& f, const rvh_params& p, const float* az,
               const float* el, const float* dop, const int32_t* off, float4* rows_g, double4_32a* rows64_g,
               const rvh_result& out);
int launch_batch(rvh_ctx* ctx, FusedArgs& a, int dim, cudaStream_t s, cudaEvent_t t0, cudaEvent_t t1);
// Grid, dynamic shared memory and item mapping (direct or work list) of a batch launch.
int prepare_launch(rvh_ctx* ctx, FusedArgs& a, int dim, int* grid, size_t* smem);

// serving loop (rvh_server.cu)
int server_create(rvh_ctx* ctx, Server** out);
void server_destroy(Server* s);
int server_submit(Server* s, const rvh_frame* f, const rvh_params* p, rvh_result* r, uint64_t* ticket);
int server_poll(Server* s, uint64_t ticket);
int server_wait(Server* s, uint64_t ticket, int64_t timeout_us);
void server_counts(Server* s, int64_t* steps, int64_t* graph_replays);

}  // namespace rvh
