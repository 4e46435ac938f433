// Internal runtime interfaces shared by the C ABI (rvh_api.cu) and the serving
// loop (rvh_server.cu).
#pragma once

#include <cstdint>
#include <string>

#include "rvh.h"
#include "rvh_kernels.h"

namespace rvh {

struct Server;

// context helpers (rvh_api.cu)
int ctx_alloc(rvh_ctx* ctx, void** p, size_t bytes);
void ctx_free(rvh_ctx* ctx, void* p, size_t bytes);
int ctx_device(rvh_ctx* ctx);
int ctx_sms(rvh_ctx* ctx);
int set_error(int code, const std::string& msg);
bool device_ptr(const void* p);
int validate_host_offsets(const int32_t* off, int32_t n, int64_t n_points);
void choose_schedule(rvh_ctx* ctx, int dim, int H, int* pw, int* hpl);
void load_tune_cache(rvh_ctx* ctx);
void fill_desc(rvh_ctx* ctx, FrameDesc& d, const rvh_frame& f, const rvh_params& p, const float* az,
               const float* el, const float* dop, const int32_t* off, float4* rows_g, double4_32a* rows64_g,
               const rvh_result& out);
int launch_batch(rvh_ctx* ctx, FusedArgs& a, int dim, cudaStream_t s, cudaEvent_t t0, cudaEvent_t t1);

// serving loop (rvh_server.cu)
int server_create(rvh_ctx* ctx, Server** out);
void server_destroy(Server* s);
int server_submit(Server* s, const rvh_frame* f, const rvh_params* p, rvh_result* r, uint64_t* ticket);
int server_poll(Server* s, uint64_t ticket);
int server_wait(Server* s, uint64_t ticket, int64_t timeout_us);

}  // namespace rvh
