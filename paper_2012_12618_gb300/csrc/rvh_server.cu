// Serving loop behind rvh_submit / rvh_poll / rvh_wait: admission by a device
// memory pool, iteration-level continuous batching (every step packs all
// frames admitted since the previous step into one persistent launch per
// model dimension), several steps in flight on separate streams, and
// completion detected with events (no device-side flags or spins).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "rvh.h"
#include "rvh_kernels.h"
#include "rvh_outputs.h"
#include "rvh_runtime.h"

namespace rvh {

namespace {

constexpr size_t kGran = 256;
// work-list capacity of one step (clusters over all frames of a launch); each
// step slot owns this scratch for the server's lifetime, so admitted frames
// can never starve a launch of its scratch
constexpr int kStepItems = 1 << 19;
size_t gran(size_t x) { return (x + kGran - 1) & ~(kGran - 1); }

// First-fit arena allocator over [0, size).
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    size_ = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = gran(std::max<size_t>(bytes, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = gran(std::max<size_t>(bytes, 1));
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0;
};

struct Req {
  uint64_t id = 0;
  rvh_frame frame{};        // device pointers after admission
  rvh_params params{};
  rvh_result user{};        // caller's outputs
  rvh_result dev{};         // where the kernel writes
  bool host_out[kOutputs] = {};
  size_t dev_off = 0, dev_bytes = 0;
  size_t pin_off = 0, pin_bytes = 0;
  size_t pin_out[kOutputs] = {};
  size_t rows64_off = 0;
  cudaEvent_t copied = nullptr;  // host inputs are on the device
  int step = -1;
  int state = 0;            // 0 queued, 1 launched, 2 done
};

struct Step {
  int id = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  size_t scratch_off = 0, scratch_bytes = 0;
  std::vector<uint64_t> reqs;
  bool busy = false;
};

}  // namespace

struct Server {
  rvh_ctx* ctx = nullptr;
  int device = 0;
  void* pool = nullptr;
  size_t pool_bytes = 0;
  Arena dev_arena;
  char* pinned = nullptr;
  size_t pinned_bytes = 0;
  Arena pin_arena;
  cudaStream_t copy_stream = nullptr;
  std::vector<Step> steps;  // ring of in-flight step slots (one stream each)
  int next_step = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread thread;
  std::string thread_error;
  // graphs of the step launch, per step slot (each slot has its own stream)
  // x model dimension x extensions x work list
  std::vector<std::unique_ptr<LaunchGraph>> graphs;
  int64_t n_steps = 0, n_graph_replays = 0;

  int finalize_step(Step& st);   // requires mu held
  void loop();
};


int server_create(rvh_ctx* ctx, Server** out) {
  Server* s = new Server();
  s->ctx = ctx;
  s->device = ctx_device(ctx);
  cudaSetDevice(s->device);
  // the device pool takes what the context's budget has left, up to 4 GiB
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  size_t want = std::min<size_t>((size_t)4 << 30, free_b / 2);
  int rc = RVH_ENOMEM;
  while (want >= ((size_t)64 << 20)) {
    rc = ctx_alloc(ctx, &s->pool, want);
    if (rc == RVH_OK) break;
    want /= 2;
  }
  if (rc) {
    delete s;
    return rc;
  }
  s->pool_bytes = want;
  s->dev_arena.reset(want);
  s->pinned_bytes = (size_t)128 << 20;
  if (cudaHostAlloc((void**)&s->pinned, s->pinned_bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    ctx_free(ctx, s->pool, s->pool_bytes);
    delete s;
    return set_error(RVH_ENOMEM, "cudaHostAlloc of the output staging area failed");
  }
  s->pin_arena.reset(s->pinned_bytes);
  cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
  s->steps.resize(3);
  for (auto& st : s->steps) {
    cudaStreamCreateWithFlags(&st.stream, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming);
    st.scratch_bytes = gran(sizeof(int2) * (size_t)kStepItems) + 256;
    if (!s->dev_arena.alloc(st.scratch_bytes, &st.scratch_off)) {
      server_destroy(s);
      return set_error(RVH_ENOMEM, "serving pool too small for the step scratch");
    }
  }
  for (size_t k = 0; k < s->steps.size() * 8; ++k) s->graphs.emplace_back(new LaunchGraph());
  s->thread = std::thread([s] { s->loop(); });
  *out = s;
  return RVH_OK;
}

void server_destroy(Server* s) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->thread.joinable()) s->thread.join();
  cudaSetDevice(s->device);
  for (auto& st : s->steps) {
    cudaStreamSynchronize(st.stream);
    cudaStreamDestroy(st.stream);
    cudaEventDestroy(st.done);
  }
  cudaStreamSynchronize(s->copy_stream);
  cudaStreamDestroy(s->copy_stream);
  s->graphs.clear();
  for (auto& kv : s->reqs)
    if (kv.second->copied) cudaEventDestroy(kv.second->copied);
  cudaFreeHost(s->pinned);
  ctx_free(s->ctx, s->pool, s->pool_bytes);
  delete s;
}

int server_submit(Server* s, const rvh_frame* f, const rvh_params* p, rvh_result* r, uint64_t* ticket) {
  cudaSetDevice(s->device);
  const int64_t np = f->n_points;
  const int32_t nc = f->n_clusters;
  const bool dim3 = p->model_dim == 3;
  if (nc > kStepItems) return set_error(RVH_EINVAL, "frame has more clusters than a serving step holds");
  if (nc > 0 && !device_ptr(f->cluster_offsets)) {
    int rc = validate_host_offsets(f->cluster_offsets, nc, np);
    if (rc) return rc;
  }
  auto q = std::make_unique<Req>();
  q->params = *p;
  q->user = *r;
  void* uo[kOutputs];
  result_ptrs(*r, uo);
  for (int i = 0; i < kOutputs; ++i) q->host_out[i] = uo[i] && !device_ptr(uo[i]);
  const bool d_az = device_ptr(f->azimuth), d_dop = device_ptr(f->doppler);
  const bool d_el = !dim3 || device_ptr(f->elevation);
  const bool d_off = nc == 0 || device_ptr(f->cluster_offsets);
  // device slot layout: [rows_g | staged inputs | staged outputs]
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += gran(b);
    return o;
  };
  const size_t o_rows = take(sizeof(float4) * (size_t)std::max<int64_t>(np, 1));
  const size_t o_rows64 = take(sizeof(double4_32a) * (size_t)std::max<int64_t>(np, 1));
  (void)o_rows;
  const size_t o_az = d_az ? 0 : take(4 * (size_t)np);
  const size_t o_el = d_el ? 0 : take(4 * (size_t)np);
  const size_t o_dop = d_dop ? 0 : take(4 * (size_t)np);
  const size_t o_off = d_off ? 0 : take(4 * (size_t)(nc + 1));
  size_t o_out[kOutputs];
  size_t pin = 0;
  for (int i = 0; i < kOutputs; ++i) {
    const size_t n = (i == kMaskOutput) ? (size_t)np : (size_t)nc;
    o_out[i] = q->host_out[i] ? take(kOutputSize[i] * std::max<size_t>(n, 1)) : 0;
    if (q->host_out[i]) {
      q->pin_out[i] = pin;
      pin += gran(kOutputSize[i] * std::max<size_t>(n, 1));
    }
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const size_t usable = s->dev_arena.size() - s->steps.size() * s->steps[0].scratch_bytes;
    if (off > usable || pin > s->pin_arena.size())
      return set_error(RVH_ENOMEM, "frame larger than the serving pool");
    if (!s->dev_arena.alloc(off, &q->dev_off)) return set_error(RVH_EAGAIN, "device pool full");
    if (pin && !s->pin_arena.alloc(pin, &q->pin_off)) {
      s->dev_arena.release(q->dev_off, off);
      return set_error(RVH_EAGAIN, "output staging full");
    }
    q->dev_bytes = off;
    q->pin_bytes = pin;
    q->rows64_off = o_rows64;
  }
  char* b = (char*)s->pool + q->dev_off;
  q->frame = *f;
  q->frame.azimuth = d_az ? f->azimuth : (const float*)(b + o_az);
  q->frame.elevation = dim3 ? (d_el ? f->elevation : (const float*)(b + o_el)) : nullptr;
  q->frame.doppler = d_dop ? f->doppler : (const float*)(b + o_dop);
  q->frame.cluster_offsets = d_off ? f->cluster_offsets : (const int32_t*)(b + o_off);
  cudaError_t e = cudaSuccess;
  if (np > 0) {
    if (!d_az) e = cudaMemcpyAsync((void*)q->frame.azimuth, f->azimuth, 4 * np, cudaMemcpyHostToDevice, s->copy_stream);
    if (e == cudaSuccess && dim3 && !d_el)
      e = cudaMemcpyAsync((void*)q->frame.elevation, f->elevation, 4 * np, cudaMemcpyHostToDevice, s->copy_stream);
    if (e == cudaSuccess && !d_dop)
      e = cudaMemcpyAsync((void*)q->frame.doppler, f->doppler, 4 * np, cudaMemcpyHostToDevice, s->copy_stream);
  }
  if (e == cudaSuccess && !d_off)
    e = cudaMemcpyAsync((void*)q->frame.cluster_offsets, f->cluster_offsets, 4 * (size_t)(nc + 1),
                        cudaMemcpyHostToDevice, s->copy_stream);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->copied, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(q->copied, s->copy_stream);
  // the caller may reuse its host input buffers once this returns
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
  void* dv[kOutputs];
  for (int i = 0; i < kOutputs; ++i) dv[i] = q->host_out[i] ? (void*)(b + o_out[i]) : uo[i];
  q->dev = result_from(dv);
  std::lock_guard<std::mutex> lk(s->mu);
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->dev_arena.release(q->dev_off, q->dev_bytes);
    if (q->pin_bytes) s->pin_arena.release(q->pin_off, q->pin_bytes);
    if (q->copied) cudaEventDestroy(q->copied);
    return set_error(RVH_ECUDA, std::string("submit copy: ") + cudaGetErrorString(e));
  }
  q->id = s->next_id++;
  *ticket = q->id;
  s->queue.push_back(q->id);
  s->reqs.emplace(q->id, std::move(q));
  s->cv.notify_all();
  return RVH_OK;
}

// Copies host outputs of a completed step to the callers and frees its memory.
int Server::finalize_step(Step& st) {
  for (uint64_t id : st.reqs) {
    auto it = reqs.find(id);
    if (it == reqs.end()) continue;
    Req& q = *it->second;
    void* uo[kOutputs];
    result_ptrs(q.user, uo);
    for (int i = 0; i < kOutputs; ++i) {
      if (!q.host_out[i]) continue;
      const size_t n = (i == kMaskOutput) ? (size_t)q.frame.n_points : (size_t)q.frame.n_clusters;
      if (n) memcpy(uo[i], pinned + q.pin_off + q.pin_out[i], kOutputSize[i] * n);
    }
    dev_arena.release(q.dev_off, q.dev_bytes);
    if (q.pin_bytes) pin_arena.release(q.pin_off, q.pin_bytes);
    if (q.copied) cudaEventDestroy(q.copied);
    q.copied = nullptr;
    q.state = 2;
  }
  st.reqs.clear();
  st.busy = false;
  return RVH_OK;
}

void Server::loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    // complete finished steps
    bool inflight = false;
    for (auto& st : steps) {
      if (!st.busy) continue;
      cudaError_t q = cudaEventQuery(st.done);
      if (q == cudaSuccess) {
        finalize_step(st);
      } else if (q == cudaErrorNotReady) {
        inflight = true;
      } else {
        thread_error = cudaGetErrorString(q);
        finalize_step(st);
      }
    }
    if (stop && queue.empty() && !inflight) break;
    if (queue.empty()) {
      if (inflight) cv.wait_for(lk, std::chrono::microseconds(20));
      else cv.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    // a free step slot (at most steps.size() launches in flight)
    Step* slot = nullptr;
    for (size_t k = 0; k < steps.size(); ++k) {
      Step& st = steps[(next_step + k) % steps.size()];
      if (!st.busy) {
        slot = &st;
        next_step = (int)((next_step + k + 1) % steps.size());
        break;
      }
    }
    if (!slot) {
      cv.wait_for(lk, std::chrono::microseconds(20));
      continue;
    }
    // iteration-level batch: everything queued now, grouped by model dimension
    std::vector<uint64_t> batch[2];
    int items[2] = {0, 0};
    std::deque<uint64_t> rest;
    for (uint64_t id : queue) {
      Req& q = *reqs[id];
      const int d = q.params.model_dim == 3;
      if ((int)batch[d].size() < kMaxBatchFrames && items[d] + q.frame.n_clusters <= kStepItems) {
        batch[d].push_back(id);
        items[d] += q.frame.n_clusters;
      } else {
        rest.push_back(id);
      }
    }
    // one dimension per step slot; the other waits for the next free slot
    int dimsel = batch[0].empty() ? 1 : 0;
    if (!batch[0].empty() && !batch[1].empty()) {
      // alternate to keep both streams of work moving
      dimsel = (slot - steps.data()) & 1;
    }
    std::vector<uint64_t>& take = batch[dimsel];
    for (uint64_t id : batch[1 - dimsel]) rest.push_front(id);
    std::sort(rest.begin(), rest.end());
    queue.assign(rest.begin(), rest.end());
    // the slot's own scratch: worklist + counter
    int n_items = 0;
    for (uint64_t id : take) n_items += reqs[id]->frame.n_clusters;
    char* sb = (char*)pool + slot->scratch_off;
    FusedArgs a;
    memset(&a, 0, sizeof(a));
    int nf = 0;
    for (uint64_t id : take) {
      Req& q = *reqs[id];
      char* b = (char*)pool + q.dev_off;
      fill_desc(ctx_trig(ctx), a.f[nf], q.frame, q.params, q.frame.azimuth, q.frame.elevation, q.frame.doppler,
                q.frame.cluster_offsets, (float4*)b, (double4_32a*)(b + q.rows64_off), q.dev);
      cudaStreamWaitEvent(slot->stream, q.copied, 0);
      if (launch_threshold_fill(q.dev.threshold, q.frame.n_clusters,
                                q.params.hypothesis_model == RVH_MODEL_PAPER_LINE, q.params.inlier_threshold,
                                slot->stream) != cudaSuccess)
        thread_error = "threshold fill failed";
      ++nf;
    }
    a.n_frames = nf;
    a.n_items = n_items;
    a.worklist = (int2*)sb;
    a.work_counter = (int*)(sb + gran(sizeof(int2) * (size_t)kStepItems));
    a.stats = nullptr;
    int Hmax = 1;
    for (int i = 0; i < nf; ++i)
      Hmax = std::max(Hmax, a.f[i].trial_block > 0 ? std::min(a.f[i].trial_block, a.f[i].H) : a.f[i].H);
    choose_schedule(ctx, dimsel ? 3 : 2, Hmax, &a.pw, &a.hpl);
    int rc = RVH_OK;
    if (n_items > 0) {
      const int dim = dimsel ? 3 : 2;
      if (ctx_graphs(ctx)) {
        // the slot's graph for this kernel instantiation and node list,
        // replayed with this step's batch
        int grid = 1;
        size_t smem = 0;
        rc = prepare_launch(ctx, a, dim, &grid, &smem);
        if (rc == RVH_OK) {
          const size_t k = (size_t)(slot - steps.data()) * 8 + (size_t)dimsel * 4 + (fused_ext(a) ? 2 : 0) +
                           (a.direct ? 0 : 1);
          LaunchGraph& g = *graphs[k];
          const int64_t r0 = g.replays;
          if (g.launch(a, dim, grid, smem, !a.direct, slot->stream) != cudaSuccess) {
            cudaGetLastError();
            rc = RVH_ECUDA;
          }
          n_graph_replays += g.replays - r0;
        }
      } else {
        rc = launch_batch(ctx, a, dim, slot->stream, nullptr, nullptr);
      }
      ++n_steps;
    }
    if (rc != RVH_OK) thread_error = "launch failed";
    // outputs that go to host memory: device -> pinned staging
    for (uint64_t id : take) {
      Req& q = *reqs[id];
      void* dv[kOutputs];
      result_ptrs(q.dev, dv);
      for (int i = 0; i < kOutputs; ++i) {
        if (!q.host_out[i]) continue;
        const size_t n = (i == kMaskOutput) ? (size_t)q.frame.n_points : (size_t)q.frame.n_clusters;
        if (n) cudaMemcpyAsync(pinned + q.pin_off + q.pin_out[i], dv[i], kOutputSize[i] * n,
                               cudaMemcpyDeviceToHost, slot->stream);
      }
      q.state = 1;
    }
    cudaEventRecord(slot->done, slot->stream);
    slot->busy = true;
    slot->reqs = take;
  }
}

void server_counts(Server* s, int64_t* steps, int64_t* graph_replays) {
  std::lock_guard<std::mutex> lk(s->mu);
  *steps = s->n_steps;
  *graph_replays = s->n_graph_replays;
}

int server_poll(Server* s, uint64_t ticket) {
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(RVH_EINVAL, "unknown ticket");
  if (it->second->state == 2) {
    s->reqs.erase(it);
    return RVH_OK;
  }
  return RVH_PENDING;
}

int server_wait(Server* s, uint64_t ticket, int64_t timeout_us) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    int rc = server_poll(s, ticket);
    if (rc != RVH_PENDING) return rc;
    if (timeout_us >= 0) {
      const auto dt = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0);
      if (dt.count() >= timeout_us) return set_error(RVH_ETIMEDOUT, "ticket not complete");
    }
    std::this_thread::sleep_for(std::chrono::microseconds(10));
  }
}

}  // namespace rvh
