// CUDA graphs of the batch launch (Eq. 4's max_trials x N_clusts trials of a
// batch in one launch, Sec. III-A): the fused kernel, optionally preceded by
// the work-list kernel, as an instantiated graph whose kernel nodes take new
// arguments before each replay.  Frames at new addresses, other sizes, other
// batches of frames and other schedules all replay the same executable graph;
// only a change of kernel instantiation (model dimension, extensions) or of
// the node list (with or without the work list) builds another one.
#include <cstring>

#include "rvh_runtime.h"

namespace rvh {

namespace {

cudaKernelNodeParams node_params(const void* fn, int grid, int block, size_t smem, void** args) {
  cudaKernelNodeParams p;
  memset(&p, 0, sizeof(p));
  p.func = const_cast<void*>(fn);
  p.gridDim = dim3((unsigned)grid);
  p.blockDim = dim3((unsigned)block);
  p.sharedMemBytes = (unsigned)smem;
  p.kernelParams = args;
  p.extra = nullptr;
  return p;
}

}  // namespace

void LaunchGraph::reset() {
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  exec = nullptr;
  graph = nullptr;
  work = fused = nullptr;
  have_last = false;
}

cudaError_t LaunchGraph::launch(const FusedArgs& a, int dim, int grid, size_t smem, bool with_work, cudaStream_t s) {
  const bool ext = fused_ext(a);
  FusedArgs arg = a;  // the node parameters are copied when set
  void* args[] = {(void*)&arg};
  const cudaKernelNodeParams pf = node_params(fused_kernel_fn(dim, ext), grid, fused_threads(), smem, args);
  const cudaKernelNodeParams pw = node_params(worklist_kernel_fn(), 1, kWorklistThreads, 0, args);
  cudaError_t e = cudaSuccess;
  if (!exec || dim_ != dim || ext_ != ext || with_work_ != with_work) {
    reset();
    e = cudaGraphCreate(&graph, 0);
    if (e == cudaSuccess && with_work) e = cudaGraphAddKernelNode(&work, graph, nullptr, 0, &pw);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&fused, graph, with_work ? &work : nullptr, with_work ? 1 : 0, &pf);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
      reset();
      return e;
    }
    dim_ = dim;
    ext_ = ext;
    with_work_ = with_work;
    ++builds;
  } else {
    const bool same = have_last && last_grid == grid && last_smem == smem && memcmp(&last, &a, sizeof(FusedArgs)) == 0;
    if (!same) {
      e = cudaGraphExecKernelNodeSetParams(exec, fused, &pf);
      if (e == cudaSuccess && with_work) e = cudaGraphExecKernelNodeSetParams(exec, work, &pw);
      if (e != cudaSuccess) {
        reset();
        return e;
      }
    }
    ++replays;
  }
  last = a;
  last_grid = grid;
  last_smem = smem;
  have_last = true;
  return cudaGraphLaunch(exec, s);
}

}  // namespace rvh
