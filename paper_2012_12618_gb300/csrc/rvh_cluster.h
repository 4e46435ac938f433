// Launch interfaces of the clustering stage (rvh_cluster.cu): DBSCAN into
// labels and the CSR of clusters, and the gather of point arrays into
// cluster order.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace rvh {

size_t cluster_scratch_bytes(int64_t n);
int64_t cluster_max_points();
cudaError_t launch_cluster(const float* feat, int64_t n, int dim, double eps, int min_pts, void* scratch,
                           int* labels, int* perm, int* offsets, int max_clusters, int* n_clusters_host,
                           int* err_host, cudaStream_t s);
cudaError_t launch_gather(const int* perm, int64_t m, const float* s0, float* d0, const float* s1, float* d1,
                          const float* s2, float* d2, cudaStream_t s);

}  // namespace rvh
