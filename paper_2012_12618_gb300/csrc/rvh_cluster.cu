// The clustering stage before the estimator (Fig. 1: point cloud ->
// clustering -> per-cluster RANSAC and least squares): DBSCAN (Ester,
// Kriegel, Sander, Xu, KDD'96) over FP32 feature vectors, and the gather of
// point attributes into cluster order.
//
// Definitions (the library's reading; rvh.h states them for the user):
// q is a neighbour of p (p itself included) when the squared Euclidean
// distance of their feature vectors, accumulated in FP64 over the components
// in order, is at most eps^2; p is a core point with at least min_pts
// neighbours; clusters are the connected components of core points, numbered
// in the order of their smallest core index; a non-core point with a core
// neighbour joins the cluster of its lowest-index core neighbour; the rest is
// noise.  Every decision is an FP64 comparison made in the same operation
// order everywhere, so the labels are exactly defined.
//
// GPU mapping: a hashed grid of cells slightly larger than eps over the first
// min(dim, 3) components (linked lists built with atomic exchange), one
// thread per point for neighbour counts, lock-free union-find over core-core
// neighbour pairs that always links the larger root under the smaller (so a
// component's root is its smallest core index), a device-wide scan for the
// numbering, and a bitonic sort of (cluster, index) keys for the CSR order.
// Every loop is bounded by the input size; the union retry loop has an
// explicit cap that raises an error flag instead of spinning.
#include <cstdint>
#include <cuda_runtime.h>

#include "rvh_cluster.h"

namespace rvh {

namespace {

constexpr int kCT = 256;                       // threads per block of the clustering kernels
constexpr int kUnionRetries = 1 << 20;         // cap on one union's compare-and-swap retries

struct ClusterArgs {
  const float* feat;  // [n * dim]
  int64_t n;
  int dim, gdim;      // components, gridded components (min(dim, 3))
  double eps2;        // eps^2 (FP64)
  float in32, out32;  // FP32 prefilter: d2_32 <= in32 certainly a neighbour, > out32 certainly not
  double inv_cell;    // 1 / cell size
  int min_pts;
  uint32_t hmask;     // hash buckets - 1 (power of two)
  int* head;          // [buckets] first point of each bucket, -1 empty
  int* next;          // [n] next point in the bucket
  int4* cellc;        // [n] cell coordinates (x, y, z, 0)
  uint8_t* core;      // [n]
  int* parent;        // [n] union-find
  int* err;           // error flag
};

__device__ __forceinline__ uint32_t cell_hash(int x, int y, int z) {
  return ((uint32_t)x * 73856093u) ^ ((uint32_t)y * 19349663u) ^ ((uint32_t)z * 83492791u);
}

// Squared Euclidean distance accumulated in FP64 over the components in order.
__device__ __forceinline__ double feat_dist2(const float* a, const float* b, int dim) {
  double s = 0.0;
  for (int k = 0; k < dim; ++k) {
    const double d = (double)a[k] - (double)b[k];
    s = s + d * d;
  }
  return s;
}

__device__ __forceinline__ int cell_coord(float v, double inv_cell) {
  const double c = floor((double)v * inv_cell);
  // far-out (or non-finite) values share the edge cells: still exact, only slower
  return c >= 1073741823.0 ? 1073741823 : (c <= -1073741823.0 ? -1073741823 : (c == c ? (int)c : 0));
}

__global__ void k_grid(ClusterArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const float* f = a.feat + i * a.dim;
  const int x = cell_coord(f[0], a.inv_cell);
  const int y = a.gdim > 1 ? cell_coord(f[1], a.inv_cell) : 0;
  const int z = a.gdim > 2 ? cell_coord(f[2], a.inv_cell) : 0;
  a.cellc[i] = make_int4(x, y, z, 0);
  a.next[i] = atomicExch(&a.head[cell_hash(x, y, z) & a.hmask], (int)i);
}

// The neighbour test.  An FP32 squared distance (differences and squares of
// FP32 values, accumulated with fmaf) is within 8u relative of the exact one
// for up to four components, and the FP64 one within 6 x 2^-53; outside
// eps^2 (1 -+ 16u) the FP32 value decides alike, inside that band (and for
// tiny values, where underflow voids the relative bound) the FP64 sum in
// component order decides.
__device__ __forceinline__ bool is_neighbour(const ClusterArgs& a, const float* fp, const float* fq) {
  float s = 0.0f;
  for (int k = 0; k < a.dim; ++k) {
    const float d = fp[k] - fq[k];
    s = fmaf(d, d, s);
  }
  if (s > a.out32) return false;  // also +inf
  if (s <= a.in32 && s >= 0x1p-100f) return true;
  return feat_dist2(fp, fq, a.dim) <= a.eps2;  // NaN: false
}

// Visits every point q within eps of point p (q = p included) until the
// visitor returns false.  Cells of the 3^gdim neighbourhood; bucket lists are
// filtered by exact cell coordinates (hash collisions) and by the distance.
template <typename Visit>
__device__ __forceinline__ void for_neighbours(const ClusterArgs& a, int64_t p, Visit visit) {
  const int4 c = a.cellc[p];
  const float* fp = a.feat + p * a.dim;
  const int ry = a.gdim > 1 ? 1 : 0, rz = a.gdim > 2 ? 1 : 0;
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -ry; dy <= ry; ++dy)
      for (int dz = -rz; dz <= rz; ++dz) {
        const int x = c.x + dx, y = c.y + dy, z = c.z + dz;
        int64_t steps = 0;
        for (int q = a.head[cell_hash(x, y, z) & a.hmask]; q >= 0 && steps <= a.n; q = a.next[q], ++steps) {
          const int4 cq = a.cellc[q];
          if (cq.x != x || cq.y != y || cq.z != z) continue;
          if (is_neighbour(a, fp, a.feat + (int64_t)q * a.dim))
            if (!visit(q)) return;
        }
      }
}

__global__ void k_core(ClusterArgs a) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  int count = 0;
  for_neighbours(a, p, [&](int) { return ++count < a.min_pts; });
  a.core[p] = count >= a.min_pts;
  a.parent[p] = (int)p;
}

// Root of x: parents always point to smaller indices, so the walk ends.
// Inside the union kernel other SMs relink roots concurrently: the loads go
// to L2 (ld.global.cg), where every compare-and-swap lands, never to a stale
// L1 line.  Path halving on the way (each visited node is pointed at its
// grandparent, which is still one of its ancestors; a node that is not a
// root never becomes one again, and links only ever touch roots) keeps the
// trees shallow.
__device__ __forceinline__ int uf_find(int* parent, int x) {
  int p = __ldcg(&parent[x]);
  while (p != x) {
    const int gp = __ldcg(&parent[p]);
    if (gp != p) __stcg(&parent[x], gp);
    x = gp;
    p = __ldcg(&parent[x]);
  }
  return x;
}

// Joins every core point with its lower-index core neighbours.  rp is p's
// root as last seen: always an ancestor of p (roots only ever gain parents),
// so a neighbour whose parent is rp, or whose root is rp, is already in p's
// set.  Otherwise the larger of the two roots is linked under the smaller; a
// failed compare-and-swap (another thread linked it first) refreshes both.
__global__ void k_union(ClusterArgs a) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n || !a.core[p]) return;
  int rp = uf_find(a.parent, (int)p);
  for_neighbours(a, p, [&](int q) {
    if (q >= p || !a.core[q]) return true;
    int rq = __ldcg(&a.parent[q]);
    if (rq == rp) return true;
    rq = uf_find(a.parent, rq);
    for (int tries = 0; rq != rp; ++tries) {
      if (tries >= kUnionRetries) {
        atomicExch(a.err, 1);
        return false;
      }
      const int hi = rq > rp ? rq : rp, lo = rq > rp ? rp : rq;
      if (atomicCAS(&a.parent[hi], hi, lo) == hi) {
        rp = lo;
        break;
      }
      rp = uf_find(a.parent, rp);
      rq = uf_find(a.parent, rq);
    }
    return true;
  });
}

// Core points: root = the component's smallest core index; border points:
// the root of their lowest-index core neighbour; noise: -1.
__global__ void k_roots(ClusterArgs a, int* root) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  if (a.core[p]) {
    root[p] = uf_find(a.parent, (int)p);
    return;
  }
  int best = 0x7fffffff;
  for_neighbours(a, p, [&](int q) {
    if (a.core[q] && q < best) best = q;
    return true;
  });
  root[p] = best == 0x7fffffff ? -1 : best;  // resolved to its root in k_label
}

// ---- device-wide exclusive scan of root flags (cluster numbering) ----------------
__global__ void k_scan_blocks(const ClusterArgs a, const int* root, int* flag_scan, int* block_sum) {
  __shared__ int s[kCT];
  const int64_t i = (int64_t)blockIdx.x * kCT + threadIdx.x;
  const int v = (i < a.n && a.core[i] && root[i] == (int)i) ? 1 : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int d = 1; d < kCT; d <<= 1) {
    const int t = threadIdx.x >= d ? s[threadIdx.x - d] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < a.n) flag_scan[i] = s[threadIdx.x] - v;  // exclusive within the block
  if (threadIdx.x == kCT - 1) block_sum[blockIdx.x] = s[kCT - 1];
}

// One block: exclusive scan of the block sums (nb <= kCT * kSumsPerThread).
constexpr int kSumsPerThread = 64;
__global__ void k_scan_sums(int* block_sum, int nb, int* total) {
  __shared__ int s[kCT];
  int loc[kSumsPerThread];
  int run = 0;
  for (int k = 0; k < kSumsPerThread; ++k) {
    const int idx = threadIdx.x * kSumsPerThread + k;
    loc[k] = idx < nb ? block_sum[idx] : 0;
    run += loc[k];
  }
  s[threadIdx.x] = run;
  __syncthreads();
  for (int d = 1; d < kCT; d <<= 1) {
    const int t = threadIdx.x >= d ? s[threadIdx.x - d] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  int base = s[threadIdx.x] - run;
  for (int k = 0; k < kSumsPerThread; ++k) {
    const int idx = threadIdx.x * kSumsPerThread + k;
    if (idx < nb) block_sum[idx] = base;
    base += loc[k];
  }
  if (threadIdx.x == kCT - 1) *total = s[kCT - 1];
}

// labels and the sort keys (cluster << 32 | index; noise sorts last)
__global__ void k_label(ClusterArgs a, const int* root, const int* flag_scan, const int* block_sum, int* labels,
                        unsigned long long* keys, int64_t n_pad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  if (i >= a.n) {
    keys[i] = ~0ull;
    return;
  }
  int lab = -1;
  int r = root[i];
  if (r >= 0) {
    if (!a.core[i]) r = root[r];  // a border point's core neighbour -> its root
    lab = flag_scan[r] + block_sum[r / kCT];
  }
  labels[i] = lab;
  keys[i] = ((unsigned long long)(uint32_t)(lab >= 0 ? lab : 0x7fffffff) << 32) | (unsigned long long)i;
}

__global__ void k_bitonic(unsigned long long* keys, int64_t n_pad, int64_t j, int64_t k) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  const int64_t l = i ^ j;
  if (l <= i) return;
  const unsigned long long x = keys[i], y = keys[l];
  const bool up = (i & k) == 0;
  if ((x > y) == up) {
    keys[i] = y;
    keys[l] = x;
  }
}

__global__ void k_csr(const unsigned long long* keys, int64_t n, int n_clustered, int* perm, int* offsets,
                      int n_clusters) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_clustered) {
    if (j == n_clustered) offsets[n_clusters] = n_clustered;
    return;
  }
  const unsigned long long kj = keys[j];
  const int c = (int)(kj >> 32);
  perm[j] = (int)(kj & 0xffffffffull);
  if (j == 0 || (int)(keys[j - 1] >> 32) != c) offsets[c] = (int)j;
  (void)n;
}

__global__ void k_count_noise(const int* labels, int64_t n, int* noise) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool nz = i < n && labels[i] < 0;
  const unsigned b = __ballot_sync(0xffffffffu, nz);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(noise, __popc(b));
}

__global__ void k_gather(const int* perm, int64_t m, const float* s0, float* d0, const float* s1, float* d1,
                         const float* s2, float* d2) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int i = perm[j];
  if (s0) d0[j] = s0[i];
  if (s1) d1[j] = s1[i];
  if (s2) d2[j] = s2[i];
}

inline unsigned grid_for(int64_t n) { return (unsigned)((n + kCT - 1) / kCT); }

}  // namespace

size_t cluster_scratch_bytes(int64_t n) {
  int64_t buckets = 1, pad = 1;
  while (buckets < 2 * n) buckets <<= 1;
  while (pad < n) pad <<= 1;
  const int64_t nb = (n + kCT - 1) / kCT;
  // ten sub-buffers, each start rounded up to 256 bytes
  return (size_t)buckets * 4 + (size_t)n * (4 + 16 + 1 + 4 + 4 + 4) + (size_t)nb * 4 + (size_t)pad * 8 + 64 + 10 * 256;
}

int64_t cluster_max_points() { return (int64_t)kCT * kSumsPerThread * kCT; }

cudaError_t launch_cluster(const float* feat, int64_t n, int dim, double eps, int min_pts, void* scratch,
                           int* labels, int* perm, int* offsets, int max_clusters, int* n_clusters_host,
                           int* err_host, cudaStream_t s) {
  int64_t buckets = 1, pad = 1;
  while (buckets < 2 * n) buckets <<= 1;
  while (pad < n) pad <<= 1;
  const int64_t nb = (n + kCT - 1) / kCT;
  char* b = (char*)scratch;
  auto take = [&](size_t bytes) {
    char* p = b;
    b += (bytes + 255) & ~(size_t)255;
    return p;
  };
  unsigned long long* keys = (unsigned long long*)take((size_t)pad * 8);
  int4* cellc = (int4*)take((size_t)n * 16);
  int* head = (int*)take((size_t)buckets * 4);
  int* next = (int*)take((size_t)n * 4);
  int* parent = (int*)take((size_t)n * 4);
  int* root = (int*)take((size_t)n * 4);
  int* flag_scan = (int*)take((size_t)n * 4);
  int* block_sum = (int*)take((size_t)nb * 4);
  uint8_t* core = (uint8_t*)take((size_t)n);
  int* small = (int*)take(64);  // err, total, noise

  ClusterArgs a;
  a.feat = feat;
  a.n = n;
  a.dim = dim;
  a.gdim = dim < 3 ? dim : 3;
  a.eps2 = eps * eps;
  {
    // FP32 certainty thresholds, rounded outward; 0 disables the in-test
    const double lo = a.eps2 * (1.0 - 16.0 * 0x1p-24), hi = a.eps2 * (1.0 + 16.0 * 0x1p-24);
    float l = (float)lo, h = (float)hi;
    if ((double)l > lo) l = nextafterf(l, 0.0f);
    if ((double)h < hi) h = nextafterf(h, __builtin_huge_valf());
    a.in32 = l;
    a.out32 = h;
    if (!(hi < 1e37)) {  // radii beyond FP32 range: every test in FP64
      a.in32 = -1.0f;
      a.out32 = __builtin_huge_valf();
    }
  }
  // cells a little larger than eps: pairs within eps stay in adjacent cells
  // whatever the rounding of the cell coordinates
  a.inv_cell = eps > 0.0 ? 1.0 / (eps * (1.0 + 0x1p-10)) : 1.0;
  a.min_pts = min_pts;
  a.hmask = (uint32_t)(buckets - 1);
  a.head = head;
  a.next = next;
  a.cellc = cellc;
  a.core = core;
  a.parent = parent;
  a.err = small;

  cudaError_t e;
  if ((e = cudaMemsetAsync(head, 0xff, (size_t)buckets * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(small, 0, 64, s)) != cudaSuccess) return e;
  k_grid<<<grid_for(n), kCT, 0, s>>>(a);
  k_core<<<grid_for(n), kCT, 0, s>>>(a);
  k_union<<<grid_for(n), kCT, 0, s>>>(a);
  k_roots<<<grid_for(n), kCT, 0, s>>>(a, root);
  k_scan_blocks<<<(unsigned)nb, kCT, 0, s>>>(a, root, flag_scan, block_sum);
  k_scan_sums<<<1, kCT, 0, s>>>(block_sum, (int)nb, small + 1);
  k_label<<<grid_for(pad), kCT, 0, s>>>(a, root, flag_scan, block_sum, labels, keys, pad);
  for (int64_t k = 2; k <= pad; k <<= 1)
    for (int64_t j = k >> 1; j > 0; j >>= 1) k_bitonic<<<grid_for(pad), kCT, 0, s>>>(keys, pad, j, k);
  k_count_noise<<<grid_for(n), kCT, 0, s>>>(labels, n, small + 2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int h[3] = {0, 0, 0};
  if ((e = cudaMemcpyAsync(h, small, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  *err_host = h[0];
  *n_clusters_host = h[1];
  if (h[0] || h[1] > max_clusters) return cudaSuccess;  // the caller reports it; no CSR written
  const int n_clustered = (int)(n - h[2]);
  k_csr<<<grid_for((int64_t)n_clustered + 1), kCT, 0, s>>>(keys, n, n_clustered, perm, offsets, h[1]);
  return cudaGetLastError();
}

cudaError_t launch_gather(const int* perm, int64_t m, const float* s0, float* d0, const float* s1, float* d1,
                          const float* s2, float* d2, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  k_gather<<<grid_for(m), kCT, 0, s>>>(perm, m, s0, d0, s1, d1, s2, d2);
  return cudaGetLastError();
}

}  // namespace rvh
