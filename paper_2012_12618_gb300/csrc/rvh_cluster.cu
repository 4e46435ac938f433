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
// GPU mapping: the first min(dim, 3) components are cut into cells slightly
// larger than eps, and cells are hashed to buckets by their coordinates
// modulo a power-of-two table (x, y, z bits side by side), so the 3^g cells
// around any cell land in 3^g distinct buckets and x - 1, x, x + 1 in
// consecutive ones.  A counting sort lays the points out bucket by bucket
// (features as float4 next to their original index): a point's candidates
// are then a few contiguous spans.  One thread per sorted point.  Neighbour
// counts look in the point's own bucket first; the points still short of
// min_pts, and the non-core points looking for their lowest-index core
// neighbour, walk alone (batched loads) when their neighbourhood is small
// and with the whole warp (coalesced tiles, ballots) when it is large.  Then
// a lock-free union-find over core-core neighbour pairs on sorted positions:
// a near-neighbour linking pass and a compression first, a root recorded
// per bucket, and a full per-thread pass that skips buckets already in the
// point's set; it links the larger root under the smaller.  An atomic
// minimum per component gives its smallest core index; a device-wide scan
// numbers the clusters.  The CSR:
// per-cluster counts, offsets by a scan, placement, and a shared-memory sort
// of each cluster's indices (a global bitonic sort of (cluster, index) keys
// when a cluster exceeds one block's capacity).
// Every loop is bounded by the input size; the union retry loop has an
// explicit cap that raises an error flag instead of spinning.
#include <cstdint>
#include <cuda_runtime.h>

#include "rvh_cluster.h"

namespace rvh {

namespace {

constexpr int kCT = 256;                       // threads per block of the clustering kernels
constexpr int kUnionRetries = 1 << 20;         // cap on one union's compare-and-swap retries
constexpr int kSumsPerThread = 64;             // block sums per thread of the one-block scan
constexpr int kBT = 1024;                      // threads of the shared-memory bitonic kernels
constexpr int kBE = 2 * kBT;                   // keys per block of those kernels

struct ClusterArgs {
  const float* feat;   // [n * dim] caller's features
  int64_t n;
  double eps2;         // eps^2 (FP64)
  float in32, out32;   // FP32 prefilter: d2_32 <= in32 certainly a neighbour, > out32 certainly not
  double inv_cell;     // 1 / cell size
  int min_pts;
  uint32_t xmask, ymask, zmask;  // table bits per gridded component (each >= 2 bits)
  int ysh, zsh;                  // bucket = x | y << ysh | z << zsh
  int* count;          // [buckets] points per bucket
  int* start;          // [buckets + 1] first sorted position of each bucket
  int2* bslot;         // [n] (bucket, slot within the bucket) of each point
  float4* sfeat;       // [n] features in sorted order, zero-padded to four
  int* sidx;           // [n] original index of each sorted position
  uint8_t* score;      // [n] core flag by sorted position
  uint8_t* core;       // [n] core flag by original index
  int* parent;         // [n] union-find over sorted positions
  int* cmin;           // [n] by root position: the component's smallest original core index
  int* broot;          // [buckets] root shared by a bucket's core points, -1 mixed, kNoCore none
  int* err;            // error flag
};

__device__ __forceinline__ int cell_coord(float v, double inv_cell) {
  const double c = floor((double)v * inv_cell);
  // far-out (or non-finite) values share the edge cells: still exact, only slower
  return c >= 1073741823.0 ? 1073741823 : (c <= -1073741823.0 ? -1073741823 : (c == c ? (int)c : 0));
}

__device__ __forceinline__ uint32_t row_bucket(const ClusterArgs& a, int y, int z) {
  return (((uint32_t)y & a.ymask) << a.ysh) | (((uint32_t)z & a.zmask) << a.zsh);
}

template <int DIM>
__device__ __forceinline__ float4 load_feat(const float* f) {
  return make_float4(f[0], DIM > 1 ? f[1] : 0.0f, DIM > 2 ? f[2] : 0.0f, DIM > 3 ? f[3] : 0.0f);
}

template <int DIM>
__device__ __forceinline__ float comp(const float4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// The neighbour test.  An FP32 squared distance (differences and squares of
// FP32 values, accumulated with fmaf) is within 8u relative of the exact one
// for up to four components, and the FP64 one within 6 x 2^-53; outside
// eps^2 (1 -+ 16u) the FP32 value decides alike, inside that band (and for
// tiny values, where underflow voids the relative bound) the FP64 sum of
// squared differences, accumulated over the components in order, decides.
template <int DIM>
__device__ __forceinline__ bool is_neighbour(const ClusterArgs& a, const float4& fp, const float4& fq) {
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const float d = comp<DIM>(fp, k) - comp<DIM>(fq, k);
    s = fmaf(d, d, s);
  }
  if (s > a.out32) return false;  // also +inf
  if (s <= a.in32 && s >= 0x1p-100f) return true;
  double s64 = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const double d = (double)comp<DIM>(fp, k) - (double)comp<DIM>(fq, k);
    s64 = s64 + d * d;
  }
  return s64 <= a.eps2;  // NaN: false
}

struct Cell {
  int x, y, z;
};

template <int DIM>
__device__ __forceinline__ Cell cell_of(const ClusterArgs& a, const float4& f) {
  constexpr int G = DIM < 3 ? DIM : 3;
  return Cell{cell_coord(f.x, a.inv_cell), G > 1 ? cell_coord(f.y, a.inv_cell) : 0,
              G > 2 ? cell_coord(f.z, a.inv_cell) : 0};
}

__device__ __forceinline__ uint32_t bucket_of(const ClusterArgs& a, const Cell& c) {
  return row_bucket(a, c.y, c.z) | ((uint32_t)c.x & a.xmask);
}

// Calls span(begin, end) for the sorted-position ranges, cut at limit, that
// hold the points of the 3^g cells around cell c, until span returns false.
// The ranges depend only on c's bucket, and each point lies in at most one:
// the cells' buckets are distinct.  Returns false when span stopped the walk.
template <int DIM, typename Span>
__device__ __forceinline__ bool for_spans(const ClusterArgs& a, const Cell& c, int limit, Span span) {
  constexpr int G = DIM < 3 ? DIM : 3;
  constexpr int RY = G > 1 ? 1 : 0, RZ = G > 2 ? 1 : 0;
  // the cell's own row first (the early exit of the neighbour count comes sooner)
  for (int iz = 0; iz <= 2 * RZ; ++iz)
    for (int iy = 0; iy <= 2 * RY; ++iy) {
      const int dz = iz == 2 ? -1 : iz, dy = iy == 2 ? -1 : iy;
      const uint32_t row = row_bucket(a, c.y + dy, c.z + dz);
      const uint32_t bx = (uint32_t)(c.x - 1) & a.xmask;
      if (bx + 2 <= a.xmask) {  // x - 1 .. x + 1 without wrap: one range of three buckets
        if (!span(a.start[row + bx], min(a.start[row + bx + 3], limit))) return false;
      } else {
        for (int dx = -1; dx <= 1; ++dx) {
          const uint32_t b = row + ((uint32_t)(c.x + dx) & a.xmask);
          if (!span(a.start[b], min(a.start[b + 1], limit))) return false;
        }
      }
    }
  return true;
}

// One thread walks its candidates kChunk at a time: chunk(t0, end) handles
// positions t0 .. min(t0 + kChunk, end) - 1, issuing their loads together.
constexpr int kChunk = 8;
constexpr int kNoCore = (int)0xfefefefe;  // bucket root before any core point (memset pattern 0xfe)
constexpr int kOwnCap = 64;  // own-bucket candidates a thread counts before the full walk
template <int DIM, typename Chunk>
__device__ __forceinline__ bool for_chunks(const ClusterArgs& a, const Cell& c, int limit, Chunk chunk) {
  return for_spans<DIM>(a, c, limit, [&](int b, int e) {
    for (int t0 = b; t0 < e; t0 += kChunk)
      if (!chunk(t0, e)) return false;
    return true;
  });
}

// Calls bucket(b) for the 3^g distinct buckets around cell c, the cell's own
// row first, until bucket returns false.
template <int DIM, typename Bucket>
__device__ __forceinline__ bool for_buckets(const ClusterArgs& a, const Cell& c, Bucket bucket) {
  constexpr int G = DIM < 3 ? DIM : 3;
  constexpr int RY = G > 1 ? 1 : 0, RZ = G > 2 ? 1 : 0;
  for (int iz = 0; iz <= 2 * RZ; ++iz)
    for (int iy = 0; iy <= 2 * RY; ++iy) {
      const int dz = iz == 2 ? -1 : iz, dy = iy == 2 ? -1 : iy;
      const uint32_t row = row_bucket(a, c.y + dy, c.z + dz);
      for (int dx = -1; dx <= 1; ++dx)
        if (!bucket(row + ((uint32_t)(c.x + dx) & a.xmask))) return false;
    }
  return true;
}

// the number of candidates of cell c (the sizes of its ranges)
template <int DIM>
__device__ __forceinline__ int cand_count(const ClusterArgs& a, const Cell& c) {
  int n = 0;
  for_spans<DIM>(a, c, 0x7fffffff, [&](int b, int e) {
    n += e - b;
    return true;
  });
  return n;
}

constexpr int kAloneMax = 64;  // a point with at most this many candidates walks them alone

constexpr unsigned kFull = 0xffffffffu;

// The whole warp walks the candidates of one point (cell cl, warp-uniform)
// kCoopW * 32 at a time: tile(base, end) runs on every lane, lane l taking
// positions base + 32 w + l below end, and returns a warp-uniform decision
// (false ends the walk).  For the few points that need a long walk alone.
constexpr int kCoopW = 4;
template <int DIM, typename Tile>
__device__ __forceinline__ void coop_walk(const ClusterArgs& a, const Cell& cl, Tile tile) {
  for_spans<DIM>(a, cl, 0x7fffffff, [&](int b, int e) {
    for (int base = b; base < e; base += 32 * kCoopW)
      if (!tile(base, e)) return false;
    return true;
  });
}

__device__ __forceinline__ float4 shfl4(const float4& v, int src) {
  return make_float4(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src), __shfl_sync(kFull, v.z, src),
                     __shfl_sync(kFull, v.w, src));
}

__device__ __forceinline__ Cell shfl_cell(const Cell& c, int src) {
  return Cell{__shfl_sync(kFull, c.x, src), __shfl_sync(kFull, c.y, src), __shfl_sync(kFull, c.z, src)};
}

template <int DIM>
__device__ __forceinline__ uint32_t point_bucket(const ClusterArgs& a, const float4& f) {
  return bucket_of(a, cell_of<DIM>(a, f));
}

// bucket and slot of every point (the slot order within a bucket is
// arbitrary; no result depends on it)
template <int DIM>
__global__ void k_grid(ClusterArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const uint32_t b = point_bucket<DIM>(a, load_feat<DIM>(a.feat + i * DIM));
  a.bslot[i] = make_int2((int)b, atomicAdd(&a.count[b], 1));
}

// start[b] = exclusive scan of the counts; start[buckets] = n
__global__ void k_starts(ClusterArgs a, const int* excl, const int* block_sum, int64_t buckets) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < buckets) a.start[b] = excl[b] + block_sum[b / kCT];
  if (b == buckets) a.start[b] = (int)a.n;
}

template <int DIM>
__global__ void k_scatter(ClusterArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int2 bs = a.bslot[i];
  const int pos = a.start[bs.x] + bs.y;
  a.sfeat[pos] = load_feat<DIM>(a.feat + i * DIM);
  a.sidx[pos] = (int)i;
}

// Neighbour counts (stopping at min_pts), one thread per sorted position.
// First each thread counts within its own bucket, which settles the points
// of dense cells (the count only needs to reach min_pts, and a subset of
// the neighbours is enough); the warp then walks the full neighbourhood of
// each point still short of min_pts together, counting by ballots.  Lanes
// past the end take the last point.
template <int DIM>
__global__ void k_core(ClusterArgs a) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  if (s - lane >= a.n) return;  // the whole warp
  const bool live = s < a.n;
  const float4 fp = a.sfeat[live ? s : a.n - 1];
  const Cell c = cell_of<DIM>(a, fp);
  int count = 0;
  if (live) {
    const uint32_t bk = bucket_of(a, c);
    const int b = a.start[bk], e = min(a.start[bk + 1], b + kOwnCap);
    for (int t0 = b; t0 < e && count < a.min_pts; t0 += kChunk) {
      float4 fq[kChunk];
#pragma unroll
      for (int u = 0; u < kChunk; ++u) fq[u] = a.sfeat[min(t0 + u, e - 1)];
#pragma unroll
      for (int u = 0; u < kChunk; ++u)
        if (t0 + u < e && is_neighbour<DIM>(a, fp, fq[u])) ++count;
    }
  }
  const bool need = live && count < a.min_pts;
  const bool alone = need && cand_count<DIM>(a, c) <= kAloneMax;
  if (alone) {  // a sparse neighbourhood: walk it alone
    count = 0;
    for_chunks<DIM>(a, c, 0x7fffffff, [&](int t0, int e) {
      float4 fq[kChunk];
#pragma unroll
      for (int u = 0; u < kChunk; ++u) fq[u] = a.sfeat[min(t0 + u, e - 1)];
#pragma unroll
      for (int u = 0; u < kChunk; ++u)
        if (t0 + u < e && is_neighbour<DIM>(a, fp, fq[u])) ++count;
      return count < a.min_pts;
    });
  }
  for (unsigned big = __ballot_sync(kFull, need && !alone); big; big &= big - 1u) {
    const int l = __ffs(big) - 1;
    const float4 fl = shfl4(fp, l);
    int n_found = 0;  // warp-uniform
    coop_walk<DIM>(a, shfl_cell(c, l), [&](int base, int e) {
      float4 fq[kCoopW];
#pragma unroll
      for (int w = 0; w < kCoopW; ++w) fq[w] = a.sfeat[min(base + 32 * w + lane, e - 1)];
#pragma unroll
      for (int w = 0; w < kCoopW; ++w)
        n_found += __popc(__ballot_sync(kFull, base + 32 * w + lane < e && is_neighbour<DIM>(a, fl, fq[w])));
      return n_found < a.min_pts;
    });
    if (lane == l) count = n_found;
  }
  if (!live) return;
  const bool core = count >= a.min_pts;
  const int p = a.sidx[s];
  a.score[s] = core;
  a.core[p] = core;
  a.parent[s] = (int)s;
  a.cmin[s] = 0x7fffffff;
}

// Root of x: parents always point to smaller positions, so the walk ends.
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

// Joins the sets of a core point (root as last seen: rp) and of a core
// neighbour whose ancestor pt was read at some moment.  rp is always an
// ancestor of the point (roots only ever gain parents), so pt == rp, or a
// common root, means the two already share a set.  Otherwise the larger
// root is linked under the smaller; a failed compare-and-swap (another
// thread linked it first) refreshes both.  False when the retry cap ran out.
__device__ __forceinline__ bool uf_union(const ClusterArgs& a, int& rp, int pt) {
  if (pt == rp) return true;
  int rq = uf_find(a.parent, pt);
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
}

// Joins every core point with its core neighbours at lower sorted positions
// (each core-core pair once), one thread per point, bucket by bucket.  rp is
// the point's root as last seen and alias the last ancestor it merged: both
// stay in its set for good.  A bucket whose core points all had root rb
// after the compression needs no look at all when rb is rp or alias, and
// otherwise only its first core neighbour: one link to rb joins them all.
// A bucket with mixed roots is walked candidate by candidate.
template <int DIM>
__global__ void k_union(ClusterArgs a) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n || !a.score[s]) return;
  const float4 fp = a.sfeat[s];
  int rp = uf_find(a.parent, (int)s);
  int alias = rp;
  for_buckets<DIM>(a, cell_of<DIM>(a, fp), [&](uint32_t b) {
    const int rb = a.broot[b];
    if (rb == kNoCore || rb == rp || rb == alias) return true;
    const int lo = a.start[b], hi = min(a.start[b + 1], (int)s);
    if (rb >= 0) {
      bool found = false;
      for (int t0 = lo; t0 < hi && !found; t0 += kChunk) {
        bool sc[kChunk];
        float4 fq[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          sc[u] = a.score[min(t0 + u, hi - 1)];
          fq[u] = a.sfeat[min(t0 + u, hi - 1)];
        }
#pragma unroll
        for (int u = 0; u < kChunk; ++u)
          if (t0 + u < hi && sc[u] && is_neighbour<DIM>(a, fp, fq[u])) found = true;
      }
      if (found) {
        if (!uf_union(a, rp, rb)) return false;
        alias = rb;
      }
      return true;
    }
    for (int t0 = lo; t0 < hi; t0 += kChunk) {
      bool sc[kChunk];
      int tag[kChunk];
#pragma unroll
      for (int u = 0; u < kChunk; ++u) {
        sc[u] = a.score[min(t0 + u, hi - 1)];
        tag[u] = __ldcg(&a.parent[min(t0 + u, hi - 1)]);
      }
#pragma unroll
      for (int u = 0; u < kChunk; ++u)
        if (t0 + u < hi && sc[u] && tag[u] != rp && tag[u] != alias && is_neighbour<DIM>(a, fp, a.sfeat[t0 + u])) {
          if (!uf_union(a, rp, tag[u])) return false;
          alias = tag[u];
        }
    }
    return true;
  });
}

// A cheap first linking pass (the sampling idea of Afforest, Sutton et al.,
// IPDPS'18): every core point joins the core neighbours among the kNear
// positions just before it, mostly points of its own cell.  After k_compress
// most points of a dense cell share one root, and the full walk of k_union
// then meets pairs whose parent already is the root.  Any subset of the
// core-core edges may be linked early: the components are the same.
constexpr int kNear = 4;
template <int DIM>
__global__ void k_union_near(ClusterArgs a) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n || !a.score[s]) return;
  const float4 fp = a.sfeat[s];
  int rp = uf_find(a.parent, (int)s);
  const int64_t lo = s > kNear ? s - kNear : 0;
  for (int64_t t = s - 1; t >= lo; --t)
    if (a.score[t] && is_neighbour<DIM>(a, fp, a.sfeat[t]))
      if (!uf_union(a, rp, __ldcg(&a.parent[t]))) return;
}

// points every core point's parent at its root (no links meanwhile)
__global__ void k_compress(ClusterArgs a) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n || !a.score[s]) return;
  a.parent[s] = uf_find(a.parent, (int)s);
}

// Per bucket, the root its core points share, or -1 (mixed): each core
// point walks to its root (no links meanwhile; parents read here are all
// ancestors), points its own parent there, and marks its bucket.
template <int DIM>
__global__ void k_bucket_roots(ClusterArgs a) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n || !a.score[s]) return;
  int x = (int)s, p = __ldcg(&a.parent[x]);
  while (p != x) {
    x = p;
    p = __ldcg(&a.parent[x]);
  }
  __stcg(&a.parent[s], x);
  int* slot = &a.broot[point_bucket<DIM>(a, a.sfeat[s])];
  const int old = atomicCAS(slot, kNoCore, x);
  if (old != kNoCore && old != x && old != -1) atomicExch(slot, -1);
}

// the smallest original core index of each component, at its root
__global__ void k_cmin(ClusterArgs a) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n || !a.score[s]) return;
  atomicMin(&a.cmin[uf_find(a.parent, (int)s)], a.sidx[s]);
}

// Core points: root = the component's smallest core index; border points:
// their lowest-index core neighbour (resolved to its root in k_label);
// noise: -1.  Written by original index.  Non-core points are few: the warp
// walks the neighbourhood of each together and takes the minimum.
template <int DIM>
__global__ void k_roots(ClusterArgs a, int* root) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  if (s - lane >= a.n) return;
  const bool live = s < a.n;
  const bool core = live && a.score[s];
  if (core) root[a.sidx[s]] = a.cmin[uf_find(a.parent, (int)s)];
  const bool need = live && !core;
  bool alone = false;
  if (need) {
    const float4 fp = a.sfeat[s];
    const Cell c = cell_of<DIM>(a, fp);
    alone = cand_count<DIM>(a, c) <= kAloneMax;
    if (alone) {  // a sparse neighbourhood: walk it alone
      int best = 0x7fffffff;
      for_chunks<DIM>(a, c, 0x7fffffff, [&](int t0, int e) {
        bool sc[kChunk];
        int q[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          sc[u] = a.score[min(t0 + u, e - 1)];
          q[u] = a.sidx[min(t0 + u, e - 1)];
        }
#pragma unroll
        for (int u = 0; u < kChunk; ++u)
          if (t0 + u < e && sc[u] && q[u] < best && is_neighbour<DIM>(a, fp, a.sfeat[t0 + u])) best = q[u];
        return true;
      });
      root[a.sidx[s]] = best == 0x7fffffff ? -1 : best;
    }
  }
  for (unsigned big = __ballot_sync(kFull, need && !alone); big; big &= big - 1u) {
    const int l = __ffs(big) - 1;
    const int64_t sl = s - lane + l;
    const float4 fl = a.sfeat[sl];
    int best = 0x7fffffff;  // warp-uniform
    coop_walk<DIM>(a, cell_of<DIM>(a, fl), [&](int base, int e) {
      int mine = 0x7fffffff;
#pragma unroll
      for (int w = 0; w < kCoopW; ++w) {
        const int t = base + 32 * w + lane, tc = min(t, e - 1);
        const bool sc = a.score[tc];
        const int q = a.sidx[tc];
        const float4 fq = a.sfeat[tc];
        if (t < e && sc && q < mine && is_neighbour<DIM>(a, fl, fq)) mine = q;
      }
      best = min(best, __reduce_min_sync(kFull, mine));
      return true;
    });
    if (lane == l) root[a.sidx[s]] = best == 0x7fffffff ? -1 : best;
  }
}

// ---- device-wide exclusive scan (bucket starts; cluster numbering) -----------------
struct CountValue {
  const int* count;
  __device__ int operator()(int64_t i) const { return count[i]; }
};
struct RootFlag {  // 1 for the root (smallest core index) of each component
  const uint8_t* core;
  const int* root;
  __device__ int operator()(int64_t i) const { return core[i] && root[i] == (int)i ? 1 : 0; }
};

template <typename Value>
__global__ void k_scan_blocks(Value value, int64_t len, int* excl, int* block_sum) {
  __shared__ int s[kCT];
  const int64_t i = (int64_t)blockIdx.x * kCT + threadIdx.x;
  const int v = i < len ? value(i) : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int d = 1; d < kCT; d <<= 1) {
    const int t = threadIdx.x >= d ? s[threadIdx.x - d] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < len) excl[i] = s[threadIdx.x] - v;  // exclusive within the block
  if (threadIdx.x == kCT - 1) block_sum[blockIdx.x] = s[kCT - 1];
}

// One block: exclusive scan of the block sums (nb <= kCT * kSumsPerThread).
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
  if (threadIdx.x == kCT - 1 && total) *total = s[kCT - 1];
}

// Labels, the points per cluster, the noise count and the sort keys of the
// large-cluster path (cluster << 32 | index; noise sorts last).  One thread
// per sorted position, so the lanes of a warp mostly share a cluster and
// add to its count once.
__global__ void k_label(ClusterArgs a, const int* root, const int* flag_scan, const int* block_sum, int* labels,
                        int* counts, int* noise, unsigned long long* keys, int64_t n_pad) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int lab = -2;  // past the end
  if (s < a.n) {
    const int i = a.sidx[s];
    lab = -1;
    int r = root[i];
    if (r >= 0) {
      if (!a.core[i]) r = root[r];  // a border point's core neighbour -> its root
      lab = flag_scan[r] + block_sum[r / kCT];
    }
    labels[i] = lab;
    keys[i] = ((unsigned long long)(uint32_t)(lab >= 0 ? lab : 0x7fffffff) << 32) | (unsigned long long)i;
  } else if (s < n_pad) {
    keys[s] = ~0ull;
  }
  const unsigned peers = __match_any_sync(kFull, lab);
  const int lane = threadIdx.x & 31;
  if (lab >= 0 && (peers & ((1u << lane) - 1u)) == 0u) atomicAdd(&counts[lab], __popc(peers));
  const unsigned nz = __ballot_sync(kFull, lab == -1);
  if (lane == 0 && nz) atomicAdd(noise, __popc(nz));
}

// the largest cluster (clusters 0 .. *total - 1)
__global__ void k_maxcount(const int* counts, int64_t n, const int* total, int* maxc) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int v = c < n && c < *total ? counts[c] : 0;
  const int m = __reduce_max_sync(kFull, v);
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(maxc, m);
}

// ---- the CSR: clusters placed by offsets, each cluster's indices sorted -----------
__global__ void k_offsets(const int* excl, const int* block_sum, int n_clusters, int n_clustered, int* offsets) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n_clusters) offsets[c] = excl[c] + block_sum[c / kCT];
  if (c == n_clusters) offsets[c] = n_clustered;
}

// places each clustered point in its cluster's range (in no particular
// order: k_segsort orders it); by sorted position, one atomic per cluster
// and warp
__global__ void k_place(const int* sidx, const int* labels, int64_t n, const int* offsets, int* cursor, int* perm) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = s < n ? sidx[s] : -1;
  const int lab = i >= 0 ? labels[i] : -1;
  const unsigned peers = __match_any_sync(kFull, lab);
  const int lane = threadIdx.x & 31, lead = __ffs(peers) - 1;
  int base = 0;
  if (lab >= 0 && lane == lead) base = atomicAdd(&cursor[lab], __popc(peers));
  base = __shfl_sync(kFull, base, lead);
  if (lab >= 0) perm[offsets[lab] + base + __popc(peers & ((1u << lane) - 1u))] = i;
}

constexpr int kSegT = 256;    // threads per cluster of the segment sort
constexpr int kSegMax = 2048;  // largest cluster the segment sort takes

// one block per cluster: bitonic sort of its indices (<= kSegMax) in shared memory
__global__ void __launch_bounds__(kSegT) k_segsort(int* perm, const int* offsets) {
  __shared__ int v[kSegMax];
  const int b = offsets[blockIdx.x], len = offsets[blockIdx.x + 1] - b;
  if (len <= 1) return;  // the whole block
  int p2 = 2;
  while (p2 < len) p2 <<= 1;
  for (int e = threadIdx.x; e < p2; e += kSegT) v[e] = e < len ? perm[b + e] : 0x7fffffff;
  __syncthreads();
  for (int k = 2; k <= p2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < p2 / 2; t += kSegT) {
        const int i = (int)(((t & ~(j - 1)) << 1) | (t & (j - 1))), l = i + j;
        const int x = v[i], y = v[l];
        if ((x > y) == ((i & k) == 0)) {
          v[i] = y;
          v[l] = x;
        }
      }
      __syncthreads();
    }
  for (int e = threadIdx.x; e < len; e += kSegT) perm[b + e] = v[e];
}

// ---- bitonic sort of the keys (n_pad a power of two) -------------------------------
// Step j of stage k compares i and i + j for every i with bit j clear, in
// ascending order where bit k of i is clear; pair number t maps to that i.
__device__ __forceinline__ int64_t pair_low(int64_t t, int64_t j) { return ((t & ~(j - 1)) << 1) | (t & (j - 1)); }

__device__ __forceinline__ void cmp_swap(unsigned long long* v, int64_t i, int64_t l, bool up) {
  const unsigned long long x = v[i], y = v[l];
  if ((x > y) == up) {
    v[i] = y;
    v[l] = x;
  }
}

// steps j = j0 .. 1 of stage k on one block's keys in shared memory
__device__ __forceinline__ void smem_steps(unsigned long long* sk, int64_t base, int len, int j0, int64_t k) {
  for (int j = j0; j > 0; j >>= 1) {
    const int t = threadIdx.x;
    if (2 * t < len) {
      const int i = (int)pair_low(t, j);
      cmp_swap(sk, i, i + j, ((base + i) & k) == 0);
    }
    __syncthreads();
  }
}

// stages k = 2 .. min(kBE, n_pad), each block on its own kBE keys
__global__ void __launch_bounds__(kBT) k_bitonic_block(unsigned long long* keys, int64_t n_pad) {
  __shared__ unsigned long long sk[kBE];
  const int64_t base = (int64_t)blockIdx.x * kBE;
  const int len = n_pad < kBE ? (int)n_pad : kBE;
  for (int e = threadIdx.x; e < len; e += kBT) sk[e] = keys[base + e];
  __syncthreads();
  for (int k = 2; k <= len; k <<= 1) smem_steps(sk, base, len, k >> 1, k);
  for (int e = threadIdx.x; e < len; e += kBT) keys[base + e] = sk[e];
}

// steps j = kBE / 2 .. 1 of a stage k > kBE: pairs stay within a block's keys
__global__ void __launch_bounds__(kBT) k_bitonic_tail(unsigned long long* keys, int64_t k) {
  __shared__ unsigned long long sk[kBE];
  const int64_t base = (int64_t)blockIdx.x * kBE;
  for (int e = threadIdx.x; e < kBE; e += kBT) sk[e] = keys[base + e];
  __syncthreads();
  smem_steps(sk, base, kBE, kBE / 2, k);
  for (int e = threadIdx.x; e < kBE; e += kBT) keys[base + e] = sk[e];
}

// one step j >= kBE of stage k, one thread per pair
__global__ void k_bitonic_step(unsigned long long* keys, int64_t n_pad, int64_t j, int64_t k) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * t >= n_pad) return;
  const int64_t i = pair_low(t, j);
  cmp_swap(keys, i, i + j, (i & k) == 0);
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

// buckets: a power of two >= 4 n (fewer far cells sharing a bucket), at
// least 64 (two bits or more per gridded component) and at most what the
// one-block scan takes, which is >= n; n_pad: the bitonic length, a power of
// two >= n
constexpr int64_t kMaxBuckets = (int64_t)kCT * kSumsPerThread * kCT;
void table_sizes(int64_t n, int64_t* buckets, int64_t* n_pad) {
  int64_t b = 64, p = 1;
  while (b < 4 * n && b < kMaxBuckets) b <<= 1;
  while (p < n) p <<= 1;
  *buckets = b;
  *n_pad = p;
}

template <int DIM>
cudaError_t launch_grid_phase(ClusterArgs& a, int64_t buckets, int* excl, int* block_sum, int* root,
                              cudaStream_t s) {
  const unsigned nbb = grid_for(buckets);
  k_grid<DIM><<<grid_for(a.n), kCT, 0, s>>>(a);
  k_scan_blocks<<<nbb, kCT, 0, s>>>(CountValue{a.count}, buckets, excl, block_sum);
  k_scan_sums<<<1, kCT, 0, s>>>(block_sum, (int)nbb, nullptr);
  k_starts<<<grid_for(buckets + 1), kCT, 0, s>>>(a, excl, block_sum, buckets);
  k_scatter<DIM><<<grid_for(a.n), kCT, 0, s>>>(a);
  k_core<DIM><<<grid_for(a.n), kCT, 0, s>>>(a);
  k_union_near<DIM><<<grid_for(a.n), kCT, 0, s>>>(a);
  k_compress<<<grid_for(a.n), kCT, 0, s>>>(a);
  // the bucket counts are consumed by now: their memory holds the bucket roots
  const cudaError_t e = cudaMemsetAsync(a.broot, 0xfe, (size_t)buckets * 4, s);
  if (e != cudaSuccess) return e;
  k_bucket_roots<DIM><<<grid_for(a.n), kCT, 0, s>>>(a);
  k_union<DIM><<<grid_for(a.n), kCT, 0, s>>>(a);
  k_cmin<<<grid_for(a.n), kCT, 0, s>>>(a);
  k_roots<DIM><<<grid_for(a.n), kCT, 0, s>>>(a, root);
  return cudaSuccess;
}

}  // namespace

size_t cluster_scratch_bytes(int64_t n) {
  int64_t buckets, pad;
  table_sizes(n, &buckets, &pad);
  const int64_t nbb = (buckets + kCT - 1) / kCT;
  // thirteen sub-buffers, each start rounded up to 256 bytes
  return (size_t)pad * 8 + (size_t)buckets * 12 + 4 + (size_t)nbb * 4 + (size_t)n * (8 + 16 + 4 + 1 + 1 + 4 + 4) +
         64 + 13 * 256;
}

int64_t cluster_max_points() { return (int64_t)kCT * kSumsPerThread * kCT; }

cudaError_t launch_cluster(const float* feat, int64_t n, int dim, double eps, int min_pts, void* scratch,
                           int* labels, int* perm, int* offsets, int max_clusters, int* n_clusters_host,
                           int* err_host, cudaStream_t s) {
  int64_t buckets, pad;
  table_sizes(n, &buckets, &pad);
  const int64_t nbb = (buckets + kCT - 1) / kCT;
  char* b = (char*)scratch;
  auto take = [&](size_t bytes) {
    char* p = b;
    b += (bytes + 255) & ~(size_t)255;
    return p;
  };
  unsigned long long* keys = (unsigned long long*)take((size_t)pad * 8);
  float4* sfeat = (float4*)take((size_t)n * 16);
  int2* bslot = (int2*)take((size_t)n * 8);
  int* count = (int*)take((size_t)buckets * 4);
  int* start = (int*)take((size_t)buckets * 4 + 4);
  // the bucket scan, then the component minima, then the root-flag scan (n <= buckets)
  int* excl = (int*)take((size_t)buckets * 4);
  int* block_sum = (int*)take((size_t)nbb * 4);
  int* sidx = (int*)take((size_t)n * 4);
  int* parent = (int*)take((size_t)n * 4);
  int* root = (int*)take((size_t)n * 4);
  uint8_t* score = (uint8_t*)take((size_t)n);
  uint8_t* core = (uint8_t*)take((size_t)n);
  int* small = (int*)take(64);  // err, total, noise

  ClusterArgs a;
  a.feat = feat;
  a.n = n;
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
  {
    int bits = 0;
    while ((int64_t{1} << bits) < buckets) ++bits;
    const int g = dim < 3 ? dim : 3;
    const int lx = (bits + g - 1) / g;
    const int ly = g > 1 ? (bits - lx + g - 2) / (g - 1) : 0;
    const int lz = bits - lx - ly;
    a.xmask = (1u << lx) - 1u;
    a.ymask = (1u << ly) - 1u;
    a.zmask = (1u << lz) - 1u;
    a.ysh = lx;
    a.zsh = lx + ly;
  }
  a.count = count;
  a.start = start;
  a.bslot = bslot;
  a.sfeat = sfeat;
  a.sidx = sidx;
  a.score = score;
  a.core = core;
  a.parent = parent;
  a.cmin = excl;
  a.broot = count;
  a.err = small;

  cudaError_t e;
  if ((e = cudaMemsetAsync(count, 0, (size_t)buckets * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(small, 0, 64, s)) != cudaSuccess) return e;
  switch (dim) {
    case 1: e = launch_grid_phase<1>(a, buckets, excl, block_sum, root, s); break;
    case 2: e = launch_grid_phase<2>(a, buckets, excl, block_sum, root, s); break;
    case 3: e = launch_grid_phase<3>(a, buckets, excl, block_sum, root, s); break;
    case 4: e = launch_grid_phase<4>(a, buckets, excl, block_sum, root, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  // per-cluster counts and placement cursors in the bucket slots (dead after k_scatter)
  int* counts = (int*)bslot;
  int* cursor = counts + n;
  if ((e = cudaMemsetAsync(counts, 0, (size_t)n * 8, s)) != cudaSuccess) return e;
  const int64_t nb = (n + kCT - 1) / kCT;
  k_scan_blocks<<<(unsigned)nb, kCT, 0, s>>>(RootFlag{core, root}, n, excl, block_sum);
  k_scan_sums<<<1, kCT, 0, s>>>(block_sum, (int)nb, small + 1);
  k_label<<<grid_for(pad), kCT, 0, s>>>(a, root, excl, block_sum, labels, counts, small + 2, keys, pad);
  k_maxcount<<<grid_for(n), kCT, 0, s>>>(counts, n, small + 1, small + 3);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int h[4] = {0, 0, 0, 0};  // err, clusters, noise, largest cluster
  if ((e = cudaMemcpyAsync(h, small, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  *err_host = h[0];
  *n_clusters_host = h[1];
  if (h[0] || h[1] > max_clusters) return cudaSuccess;  // the caller reports it; no CSR written
  const int nc = h[1], n_clustered = (int)(n - h[2]);
  if (h[3] <= kSegMax) {
    if (nc > 0) {
      const int64_t nbc = (nc + kCT - 1) / kCT;
      k_scan_blocks<<<(unsigned)nbc, kCT, 0, s>>>(CountValue{counts}, nc, excl, block_sum);
      k_scan_sums<<<1, kCT, 0, s>>>(block_sum, (int)nbc, nullptr);
    }
    k_offsets<<<grid_for((int64_t)nc + 1), kCT, 0, s>>>(excl, block_sum, nc, n_clustered, offsets);
    if (nc > 0) {
      k_place<<<grid_for(n), kCT, 0, s>>>(sidx, labels, n, offsets, cursor, perm);
      k_segsort<<<(unsigned)nc, kSegT, 0, s>>>(perm, offsets);
    }
  } else {  // a cluster too large for one block: sort all (cluster, index) keys
    k_bitonic_block<<<(unsigned)(pad > kBE ? pad / kBE : 1), kBT, 0, s>>>(keys, pad);
    for (int64_t k = 2 * kBE; k <= pad; k <<= 1) {
      for (int64_t j = k >> 1; j >= kBE; j >>= 1) k_bitonic_step<<<grid_for(pad / 2), kCT, 0, s>>>(keys, pad, j, k);
      k_bitonic_tail<<<(unsigned)(pad / kBE), kBT, 0, s>>>(keys, k);
    }
    k_csr<<<grid_for((int64_t)n_clustered + 1), kCT, 0, s>>>(keys, n, n_clustered, perm, offsets, nc);
  }
  return cudaGetLastError();
}

cudaError_t launch_gather(const int* perm, int64_t m, const float* s0, float* d0, const float* s1, float* d1,
                          const float* s2, float* d2, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  k_gather<<<grid_for(m), kCT, 0, s>>>(perm, m, s0, d0, s1, d1, s2, d2);
  return cudaGetLastError();
}

}  // namespace rvh
