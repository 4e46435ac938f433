/*
 * rvh.h -- radar velocity and heading: C ABI of the GB300 (sm_103a) library.
 *
 * The library estimates, for every cluster of an imaging-radar point cloud,
 * the rigid-body velocity and heading of the object behind it, following
 * Singh, Sil and Sharma, "Parallelized Instantaneous Velocity and Heading
 * Estimation of Objects using Single Imaging Radar" (arXiv 2012.12618):
 *
 *   1. robust inlier detection by RANSAC (Sec. III-A, Alg. 1), one hypothesis
 *      per trial, "max_trials x N_clusts" trials in parallel (Eq. 4);
 *      the winning trial is the one with the most points within the
 *      threshold, and the frame's inlier mask is the union of the per-cluster
 *      masks (Sec. III-A, last paragraph);
 *   2. the least-squares velocity v_i = A_i^+ v_r,i on the inliers
 *      (Eq. LSQ_eq, Eq. eq:LSQPerCluster, Alg. 2);
 *   3. the heading phi_i of (vx, vy) (Sec. III-B).
 *
 * Readings of the paper fixed by this interface:
 *   - the hypothesis model is Eq. LSQ_eq itself, v_d = vx cos t + vy sin t
 *     (2D), or vx cos t cos e + vy sin t cos e + vz sin e with an elevation e
 *     (3D); a trial solves it exactly on 2 (3) points drawn without
 *     replacement;
 *   - a point is an inlier of a trial iff |v_d - a.v| <= inlier_threshold;
 *   - the random minimal sets come from Philox4x32-10 (Salmon et al., SC'11)
 *     with key (seed low word, seed high word) and counter
 *     (hypothesis, first_cluster + cluster index within the frame, 0, 0); the first index is
 *     floor(w0 * N / 2^32), the second floor(w1 * (N-1) / 2^32) skipping
 *     the first, the third floor(w2 * (N-2) / 2^32) skipping the smaller and
 *     then the larger of the two taken;
 *   - a minimal set is rejected when |det| < cond_eps (its rows are unit
 *     vectors, so |det| <= 1); rejected trials count -1;
 *   - ties in the inlier count go to the lowest hypothesis index;
 *   - the pseudo-inverse is taken through the FP64 normal equations of the
 *     inliers; with fewer than k inliers, or |det(A^T A)| <= 1e-12 trace^k,
 *     the winning minimal-set velocity is returned with RVH_STATUS_LSQ_FALLBACK;
 *   - the heading is atan2(vy, vx) in (-pi, pi].
 * Every inlier decision, count and winner index equals that of an FP64
 * evaluation of the same formulas: scoring runs in FP32 with a rigorous
 * per-trial error bound, and points whose FP32 residual is within the bound
 * of the threshold are re-decided in FP64.
 *
 * Conventions: all functions return an RVH_* code (0 = success) unless noted.
 * No function throws or aborts; no device-side trap or assert is used.
 * Pointers may be host or device memory (detected per pointer); sizes are
 * element counts.
 */
#ifndef RVH_H
#define RVH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------------------- */
#define RVH_OK 0
#define RVH_PENDING 1        /* rvh_poll: the ticket has not completed yet */
#define RVH_EINVAL (-1)      /* invalid argument; nothing was launched */
#define RVH_ENOMEM (-2)      /* the request does not fit the context's memory budget */
#define RVH_EAGAIN (-3)      /* serving: budget or queue full right now; retry later */
#define RVH_ECUDA (-4)       /* a CUDA call failed; rvh_last_error() has the message */
#define RVH_ETIMEDOUT (-5)   /* rvh_wait: the ticket did not complete in time */

/* ---- per-cluster status bits (rvh_result.status) --------------------------------- */
#define RVH_STATUS_TOO_FEW_POINTS 1  /* N < k: no trial possible; outputs NaN, best -1 */
#define RVH_STATUS_ALL_DEGENERATE 2  /* every minimal set failed the conditioning test */
#define RVH_STATUS_LSQ_FALLBACK 4    /* normal equations singular or n_in < k */
#define RVH_STATUS_BAD_OFFSETS 8     /* device-side CSR check failed for this cluster */

typedef struct rvh_ctx rvh_ctx;

/* One radar frame: structure-of-arrays points, grouped into clusters by CSR
 * offsets (the clustering stage of Fig. 1 precedes this library).
 * Cluster i owns points cluster_offsets[i] .. cluster_offsets[i+1]-1.
 * Requirements: cluster_offsets[0] == 0, non-decreasing, and
 * cluster_offsets[n_clusters] == n_points.  Host offsets are checked before
 * any launch (RVH_EINVAL); device offsets are checked per cluster on the
 * device (RVH_STATUS_BAD_OFFSETS, no out-of-range access). */
typedef struct {
  const float* azimuth;            /* [n_points] radians, measured from +x toward +y */
  const float* elevation;          /* [n_points] radians, or NULL for the 2D model */
  const float* doppler;            /* [n_points] m/s, the projected velocity v_r */
  const int32_t* cluster_offsets;  /* [n_clusters + 1] */
  int32_t n_clusters;              /* >= 0 */
  int64_t n_points;                /* >= 0, < 2^31 */
} rvh_frame;

typedef struct {
  int32_t model_dim;         /* 2 or 3; 3 requires elevation != NULL, 2 requires NULL */
  int32_t num_hypotheses;    /* H >= 1: trials per cluster ("max_trials", Eq. 4) */
  double inlier_threshold;   /* tau >= 0, m/s; inlier iff |residual| <= tau */
  uint64_t seed;             /* Philox key */
  double cond_eps;           /* minimal-set rejection; <= 0 selects 1e-4 (2D) / 1e-6 (3D) */
  int32_t first_cluster;     /* cluster i of this frame draws as cluster first_cluster + i
                                (0 normally; a shard of a larger frame passes the index of
                                its first cluster there, so its results equal the whole's) */
  int32_t refine_iterations; /* local-optimisation rounds after the refine, 0 (none) ..
                                RVH_MAX_REFINE_ITERATIONS; see below */
  double confidence;         /* 0: every cluster runs all num_hypotheses trials;
                                in (0, 1): adaptive trial count, see below */
  int32_t trial_block;       /* adaptive: trials between stopping checks, a multiple of 32
                                in [32, 1024]; 0 selects 128.  Ignored when confidence is 0 */
  int32_t hypothesis_model;  /* RVH_MODEL_VELOCITY_PROFILE (0) or RVH_MODEL_PAPER_LINE (1) */
} rvh_params;

/* Hypothesis models.
 * RVH_MODEL_VELOCITY_PROFILE: trials are exact solves of Eq. LSQ_eq on
 *   k = 2 (3) points, inliers |v_d - a.v| <= inlier_threshold (above).
 * RVH_MODEL_PAPER_LINE: Alg. 1 as printed, 2D only.  Each cluster's
 *   (azimuth, Doppler) points are normalised (the paper does not define
 *   normalize(); here min-max scaling to [0, 1], x = (t - t_min) *
 *   (1 / (t_max - t_min)), 0 for an empty range); a trial fits the line
 *   y = m x + c through its two seed points (rejected when they share x);
 *   a point is an inlier when its perpendicular distance |aa x + bb y + cc| /
 *   sqrt(aa^2 + bb^2), aa = -m, bb = 1, cc = -c, evaluated in FP64 left to
 *   right as printed, is at most the cluster's threshold: the median
 *   absolute deviation of the normalised Doppler (Eq. eq:MAD prints the mean
 *   of signed deviations from the median; read as med |y - med y|, the mean
 *   of the two middle values for even counts).  inlier_threshold is unused.
 *   The velocity is the least-squares refine of Eq. eq:LSQPerCluster on the
 *   winner's inliers; when it is singular the velocity and heading are NaN
 *   (RVH_STATUS_LSQ_FALLBACK).  Combines with the adaptive trial count, not
 *   with refine_iterations (RVH_EINVAL). */
#define RVH_MODEL_VELOCITY_PROFILE 0
#define RVH_MODEL_PAPER_LINE 1

/* Adaptive trial count (confidence p > 0).  Sec. III-A tunes max_trials to
 * the hardware and cites work on optimal RANSAC; here each cluster runs its
 * trials in index order in blocks of trial_block, and after a block stops
 * once (1 - eps^k)^m <= 1 - p, where m is the number of trials run and eps
 * the best inlier count so far divided by the cluster's N: the standard
 * bound on the chance that every trial so far drew an outlier.  The power
 * is evaluated by binary exponentiation (lowest bit first), one FP64
 * rounding per operation, so the decision is reproducible.  The winner is
 * the lowest-index trial with the largest count among the trials run;
 * rvh_stats.hypotheses / pair_evals count the trials actually run.  Not
 * supported by rvh_estimate_baseline (RVH_EINVAL). */

/* Local optimisation (refine_iterations > 0).  Sec. III-B computes the
 * velocity "subsequent to" inlier detection; these rounds repeat that step.
 * Each round solves the normal equations of the current inlier set,
 * re-thresholds every point of the cluster against that velocity with the
 * same test |v_d - a.v| <= inlier_threshold (decided exactly as in FP64),
 * and keeps the new set when its normal equations are solvable (at least k
 * rows, |det| > 1e-12 trace^k); a round that changes no point, or whose new
 * set is not solvable (the previous set then stands), ends the loop.
 * inlier_mask, inlier_count and the velocity are those of the final set;
 * best_hypothesis stays the RANSAC winner.  A cluster whose first refine
 * fell back (RVH_STATUS_LSQ_FALLBACK) is left as it is.  Not supported by
 * rvh_estimate_baseline (RVH_EINVAL). */
#define RVH_DEFAULT_TRIAL_BLOCK 128
#define RVH_MAX_REFINE_ITERATIONS 64

/* Caller-owned, caller-sized outputs.  Per-cluster arrays have n_clusters
 * entries, inlier_mask has n_points.  vz may be NULL (it is written with 0
 * for the 2D model when given). */
typedef struct {
  double* vx;                /* m/s, longitudinal (Sec. III-B) */
  double* vy;                /* m/s, lateral */
  double* vz;                /* m/s, vertical (3D model) */
  double* heading;           /* rad, atan2(vy, vx) */
  int32_t* inlier_count;     /* inliers of the winning trial */
  int32_t* best_hypothesis;  /* winning trial index h, -1 if none */
  int32_t* status;           /* RVH_STATUS_* bits */
  uint8_t* inlier_mask;      /* 1 = inlier of its cluster's winning trial */
  double* threshold;         /* optional, NULL: not written.  The inlier threshold
                                each cluster used: tau, or with
                                RVH_MODEL_PAPER_LINE the cluster's MAD threshold
                                in the normalised plane (Eq. eq:MAD as
                                med |y - med y|; NaN for a cluster with fewer
                                than 2 points) */
} rvh_result;

/* Creates a context on CUDA device `device` with its own stream.
 * mem_budget_bytes (0 selects 4 GiB) caps the device memory the context
 * allocates for scratch, staging and serving slots.  *out receives the
 * context, or NULL on failure. */
int rvh_create(rvh_ctx** out, int device, size_t mem_budget_bytes);

/* Waits for the context's work, frees its memory, streams and events.
 * NULL is ignored. */
void rvh_destroy(rvh_ctx* ctx);

/* Estimates one frame with the fused FP32/FP64-band persistent kernel.
 * stream: a cudaStream_t, or NULL for the context's stream.
 * Each input and output may be device memory, page-locked host memory
 * (cudaHostAlloc / cudaHostRegister, mapped for the device) or pageable
 * host memory.  Device buffers are used where they are.  Host inputs are
 * copied into the context's scratch, one bulk copy per array, inside the
 * call.  Page-locked outputs are written in place by the kernels over the
 * CPU-GPU link; pageable outputs are staged in the context's scratch and
 * copied back inside the call.  When every output is device memory the call is stream-ordered: it
 * returns once the work is enqueued, and the results are valid after the
 * stream reaches this point.  When any output is host memory the call
 * returns after the stream has completed, with the results in place.  Host
 * inputs must stay unchanged until the call returns.  A context's scratch is
 * reused across calls; calls on one context are serialised on the device (a
 * later call waits for the previous one).  On a stream that is not being
 * captured, the fused kernel runs as an instantiated CUDA graph, one per
 * kernel instantiation, which every later call replays with its own
 * arguments (frame addresses and sizes may change from call to call;
 * environment RVH_GRAPHS=0 launches plainly instead). */
int rvh_estimate(rvh_ctx* ctx, const rvh_frame* frame, const rvh_params* params,
                 rvh_result* result, void* stream);

/* The same computation and outputs with a plain all-FP64 GPU kernel, one
 * launch per cluster (the baseline the fused kernel is measured against). */
int rvh_estimate_baseline(rvh_ctx* ctx, const rvh_frame* frame, const rvh_params* params,
                          rvh_result* result, void* stream);

/* ---- allocation-free estimate ----------------------------------------------------- */
/* The paper has no counterpart to this entry point.  It is rvh_estimate for
 * callers that may not allocate device memory once they are running: for
 * example real-time perception stacks that forbid any allocation after
 * start-up, or plugins whose host framework owns all device memory.  It needs
 * no context and calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Its scratch (work list, work counter, FP32 and FP64 point rows) and the
 * FP64 row table live in file-scope device arrays of fixed size:
 * RVH_NOALLOC_MAX_CLUSTERS clusters and RVH_NOALLOC_MAX_POINTS points, about
 * 48.5 MiB, which every GPU that loads the library holds until the process
 * exits.  Larger frames are rejected with RVH_EINVAL and a message.
 *
 * The first call on a device sets that device up (device addresses of the
 * arrays, the row table upload, the kernels' shared-memory opt-in), with the
 * device current.  Under CUDA's lazy module loading (the default) that first
 * call is also when the driver commits the arrays' device memory, so make it
 * during start-up, before the caller's no-allocation phase begins and before
 * any stream capture; later calls leave the device's free memory unchanged.
 * All inputs and outputs must be device memory; the call is stream-ordered on
 * `stream` (a cudaStream_t, NULL = the legacy default stream) and returns once
 * the work is enqueued.  Every call shares the arrays, which keep the last
 * call's contents (each call resets the work counter it needs zeroed), so
 * calls that overlap on the GPU race: order them on one stream or with events.
 * Argument checks are rvh_estimate's (plus the limits above and device
 * memory for every array the launch touches), and results equal
 * rvh_estimate's: the same kernels with the same per-frame settings. */
#define RVH_NOALLOC_MAX_POINTS 1048576
#define RVH_NOALLOC_MAX_CLUSTERS 65536
int rvh_estimate_noalloc(const rvh_frame* frame, const rvh_params* params, rvh_result* result, void* stream);

/* ---- clustering stage ------------------------------------------------------------ */
/* The clustering that precedes the estimator in Fig. 1 (the paper names NN,
 * DBSCAN and grid DBSCAN): DBSCAN (Ester, Kriegel, Sander, Xu, KDD'96) over
 * caller-chosen FP32 feature vectors, e.g. point positions.
 *   - q is a neighbour of p (p itself included) when the squared Euclidean
 *     distance of their feature vectors, accumulated in FP64 over the
 *     components in order, is at most eps^2;
 *   - p is a core point when it has at least min_pts neighbours;
 *   - clusters are the connected components of core points under the
 *     neighbour relation, numbered 0.. in the order of their smallest core
 *     point index;
 *   - a non-core point with a core neighbour joins the cluster of its
 *     lowest-index core neighbour (DBSCAN itself leaves this to the visit
 *     order); every other point is noise, label -1.
 * features: [n_points * dim] row-major, dim in 1..4, device memory.
 * labels [n_points], perm [n_points] and offsets [max_clusters + 1]: device
 * memory, caller-owned.  perm lists the clustered points cluster by
 * cluster, each cluster's points in increasing index order (noise omitted);
 * offsets is its CSR: cluster c owns perm[offsets[c] .. offsets[c+1]-1], so
 * offsets[n_clusters] is the number of clustered points.  *n_clusters (host
 * memory) receives the cluster count.  n_points <= 4,194,304.  The call is
 * ordered on `stream` (NULL: the context's stream) and returns after it has
 * completed (it reads the cluster count back).  More than max_clusters
 * clusters: RVH_EINVAL with *n_clusters and labels set, perm and offsets
 * not written.  The context's memory budget covers the scratch: about 38
 * bytes per point, 8 bytes per point rounded up to a power of two, and 12
 * bytes per bucket of the cell table (a power of two >= 4 x n_points, at
 * most 4,194,304 buckets). */
int rvh_cluster(rvh_ctx* ctx, const float* features, int64_t n_points, int32_t dim, double eps, int32_t min_pts,
                int32_t* labels, int32_t* perm, int32_t* offsets, int32_t max_clusters, int32_t* n_clusters,
                void* stream);

/* Gathers up to three FP32 point arrays into cluster order: dst_k[j] =
 * src_k[perm[j]] for j < m (a NULL src_k skips that array).  All pointers
 * device memory; ordered on `stream` (NULL: the context's stream), returns
 * once the work is enqueued.  With perm and offsets from rvh_cluster the
 * gathered azimuth / elevation / Doppler arrays and offsets form the
 * rvh_frame of the clustered points. */
int rvh_gather(rvh_ctx* ctx, const int32_t* perm, int64_t m, const float* src0, float* dst0, const float* src1,
               float* dst1, const float* src2, float* dst2, void* stream);

/* ---- streaming (serving) -------------------------------------------------------- */
/* Queues a frame for continuous batching.  Host inputs are copied into the
 * context's device pool before the call returns; device inputs must stay
 * valid until the ticket completes.  Results are written to the caller's
 * buffers (host or device) when the ticket completes.  RVH_EAGAIN: the pool
 * or queue is full right now.  The frame is estimated with the same
 * per-frame seed and cluster indices as rvh_estimate, so its results do not
 * depend on which other frames share its batch. */
int rvh_submit(rvh_ctx* ctx, const rvh_frame* frame, const rvh_params* params,
               rvh_result* result, uint64_t* ticket);

/* RVH_OK when the ticket has completed (its outputs are written), RVH_PENDING
 * while it has not, RVH_EINVAL for an unknown ticket.  Never blocks. */
int rvh_poll(rvh_ctx* ctx, uint64_t ticket);

/* Blocks until the ticket completes or timeout_us passes (< 0: no limit);
 * RVH_OK or RVH_ETIMEDOUT. */
int rvh_wait(rvh_ctx* ctx, uint64_t ticket, int64_t timeout_us);

/* Message of the last failing call on this thread ("" if none).  ctx may be NULL. */
const char* rvh_last_error(rvh_ctx* ctx);

/* ---- measurement and tuning ------------------------------------------------------ */
typedef struct {
  int64_t hypotheses;          /* trials run: n_clusters x H for the plain method; with an extension
                                  (adaptive count, local optimisation, line model) the kernel's count,
                                  over clusters with N >= k, of the trials actually run */
  int64_t pair_evals;          /* trial x point evaluations (n_points x H, or the kernel's sum of trials x N) */
  int64_t candidates;          /* trials re-scored exactly (upper bound reached the lead) */
  int64_t band_points;         /* point decisions taken in FP64 (inside the error band) */
  int64_t fp64_hypotheses;     /* trials whose conditioning or bound needed FP64 */
  float kernel_ms;             /* device time of the last fused launch (events) */
  int32_t grid;                /* persistent CTAs of the last launch */
  int32_t points_per_warp;     /* schedule of the last launch */
  int32_t hyps_per_lane;
  /* SM cycles summed over CTAs, per stage of the fused kernel: rows,
   * hypotheses (draw + solve + bound), scoring pass, exact re-scoring,
   * winner mask + refine, scheduling/other. */
  int64_t phase_cycles[6];
  int64_t refined_hypotheses;  /* trials whose FP32 solve took one refinement step */
  int64_t graph_replays;       /* rvh_estimate calls that replayed an instantiated CUDA graph of the fused
                                  launch, its kernel node given the call's arguments (new frame addresses,
                                  sizes and schedules replay the same graph) */
  int32_t kernel_launches;     /* the library's kernels launched by the last call (work list + fused) */
  int64_t graph_builds;        /* graphs of the fused launch built by rvh_estimate calls (one per kernel
                                  instantiation: model dimension, with or without the extensions) */
  int64_t serving_steps;       /* serving steps launched by the context's request loop (rvh_submit) */
  int64_t serving_graph_replays; /* serving steps that replayed an instantiated graph (work list + fused
                                    kernel) with that step's batch of frames */
  int64_t pairs_scored;        /* trial x point pairs the scoring pass of the last rvh_estimate evaluated:
                                  pair_evals without pruning, fewer with it (rvh_set_pruning) */
} rvh_stats;

/* Counters of the last rvh_estimate on this context (synchronises its stream). */
int rvh_get_stats(rvh_ctx* ctx, rvh_stats* out);

/* Fixes the scoring schedule: points_per_warp in {1, 8, 32} (lanes over points
 * per trial group) and hyps_per_lane in {4, 8}; 0 restores the automatic
 * choice. */
int rvh_set_schedule(rvh_ctx* ctx, int32_t points_per_warp, int32_t hyps_per_lane);

/* Staged scoring with exact pruning (default on): the scoring pass of a
 * cluster of at least 512 points whose rows fit shared memory (the
 * lanes-over-trials schedule, points_per_warp 1) runs in stages, the first
 * of 128 points and each later one half as long again; after the first,
 * the trial with the highest partial count is
 * counted exactly and leads, and after each stage a trial whose partial
 * count plus the points still to come cannot beat the lead's (count, lower
 * index) key is dropped.  Counts only grow by one per point and the exact
 * count never exceeds the upper-bound count, so no dropped trial can win:
 * every output equals the unpruned pass's (the winner of Sec. III-A over
 * all trials of Alg. 1), with fewer (trial, point) evaluations
 * (rvh_stats.pairs_scored).  enabled: 1 on, 0 off. */
int rvh_set_pruning(rvh_ctx* ctx, int32_t enabled);

/* A scoring schedule and its measured fused-kernel time. */
typedef struct {
  int32_t points_per_warp;
  int32_t hyps_per_lane;
  float kernel_ms;
} rvh_schedule;

/* Autotuner: runs the fused kernel on this frame with every scoring schedule
 * (points_per_warp in {1, 8, 32} x hyps_per_lane in {4, 8}), the schedules
 * taking turns for one untimed and then `reps` timed rounds (CUDA events on
 * the context's stream), and keeps the one with the lowest median time for
 * frames of this model dimension and trial-count bucket (floor(log2) of the
 * trials scored together: H, or the adaptive trial_block); later calls pick
 * it automatically unless
 * rvh_set_schedule fixed one.  `result` receives the frame's outputs.  When
 * the environment variable RVH_TUNE_CACHE names a file, choices are loaded
 * from it by rvh_create (entries keyed by GPU name, SM count, model and
 * bucket) and saved to it here.  *best (may be NULL) receives the choice. */
int rvh_autotune(rvh_ctx* ctx, const rvh_frame* frame, const rvh_params* params, rvh_result* result,
                 int32_t reps, rvh_schedule* best);

#ifdef __cplusplus
}
#endif

#endif /* RVH_H */
