/*
 * rvh oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU restatement of the per-cluster
 * velocity-profile RANSAC + least-squares refine of Singh, Sil and Sharma,
 * "Parallelized Instantaneous Velocity and Heading Estimation of Objects
 * using Single Imaging Radar" (arXiv 2012.12618):
 *   - Alg. 1 (RANSAC kernel) and the winner rule of Sec. III-A, with the
 *     cosine velocity-profile model of Eq. (LSQ_eq) as the hypothesis model;
 *   - Eq. (LSQ_eq), Eq. (eq:LSQPerCluster) and Alg. 2 for the refine and the
 *     heading.
 *
 * Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * may load or call this library.  The CUDA product path shares no code with
 * it and never calls it.
 *
 * Readings of the paper used here:
 *   - hypotheses are exact minimal-set solves of the cosine model (2 points in
 *     2D, 3 points in 3D), not the line fit in a normalised plane of Alg. 1;
 *   - the residual is the Doppler residual |v_d - a.v| with the test
 *     "|r| <= tau" (Alg. 1 thresholds with "<="), tau a fixed m/s value;
 *   - the minimal sets come from Philox4x32-10 (Salmon et al., SC'11) keyed by
 *     the seed, with counter (hypothesis, cluster, 0, 0), in place of the
 *     host-side random index arrays that Alg. 1 requires;
 *   - ties between trials go to the lowest hypothesis index (Sec. III-A picks
 *     "the" trial with the most inliers and does not say which);
 *   - the pseudo-inverse of Eq. (eq:LSQPerCluster) is computed through the
 *     normal equations, with a fallback to the winning minimal-set velocity
 *     when they are singular or have fewer than k rows;
 *   - the heading is atan2(vy, vx) (Sec. III-B writes arctan(vy/vx));
 *   - optional local optimisation (refine_iterations > 0): the velocity of
 *     Sec. III-B is computed "subsequent to" inlier detection; here that is
 *     repeated: every point of the cluster is re-thresholded against the
 *     current least-squares velocity and the normal equations of the new
 *     inlier set are solved again, until the set stops changing, its system
 *     is singular or short (the last accepted velocity and set then stand),
 *     or the round limit is reached;
 *   - optional adaptive trial count (confidence p in (0, 1)): Sec. III-A
 *     sets max_trials per hardware and cites work on optimal RANSAC; here
 *     trials run in index order in blocks of B, and after each block the
 *     count stops once (1 - eps^k)^m <= 1 - p, where m is the number of
 *     trials run and eps = best count / N the best inlier ratio so far (the
 *     standard bound on the chance that every trial drew an outlier).  The
 *     power is taken by binary exponentiation in a fixed order, so that any
 *     IEEE implementation decides the same way;
 *   - line_model = 1 follows Alg. 1 as printed instead of the cosine model:
 *     each point's (azimuth, Doppler) is normalised per cluster (the paper
 *     does not define normalize(); here min-max scaling to [0, 1]:
 *     x = (t - t_min) * (1 / (t_max - t_min)), 0 when the range is 0), a
 *     trial fits the line y = m x + c through its two seed points (rejected
 *     when they share x), and a point is an inlier when its perpendicular
 *     distance |aa x + bb y + cc| / sqrt(aa^2 + bb^2), aa = -m, bb = 1,
 *     cc = -c, evaluated left to right as printed, is within thresh[cluster];
 *     the threshold is the median absolute deviation of the normalised
 *     Doppler (Eq. eq:MAD prints the mean of signed deviations from the
 *     median, which is not a dispersion; read as med(|y - med(y)|), medians
 *     of even counts the mean of the two middle values).  The refine is
 *     Eq. eq:LSQPerCluster on the winner's inliers as before; when it is
 *     singular the outputs are NaN (a line has no velocity to fall back to).
 */
#ifndef RVH_ORACLE_H
#define RVH_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_TOO_FEW_POINTS 1
#define ORC_ALL_DEGENERATE 2
#define ORC_LSQ_FALLBACK 4

typedef struct {
  int32_t model_dim;      /* 2 or 3 */
  int32_t num_hypotheses; /* H >= 1 */
  double tau;             /* inlier iff |r| <= tau */
  uint64_t seed;
  double cond_eps;        /* minimal set rejected unless |det| >= cond_eps */
  int32_t enumerate;      /* 0: Philox draws; 1: h-th k-subset, lexicographic */
  int32_t refine_iterations; /* >= 0: re-threshold + re-fit rounds after the refine */
  double confidence;      /* 0: all H trials; in (0, 1): adaptive trial count */
  int32_t trial_block;    /* adaptive: trials between stopping checks (B >= 1) */
  int32_t line_model;     /* 1: Alg. 1 as printed (2D only): normalised line fits,
                             perpendicular distance, MAD threshold; tau unused */
  int32_t first_cluster;  /* the frame index of cluster 0 of these arrays: a shard
                             of a frame draws its minimal sets with counter
                             (h, first_cluster + cluster, 0, 0), as the whole frame */
} orc_params;

/* Philox4x32 with 10 rounds: out = Philox(ctr; key). */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The k distinct point indices (k = 2 or 3) of hypothesis h of a cluster of
 * n points; q[0..k-1] in draw order.  Returns 0, or -1 if n < k. */
int oracle_draw(uint64_t seed, int32_t cluster, int32_t h, int32_t n, int32_t k, int32_t* q);

/* Estimate every cluster listed in `subset` (all clusters when subset is NULL).
 * Inputs are FP64 (FP32 data widens exactly).  elevation == NULL means 2D.
 * Per-cluster outputs are written at the cluster's position in the subset
 * (its index when subset is NULL); mask is indexed by global point index and
 * only the points of processed clusters are written.
 * hyp_counts (optional) receives [n_out * H] exact counts (-1 = rejected).
 * fragile (optional) receives 1 for a cluster where some decision that can
 * change the outputs lies within rounding distance of its threshold.
 * trials_used (optional) receives the number of trials run per cluster.
 * threshold (optional) receives the inlier threshold each cluster used: tau,
 * or with line_model the cluster's MAD threshold (NaN for a cluster with
 * fewer than k points, which has none).
 * Returns 0, or -1 on invalid arguments. */
int oracle_estimate(const double* azimuth, const double* elevation, const double* doppler,
                    const int32_t* offsets, int32_t n_clusters,
                    const int32_t* subset, int32_t n_subset, const orc_params* p,
                    double* vx, double* vy, double* vz, double* heading,
                    int32_t* inlier_count, int32_t* best_hypothesis, int32_t* status,
                    uint8_t* mask, int32_t* hyp_counts, uint8_t* fragile, int32_t* trials_used,
                    double* threshold);

/* DBSCAN over n feature vectors of `dim` (1..4) FP64 components (row-major):
 * the clustering stage of Fig. 1 that forms the clusters the estimator takes.
 * labels[n] receives cluster ids 0..n_clusters-1 (numbered in the order of
 * their smallest core-point index) or -1 for noise; core[n] (optional)
 * receives 1 for core points.  Returns 0, or -1 on invalid arguments. */
int oracle_dbscan(const double* feat, int64_t n, int32_t dim, double eps, int32_t min_pts,
                  int32_t* labels, uint8_t* core, int32_t* n_clusters);

#ifdef __cplusplus
}
#endif

#endif
