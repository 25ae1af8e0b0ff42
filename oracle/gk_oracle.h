/*
 * gk_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-pass-at-a-time FP64 CPU restatement of balanced k-means
 * for geometric partitioning ("Balanced k-means for Parallel Geometric
 * Partitioning", Sections 4.1-4.5, Algorithms 1 and 2, Eq. 1-3).  It exists so
 * that the CUDA library can be checked against something written straight from
 * the paper.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never does.
 *
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Conventions:
 *   - points are n x d row-major FP64 (FP32 inputs are widened exactly by the
 *     caller, except for the Hilbert quantisation, which has an FP32 variant
 *     because its subtraction is done in the input precision);
 *   - weights may be NULL (unit weights);
 *   - block ids are int32 in [0, k).
 */
#ifndef GK_ORACLE_H
#define GK_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes of the oracle's full run (same meaning as the library's). */
#define OR_OK 0
#define OR_INVALID 1
#define OR_NOT_BALANCED 4

typedef struct {
    int32_t max_iter;           /* movement iterations (Algorithm 2 main loop)   */
    int32_t max_balance_iter;   /* balance passes per movement (Algorithm 1)     */
    int32_t final_balance_iter; /* extra balance passes with centers fixed       */
    int32_t erosion;            /* 1: apply influence erosion (Eq. 2-3)          */
    double delta_threshold;     /* absolute; < 0 selects 1e-4 * bbox extent      */
    int32_t threads;            /* OpenMP threads for the per-point argmin only  */
} or_options;

typedef struct {
    int32_t status;
    int32_t iterations;         /* movement phases executed                      */
    int32_t balance_passes;     /* assignment passes executed (all phases)       */
    int32_t converged;          /* 1 if max delta < threshold ended the loop     */
    int32_t balanced;           /* 1 if the returned assignment meets the bound  */
    double max_imbalance;       /* max_c S_c / ceil(W/k) - 1                      */
    double max_delta;           /* max center movement of the last movement      */
    double delta_threshold;     /* the absolute threshold used                   */
} or_result;

int64_t or_version(void);

/* Axis-aligned bounding box (the "bb" of Algorithm 1; Section 4.4). */
void or_bbox(const double *x, int64_t n, int d, double *lo, double *hi);

/* Hilbert curve index of one cell q[0..d-1] (each < 2^b) by level-by-level
 * descent (Section 3.1 / Algorithm 2 "sfcIndex").  d in {2,3}, d*b <= 64. */
uint64_t or_hilbert_index(const uint32_t *q, int d, int b);

/* Quantisation of every point to the 2^b grid over its bounding box followed by
 * or_hilbert_index (b = 32 for d = 2, 21 for d = 3).  q_out (nullable) receives
 * the n x d grid cells. */
void or_hilbert_keys_f64(const double *x, int64_t n, int d, uint64_t *keys, uint32_t *q_out);
void or_hilbert_keys_f32(const float *x, int64_t n, int d, uint64_t *keys, uint32_t *q_out);

/* Stable ascending sort by key: perm[i] = input index of the i-th point. */
void or_sort_keys(const uint64_t *keys, int64_t n, int64_t *perm);

/* Initial centers at ranks i*n/k + n/(2k) of the sorted points (Algorithm 2). */
void or_sfc_centers(const double *x_sorted, int64_t n, int d, int k, double *centers);

/* Effective-distance assignment (Section 4.2; Algorithm 1 inner loop without
 * its accelerations): A[p] = argmin_c dist(p, C_c) / I_c, ties to the lowest c.
 * best/second (nullable) receive the two smallest effective distances. */
void or_assign(const double *x, int64_t n, int d, const double *C, const double *I, int k,
               int32_t *A, double *best, double *second, int threads);

/* Block weights S_c = sum of w_p over A[p] = c (Algorithm 1, block sizes).
 * Returns W = sum of all weights. */
double or_block_weights(const int32_t *A, const double *w, int64_t n, int k, double *S);

/* Balance bound L_max = (1 + eps) * ceil(W / k) (Section 2). */
double or_balance_bound(double W, int k, double eps);

/* Balance test and influence adaptation (Section 4.2, Eq. 1 as read: the
 * influence of an oversized block shrinks).  Returns 1 when max_c S_c <= L_max
 * (I untouched), else 0 after I_c <- I_c * clamp((W/k / S_c)^(1/d), 0.95, 1.05).
 * imbalance (nullable) receives max_c S_c / ceil(W/k) - 1. */
int or_balance_update(const double *S, double W, int k, int d, double eps, double *I,
                      double *imbalance);

/* Center movement (Algorithm 2): weighted means of the assigned points (empty
 * block: center unchanged), the distance each center moved, and the average
 * block diameter beta (mean over non-empty blocks of the diagonal of the
 * block's bounding box). */
void or_move_centers(const double *x, const double *w, const int32_t *A, int64_t n, int d,
                     int k, const double *C, double *C_new, double *delta, double *beta);

/* Influence erosion (Section 4.2, Eq. 2-3). */
void or_erosion(const double *delta, double beta, int k, double *I);

void or_default_options(or_options *o);

/* Algorithm 2 (with Algorithm 1) on points given in processing order, from the
 * given centers and influence.  On return C holds the centers under which A
 * was computed, I_used the influence under which A was computed, I the
 * influence state after the last update, C_moved (nullable) the last computed
 * weighted means. */
int or_balanced_kmeans(const double *x, const double *w, int64_t n, int d, int k, double eps,
                       const or_options *opt, double *C, double *I, double *I_used,
                       double *C_moved, int32_t *A, or_result *res);

/* The whole partitioner: bounding box, Hilbert keys, stable sort, initial
 * centers, Algorithm 2, and the block ids returned in input order.  x is FP64
 * when is_f32 == 0, else FP32 (passed as const void*). */
int or_partition(const void *x, int is_f32, const double *w, int64_t n, int d, int k, double eps,
                 const or_options *opt, int32_t *A_out, double *C_out, double *I_out,
                 or_result *res);

/* Section 4.5, random initialization: the first rounds of Algorithm 2 on a random
 * sample of the points (round r: the first m0 * 2^r entries of order, a permutation of
 * the input indices, in curve order), then Algorithm 2 on all points.  m0 =
 * or_sample_first(n, k, sample0) (sample0 <= 0: 100 k; at least k; at most n);
 * or_sample_rounds gives the number of sample rounds. */
int64_t or_sample_first(int64_t n, int k, int64_t sample0);
int or_sample_rounds(int64_t n, int64_t m0, int max_iter);
int or_partition_sampled(const void *x, int is_f32, const double *w, int64_t n, int d, int k,
                         double eps, const int64_t *order, int64_t sample0, const or_options *opt,
                         int32_t *A_out, double *C_out, double *I_out, or_result *res);

#ifdef __cplusplus
}
#endif
#endif
