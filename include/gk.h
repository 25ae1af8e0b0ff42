/*
 * gk.h -- C ABI of the GB300 (sm_103a) balanced k-means geometric partitioner.
 *
 * The library implements the data-parallel path of "Balanced k-means for
 * Parallel Geometric Partitioning": the Hilbert space-filling-curve bootstrap
 * (Section 4.1; Algorithm 2, the sfcIndex / sortGlobal / initial-center steps)
 * and the balanced k-means iteration (Section 4.2, Eq. 1-3; Algorithm 1
 * AssignAndBalance; Algorithm 2 BalancedKMeans), as hand-written CUDA kernels
 * for one GPU.
 *
 * Conventions for every entry point:
 *   - coords: n x d row-major (point p's coordinates at coords[p*d .. p*d+d-1]),
 *     element type given by dtype (GK_F32 or GK_F64), d in {2, 3}.
 *   - weights: n values of the same dtype as coords, or NULL for unit weights;
 *     every weight must be finite and > 0 (Section 4: w maps points to R+).
 *   - Every pointer may address host memory or device memory of the current
 *     device; the library looks at each one and stages host buffers through
 *     its workspace (host<->device copies then happen inside the call).
 *   - The caller owns every pointer it passes.  The library keeps a device
 *     workspace that grows on demand and is reused across calls; gk_release()
 *     frees it.
 *   - stream: a cudaStream_t (passed as void*; NULL = legacy default stream).
 *     Work is enqueued on it, and every entry point synchronises it before
 *     returning, so outputs and the returned status are final on return.
 *   - Errors: invalid arguments are reported as GK_ERR_INVALID_ARG before any
 *     kernel launch; a failing CUDA call as GK_ERR_CUDA; an allocation failure
 *     as GK_ERR_OOM.  Outputs are unspecified after an error, except
 *     GK_ERR_NOT_BALANCED, which still returns a valid assignment.
 *   - Not thread-safe: calls must not overlap (one workspace per process).
 */
#ifndef GK_H
#define GK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GK_ABI_VERSION 3

typedef enum gk_status {
    GK_OK = 0,
    GK_ERR_INVALID_ARG = 1,
    GK_ERR_CUDA = 2,
    GK_ERR_OOM = 3,
    GK_ERR_NOT_BALANCED = 4, /* assignment returned, but a block exceeds (1+eps)*ceil(W/k) */
    GK_ERR_TIMEOUT = 5       /* a bounded device-side wait gave up */
} gk_status;

typedef enum gk_dtype { GK_F32 = 0, GK_F64 = 1 } gk_dtype;

/* Tuning parameters of Algorithms 1 and 2 (the paper leaves their values open). */
typedef struct gk_options {
    int32_t max_iter;           /* movement phases of Algorithm 2 (default 50)             */
    int32_t max_balance_iter;   /* assignment passes per phase, Algorithm 1 (default 50)   */
    int32_t final_balance_iter; /* extra passes with centers fixed if still unbalanced
                                   after the last phase (default 500)                     */
    int32_t erosion;            /* 1: influence erosion of Eq. 2-3 after each move (default) */
    double delta_threshold;     /* stop when every center moved less than this (input
                                   units); < 0 selects 1e-4 * largest bounding-box extent */
    int32_t assign_dtype;       /* GK_F64 (default): the assignment is the FP64 argmin of
                                   the effective distance (FP32 search certified by an
                                   error bound, FP64 re-decision of the rest).  GK_F32:
                                   plain FP32 argmin on box-normalised coordinates.       */
    int32_t use_graph;          /* 1 (default): the iteration loop runs as one CUDA graph
                                   with conditional while-nodes; 0: host-driven loop       */
    int32_t timing;             /* 1: with use_graph = 0, time every kernel of the loop with
                                   CUDA events (fills the time_*_ms fields of gk_result)  */
    int32_t bounds;             /* 1: per-point bounds in the spirit of Section 4.3, adapted
                                   to changing influence: while the centers stay fixed, a
                                   point is not evaluated again when its recorded ratio
                                   (other centers' smallest effective distance over its
                                   own) exceeds the largest growth of any center's 1/I^2
                                   over the smallest since then.  Results are identical to
                                   0 (default: every point evaluated every pass); on the
                                   benchmark workloads about a third of the point
                                   evaluations remain, but the bookkeeping makes a pass
                                   slower on this GPU, hence the default.                  */
    int32_t supertile_tiles;    /* tiles of 256 curve-consecutive points per supertile, the
                                   unit of the candidate filter's first level (Section 4.4's
                                   bounding-box pruning) and one warp of it: 16 or 32; 0
                                   (default): chosen by the launch-shape tuner            */
    int32_t assign_ctas_per_sm; /* resident CTAs per SM of the persistent assignment kernel
                                   (4 warps each, a tile of 256 points per warp and stage):
                                   1 .. the kernel's maximum (larger values are clamped);
                                   0 (default): chosen by the tuner                        */
    int32_t hypertiles;         /* the filter's first level per hypertile of 16 supertiles,
                                   each supertile's list then taken from its hypertile's
                                   (same lists, less work for large k): 1 off, 2 on;
                                   0 (default): chosen by the tuner                        */
    int32_t reserved[1];        /* must be zero                                           */
} gk_options;

/* Outcome and counters of one call. */
typedef struct gk_result {
    int32_t status;             /* same value as returned                                  */
    int32_t iterations;         /* movement phases executed                                */
    int32_t balance_passes;     /* assignment passes executed (all phases)                 */
    int32_t converged;          /* 1 if max center movement < threshold ended the loop     */
    int32_t balanced;           /* 1 if the returned assignment meets the balance bound    */
    int32_t reserved0;
    double max_imbalance;       /* max_c S_c / ceil(W/k) - 1 of the returned assignment    */
    double max_delta;           /* largest center movement of the last movement phase      */
    double delta_threshold;     /* absolute threshold used                                 */
    double avg_candidates;      /* mean candidate centers evaluated per point and pass     */
    int64_t rechecked_points;   /* point-passes re-decided in FP64 (GK_F64 assignment)     */
    int64_t kernel_launches;    /* kernels executed by this call (graph nodes included)    */
    double time_bootstrap_ms;   /* device time: bounding box, keys, sort, gather, centers  */
    double time_kmeans_ms;      /* device time: the iteration loop                          */
    double time_total_ms;       /* device time of the whole call                           */
    double time_filter_ms;      /* CUDA-event sums per kernel kind (gk_options.timing = 1) */
    double time_assign_ms;
    double time_balance_ms;
    double time_move_ms;        /* centroid accumulation + finalize                        */
    int64_t filter_launches;
    int64_t assign_launches;
    int64_t balance_launches;
    int64_t move_launches;
    double assign_live_ms;      /* device-clock (globaltimer) sum of the assignment kernel
                                   launches, any mode (graph included)                    */
    int64_t assign_live_launches;
    int64_t evaluated_points;   /* point evaluations over all passes on all points (equal to
                                   n x passes without bounds)                               */
    int32_t supertile_tiles;    /* the launch shapes used (given or tuned)                 */
    int32_t assign_ctas_per_sm;
    int32_t hypertiles;         /* 1 off, 2 on                                             */
    int32_t reserved1;
    double tune_ms;             /* device time the tuner spent measuring (0: shapes given or
                                   taken from its cache)                                   */
} gk_result;

/*
 * Launch-shape tuner.  A field of gk_options left 0 is chosen by measurement: on the first
 * call for a kind of problem (d, input and assignment precision, weights, bounds, and the
 * powers of two of n and k), after the bootstrap, the filter and assignment of the
 * problem's first pass run once per candidate shape (supertiles of 16 or 32 tiles, with
 * and without the hypertile level; the assignment's largest CTA count per SM and the one
 * below it), the state is restored,
 * and the fastest shape is kept in a process-wide cache for later calls of that kind.
 * gk_partition_batched tunes every instance by its own kind.  The shapes change the
 * speed only: every shape gives the same results.
 */

/* Fills *opt with the defaults listed above. */
void gk_default_options(gk_options *opt);

/* Human-readable name of a gk_status value (static string). */
const char *gk_status_string(int32_t status);

/* GK_ABI_VERSION of the loaded library. */
int32_t gk_abi_version(void);

/*
 * Self-check of the library's failure detection (no counterpart in the paper).  Every
 * wait in the library's kernels (the assignment waits on an mbarrier for the bulk copies of
 * its tiles) is bounded: after 2 s of device time (or 2^26 polls) it gives up, records
 * GK_ERR_TIMEOUT, waits (bounded) for its own copies still in flight and returns, so the
 * CUDA context stays usable and the call returns GK_ERR_TIMEOUT.  This call runs one such
 * wait, limited to limit_us microseconds of device time, on an mbarrier that nothing
 * completes (no copy is issued on it), so that the path can be exercised without a fault.
 *   limit_us: 1 .. 10,000,000, else GK_ERR_INVALID_ARG;
 *   waited_us (nullable, host memory): the device time the wait took, in microseconds.
 * Returns GK_ERR_TIMEOUT when the wait gave up (the expected result), GK_OK if it
 * completed, GK_ERR_CUDA on a CUDA error.  Waits for its stream before it returns.
 * Calls whose GPU work overlaps (other streams, other host threads) share one status
 * word in device memory and race on it.
 */
gk_status gk_check_wait_timeout(int64_t limit_us, int64_t *waited_us, void *stream);

/*
 * Hilbert index of every point (Algorithm 2 "sfcIndex"; Section 4.1).
 * Each coordinate is mapped to a 2^b cell grid (b = 32 for d = 2, 21 for
 * d = 3) over the points' bounding box made isotropic with side 2^E, the
 * smallest power of two not below the largest extent; cell =
 * floor((x - lo) * 2^(b-E)) clamped to 2^b - 1, the subtraction done once in
 * the input precision.  The key is the index of that cell on the Hilbert curve
 * of J. Skilling ("Programming the Hilbert curve", 2004), most significant
 * level first, axis 0 first inside a level.
 *   keys_out: n uint64 (host or device), written in input order.
 */
gk_status gk_hilbert_keys(const void *coords, int32_t dtype, int64_t n, int32_t d,
                          uint64_t *keys_out, void *stream);

/*
 * Space-filling-curve bootstrap (Algorithm 2, sfcIndex / sortGlobal / initial
 * centers): keys as gk_hilbert_keys, a stable sort by key (equal keys keep input
 * order), and the initial centers C[i] = sorted point i*n/k + n/(2k).
 *   perm_out:    n int64, perm_out[i] = input index of the i-th point on the curve
 *                (nullable).
 *   centers_out: k x d FP64 in input units (nullable).
 * Requires 1 <= k <= n.
 */
gk_status gk_sfc_init(const void *coords, int32_t dtype, int64_t n, int32_t d, int32_t k,
                      int64_t *perm_out, double *centers_out, void *stream);

/*
 * One assignment pass (Section 4.2; the inner loop of Algorithm 1): every point
 * goes to the center c minimising dist(p, C_c) / influence_c (ties: lowest c),
 * and the block weights S_c = sum of w_p over the points of block c are formed.
 *   centers:   k x d FP64 (input units);  influence: k FP64 > 0.
 *   assign_dtype: GK_F64 (FP64 argmin) or GK_F32 (see gk_options).
 *   block_out: n int32 in input order.  block_weights_out: k FP64 (nullable).
 * Points are processed in the order given; it is fastest on curve-sorted points.
 */
gk_status gk_assign(const void *coords, int32_t dtype, const void *weights, int64_t n, int32_t d,
                    int32_t k, const double *centers, const double *influence,
                    int32_t assign_dtype, int32_t *block_out, double *block_weights_out,
                    void *stream);

/*
 * Center movement (Algorithm 2, the weighted means after AssignAndBalance):
 * centers_out[c] = sum w_p x_p / sum w_p over the points with block[p] = c
 * (an empty block keeps centers[c]); delta_out[c] = distance moved (nullable);
 * *beta_out = mean over non-empty blocks of the diagonal of the block's
 * bounding box, the block diameter used by the erosion of Eq. 2 (nullable).
 *   block: n int32 in [0, k).  centers: k x d FP64.  centers_out: k x d FP64.
 */
gk_status gk_move_centers(const void *coords, int32_t dtype, const void *weights, int64_t n,
                          int32_t d, int32_t k, const int32_t *block, const double *centers,
                          double *centers_out, double *delta_out, double *beta_out,
                          void *stream);

/*
 * Balanced k-means from given centers and influence (Algorithm 2 from its main
 * loop on, with Algorithm 1): repeated assignment passes with the influence
 * update of Eq. 1 (influence *= clamp((W/k / S_c)^(1/d), 0.95, 1.05) while some
 * block exceeds (1+eps)*ceil(W/k)), weighted-mean center movement, the erosion of
 * Eq. 2-3, until the centers move less than the threshold or max_iter phases ran;
 * then, if the assignment is still unbalanced, up to final_balance_iter passes
 * with the centers fixed.
 *   centers_inout:   k x d FP64; in: initial centers; out: the centers the
 *                    returned assignment was computed with.
 *   influence_inout: k FP64; in: initial influence (e.g. all 1); out: the
 *                    influence the returned assignment was computed with.
 *   block_out:       n int32 in input order.
 *   opt: NULL = defaults.  result: nullable.
 * Points are processed in the given order (curve-sorted points are fastest).
 */
gk_status gk_balanced_kmeans(const void *coords, int32_t dtype, const void *weights, int64_t n,
                             int32_t d, int32_t k, double eps, double *centers_inout,
                             double *influence_inout, int32_t *block_out, const gk_options *opt,
                             gk_result *result, void *stream);

/*
 * The whole partitioner (Algorithm 2): Hilbert bootstrap, balanced k-means on
 * the curve-sorted points from the curve centers with influence 1, and one
 * block id per input point.
 *   block_out:     n int32 in input order.
 *   centers_out:   k x d FP64 (nullable): centers of the returned assignment.
 *   influence_out: k FP64 (nullable): influence of the returned assignment.
 */
gk_status gk_partition(const void *coords, int32_t dtype, const void *weights, int64_t n,
                       int32_t d, int32_t k, double eps, const gk_options *opt,
                       int32_t *block_out, double *centers_out, double *influence_out,
                       gk_result *result, void *stream);

/*
 * gk_partition with the random initialization of Section 4.5: the first
 * iterations of Algorithm 2 run on random samples of the points that double
 * after every movement, then Algorithm 2 continues on all points.
 *   order:   n int64 (host or device), a permutation of [0, n): the random order
 *            of the points.  Round r's sample is the points order[0 .. m0*2^r),
 *            taken in curve order; its balance bound is (1+eps)*ceil(W_r/k) with
 *            W_r the sample's total weight; every round moves the centers and
 *            applies the erosion, whatever their movement.
 *   sample0: m0, the first sample's size; <= 0 selects 100*k (the paper's 100
 *            points per process with as many processes as blocks); raised to k,
 *            capped at n.
 * The rounds number ceil(log2(n/m0)), at most max_iter - 1; they count as
 * iterations (result->iterations and ->balance_passes include them) and the
 * iterations on all points are at most max_iter minus the rounds.  An order that
 * is not a permutation gives GK_ERR_INVALID_ARG, found on the device after the
 * bootstrap.  Other arguments and outputs as gk_partition.
 */
gk_status gk_partition_sampled(const void *coords, int32_t dtype, const void *weights, int64_t n,
                               int32_t d, int32_t k, double eps, const int64_t *order,
                               int64_t sample0, const gk_options *opt, int32_t *block_out,
                               double *centers_out, double *influence_out, gk_result *result,
                               void *stream);

/* One problem of a batch (gk_partition_batched). */
typedef struct gk_instance {
    const void *coords;     /* n x d row-major, dtype; device memory                 */
    const void *weights;    /* n values of dtype, or NULL (unit weights); device     */
    int64_t n;
    int32_t d;              /* 2 or 3                                                */
    int32_t dtype;          /* GK_F32 or GK_F64                                      */
    int32_t k;              /* 1 <= k <= n                                           */
    int32_t reserved;       /* must be 0                                             */
    double eps;             /* >= 0                                                  */
    int32_t *block_out;     /* n int32 in input order; device memory                 */
    double *centers_out;    /* k x d FP64, nullable; host or device                  */
    double *influence_out;  /* k FP64, nullable; host or device                      */
} gk_instance;

/*
 * gk_partition for count independent problems of any mix of n, d, dtype and k
 * (Algorithm 2 for each; the paper partitions one point set at a time, so there
 * is no counterpart of the batch itself).  The bootstraps run in turn, then the
 * k-means loops of all problems run as one CUDA graph launch with one chain per
 * problem, so that small problems proceed beside large ones.  Every instance's
 * coords, weights and block_out must be device memory of the current device.
 *   opt: NULL = defaults, shared by all instances.
 *   results: count entries (nullable); results[i].status is instance i's status;
 *            the times are those of the whole batch.
 * Returns GK_OK when every instance succeeded; otherwise GK_ERR_INVALID_ARG
 * (before any launch), GK_ERR_CUDA / GK_ERR_OOM, else GK_ERR_TIMEOUT if an
 * instance timed out, else GK_ERR_NOT_BALANCED if an instance ended unbalanced.
 */
gk_status gk_partition_batched(const gk_instance *inst, int32_t count, const gk_options *opt,
                               gk_result *results, void *stream);

/* Quality of a partition (Section 5 measures). */
typedef struct gk_quality {
    int64_t edge_cut;           /* edges whose ends lie in different blocks                  */
    int64_t total_comm_volume;  /* sum over blocks of comm(V_i)                              */
    int64_t max_comm_volume;    /* max over blocks of comm(V_i)                              */
    int64_t max_ext;            /* max over blocks of ext(V_i)                               */
    int64_t boundary_vertices;  /* vertices with a neighbour in another block                */
} gk_quality;

/*
 * Edge cut and communication volume of a partition of a graph (Section 5): for block
 * V_i, ext(V_i) = edges {u, v} with u in V_i and v outside, and comm(V_i) = sum over
 * v in V_i of the number of blocks other than V_i holding a neighbour of v (the printed
 * definition does not exclude V_i; counting it would add the block's size); the edge
 * cut is sum_i ext(V_i) / 2.
 *   row_ptr: n + 1 int64 offsets into col (row_ptr[0] = 0, row_ptr[n] = nnz);
 *   col:     nnz int32 neighbours in [0, n); every undirected edge stored in both rows
 *            (self-loops are ignored, repeated entries count as parallel edges);
 *   block:   n int32 block ids in [0, k);
 *   ext_out, comm_out: k int64 each (nullable);  quality: nullable.
 * Every pointer may be host or device memory.  Malformed input (row ranges outside
 * [0, nnz], neighbours outside [0, n), block ids outside [0, k)) is found on the device
 * and gives GK_ERR_INVALID_ARG.  Requires 1 <= n < 2^31, nnz >= 0, k >= 1.
 */
gk_status gk_partition_quality(const int64_t *row_ptr, const int32_t *col, int64_t n, int64_t nnz,
                               const int32_t *block, int32_t k, int64_t *ext_out,
                               int64_t *comm_out, gk_quality *quality, void *stream);

/* Block diameters of a partition (Section 5). */
typedef struct gk_diameter {
    int64_t max_diameter;         /* largest bound over the connected blocks (0 if none)       */
    int64_t disconnected_blocks;  /* blocks whose induced subgraph is not connected            */
    int64_t bfs_levels;           /* breadth-first levels run, over all sweeps                 */
    double harmonic_mean;         /* over the blocks of >= 2 vertices, a disconnected block
                                     adding 1/inf = 0 to the sum of reciprocals; +inf if the
                                     sum is 0, 0 if there is no such block                    */
} gk_diameter;

/* Largest number of sweeps gk_block_diameter accepts. */
#define GK_MAX_SWEEPS 64

/*
 * Lower bounds of the block diameters of a partition (Section 5): diam(V_i) is the largest
 * distance between two vertices of V_i in the subgraph V_i induces (infinite when that
 * subgraph is not connected).  The paper evaluates a lower bound from the first rounds of
 * iFUB; this call runs `sweeps` breadth-first searches inside every block (all blocks in
 * parallel), the first from the block's smallest vertex index, each later one from the
 * smallest vertex index at the largest distance of the previous one, and returns the
 * largest eccentricity seen.  Every sweep's eccentricity lies in [diam/2, diam]; on a tree
 * two sweeps give diam exactly.
 *   row_ptr, col, block, n, nnz, k: as for gk_partition_quality;
 *   sweeps:   1 .. GK_MAX_SWEEPS (3 is the usual choice);
 *   diam_out: k int32 (nullable): the bound of each block, -1 for a block that is not
 *             connected, 0 for an empty block;
 *   summary:  nullable.
 * Every pointer may be host or device memory.  The host enqueues 16 breadth-first levels at
 * a time (each reads its frontier's length on the device) and reads the length of the
 * next frontier after them; the call returns with its work done.
 * Malformed input gives GK_ERR_INVALID_ARG (found on the device, before any search).
 * Requires 1 <= n < 2^31, nnz >= 0, k >= 1.
 */
gk_status gk_block_diameter(const int64_t *row_ptr, const int32_t *col, int64_t n, int64_t nnz,
                            const int32_t *block, int32_t k, int32_t sweeps, int32_t *diam_out,
                            gk_diameter *summary, void *stream);

/*
 * Sharded runs: the points split over several processes (one GPU each), as in the
 * paper's distributed design (Section 4.1; Algorithm 2: sortGlobal and the
 * redistribution give each process a contiguous range of the curve-sorted points;
 * centers and influence are replicated; Algorithm 1 globalSumVector and Algorithm 2
 * globalWeightedMeanVector are the only exchanges of the loop).  The caller moves the
 * points between the processes (a splitter-based sample sort on the Hilbert keys and a
 * redistribution into equal ranges); the library computes every step on each shard and
 * calls the caller's reduction wherever the method needs a sum over all shards.
 */
#define GK_REDUCE_SUM 0
#define GK_REDUCE_MIN 1
#define GK_REDUCE_MAX 2
/*
 * The caller's reduction over all shards: replaces buf[0 .. count) (host memory) by the
 * element-wise sum (GK_REDUCE_SUM), minimum or maximum over every shard's buf, as
 * int64; returns 0 on success.  Every shard's call passes the same count and op, in the
 * same order (a collective such as MPI_Allreduce or torch.distributed.all_reduce).
 * The library sends exact integers only: 128-bit fixed-point sums as four 32-bit limbs
 * (no overflow below 2^31 shards) and ordered keys of floating-point values.
 */
typedef int32_t (*gk_reduce_fn)(int64_t *buf, int64_t count, int32_t op, void *ctx);

/*
 * Bounding box of the points (Algorithm 2 sfcIndex needs the box of all points; a shard
 * reduces its box with the other shards' by minimum and maximum).
 *   lo_out, hi_out: d FP64 each, host memory.  Coordinates that are not finite give
 *   GK_ERR_INVALID_ARG.
 */
gk_status gk_bounding_box(const void *coords, int32_t dtype, int64_t n, int32_t d, double *lo_out,
                          double *hi_out, void *stream);

/*
 * gk_hilbert_keys with the bounding box given (lo, hi: d FP64 each, host memory) instead
 * of taken from the points: a shard's keys on the box of all shards' points are the keys
 * the whole point set would get.  Every point must lie inside [lo, hi] (else
 * GK_ERR_INVALID_ARG).  With the points' own box the keys equal gk_hilbert_keys'.
 */
gk_status gk_hilbert_keys_in_box(const void *coords, int32_t dtype, int64_t n, int32_t d,
                                 const double *lo, const double *hi, uint64_t *keys_out,
                                 void *stream);

/*
 * Stable sort of Hilbert keys (Algorithm 2 sortGlobal, the local part): perm_out[i] =
 * index of the i-th smallest key; equal keys keep their order.  The same LSD radix sort
 * as the bootstrap of gk_partition (64 key bits for d = 2, 63 for d = 3).
 *   keys: n uint64 (host or device); perm_out: n int64 (host or device).
 *   1 <= n < 2^32.
 */
gk_status gk_sort_keys(const uint64_t *keys, int64_t n, int32_t d, int64_t *perm_out, void *stream);

/*
 * gk_balanced_kmeans on one shard: this process's points are a contiguous range of the
 * curve-sorted points of a problem of n_global points in all (every shard calls this
 * with its own range, the same k, eps, options and initial centers and influence).
 * Every step runs on the shard's points; the bounding box, the total weight, the block
 * weights of every pass and the coordinate sums and block boxes of every movement go
 * through `reduce` (see gk_reduce_fn), so that every shard takes the same decisions and
 * ends with the same centers and influence.  All sums are exact integers, so the result
 * does not depend on how the points are split: with the FP64 assignment the block ids
 * are those of gk_balanced_kmeans on all points in curve order, bit for bit.  The loop
 * is host-driven (use_graph is ignored).
 *   n_local >= 1, n_global >= n_local, 1 <= k <= n_global; block_out: n_local int32;
 *   other arguments as gk_balanced_kmeans.  A failed reduction gives GK_ERR_CUDA.
 *   An argument error found on one shard before its first reduction leaves the other
 *   shards waiting in theirs: the caller's collective decides how long.
 */
gk_status gk_balanced_kmeans_sharded(const void *coords, int32_t dtype, const void *weights,
                                     int64_t n_local, int64_t n_global, int32_t d, int32_t k,
                                     double eps, double *centers_inout, double *influence_inout,
                                     int32_t *block_out, const gk_options *opt, gk_result *result,
                                     gk_reduce_fn reduce, void *reduce_ctx, void *stream);

/* Frees the device workspace and cached graphs of the current device. */
void gk_release(void);

/*
 * Caller-supplied device memory for the library's workspace (for instance a framework's
 * caching allocator).  alloc(bytes, ctx) returns device memory of the current device,
 * 256-byte aligned (anything else counts as a failed allocation: GK_ERR_OOM), or NULL;
 * free(ptr, bytes, ctx) takes back a block alloc returned.  The library synchronises the
 * device before it calls free.  Passing NULL for both restores cudaMalloc / cudaFree;
 * passing exactly one NULL gives GK_ERR_INVALID_ARG.  The current workspace is released
 * first, to whoever provided it.  The pinned host control block and the scratch of
 * gk_move_centers_noalloc do not come from this allocator.
 */
typedef void *(*gk_alloc_fn)(size_t bytes, void *ctx);
typedef void (*gk_free_fn)(void *ptr, size_t bytes, void *ctx);
gk_status gk_set_allocator(gk_alloc_fn alloc, gk_free_fn free_fn, void *ctx);

/* Largest k accepted by gk_move_centers_noalloc. */
#define GK_NOALLOC_MAX_K 4096

/*
 * gk_move_centers without any memory allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory while
 * they run -- processes whose device memory belongs to their own pool or allocator
 * (a library cudaMalloc could fail there or fragment it) and latency-critical loops
 * that cannot afford the device synchronisation a cudaMalloc/cudaFree may cause.
 * It calls no allocation routine of CUDA or of any other library.
 *
 * Same results as gk_move_centers (exact fixed-point sums, the same diagonal mean).
 * Its scratch is one fixed array of about 450 KB in the library's device memory,
 * held by every GPU that loads the library until the process exits; hence the limit
 * 1 <= k <= GK_NOALLOC_MAX_K (larger k: GK_ERR_INVALID_ARG).  The first call on a
 * device looks up the array's device address (set-up).  Every call reuses the array
 * and clears it first; calls whose GPU work overlaps (other streams, other host
 * threads) race on it.  The call waits for its stream before it returns (it reads the
 * input check and beta back), so it cannot be captured into a CUDA graph.
 *   coords, weights (nullable), block, centers, centers_out, delta_out (nullable):
 *   device memory of the current device; beta_out (nullable): host memory or device
 *   memory of the current device (written by a copy on the stream).
 *   Block ids outside [0, k), a coordinate that is not finite and a weight that is not
 *   finite and > 0 give GK_ERR_INVALID_ARG (found on the device; outputs unspecified).
 */
gk_status gk_move_centers_noalloc(const void *coords, int32_t dtype, const void *weights,
                                  int64_t n, int32_t d, int32_t k, const int32_t *block,
                                  const double *centers, double *centers_out, double *delta_out,
                                  double *beta_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GK_H */
