/*
 * gk_oracle.c -- TEST INFRASTRUCTURE ONLY (see gk_oracle.h).
 *
 * Plain FP64 CPU restatement of the balanced k-means partitioner of
 * "Balanced k-means for Parallel Geometric Partitioning": Hilbert-curve
 * bootstrap (Section 4.1, Algorithm 2), effective-distance assignment and
 * balancing (Section 4.2, Eq. 1, Algorithm 1), center movement and influence
 * erosion (Section 4.2, Eq. 2-3, Algorithm 2).
 *
 * Deliberately naive: every assignment is a brute-force scan over all k
 * centers in FP64 (the bounding-box and Hamerly accelerations of Sections
 * 4.3-4.4 are exact in real arithmetic and therefore left out), every sum is a
 * sequential FP64 loop.  Readings of points the paper leaves open are marked
 * "Reading:" where they are applied.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no FMA contraction,
 * so each FP64 operation is the single IEEE operation written here).
 */
#include "gk_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int64_t or_version(void) { return 1; }

/* ------------------------------------------------------------------------ */
/* Bounding box (Algorithm 1 "bb"; Section 4.4).                             */
/* ------------------------------------------------------------------------ */
void or_bbox(const double *x, int64_t n, int d, double *lo, double *hi) {
    for (int j = 0; j < d; ++j) {
        lo[j] = INFINITY;
        hi[j] = -INFINITY;
    }
    for (int64_t p = 0; p < n; ++p) {
        for (int j = 0; j < d; ++j) {
            double v = x[p * d + j];
            if (v < lo[j]) lo[j] = v;
            if (v > hi[j]) hi[j] = v;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Hilbert curve index (Section 3.1; Algorithm 2 "sfcIndex").                */
/*                                                                          */
/* Reading: the curve is the one of J. Skilling, "Programming the Hilbert     */
/* curve" (AIP Conf. Proc. 707, 2004), with the index digits taken most       */
/* significant level first and, inside a level, axis 0 (x) as the most        */
/* significant bit.  It is computed here by descending the levels of the     */
/* 2^b grid one at a time, carrying the orientation of the current sub-cube   */
/* as a signed axis permutation (slot i reads axis perm[i], mirrored when     */
/* flip[i] is set) plus the running parity that turns the per-level bit       */
/* vector into its Gray-code rank.                                            */
/* ------------------------------------------------------------------------ */
uint64_t or_hilbert_index(const uint32_t *q, int d, int b) {
    int perm[3] = {0, 1, 2};
    int flip[3] = {0, 0, 0};
    int parity_above = 0; /* XOR of the level parities of all coarser levels */
    uint64_t key = 0;
    for (int level = b - 1; level >= 0; --level) {
        int v[3];
        for (int i = 0; i < d; ++i) v[i] = (int)((q[perm[i]] >> level) & 1u) ^ flip[i];
        /* rank of this sub-cube along the curve: Gray-code inverse of v */
        int prefix = 0;
        uint64_t digit = 0;
        for (int i = 0; i < d; ++i) {
            prefix ^= v[i];
            digit = (digit << 1) | (uint64_t)(prefix ^ parity_above);
        }
        parity_above ^= prefix;
        key = (key << d) | digit;
        /* orientation of the chosen sub-cube for the finer levels */
        for (int i = 0; i < d; ++i) {
            if (v[i]) {
                flip[0] ^= 1; /* mirror slot 0 */
            } else {          /* exchange slots 0 and i */
                int tp = perm[0];
                perm[0] = perm[i];
                perm[i] = tp;
                int tf = flip[0];
                flip[0] = flip[i];
                flip[i] = tf;
            }
        }
    }
    return key;
}

static int hilbert_bits(int d) { return d == 2 ? 32 : 21; }

/* Reading (the paper does not define the grid): the box is the points'
 * bounding box, made isotropic with side 2^E, the smallest power of two not
 * below the largest extent s = max_j (hi_j - lo_j).  A coordinate maps to
 * cell floor((x_j - lo_j) * 2^(b - E)), clamped to 2^b - 1, where the
 * subtraction is one IEEE operation in the input precision and the scaling by
 * a power of two is exact. */
static int grid_exponent(double s) {
    if (!(s > 0.0)) return 0;
    int e;
    double f = frexp(s, &e); /* s = f * 2^e, f in [0.5, 1) */
    return (f == 0.5) ? e - 1 : e;
}

static uint32_t quantise(double v, int m, int b) {
    double scaled = ldexp(v, m);
    double top = ldexp(1.0, b);
    if (scaled >= top) return (uint32_t)(top - 1.0);
    return (uint32_t)floor(scaled);
}

void or_hilbert_keys_f64(const double *x, int64_t n, int d, uint64_t *keys, uint32_t *q_out) {
    double lo[3], hi[3];
    or_bbox(x, n, d, lo, hi);
    double s = 0.0;
    for (int j = 0; j < d; ++j)
        if (hi[j] - lo[j] > s) s = hi[j] - lo[j];
    int b = hilbert_bits(d);
    int m = b - grid_exponent(s);
    for (int64_t p = 0; p < n; ++p) {
        uint32_t q[3];
        for (int j = 0; j < d; ++j) {
            double v = x[p * d + j] - lo[j];
            q[j] = quantise(v, m, b);
            if (q_out) q_out[p * d + j] = q[j];
        }
        keys[p] = or_hilbert_index(q, d, b);
    }
}

void or_hilbert_keys_f32(const float *x, int64_t n, int d, uint64_t *keys, uint32_t *q_out) {
    float lo[3], hi[3];
    for (int j = 0; j < d; ++j) {
        lo[j] = INFINITY;
        hi[j] = -INFINITY;
    }
    for (int64_t p = 0; p < n; ++p)
        for (int j = 0; j < d; ++j) {
            float v = x[p * d + j];
            if (v < lo[j]) lo[j] = v;
            if (v > hi[j]) hi[j] = v;
        }
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double e = (double)hi[j] - (double)lo[j];
        if (e > s) s = e;
    }
    int b = hilbert_bits(d);
    int m = b - grid_exponent(s);
    for (int64_t p = 0; p < n; ++p) {
        uint32_t q[3];
        for (int j = 0; j < d; ++j) {
            float v = x[p * d + j] - lo[j]; /* one FP32 subtraction */
            q[j] = quantise((double)v, m, b);
            if (q_out) q_out[p * d + j] = q[j];
        }
        keys[p] = or_hilbert_index(q, d, b);
    }
}

/* ------------------------------------------------------------------------ */
/* Stable sort by key (Algorithm 2 "sortGlobal"; Section 4.1).               */
/* Reading: equal keys keep input order.  Top-down merge sort.               */
/* ------------------------------------------------------------------------ */
static void merge_sort(const uint64_t *keys, int64_t *a, int64_t *tmp, int64_t lo, int64_t hi) {
    if (hi - lo < 2) return;
    int64_t mid = lo + (hi - lo) / 2;
    merge_sort(keys, a, tmp, lo, mid);
    merge_sort(keys, a, tmp, mid, hi);
    int64_t i = lo, j = mid, o = lo;
    while (i < mid && j < hi) {
        if (keys[a[j]] < keys[a[i]])
            tmp[o++] = a[j++];
        else
            tmp[o++] = a[i++]; /* equal keys: left run first -> stable */
    }
    while (i < mid) tmp[o++] = a[i++];
    while (j < hi) tmp[o++] = a[j++];
    memcpy(a + lo, tmp + lo, (size_t)(hi - lo) * sizeof(int64_t));
}

void or_sort_keys(const uint64_t *keys, int64_t n, int64_t *perm) {
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    int64_t *tmp = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    merge_sort(keys, perm, tmp, 0, n);
    free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Initial centers (Algorithm 2): C[i] = sortedPoints[i*n/k + n/2k].         */
/* Reading: 64-bit integer arithmetic, i*n/k + n/(2k).                        */
/* ------------------------------------------------------------------------ */
void or_sfc_centers(const double *x_sorted, int64_t n, int d, int k, double *centers) {
    for (int64_t i = 0; i < k; ++i) {
        int64_t idx = i * n / k + n / (2 * (int64_t)k);
        for (int j = 0; j < d; ++j) centers[i * d + j] = x_sorted[idx * d + j];
    }
}

/* ------------------------------------------------------------------------ */
/* Assignment by effective distance dist(p, C_c) / influence(c)              */
/* (Section 4.2; Algorithm 1).  Brute force over all k centers; the first    */
/* strictly smaller value wins, so ties go to the lowest center index.       */
/* ------------------------------------------------------------------------ */
void or_assign(const double *x, int64_t n, int d, const double *C, const double *I, int k,
               int32_t *A, double *best_out, double *second_out, int threads) {
#ifdef _OPENMP
    int nt = threads > 0 ? threads : 1;
#pragma omp parallel for schedule(static) num_threads(nt)
#endif
    for (int64_t p = 0; p < n; ++p) {
        double best = INFINITY, second = INFINITY;
        int32_t arg = 0;
        for (int c = 0; c < k; ++c) {
            double ss = 0.0;
            for (int j = 0; j < d; ++j) {
                double diff = x[p * d + j] - C[c * d + j];
                ss += diff * diff;
            }
            double eff = sqrt(ss) / I[c];
            if (eff < best) {
                second = best;
                best = eff;
                arg = c;
            } else if (eff < second) {
                second = eff;
            }
        }
        A[p] = arg;
        if (best_out) best_out[p] = best;
        if (second_out) second_out[p] = second;
    }
    (void)threads;
}

/* Block weights (Algorithm 1 "localBlockSizes" + "globalSumVector"). */
double or_block_weights(const int32_t *A, const double *w, int64_t n, int k, double *S) {
    for (int c = 0; c < k; ++c) S[c] = 0.0;
    double W = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        double wp = w ? w[p] : 1.0;
        S[A[p]] += wp;
        W += wp;
    }
    return W;
}

/* Balance constraint of Section 2: |V_i| <= (1 + eps) * ceil(|V| / k).
 * Reading: with weights, |V| is the total weight W and the ceiling is taken
 * of the FP64 quotient. */
double or_balance_bound(double W, int k, double eps) { return (1.0 + eps) * ceil(W / (double)k); }

/* Balance test and influence adaptation (Section 4.2, Eq. 1; Algorithm 1).
 * Reading: gamma(c) = target / current with target = W/k; the influence is
 * multiplied by gamma^(1/d) (so an oversized block, gamma < 1, loses
 * influence, as the text of Section 4.2 requires), and the factor is clamped
 * to [0.95, 1.05] (the 5% limit).  An empty block has gamma = +inf and gets
 * the largest allowed growth.  Balanced means max S <= L_max. */
int or_balance_update(const double *S, double W, int k, int d, double eps, double *I,
                      double *imbalance) {
    double ceil_avg = ceil(W / (double)k);
    double bound = or_balance_bound(W, k, eps);
    double max_s = 0.0;
    for (int c = 0; c < k; ++c)
        if (S[c] > max_s) max_s = S[c];
    if (imbalance) *imbalance = max_s / ceil_avg - 1.0;
    if (max_s <= bound) return 1;
    double target = W / (double)k;
    for (int c = 0; c < k; ++c) {
        double factor;
        if (S[c] > 0.0) {
            double gamma = target / S[c];
            if (d == 2)
                factor = sqrt(gamma);
            else if (d == 3)
                factor = cbrt(gamma);
            else
                factor = pow(gamma, 1.0 / (double)d);
        } else {
            factor = INFINITY;
        }
        if (factor < 0.95) factor = 0.95;
        if (factor > 1.05) factor = 1.05;
        I[c] = I[c] * factor;
    }
    return 0;
}

/* Center movement (Algorithm 2): new center = weighted mean of the block's
 * points; an empty block keeps its center (Reading).  delta_c is the
 * Euclidean distance moved.  beta is the average block diameter used by the
 * erosion; Reading: the diameter of a block is the diagonal of the bounding
 * box of its points, averaged over the non-empty blocks. */
void or_move_centers(const double *x, const double *w, const int32_t *A, int64_t n, int d,
                     int k, const double *C, double *C_new, double *delta, double *beta) {
    double *sw = (double *)calloc((size_t)k, sizeof(double));
    double *sx = (double *)calloc((size_t)k * d, sizeof(double));
    double *blo = (double *)malloc((size_t)k * d * sizeof(double));
    double *bhi = (double *)malloc((size_t)k * d * sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    for (int64_t i = 0; i < (int64_t)k * d; ++i) {
        blo[i] = INFINITY;
        bhi[i] = -INFINITY;
    }
    for (int64_t p = 0; p < n; ++p) {
        int c = A[p];
        double wp = w ? w[p] : 1.0;
        sw[c] += wp;
        cnt[c] += 1;
        for (int j = 0; j < d; ++j) {
            double v = x[p * d + j];
            sx[c * d + j] += wp * v;
            if (v < blo[c * d + j]) blo[c * d + j] = v;
            if (v > bhi[c * d + j]) bhi[c * d + j] = v;
        }
    }
    double diam_sum = 0.0;
    int64_t nonempty = 0;
    for (int c = 0; c < k; ++c) {
        if (cnt[c] == 0) {
            for (int j = 0; j < d; ++j) C_new[c * d + j] = C[c * d + j];
            delta[c] = 0.0;
            continue;
        }
        double dd = 0.0, diag = 0.0;
        for (int j = 0; j < d; ++j) {
            C_new[c * d + j] = sx[c * d + j] / sw[c];
            double m = C_new[c * d + j] - C[c * d + j];
            dd += m * m;
            double e = bhi[c * d + j] - blo[c * d + j];
            diag += e * e;
        }
        delta[c] = sqrt(dd);
        diam_sum += sqrt(diag);
        nonempty += 1;
    }
    *beta = nonempty > 0 ? diam_sum / (double)nonempty : 0.0;
    free(sw);
    free(sx);
    free(blo);
    free(bhi);
    free(cnt);
}

/* Influence erosion (Section 4.2, Eq. 2-3), as printed:
 *   alpha = 2 / (1 + exp(min(-delta/beta, 0))) - 1,
 *   influence <- exp((1 - alpha) * log(influence)).
 * Reading for beta = 0 (every block a single point or a set of equal points):
 * alpha = 1 when the center moved, 0 otherwise. */
void or_erosion(const double *delta, double beta, int k, double *I) {
    for (int c = 0; c < k; ++c) {
        double alpha;
        if (beta > 0.0) {
            double t = -delta[c] / beta;
            if (t > 0.0) t = 0.0;
            alpha = 2.0 / (1.0 + exp(t)) - 1.0;
        } else {
            alpha = delta[c] > 0.0 ? 1.0 : 0.0;
        }
        I[c] = exp((1.0 - alpha) * log(I[c]));
    }
}

void or_default_options(or_options *o) {
    o->max_iter = 50;
    o->max_balance_iter = 50;
    o->final_balance_iter = 500;
    o->erosion = 1;
    o->delta_threshold = -1.0;
    o->threads = 1;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2 with Algorithm 1 inlined.                                     */
/*                                                                          */
/* Reading of the loop bounds: maxIter movement phases, maxBalanceIter       */
/* assignment passes per phase.  The last phase does not move the centers   */
/* (no assignment would follow).  If the final assignment is still outside  */
/* the balance bound, up to final_balance_iter more passes of Algorithm 1   */
/* run with the centers fixed (an extension; the status reports the         */
/* outcome).                                                                */
/* ------------------------------------------------------------------------ */
int or_balanced_kmeans(const double *x, const double *w, int64_t n, int d, int k, double eps,
                       const or_options *opt, double *C, double *I, double *I_used,
                       double *C_moved, int32_t *A, or_result *res) {
    or_options dflt;
    if (!opt) {
        or_default_options(&dflt);
        opt = &dflt;
    }
    memset(res, 0, sizeof(*res));
    if (n < 1 || k < 1 || k > n || (d != 2 && d != 3) || !(eps >= 0.0)) {
        res->status = OR_INVALID;
        return OR_INVALID;
    }
    double lo[3], hi[3];
    or_bbox(x, n, d, lo, hi);
    double extent = 0.0;
    for (int j = 0; j < d; ++j)
        if (hi[j] - lo[j] > extent) extent = hi[j] - lo[j];
    double thr = opt->delta_threshold >= 0.0 ? opt->delta_threshold : 1e-4 * extent;
    res->delta_threshold = thr;

    double *S = (double *)malloc((size_t)k * sizeof(double));
    double *C_new = (double *)malloc((size_t)k * d * sizeof(double));
    double *delta = (double *)malloc((size_t)k * sizeof(double));
    double W = 0.0;
    int balanced = 0;
    double imbalance = 0.0;
    for (int c = 0; c < k; ++c) I_used[c] = I[c];

    for (int it = 0; it < opt->max_iter; ++it) {
        /* Algorithm 1: assign, sum block weights, test, adapt influence */
        for (int bp = 0; bp < opt->max_balance_iter; ++bp) {
            or_assign(x, n, d, C, I, k, A, NULL, NULL, opt->threads);
            W = or_block_weights(A, w, n, k, S);
            res->balance_passes += 1;
            for (int c = 0; c < k; ++c) I_used[c] = I[c];
            balanced = or_balance_update(S, W, k, d, eps, I, &imbalance);
            if (balanced) break;
        }
        /* Algorithm 2: move centers to the weighted means */
        double beta = 0.0;
        or_move_centers(x, w, A, n, d, k, C, C_new, delta, &beta);
        res->iterations += 1;
        double max_delta = 0.0;
        for (int c = 0; c < k; ++c)
            if (delta[c] > max_delta) max_delta = delta[c];
        res->max_delta = max_delta;
        if (C_moved) memcpy(C_moved, C_new, (size_t)k * d * sizeof(double));
        if (max_delta < thr) {
            res->converged = 1;
            break;
        }
        if (it == opt->max_iter - 1) break;
        memcpy(C, C_new, (size_t)k * d * sizeof(double));
        if (opt->erosion) or_erosion(delta, beta, k, I);
    }
    if (!balanced) {
        for (int fp = 0; fp < opt->final_balance_iter; ++fp) {
            or_assign(x, n, d, C, I, k, A, NULL, NULL, opt->threads);
            W = or_block_weights(A, w, n, k, S);
            res->balance_passes += 1;
            for (int c = 0; c < k; ++c) I_used[c] = I[c];
            balanced = or_balance_update(S, W, k, d, eps, I, &imbalance);
            if (balanced) break;
        }
    }
    res->balanced = balanced;
    res->max_imbalance = imbalance;
    res->status = balanced ? OR_OK : OR_NOT_BALANCED;
    free(S);
    free(C_new);
    free(delta);
    return res->status;
}

int or_partition(const void *x, int is_f32, const double *w, int64_t n, int d, int k, double eps,
                 const or_options *opt, int32_t *A_out, double *C_out, double *I_out,
                 or_result *res) {
    memset(res, 0, sizeof(*res));
    if (n < 1 || k < 1 || k > n || (d != 2 && d != 3) || !(eps >= 0.0)) {
        res->status = OR_INVALID;
        return OR_INVALID;
    }
    double *xd = (double *)malloc((size_t)n * d * sizeof(double));
    uint64_t *keys = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    int64_t *perm = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (is_f32) {
        const float *xf = (const float *)x;
        for (int64_t i = 0; i < n * d; ++i) xd[i] = (double)xf[i];
        or_hilbert_keys_f32(xf, n, d, keys, NULL);
    } else {
        memcpy(xd, x, (size_t)n * d * sizeof(double));
        or_hilbert_keys_f64(xd, n, d, keys, NULL);
    }
    or_sort_keys(keys, n, perm);
    double *xs = (double *)malloc((size_t)n * d * sizeof(double));
    double *ws = w ? (double *)malloc((size_t)n * sizeof(double)) : NULL;
    for (int64_t i = 0; i < n; ++i) {
        for (int j = 0; j < d; ++j) xs[i * d + j] = xd[perm[i] * d + j];
        if (ws) ws[i] = w[perm[i]];
    }
    double *I = (double *)malloc((size_t)k * sizeof(double));
    int32_t *As = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    or_sfc_centers(xs, n, d, k, C_out);
    for (int c = 0; c < k; ++c) I[c] = 1.0;
    int st = or_balanced_kmeans(xs, ws, n, d, k, eps, opt, C_out, I, I_out, NULL, As, res);
    for (int64_t i = 0; i < n; ++i) A_out[perm[i]] = As[i];
    free(xd);
    free(keys);
    free(perm);
    free(xs);
    free(ws);
    free(I);
    free(As);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Random initialization (Section 4.5): the first rounds of Algorithm 2 run  */
/* on a random sample of the points that doubles after every round with     */
/* center movement; then Algorithm 2 continues on all points.               */
/*                                                                          */
/* Readings: the random order of the points is an input (order, a           */
/* permutation of the input indices; the sample of a round is its first m   */
/* points, taken in curve order).  The paper's first sample is 100 points   */
/* per process with as many processes as blocks (Section 5), so one         */
/* process holding all points starts from m0 = 100 k (sample0 <= 0), and    */
/* never from fewer than k points; the rounds number ceil(log2(n / m0)),    */
/* the paper's count with n_local = n / k.  The rounds are the first        */
/* iterations of Algorithm 2 (they count towards maxIter; at least one      */
/* iteration on all points remains); a sample round always moves the        */
/* centers (no convergence stop) and applies the erosion; its balance       */
/* bound is that of the sample's own total weight.                          */
/* ------------------------------------------------------------------------ */
int64_t or_sample_first(int64_t n, int k, int64_t sample0) {
    int64_t m0 = sample0 > 0 ? sample0 : 100 * (int64_t)k;
    if (m0 < k) m0 = k;
    return m0 < n ? m0 : n;
}

int or_sample_rounds(int64_t n, int64_t m0, int max_iter) {
    int r = 0;
    while (r < 62 && (m0 << r) < n) ++r;
    if (r > max_iter - 1) r = max_iter - 1;
    return r < 0 ? 0 : r;
}

int or_partition_sampled(const void *x, int is_f32, const double *w, int64_t n, int d, int k,
                         double eps, const int64_t *order, int64_t sample0, const or_options *opt,
                         int32_t *A_out, double *C_out, double *I_out, or_result *res) {
    memset(res, 0, sizeof(*res));
    if (n < 1 || k < 1 || k > n || (d != 2 && d != 3) || !(eps >= 0.0) || !order) {
        res->status = OR_INVALID;
        return OR_INVALID;
    }
    {   /* order must be a permutation of [0, n) */
        unsigned char *seen = (unsigned char *)calloc((size_t)n, 1);
        int bad = 0;
        for (int64_t i = 0; i < n && !bad; ++i) {
            if (order[i] < 0 || order[i] >= n || seen[order[i]])
                bad = 1;
            else
                seen[order[i]] = 1;
        }
        free(seen);
        if (bad) {
            res->status = OR_INVALID;
            return OR_INVALID;
        }
    }
    or_options dflt;
    if (!opt) {
        or_default_options(&dflt);
        opt = &dflt;
    }
    double *xd = (double *)malloc((size_t)n * d * sizeof(double));
    uint64_t *keys = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    int64_t *perm = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (is_f32) {
        const float *xf = (const float *)x;
        for (int64_t i = 0; i < n * d; ++i) xd[i] = (double)xf[i];
        or_hilbert_keys_f32(xf, n, d, keys, NULL);
    } else {
        memcpy(xd, x, (size_t)n * d * sizeof(double));
        or_hilbert_keys_f64(xd, n, d, keys, NULL);
    }
    or_sort_keys(keys, n, perm);
    double *xs = (double *)malloc((size_t)n * d * sizeof(double));
    double *ws = w ? (double *)malloc((size_t)n * sizeof(double)) : NULL;
    int64_t *rank = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        for (int j = 0; j < d; ++j) xs[i * d + j] = xd[perm[i] * d + j];
        if (ws) ws[i] = w[perm[i]];
        rank[perm[i]] = i;
    }
    double *I = (double *)malloc((size_t)k * sizeof(double));
    int32_t *As = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    or_sfc_centers(xs, n, d, k, C_out);
    for (int c = 0; c < k; ++c) I[c] = 1.0;

    const int64_t m0 = or_sample_first(n, k, sample0);
    const int R = or_sample_rounds(n, m0, opt->max_iter);
    unsigned char *mark = (unsigned char *)calloc((size_t)n, 1);
    double *xr = (double *)malloc((size_t)n * d * sizeof(double));
    double *wr = ws ? (double *)malloc((size_t)n * sizeof(double)) : NULL;
    double *S = (double *)malloc((size_t)k * sizeof(double));
    double *C_new = (double *)malloc((size_t)k * d * sizeof(double));
    double *delta = (double *)malloc((size_t)k * sizeof(double));
    int passes = 0;
    for (int r = 0; r < R; ++r) {
        const int64_t m = m0 << r; /* < n: r < R */
        memset(mark, 0, (size_t)n);
        for (int64_t i = 0; i < m; ++i) mark[rank[order[i]]] = 1;
        int64_t j = 0;
        for (int64_t pos = 0; pos < n; ++pos) {
            if (!mark[pos]) continue;
            for (int a = 0; a < d; ++a) xr[j * d + a] = xs[pos * d + a];
            if (wr) wr[j] = ws[pos];
            ++j;
        }
        double imbalance = 0.0;
        for (int bp = 0; bp < opt->max_balance_iter; ++bp) {
            or_assign(xr, j, d, C_out, I, k, As, NULL, NULL, opt->threads);
            const double W = or_block_weights(As, wr, j, k, S);
            passes += 1;
            if (or_balance_update(S, W, k, d, eps, I, &imbalance)) break;
        }
        double beta = 0.0;
        or_move_centers(xr, wr, As, j, d, k, C_out, C_new, delta, &beta);
        memcpy(C_out, C_new, (size_t)k * d * sizeof(double));
        if (opt->erosion) or_erosion(delta, beta, k, I);
    }
    or_options rest = *opt;
    rest.max_iter = opt->max_iter - R;
    int st = or_balanced_kmeans(xs, ws, n, d, k, eps, &rest, C_out, I, I_out, NULL, As, res);
    res->iterations += R;
    res->balance_passes += passes;
    for (int64_t i = 0; i < n; ++i) A_out[perm[i]] = As[i];
    free(xd);
    free(keys);
    free(perm);
    free(xs);
    free(ws);
    free(rank);
    free(I);
    free(As);
    free(mark);
    free(xr);
    free(wr);
    free(S);
    free(C_new);
    free(delta);
    return st;
}
