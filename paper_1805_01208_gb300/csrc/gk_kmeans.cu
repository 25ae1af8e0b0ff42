// gk_kmeans.cu -- the balanced k-means iteration (Algorithm 1 AssignAndBalance and the
// movement / erosion steps of Algorithm 2; Section 4.2 Eq. 1-3; Section 4.4).
//
//   init_a/init_b     influence state, center data, totals, loop state
//   filter_kernel     candidate centers per tile from bounding boxes (Section 4.4):
//                     a supertile against all centers, then each tile against the
//                     supertile's list; writes each tile's coefficient table
//   assign_kernel     effective-distance argmin over the tile's candidates + block
//                     weight histogram (Algorithm 1 inner loop, localBlockSizes)
//   balance_kernel    global block weights, balance test, influence update (Eq. 1)
//   centroid_kernel   weighted coordinate sums and block bounding boxes (Algorithm 2)
//   finalize_a/b      new centers, movement, average block diameter, convergence test,
//                     erosion (Eq. 2-3)
//
// Effective distances are compared squared: dist^2 / influence^2 orders the centers
// exactly as dist / influence does.  The k-sized FP64 work (cbrt, divisions, exp, log)
// is spread over ceil(k/32) CTAs; the CTA that finishes last takes the global
// decisions (no grid-wide waiting).  The influence is double-buffered: a pass writes
// the updated influence into the other buffer and the decision flips the buffer index.
#include "gk_common.cuh"
#include "gk_internal.h"

namespace gk {

constexpr float kU = 5.9604644775390625e-8f;  // 2^-24, unit roundoff of FP32
constexpr int kFilterWarps = 8;                   // supertiles per CTA of the filter
constexpr int kFilterThreads = kFilterWarps * 32;
constexpr int kAssignWarps = 8;

__device__ __forceinline__ int exponent_above(double v) {  // smallest e with |v| < 2^e
    if (v == 0.0) return 0;
    int e;
    frexp(fabs(v), &e);
    return e;
}

// Frame coordinates of center c (FP64) split into an FP32 pair hi + lo.
__device__ __forceinline__ void frame_center(const Prob &p, int c, float hi[3], float lo[3]) {
    for (int j = 0; j < 3; ++j) {
        hi[j] = 0.f;
        lo[j] = 0.f;
    }
    for (int j = 0; j < p.d; ++j) {
        double f = (p.C[c * p.d + j] - p.origin[j]) * p.scale;
        hi[j] = __double2float_rn(f);
        lo[j] = __double2float_rn(f - (double)hi[j]);
    }
}

__device__ __forceinline__ float scaled_g32(double g, int gshift) {
    return __double2float_rn(ldexp(g, -gshift));
}

// log2 of a center's g for the per-point bounds (FP32; error far below kLgMargin).  An
// infinite or zero g gives +-inf, which makes every threshold that uses it NaN or infinite,
// so that no point is skipped on it.
constexpr float kLgMargin = 6.103515625e-5f;   // 2^-14: covers the rounding of two log2 values
constexpr float kLqMargin = 2.44140625e-4f;    // 2^-12: that and two fast log2 of the bound
__device__ __forceinline__ float lg_of(double g) { return log2f(__double2float_rn(g)); }

// Record of the group of kGroup consecutive centers handled by this CTA (called by all
// of its threads; lanes without a center pass valid = false): the box of the centers'
// FP32 frame coordinates, rounded outwards and widened by 8 u R (the lo parts and the
// rounding of the tests that use it), and the range of their g32.  A NaN g32 widens
// the range to [0, inf], so the group is never pruned.
__device__ __forceinline__ void write_group(const Prob &p, float4 *gd, bool valid, const float hi[3],
                                            float g32) {
    float mn[3], mx[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        mn[j] = valid ? hi[j] : INFINITY;
        mx[j] = valid ? hi[j] : -INFINITY;
    }
    float gmn = valid ? g32 : INFINITY, gmx = valid ? g32 : 0.0f;
    const bool nan = __any_sync(0xffffffffu, valid && isnan(g32));
    for (int off = 16; off; off >>= 1) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            mn[j] = fminf(mn[j], __shfl_xor_sync(0xffffffffu, mn[j], off));
            mx[j] = fmaxf(mx[j], __shfl_xor_sync(0xffffffffu, mx[j], off));
        }
        gmn = fminf(gmn, __shfl_xor_sync(0xffffffffu, gmn, off));
        gmx = fmaxf(gmx, __shfl_xor_sync(0xffffffffu, gmx, off));
    }
    if (threadIdx.x == 0) {
        if (nan) {
            gmn = 0.0f;
            gmx = INFINITY;
        }
        const float wide = 8.0f * 5.9604644775390625e-8f * p.R;
        float mid[3], half[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            mid[j] = 0.5f * mn[j] + 0.5f * mx[j];
            half[j] = __fadd_ru(fmaxf(__fsub_ru(mx[j], mid[j]), __fsub_ru(mid[j], mn[j])), wide);
        }
        gd[2 * blockIdx.x] = make_float4(mid[0], mid[1], mid[2], gmn);
        gd[2 * blockIdx.x + 1] = make_float4(half[0], half[1], half[2], gmx);
    }
}

// Supergroup record sg (one CTA of 32 threads, lane = group): union of the boxes of its
// groups' records in the current buffer (rounded outwards) and the range of their g.
__global__ void __launch_bounds__(kSuperGroup) supergroup_kernel(Prob p) {
    count_launch(p.ctl);
    const int lane = threadIdx.x;
    const int g = blockIdx.x * kSuperGroup + lane;
    const float4 *gd = p.gdata2 + (size_t)p.ctl->isel * 2 * p.ngroups;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float gmn = INFINITY, gmx = 0.0f;
    if (g < p.ngroups) {
        const float4 m = gd[2 * g], h = gd[2 * g + 1];
        const float mm[3] = {m.x, m.y, m.z}, hh[3] = {h.x, h.y, h.z};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            lo[j] = __fsub_rd(mm[j], hh[j]);
            hi[j] = __fadd_ru(mm[j], hh[j]);
        }
        gmn = m.w;
        gmx = h.w;
    }
    for (int off = 16; off; off >>= 1) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            lo[j] = fminf(lo[j], __shfl_xor_sync(0xffffffffu, lo[j], off));
            hi[j] = fmaxf(hi[j], __shfl_xor_sync(0xffffffffu, hi[j], off));
        }
        gmn = fminf(gmn, __shfl_xor_sync(0xffffffffu, gmn, off));
        gmx = fmaxf(gmx, __shfl_xor_sync(0xffffffffu, gmx, off));
    }
    if (lane == 0) {
        float mid[3], half[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            mid[j] = 0.5f * lo[j] + 0.5f * hi[j];
            half[j] = fmaxf(__fsub_ru(hi[j], mid[j]), __fsub_ru(mid[j], lo[j]));
        }
        p.sgdata[2 * blockIdx.x] = make_float4(mid[0], mid[1], mid[2], gmn);
        p.sgdata[2 * blockIdx.x + 1] = make_float4(half[0], half[1], half[2], gmx);
    }
}

template <typename T>
__device__ __forceinline__ T block_reduce_max(T v, T *red) {  // all threads get the result
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int off = 16; off; off >>= 1) {
        T o = __shfl_xor_sync(0xffffffffu, v, off);
        v = o > v ? o : v;
    }
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T m = red[0];
    for (int i = 1; i < nw; ++i) m = red[i] > m ? red[i] : m;
    return m;
}

// ------------------------------------------------------------------------------
// Initial state (two kernels over ceil(k/32) CTAs).
// ------------------------------------------------------------------------------
__global__ void __launch_bounds__(kKThreads) init_a_kernel(Prob p, cudaGraphConditionalHandle h_move,
                                                           cudaGraphConditionalHandle h_bal) {
    count_launch(p.ctl);
    __shared__ double red[32];
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    double g = 0.0;
    if (c < p.k) {
        double I = p.Iin[c];
        g = 1.0 / (I * I);
        p.I2[c] = I;
        p.g64_2[c] = g;
        if (p.bounds) p.lg[c] = lg_of(g);
        float hi[3], lo[3];
        frame_center(p, c, hi, lo);
        for (int b = 0; b < 2; ++b) {
            float4 *cd = p.cdata2 + (size_t)b * 2 * p.k;
            cd[2 * c] = make_float4(hi[0], hi[1], hi[2], 0.0f);
            cd[2 * c + 1] = make_float4(lo[0], lo[1], lo[2], 0.0f);
        }
    }
    double m = block_reduce_max(g, red);
    if (threadIdx.x == 0) atomicMax(&p.ctl->maxg_key, okey_f64(m));
    if (last_block(p.ctl) && threadIdx.x == 0) {
        Ctl *ctl = p.ctl;
        double gmax = okey_to_f64(atomicOr(&ctl->maxg_key, 0ull));
        ctl->maxg_key = 0ull;
        ctl->gshift = exponent_above(gmax);
        if (p.weighted)
            ctl->W = i128_to_f64(ctl->wsum_lo, ctl->wsum_hi, p.Fw);
        else
            ctl->W = (double)p.n_global;  // all points of the problem (every shard's)
        ctl->target = ctl->W / (double)p.k;
        ctl->ceil_avg = ceil(ctl->W / (double)p.k);
        ctl->bound = (1.0 + p.eps) * ctl->ceil_avg;
        ctl->isel = 0;
        ctl->iused_sel = 0;
        ctl->balanced = 0;
        ctl->converged = 0;
        ctl->pass_in_phase = 0;
        ctl->iter = 0;
        ctl->passes = 0;
        ctl->final_passes = 0;
        ctl->cont_balance = 1;
        ctl->cont_move = 1;
        ctl->cont_final = 0;
        ctl->max_delta = 0.0;
        ctl->maxS_key = 0ull;
        ctl->maxd_key = 0ull;
        ctl->nonempty = 0;
        ctl->coop_cnt = 0u;
        ctl->big_cnt = 0u;
        ctl->multi_cnt = 0u;
        ctl->jump_cnt = 0u;
        ctl->phase_pass = 0;
        ctl->min_lr_key = 0xffffffffu;
        ctl->max_lr_key = 0u;
        if (p.bounds) {
            p.cumm[0] = 0.0;
            p.dm[0] = 0.0f;
        }
        if (h_move) cudaGraphSetConditional(h_move, 1u);
        if (h_bal) cudaGraphSetConditional(h_bal, 1u);
    }
}

__global__ void __launch_bounds__(kKThreads) init_b_kernel(Prob p) {
    count_launch(p.ctl);
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = c < p.k;
    float4 hc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        hc = p.cdata2[2 * c];
        hc.w = scaled_g32(p.g64_2[c], p.ctl->gshift);
        p.cdata2[2 * c] = hc;
    }
    const float hi[3] = {hc.x, hc.y, hc.z};
    write_group(p, p.gdata2, valid, hi, hc.w);
}

__global__ void final_begin_kernel(Prob p, cudaGraphConditionalHandle h_fin) {
    count_launch(p.ctl);
    Ctl *ctl = p.ctl;
    int cont = (!ctl->balanced && p.final_balance_iter > 0 && ctl->status == kOk) ? 1 : 0;
    ctl->cont_final = cont;
    if (h_fin) cudaGraphSetConditional(h_fin, (unsigned)cont);
}

// Influence the last assignment was computed with -> Iin (output staging).
__global__ void export_kernel(Prob p) {
    count_launch(p.ctl);
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < p.k) p.Iin[c] = p.I2[(size_t)p.ctl->iused_sel * p.k + c];
}

// ------------------------------------------------------------------------------
// Candidate filter (Section 4.4).  For a box B (origin o, half extents h) and a
// center c (frame coordinates, q = c - o):
//   UB_c = g_c * maxDist(B, c)^2,  LB_c = g_c * minDist(B, c)^2,  tau = min_c UB_c.
// Every point of B has effective distance <= tau to its best center, so c can only
// win if LB_c <= tau.  Boxes are widened by 4 u R and tau by 64 u so that FP32
// rounding of points, centers and this arithmetic never drops the FP64 winner;
// comparisons are written so that a NaN keeps the center.
//
// Level 1: the supertile box against the group records (box of 32 consecutive
// centers and their g range): a group whose lower bound exceeds the smallest group
// upper bound holds no center that passes the test below, nor the center that attains
// tau; then tau and the supertile's candidate list from the centers of the remaining
// groups.  Level 2: each tile of the supertile against that list, written to the
// tile's record in ascending center order.
// ------------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void box_bounds(const float4 &ch, const float4 &cl, const float o[3],
                                           const float h[3], float &lb, float &ub) {
    float sl = 0.f, su = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        float cj = j == 0 ? ch.x : (j == 1 ? ch.y : ch.z);
        float lj = j == 0 ? cl.x : (j == 1 ? cl.y : cl.z);
        float a = fabsf((cj - o[j]) + lj);
        float l = fmaxf(a - h[j], 0.0f);
        float u = a + h[j];
        sl = fmaf(l, l, sl);
        su = fmaf(u, u, su);
    }
    lb = ch.w * sl;
    ub = ch.w * su;
}

// The same bounds for a group record {mid, gmin}, {half, gmax}: LB with the smallest
// g and the box-to-box minimum distance, UB with the largest g and the maximum one.
template <int D>
__device__ __forceinline__ void group_bounds(const float4 &gm, const float4 &gh, const float o[3],
                                             const float h[3], float &lb, float &ub) {
    float sl = 0.f, su = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        float mj = j == 0 ? gm.x : (j == 1 ? gm.y : gm.z);
        float hj = j == 0 ? gh.x : (j == 1 ? gh.y : gh.z);
        float a = fabsf(mj - o[j]);
        float hs = __fadd_ru(h[j], hj);
        float l = fmaxf(a - hs, 0.0f);
        float u = a + hs;
        sl = fmaf(l, l, sl);
        su = fmaf(u, u, su);
    }
    lb = gm.w * sl;
    ub = gh.w * su;
}


// Level 1 of the filter for supertile s, by one warp: writes the ascending list of
// the supertile's candidates to glist_out (kWarpList entries, global) and its first
// kLaneMax entries to list (shared), and returns its length (> kWarpList: the list
// did not fit, every center is a candidate); gall gets the largest g of all centers.
//
// tau is first bounded by the exact upper bounds of the centers of the nearest group
// (the group with the smallest lower bound, found inside the nearest supergroup when
// there are supergroups): every supergroup and group whose lower bound exceeds that
// bound is dropped (it holds no center that passes the test below, nor the center
// that attains tau).  Then tau and the list from the remaining groups' centers.
constexpr int kGroupRegs = 8;   // group chunks whose bounds stay in registers
constexpr int kCenterRegs = 8;  // kept groups whose center bounds stay in registers

// lamS gets the smallest lower bound of the supergroups, groups and centers the level
// drops (+inf when none): every center outside the list has E >= lamS on the supertile.
// box: the 2 float4 of the box (a supertile's, or a hypertile's for the level above).
// split > 0: when the level keeps more than split groups (or more than kWarpSG
// supergroups), it stops before the center sweeps and returns kSplit: the box is too large
// for one warp's list to be cheap (a curve jump across sparse space), and the caller
// builds each tile's list from its own box instead.  gcap: entries of glist_out.  Only the
// boxes whose level 1 would sweep every center are split: at 1e9 points a few dozen
// supertiles, each of which had taken 300-600 us alone; splitting the 3.5 % of supertiles
// with more than 16 kept groups instead cost more work than it saved.
constexpr int kSplitGroups = kWarpGroups;
constexpr int kSplit = -2;
template <int D>
__device__ __forceinline__ int supertile_list(const Prob &p, const float4 *box, const float4 *cd,
                                              const float4 *gd, int *list, float4 *lcd, int *glist,
                                              int *sglist, int *glist_out, float &gall, float &lamS,
                                              int split = 0, int gcap = kWarpList) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int ng = p.ngroups;
    const float infl = 4.0f * kU * p.R;
    float so[3], sh[3];
    {
        const float4 a = box[0], b = box[1];
        so[0] = a.x;
        so[1] = a.y;
        so[2] = a.z;
        sh[0] = __fadd_ru(b.x, infl);
        sh[1] = __fadd_ru(b.y, infl);
        sh[2] = __fadd_ru(b.z, infl);
    }
    // warp-wide argmin of (value, index), the smallest index on ties
    auto argmin = [&](float &v, int &i) {
        for (int off = 16; off; off >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, v, off);
            const int oi = __shfl_xor_sync(0xffffffffu, i, off);
            if (ov < v || (ov == v && oi < i)) {
                v = ov;
                i = oi;
            }
        }
    };
    float ga = 0.0f;
    const int nsg = p.nsgroups;
    float sglb = INFINITY;  // lane's supergroup lower bound (supergroup index = lane)
    int g0 = 0, g1 = ng;    // groups searched for the nearest one
    if (nsg > 0) {
        float nl = INFINITY;
        int ni = 0x7fffffff;
        for (int si = lane; si < nsg; si += 32) {
            const float4 m = __ldg(&p.sgdata[2 * si]), h = __ldg(&p.sgdata[2 * si + 1]);
            float lb, ub;
            group_bounds<D>(m, h, so, sh, lb, ub);
            ga = fmaxf(ga, h.w);
            if (si == lane) sglb = lb;
            if (lb < nl) {
                nl = lb;
                ni = si;
            }
        }
        argmin(nl, ni);
        if (ni != 0x7fffffff) {
            g0 = ni * kSuperGroup;
            g1 = min(ng, g0 + kSuperGroup);
        }
    }
    // the nearest group: sweep of all groups (or of the nearest supergroup's groups),
    // with the bounds of the first chunks kept in registers for the keep pass
    float glb[kGroupRegs];
#pragma unroll
    for (int r = 0; r < kGroupRegs; ++r) glb[r] = INFINITY;
    float tg = INFINITY, nl = INFINITY;
    int ni = 0x7fffffff;
#pragma unroll 4
    for (int r = 0; g0 + r * 32 < g1; ++r) {
        const int gi = g0 + r * 32 + lane;
        if (gi < g1) {
            const float4 gm = __ldg(&gd[2 * gi]), gh = __ldg(&gd[2 * gi + 1]);
            float lb, ub;
            group_bounds<D>(gm, gh, so, sh, lb, ub);
            tg = fminf(tg, ub);
            if (nsg == 0) ga = fmaxf(ga, gh.w);
            if (lb < nl) {
                nl = lb;
                ni = gi;
            }
#pragma unroll
            for (int q = 0; q < kGroupRegs; ++q)
                if (q == r) glb[q] = lb;
        }
    }
    for (int off = 16; off; off >>= 1) {
        tg = fminf(tg, __shfl_xor_sync(0xffffffffu, tg, off));
        ga = fmaxf(ga, __shfl_xor_sync(0xffffffffu, ga, off));
    }
    argmin(nl, ni);
    gall = ga;
    if (ni != 0x7fffffff) {
        const int c = ni * kGroup + lane;
        float t1 = INFINITY;
        if (c < p.k) {
            float lb, ub;
            box_bounds<D>(__ldg(&cd[2 * c]), __ldg(&cd[2 * c + 1]), so, sh, lb, ub);
            t1 = ub;
        }
        for (int off = 16; off; off >>= 1) t1 = fminf(t1, __shfl_xor_sync(0xffffffffu, t1, off));
        tg = fminf(tg, t1);
    }
    const float tauG = __fmul_ru(tg, 1.0f + 256.0f * kU);
    float lam = INFINITY, lamg = INFINITY;  // dropped supergroups / centers, dropped groups
    // chunks of 32 groups to test: all groups, or those of the kept supergroups
    int nchunk = (ng + 31) / 32;
    bool by_sg = false;
    if (nsg > 0) {
        int nks = 0;
        for (int r = 0; r * 32 < nsg; ++r) {
            const int si = r * 32 + lane;
            bool keep = false;
            if (si < nsg) {
                float lb = sglb;
                if (r > 0) {
                    float ub;
                    group_bounds<D>(__ldg(&p.sgdata[2 * si]), __ldg(&p.sgdata[2 * si + 1]), so, sh, lb, ub);
                }
                keep = !(lb > tauG);
                if (!keep) lamg = fminf(lamg, lb);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            const int pos = nks + __popc(bal & lt);
            if (keep && pos < kWarpSG) sglist[pos] = si;
            nks += __popc(bal);
        }
        __syncwarp();
        if (nks <= kWarpSG) {
            by_sg = true;
            nchunk = nks;
        } else {
            if (split > 0) return kSplit;
            lamg = INFINITY;  // every group is tested below
        }
    }
    int ngk = 0;  // kept groups, ascending
    for (int r = 0; r < nchunk; ++r) {
        const int gi = (by_sg ? sglist[r] * kSuperGroup : r * 32) + lane;
        bool keep = false;
        if (gi < ng) {
            float lb = INFINITY;
            if (!by_sg && nsg == 0 && r < kGroupRegs) {
#pragma unroll
                for (int q = 0; q < kGroupRegs; ++q)
                    if (q == r) lb = glb[q];
            } else {
                float ub;
                group_bounds<D>(__ldg(&gd[2 * gi]), __ldg(&gd[2 * gi + 1]), so, sh, lb, ub);
            }
            keep = !(lb > tauG);
            if (!keep) lamg = fminf(lamg, lb);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int pos = ngk + __popc(bal & lt);
        if (keep && pos < kWarpGroups) glist[pos] = gi;
        ngk += __popc(bal);
    }
    __syncwarp();
    if (split > 0 && ngk > split) return kSplit;
    const bool gover = ngk > kWarpGroups;  // too many groups: sweep every center
    if (!gover) lam = lamg;                // (a sweep of every center tests them one by one)
    // tau of the supertile over the centers of the kept groups (lane = center of the group)
    float tc = INFINITY;
    float clb[kCenterRegs];
#pragma unroll
    for (int r = 0; r < kCenterRegs; ++r) clb[r] = INFINITY;
    const int nsweep = gover ? (p.k + 31) / 32 : ngk;
#pragma unroll 4
    for (int i = 0; i < nsweep; ++i) {
        const int c = (gover ? i : glist[i]) * kGroup + lane;
        if (c < p.k) {
            float lb, ub;
            box_bounds<D>(__ldg(&cd[2 * c]), __ldg(&cd[2 * c + 1]), so, sh, lb, ub);
            tc = fminf(tc, ub);
#pragma unroll
            for (int q = 0; q < kCenterRegs; ++q)
                if (q == i) clb[q] = lb;
        }
    }
    for (int off = 16; off; off >>= 1) tc = fminf(tc, __shfl_xor_sync(0xffffffffu, tc, off));
    const float tauS = __fmul_ru(tc, 1.0f + 64.0f * kU);
    int L = 0;
    for (int i = 0; i < nsweep; ++i) {
        const int c = (gover ? i : glist[i]) * kGroup + lane;
        bool keep = false;
        if (c < p.k) {
            float lb = INFINITY;
            if (i < kCenterRegs) {
#pragma unroll
                for (int q = 0; q < kCenterRegs; ++q)
                    if (q == i) lb = clb[q];
            } else {
                float ub;
                box_bounds<D>(__ldg(&cd[2 * c]), __ldg(&cd[2 * c + 1]), so, sh, lb, ub);
            }
            keep = !(lb > tauS);
            if (!keep) lam = fminf(lam, lb);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int pos = L + __popc(bal & lt);
        if (keep && pos < gcap) glist_out[pos] = c;
        if (keep && pos < kLaneMax) list[pos] = c;
        L += __popc(bal);
    }
    __syncwarp();
    // the center data of the short list, copied after the pass so that the loads of all
    // its entries are in flight together
    if (L <= kLaneMax) {
        for (int i = lane; i < L; i += 32) {
            const int c = list[i];
            const float4 ch = __ldg(&cd[2 * c]), cl = __ldg(&cd[2 * c + 1]);
            lcd[2 * i] = ch;
            lcd[2 * i + 1] = cl;
        }
        __syncwarp();
    }
    for (int off = 16; off; off >>= 1) lam = fminf(lam, __shfl_xor_sync(0xffffffffu, lam, off));
    lamS = lam;
    return L;
}

// A supertile's level-1 list from its hypertile's list (one warp; lanes over the list's
// centers, ascending): the supertile box lies inside the hypertile box, so a center the
// hypertile level left out has a lower bound on the supertile at least as large, above
// the hypertile's tau and so above the supertile's; the center that attains the
// supertile's tau passes the hypertile's test.  tau over the hypertile list is therefore
// the supertile's tau, and the centers of the list that pass its test are the list a
// level 1 over all centers builds.  lamS: the smallest lower bound of what is left out
// (the hypertile's bound, and the list's centers that fail).  Returns the list length.
template <int D>
__device__ __forceinline__ int list_from_hyper(const Prob &p, const float4 *box, const float4 *cd,
                                               const int *hl, int Lh, float lamH, int *list, float4 *lcd,
                                               int *glist_out, float &lamS) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const float infl = 4.0f * kU * p.R;
    float so[3], sh[3];
    {
        const float4 a = box[0], b = box[1];
        so[0] = a.x;
        so[1] = a.y;
        so[2] = a.z;
        sh[0] = __fadd_ru(b.x, infl);
        sh[1] = __fadd_ru(b.y, infl);
        sh[2] = __fadd_ru(b.z, infl);
    }
    // one pass of loads: the lane's list entries (at most kHyperList / 32) and their
    // bounds stay in registers for the keep pass
    constexpr int kR = kHyperList / 32;
    int cs[kR];
    float lbs[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int i = r * 32 + lane;
        cs[r] = i < Lh ? hl[i] : -1;
    }
    float tc = INFINITY;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        lbs[r] = INFINITY;
        if (cs[r] >= 0) {
            float lb, ub;
            box_bounds<D>(__ldg(&cd[2 * cs[r]]), __ldg(&cd[2 * cs[r] + 1]), so, sh, lb, ub);
            lbs[r] = lb;
            tc = fminf(tc, ub);
        }
    }
    for (int off = 16; off; off >>= 1) tc = fminf(tc, __shfl_xor_sync(0xffffffffu, tc, off));
    const float tauS = __fmul_ru(tc, 1.0f + 64.0f * kU);
    float lam = lamH;
    int L = 0;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        if (r * 32 >= Lh) break;
        const int c = cs[r];
        const bool keep = c >= 0 && !(lbs[r] > tauS);  // a NaN bound keeps the center
        if (c >= 0 && !keep) lam = fminf(lam, lbs[r]);
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int pos = L + __popc(bal & lt);
        if (keep) {
            glist_out[pos] = c;  // L <= Lh <= kHyperList <= kWarpList
            if (pos < kLaneMax) {
                list[pos] = c;
                lcd[2 * pos] = __ldg(&cd[2 * c]);
                lcd[2 * pos + 1] = __ldg(&cd[2 * c + 1]);
            }
        }
        L += __popc(bal);
    }
    __syncwarp();
    for (int off = 16; off; off >>= 1) lam = fminf(lam, __shfl_xor_sync(0xffffffffu, lam, off));
    lamS = lam;
    return L;
}
static_assert(kHyperList <= kWarpList, "a list built from a hypertile list fits the supertile's");

// Level 1 for every hypertile (one warp each, the same as for a supertile): its list of
// candidate centers, for the supertiles inside it.
template <int D>
__global__ void __launch_bounds__(kFilterThreads) hyper_kernel(Prob p) {
    count_launch(p.ctl);
    __shared__ int s_list[kFilterWarps][kLaneMax];
    __shared__ float4 s_lcd[kFilterWarps][2 * kLaneMax];
    __shared__ int s_grp[kFilterWarps][kWarpGroups];
    __shared__ int s_sg[kFilterWarps][kWarpSG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int h = blockIdx.x * kFilterWarps + warp;
    if (h >= p.nhypers) return;
    const int sel = p.ctl->isel;
    const float4 *cd = p.cdata2 + (size_t)sel * 2 * p.k;
    const float4 *gd = p.gdata2 + (size_t)sel * 2 * p.ngroups;
    float gall, lam;
    const int L = supertile_list<D>(p, p.hypers + 2 * h, cd, gd, s_list[warp], s_lcd[warp], s_grp[warp],
                                    s_sg[warp], p.hlists + (size_t)h * kWarpList, gall, lam, kSplitGroups);
    if (lane == 0) {  // a split or overlong list: the supertiles build their own
        p.hlen[h] = L >= 0 && L <= kWarpList ? L : -1;
        p.hlam[h] = lam;
    }
}

// Header of tile t's record (count, -1: scan all centers; the largest g the tile can
// meet) and, for a tile with more than kCoopCands candidates, its entry in the
// cooperative list (one thread per tile).
// lam: smallest lower bound of the centers left out of the tile's list, which the
// record keeps lowered by 16 u (the rounding of the bound's own arithmetic), as a lower
// bound of every left-out center's E on the tile (+inf when all centers are evaluated).
// uid: the tile's stored-id marker (the w of its second box word), handed to the
// assignment in the header's w.  Returns the tile's candidates x points (the caller adds
// it to the statistics).
__device__ __forceinline__ unsigned long long finish_tile(const Prob &p, int t, int cnt, float gkept,
                                                          float gall, const float4 &tb0, float lam,
                                                          float uid) {
    const bool over = cnt > kCap;
    float4 *rec = p.trec + (size_t)t * kRecF4;
    const float lamr = over ? INFINITY : __fmul_rd(lam, 1.0f - 16.0f * kU);
    rec[0] = make_float4(__int_as_float(over ? -1 : cnt), over ? gall : gkept, lamr, uid);
    rec[1] = tb0;
    const bool coop = over || cnt > kCoopCands;
    if (coop) p.coop[atomicAdd(&p.ctl->coop_cnt, 1u)] = t;
    if (over) atomicAdd(&p.ctl->overflow_tiles, 1ull);
    long long nv = p.n - (long long)t * kTile;
    nv = nv > kTile ? kTile : nv;
    const unsigned long long used = over ? (unsigned long long)p.k : (unsigned long long)cnt;
    return used * (unsigned long long)nv;
}
__device__ __forceinline__ void add_candidates(const Prob &p, int stripe, unsigned long long v) {
    if (v) atomicAdd(&p.ctl->cand_stripes[(stripe % kStripes) * kStripeStride], v);
}

// Block weights of a tile all of whose points went to block b (called by lane 0): the
// tile's point count, or its weight sum formed at the bootstrap with the same fixed-point
// conversion of every weight as tile_histogram uses.
__device__ __forceinline__ void tile_weight_to(const Prob &p, int t, int b) {
    if (p.weighted) {
        red_add_u64(&p.Sfix[2 * b], p.tws[t]);
    } else {
        const long long nv = p.n - (long long)t * kTile;
        atomicAdd(&p.Sfix[2 * b], (unsigned long long)(nv < kTile ? nv : kTile));
    }
}

// A tile whose only candidate is c1 (without per-point bounds to keep up) is finished by
// the filter, and the assignment never sees it: every point of the tile goes to c1, so
// its stored ids are written only when its marker (every stored 16-bit id equal to it)
// does not already name c1.  The tile's point count (or weight sum) goes to block c1:
// here when add_weight, else the caller adds it (single_weight).  One thread; returns
// the tile's points.
__device__ __forceinline__ unsigned long long single_weight(const Prob &p, int t) {
    if (p.weighted) return p.tws[t];
    const long long nv = p.n - (long long)t * kTile;
    return (unsigned long long)(nv < kTile ? nv : kTile);
}
__device__ __forceinline__ long long single_tile_finish(const Prob &p, int t, int c1, int marker,
                                                        bool add_weight = true) {
    if (add_weight) tile_weight_to(p, t, c1);
    const long long i0 = (long long)t * kTile;
    long long nv = p.n - i0;
    nv = nv > kTile ? kTile : nv;
    if (p.a16) {
        if (marker == c1) return nv;
        if (nv == kTile) {
            const unsigned u = (unsigned)c1 | ((unsigned)c1 << 16);
            uint4 *dst = reinterpret_cast<uint4 *>(p.A16 + i0);
#pragma unroll 4
            for (int q = 0; q < kTile / 8; ++q) dst[q] = make_uint4(u, u, u, u);
        } else {
            for (int q = 0; q < (int)nv; ++q) p.A16[i0 + q] = (unsigned short)c1;
        }
        reinterpret_cast<int *>(p.tiles)[8 * t + 7] = c1;
    } else if (nv == kTile) {
        int4 *dst = reinterpret_cast<int4 *>(p.A + i0);
#pragma unroll 4
        for (int q = 0; q < kTile / 4; ++q) dst[q] = make_int4(c1, c1, c1, c1);
    } else {
        for (int q = 0; q < (int)nv; ++q) p.A[i0 + q] = c1;
    }
    return nv;
}

// One warp per supertile, with no block-wide synchronisation: level 1; then, for a
// list of at most kLaneMax centers, level 2 with one lane per tile (lanes 0-15), each
// walking the list.  A longer list is handed to filter_big_kernel.
template <int D>
__global__ void __launch_bounds__(kFilterThreads) filter_kernel(Prob p) {
    count_launch(p.ctl);
    __shared__ int s_list[kFilterWarps][kLaneMax];     // short level-1 lists
    __shared__ float4 s_lcd[kFilterWarps][2 * kLaneMax];  // their center data
    __shared__ int s_grp[kFilterWarps][kWarpGroups];   // kept groups (scratch of level 1)
    __shared__ int s_sg[kFilterWarps][kWarpSG];        // kept supergroups (scratch of level 1)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x < kQueues) p.ctl->tile_q[threadIdx.x * kQueueStride] = 0u;
    const int s = blockIdx.x * kFilterWarps + warp;
    if (s >= p.nsupers) return;
    const int sel = p.ctl->isel;
    const float4 *cd = p.cdata2 + (size_t)sel * 2 * p.k;
    const float4 *gd = p.gdata2 + (size_t)sel * 2 * p.ngroups;
    const float infl = 4.0f * kU * p.R;
    // this lane's tile box, loaded while level 1 runs
    const int t = s * p.stiles + lane;
    const bool has_tile = lane < p.stiles && t < p.ntiles;
    float4 tb0 = make_float4(0.f, 0.f, 0.f, 0.f), tb1 = tb0;
    if (has_tile) {
        tb0 = p.tiles[2 * t];
        tb1 = p.tiles[2 * t + 1];
    }
    float gall = 0.0f, lamS = INFINITY;
    int *gl_out = p.blists + (size_t)s * kWarpList;
    int L = -1;
    if (p.hyper) {  // from the hypertile's list, when it is short enough
        const int h = s / kHyperSupers;
        const int Lh = p.hlen[h];
        if (Lh >= 0 && Lh <= kHyperList)
            L = list_from_hyper<D>(p, p.supers + 2 * s, cd, p.hlists + (size_t)h * kWarpList, Lh,
                                   p.hlam[h], s_list[warp], s_lcd[warp], gl_out, lamS);
    }
    if (L < 0)
        L = supertile_list<D>(p, p.supers + 2 * s, cd, gd, s_list[warp], s_lcd[warp], s_grp[warp],
                              s_sg[warp], gl_out, gall, lamS, kSplitGroups);
    if (L > kLaneMax || L == kSplit) {  // hand the supertile to the warp-per-tile kernel
        if (lane == 0) {
            const int slot = (int)atomicAdd(&p.ctl->big_cnt, 1u);
            p.bigs[4 * slot] = s;
            p.bigs[4 * slot + 1] = L;
            p.bigs[4 * slot + 2] = __float_as_int(gall);
            p.bigs[4 * slot + 3] = __float_as_int(L > kWarpList ? INFINITY : lamS);
        }
        return;
    }
    // level 2, short list: lane = tile
    unsigned long long cs = 0;  // candidates x points of the lane's tile
    long long ev = 0;           // points of a tile finished here (one candidate)
    int sb = -1;                // its block
    int cnt_t = 0;              // the lane's candidate count
    bool multi = false;         // the lane's tile goes to the assignment's work list
    const int *list = s_list[warp];
    const float4 *lcd = s_lcd[warp];
    if (has_tile) {
        const float o[3] = {tb0.x, tb0.y, tb0.z};
        const float h[3] = {__fadd_ru(tb1.x, infl), __fadd_ru(tb1.y, infl), __fadd_ru(tb1.z, infl)};
        float tt = INFINITY;
#pragma unroll 4
        for (int i = 0; i < L; ++i) {
            float lb, ub;
            box_bounds<D>(lcd[2 * i], lcd[2 * i + 1], o, h, lb, ub);
            tt = fminf(tt, ub);
        }
        const float tauT = __fmul_ru(tt, 1.0f + 64.0f * kU);
        int cnt = 0, c1 = -1;
        float gkept = 0.0f, lamT = lamS;
        float4 *rec = p.trec + (size_t)t * kRecF4;
        float4 e0 = make_float4(0.f, 0.f, 0.f, 0.f);  // the first candidate's entry, written
                                                       // once the tile is known to need it
        for (int i = 0; i < L; ++i) {
            const int c = list[i];
            const float4 ch = lcd[2 * i], cl = lcd[2 * i + 1];
            float lb, ub;
            box_bounds<D>(ch, cl, o, h, lb, ub);
            if (lb > tauT) lamT = fminf(lamT, lb);
            if (!(lb > tauT)) {  // L <= kLaneMax <= kCap: always stored
                const float q0 = (ch.x - o[0]) + cl.x;
                const float q1 = (ch.y - o[1]) + cl.y;
                const float q2 = D == 3 ? (ch.z - o[2]) + cl.z : 0.0f;
                if (cnt == 0) {
                    e0 = make_float4(q0, q1, q2, ch.w);
                    c1 = c;
                } else {
                    rec[2 + 2 * cnt] = make_float4(q0, q1, q2, ch.w);
                    rec[3 + 2 * cnt] = make_float4(__int_as_float(c), 0.0f, 0.0f, 0.0f);
                }
                gkept = fmaxf(gkept, ch.w);
                ++cnt;
            }
        }
        cnt_t = cnt;
        if (!p.bounds && cnt == 1) {
            // finished here: the record is never read, so it is not written
            cs = (unsigned long long)single_tile_finish(p, t, c1, __float_as_int(tb1.w), false);
            ev = (long long)cs;
            sb = c1;
        } else {
            if (cnt > 0) {
                rec[2] = e0;
                rec[3] = make_float4(__int_as_float(c1), 0.0f, 0.0f, 0.0f);
            }
            cs = finish_tile(p, t, cnt, gkept, gall, tb0, lamT, tb1.w);
            multi = cnt <= kCoopCands;  // L <= kLaneMax <= kCap: never an overflowed list
        }
    }
    // block weights of the one-candidate tiles: neighbouring tiles mostly share the block,
    // so runs of equal blocks over the lanes are summed first (low and high 32-bit parts
    // apart, the carry-free form), then one atomic per run
    {
        const unsigned long long wv = sb >= 0 ? single_weight(p, t) : 0ull;
        unsigned long long wlo = wv & 0xffffffffull, whi = wv >> 32;
        const int prev = __shfl_up_sync(0xffffffffu, sb, 1);
        const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || sb != prev);
        const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long a = __shfl_up_sync(0xffffffffu, wlo, off);
            const unsigned long long b = __shfl_up_sync(0xffffffffu, whi, off);
            if (lane - off >= start) {
                wlo += a;
                whi += b;
            }
        }
        const bool end = lane == 31 || ((heads >> (lane + 1)) & 1u);
        if (end && sb >= 0) {
            atomicAdd(&p.Sfix[2 * sb], wlo);
            if (whi) atomicAdd(&p.Sfix[2 * sb + 1], whi);
        }
    }
    // the work list: one atomic per supertile
    const unsigned mb = __ballot_sync(0xffffffffu, multi);
    if (mb) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&p.ctl->multi_cnt, (unsigned)__popc(mb));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (multi) p.mlist[base + __popc(mb & ((1u << lane) - 1u))] = make_int2(t, cnt_t);
    }
    // the statistics: one atomic per supertile (one per tile contended at 1e9 points)
    for (int off = 16; off; off >>= 1) {
        cs += __shfl_xor_sync(0xffffffffu, cs, off);
        ev += __shfl_xor_sync(0xffffffffu, ev, off);
    }
    if (lane == 0) {
        add_candidates(p, s, cs);
        if (ev) atomicAdd(&p.ctl->evaluated, (unsigned long long)ev);
    }
}
static_assert(kLaneMax <= kCap, "a short list always fits the tile record");
static_assert(kMaxSuperTiles <= 32, "level 2 of the filter takes one lane per tile");

// Whether filter_tile_kernel runs: with at most kWarpGroups groups (k <= 2048) no supertile
// is split, and a tile whose list does not fit its record takes every center (an
// overflowed record), as it costs little at that k; the launch is then left out.
__host__ __device__ __forceinline__ bool filter_tile_needed(const Prob &p) { return p.ngroups > kWarpGroups; }

// A tile of filter_big_kernel once its record is written (lane 0): finished here with one
// candidate c1, or put on the assignment's work list.
__device__ __forceinline__ void big_tile_done(const Prob &p, int t, int cnt, int c1, int marker) {
    if (!p.bounds && cnt == 1) {
        atomicAdd(&p.ctl->evaluated, (unsigned long long)single_tile_finish(p, t, c1, marker));
    } else if (cnt <= kCoopCands) {
        p.mlist[atomicAdd(&p.ctl->multi_cnt, 1u)] = make_int2(t, cnt);
    }
}

// Level 2 of the supertiles with long lists: one warp per tile, lanes over chunks
// of 32 candidates (tau pass, then the ascending keep pass with ballots).  A split
// supertile (kSplit: level 1 on its box would keep too many groups) gets level 1 on each
// tile's own box instead, whose list is the tile's candidates: the tile's tau is the
// smallest upper bound over all centers either way, and the kept centers are those whose
// lower bound on the tile passes it.
template <int D>
__global__ void __launch_bounds__(kFilterThreads) filter_big_kernel(Prob p) {
    count_launch(p.ctl);
    __shared__ int s_list[kFilterWarps][kLaneMax];
    __shared__ float4 s_lcd[kFilterWarps][2 * kLaneMax];
    __shared__ int s_grp[kFilterWarps][kWarpGroups];
    __shared__ int s_sg[kFilterWarps][kWarpSG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int total = (int)p.ctl->big_cnt * p.stiles;
    const int sel = p.ctl->isel;
    const float4 *cd = p.cdata2 + (size_t)sel * 2 * p.k;
    const float4 *gd = p.gdata2 + (size_t)sel * 2 * p.ngroups;
    const float infl = 4.0f * kU * p.R;
    const int TW = gridDim.x * kFilterWarps;
    for (int item = blockIdx.x * kFilterWarps + warp; item < total; item += TW) {
        const int slot = item / p.stiles;
        const int s = p.bigs[4 * slot], Lr = p.bigs[4 * slot + 1];
        const int t = s * p.stiles + item % p.stiles;
        if (t >= p.ntiles) continue;
        if (Lr == kSplit) {  // level 1 on the tile's own box, in filter_tile_kernel
            if (lane == 0) p.tlist[atomicAdd(&p.ctl->jump_cnt, 1u)] = t;
            continue;
        }
        const float gall = __int_as_float(p.bigs[4 * slot + 2]);
        float lamT = __int_as_float(p.bigs[4 * slot + 3]);
        const bool all = Lr > kWarpList;
        const int L = all ? p.k : Lr;
        const int *list = p.blists + (size_t)s * kWarpList;
        const float4 tb0 = p.tiles[2 * t], tb1 = p.tiles[2 * t + 1];
        const float o[3] = {tb0.x, tb0.y, tb0.z};
        const float h[3] = {__fadd_ru(tb1.x, infl), __fadd_ru(tb1.y, infl), __fadd_ru(tb1.z, infl)};
        auto center = [&](int i, int &c, float4 &ch, float4 &cl) {
            c = all ? i : list[i];
            ch = __ldg(&cd[2 * c]);
            cl = __ldg(&cd[2 * c + 1]);
        };
        float tt = INFINITY;
#pragma unroll 4
        for (int i = lane; i < L; i += 32) {  // several chunks' loads in flight together
            int c;
            float4 ch, cl;
            center(i, c, ch, cl);
            float lb, ub;
            box_bounds<D>(ch, cl, o, h, lb, ub);
            tt = fminf(tt, ub);
        }
        for (int off = 16; off; off >>= 1) tt = fminf(tt, __shfl_xor_sync(0xffffffffu, tt, off));
        const float tauT = __fmul_ru(tt, 1.0f + 64.0f * kU);
        int cnt = 0, c1 = -1;
        float gkept = 0.0f;
        float4 *rec = p.trec + (size_t)t * kRecF4;
#pragma unroll 2
        for (int base = 0; base < L; base += 32) {
            const int i = base + lane;
            bool keep = false;
            int c = 0;
            float4 ch = make_float4(0.f, 0.f, 0.f, 0.f), cl = ch;
            if (i < L) {
                center(i, c, ch, cl);
                float lb, ub;
                box_bounds<D>(ch, cl, o, h, lb, ub);
                keep = !(lb > tauT);
                if (lb > tauT) lamT = fminf(lamT, lb);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            const int pos = cnt + __popc(bal & lt);
            if (keep && pos < kCap) {
                const float q0 = (ch.x - o[0]) + cl.x;
                const float q1 = (ch.y - o[1]) + cl.y;
                const float q2 = D == 3 ? (ch.z - o[2]) + cl.z : 0.0f;
                rec[2 + 2 * pos] = make_float4(q0, q1, q2, ch.w);
                rec[3 + 2 * pos] = make_float4(__int_as_float(c), 0.0f, 0.0f, 0.0f);
            }
            if (keep) gkept = fmaxf(gkept, ch.w);
            if (keep && pos == 0) c1 = c;
            cnt += __popc(bal);
        }
        c1 = __reduce_max_sync(0xffffffffu, c1);  // the first kept center
        if (cnt > kCap && filter_tile_needed(p)) {  // the tile's own level 1 rewrites the record
            if (lane == 0) p.tlist[atomicAdd(&p.ctl->jump_cnt, 1u)] = t;
            continue;
        }
        for (int off = 16; off; off >>= 1) {
            gkept = fmaxf(gkept, __shfl_xor_sync(0xffffffffu, gkept, off));
            lamT = fminf(lamT, __shfl_xor_sync(0xffffffffu, lamT, off));
        }
        if (lane == 0) {
            add_candidates(p, t, finish_tile(p, t, cnt, gkept, gall, tb0, lamT, tb1.w));
            big_tile_done(p, t, cnt, c1, __float_as_int(tb1.w));
        }
    }
}

// Level 1 on a tile's own box, by a whole CTA per tile, for the tiles filter_big_kernel
// listed: the tiles of a split supertile and the tiles whose list from their supertile's
// list does not fit the record.  At 1e9 points these are the tiles of the sparse
// background next to a dense spot: the nearest centers are far, so hundreds of the spot's
// small groups pass the group test, yet the final list fits the record.  One warp sweeping
// them took 300-600 us; handing such a tile every center made the assignment's
// cooperative CTAs pay 0.29 ms per pass.  Here the eight warps share the sweeps:
// 1. every group's bounds (threads over groups): tau_G = the smallest group upper bound
//    (each group's bounds every member's, so tau_G >= tau), kept: the groups whose lower
//    bound passes tau_G, in ascending order;
// 2. tau = the smallest upper bound over the kept groups' centers (warps over groups);
// 3. the kept centers (lower bound <= tau): each warp a contiguous range of the kept
//    groups, then the warps' lists in order: the ascending list.
// The center attaining tau lies in a kept group (its group's lower bound <= its own <=
// tau <= tau_G), as does every center that passes tau, so the list is the one level 1
// over all centers gives.  More than kTileGroups kept groups, or more than kCap
// candidates: every center (an overflowed record).
constexpr int kTileGroups = 2048;
template <int D>
__global__ void __launch_bounds__(kFilterThreads) filter_tile_kernel(Prob p) {
    count_launch(p.ctl);
    __shared__ int s_grp[kTileGroups];
    __shared__ int s_cent[kFilterWarps][kCap];
    __shared__ int s_cnt[kFilterWarps];
    __shared__ float s_red[kFilterWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int total = (int)p.ctl->jump_cnt;
    const int sel = p.ctl->isel;
    const float4 *cd = p.cdata2 + (size_t)sel * 2 * p.k;
    const float4 *gd = p.gdata2 + (size_t)sel * 2 * p.ngroups;
    const float infl = 4.0f * kU * p.R;
    const int ng = p.ngroups;
    // CTA-wide minimum (op 0) or maximum (op 1) of one value per thread
    auto cta_red = [&](float v, int op) -> float {
        for (int off = 16; off; off >>= 1) {
            const float o = __shfl_xor_sync(0xffffffffu, v, off);
            v = op ? fmaxf(v, o) : fminf(v, o);
        }
        __syncthreads();
        if (lane == 0) s_red[warp] = v;
        __syncthreads();
        float r = s_red[0];
        for (int w = 1; w < kFilterWarps; ++w) r = op ? fmaxf(r, s_red[w]) : fminf(r, s_red[w]);
        return r;
    };
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int t = p.tlist[item];
        const float4 tb0 = p.tiles[2 * t], tb1 = p.tiles[2 * t + 1];
        const float so[3] = {tb0.x, tb0.y, tb0.z};
        const float sh[3] = {__fadd_ru(tb1.x, infl), __fadd_ru(tb1.y, infl), __fadd_ru(tb1.z, infl)};
        // 1. groups
        float tg = INFINITY, ga = 0.0f;
        for (int gi = tid; gi < ng; gi += kFilterThreads) {
            float lb, ub;
            const float4 gm = __ldg(&gd[2 * gi]), gh = __ldg(&gd[2 * gi + 1]);
            group_bounds<D>(gm, gh, so, sh, lb, ub);
            tg = fminf(tg, ub);
            ga = fmaxf(ga, gh.w);
        }
        const float gall = cta_red(ga, 1);
        const float tauG = __fmul_ru(cta_red(tg, 0), 1.0f + 256.0f * kU);
        float lam = INFINITY;
        int ngk = 0;
        for (int base = 0; base < ng; base += kFilterThreads) {  // ascending, a CTA round at a time
            const int gi = base + tid;
            bool keep = false;
            if (gi < ng) {
                float lb, ub;
                group_bounds<D>(__ldg(&gd[2 * gi]), __ldg(&gd[2 * gi + 1]), so, sh, lb, ub);
                keep = !(lb > tauG);
                if (!keep) lam = fminf(lam, lb);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) s_cnt[warp] = __popc(bal);
            __syncthreads();
            int before = ngk;
            for (int w = 0; w < warp; ++w) before += s_cnt[w];
            int round = 0;
            for (int w = 0; w < kFilterWarps; ++w) round += s_cnt[w];
            const int pos = before + __popc(bal & lt);
            if (keep && pos < kTileGroups) s_grp[pos] = gi;
            ngk += round;
            __syncthreads();
        }
        bool over = ngk > kTileGroups;
        int L = 0;
        if (!over) {
            // 2. tau over the kept groups' centers (warp w: groups w, w + 8, ...)
            float tc = INFINITY;
            for (int i = warp; i < ngk; i += kFilterWarps) {
                const int c = s_grp[i] * kGroup + lane;
                if (c < p.k) {
                    float lb, ub;
                    box_bounds<D>(__ldg(&cd[2 * c]), __ldg(&cd[2 * c + 1]), so, sh, lb, ub);
                    tc = fminf(tc, ub);
                }
            }
            const float tauS = __fmul_ru(cta_red(tc, 0), 1.0f + 64.0f * kU);
            // 3. the kept centers, warp w over kept groups [w ngk / 8, (w + 1) ngk / 8)
            const int g0 = (int)((long long)warp * ngk / kFilterWarps);
            const int g1 = (int)((long long)(warp + 1) * ngk / kFilterWarps);
            int cw = 0;
            for (int i = g0; i < g1; ++i) {
                const int c = s_grp[i] * kGroup + lane;
                bool keep = false;
                if (c < p.k) {
                    float lb, ub;
                    box_bounds<D>(__ldg(&cd[2 * c]), __ldg(&cd[2 * c + 1]), so, sh, lb, ub);
                    keep = !(lb > tauS);
                    if (!keep) lam = fminf(lam, lb);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                const int pos = cw + __popc(bal & lt);
                if (keep && pos < kCap) s_cent[warp][pos] = c;
                cw += __popc(bal);
            }
            if (lane == 0) s_cnt[warp] = cw;
            __syncthreads();
            int before = 0;
            for (int w = 0; w < warp; ++w) before += s_cnt[w];
            for (int w = 0; w < kFilterWarps; ++w) L += s_cnt[w];
            over = L > kCap;
            float gkept = 0.0f;
            if (!over) {
                float4 *rec = p.trec + (size_t)t * kRecF4;
                for (int j = lane; j < cw; j += 32) {
                    const int c = s_cent[warp][j];
                    const float4 ch = __ldg(&cd[2 * c]), cl = __ldg(&cd[2 * c + 1]);
                    const float q0 = (ch.x - so[0]) + cl.x;
                    const float q1 = (ch.y - so[1]) + cl.y;
                    const float q2 = D == 3 ? (ch.z - so[2]) + cl.z : 0.0f;
                    rec[2 + 2 * (before + j)] = make_float4(q0, q1, q2, ch.w);
                    rec[3 + 2 * (before + j)] = make_float4(__int_as_float(c), 0.0f, 0.0f, 0.0f);
                    gkept = fmaxf(gkept, ch.w);
                }
            }
            gkept = cta_red(gkept, 1);
            lam = cta_red(lam, 0);
            if (tid == 0) {
                int c1 = -1;
                for (int w = 0; w < kFilterWarps && c1 < 0; ++w)
                    if (s_cnt[w] > 0) c1 = s_cent[w][0];
                const int cnt = over ? p.k + kCap + 1 : L;  // more than kCap: overflowed
                add_candidates(p, t, finish_tile(p, t, cnt, gkept, gall, tb0, lam, tb1.w));
                big_tile_done(p, t, cnt, c1, __float_as_int(tb1.w));
            }
        } else {
            lam = cta_red(lam, 0);
            if (tid == 0) {
                const int cnt = p.k + kCap + 1;
                add_candidates(p, t, finish_tile(p, t, cnt, 0.0f, gall, tb0, lam, tb1.w));
                big_tile_done(p, t, cnt, -1, __float_as_int(tb1.w));
            }
        }
        __syncthreads();  // the shared lists are reused by the next tile
    }
}

// ------------------------------------------------------------------------------
// Warp segmented reduction of per-lane (id, value) runs whose ids are laid out in
// lane order; the last lane of each segment adds the segment's sum to acc[2*id].
// Lanes with id < 0 contribute nothing.
// ------------------------------------------------------------------------------
__device__ __forceinline__ void seg_flush_u64(int id, unsigned long long v, unsigned long long *acc,
                                              bool wide) {
    const int lane = threadIdx.x & 31;
    int prev = __shfl_up_sync(0xffffffffu, id, 1);
    bool head = lane == 0 || id != prev;
    unsigned heads = __ballot_sync(0xffffffffu, head);
    int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, v, off);
        if (lane - off >= start) v += y;
    }
    bool end = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (end && id >= 0) {
        if (wide)
            red_add_u64(&acc[2 * id], v);
        else
            atomicAdd(&acc[2 * id], v);
    }
}

// ------------------------------------------------------------------------------
// Assignment + block-weight histogram (Section 4.2; Algorithm 1 inner loop).
//
// One warp per tile of 256 curve-consecutive points; lane l owns points 8l..8l+7.
// With tile-local frame coordinates x' = x - o and the candidate's frame center
// relative to the tile origin q, the squared effective distance is
//     E = g |x' - q|^2   (g = scaled 1/I^2; two points per packed f32x2 operation).
// FP64 mode: the FP32 winner b is kept when the FP32 gap to the runner-up exceeds
// twice a rigorous bound B on |E_fp32 - E_exact| (rounding of the stored point, of
// the tile-local differences and of the hi/lo center, and of the squares, the sum
// and g; per point, with the largest g of the tile's candidates; doubled for safety);
// a point with a single candidate is decided by the filter alone.  Every other point
// is decided again in FP64 from the raw coordinates, over the candidates whose FP32
// value lies within the margin.  The result is the FP64 argmin up to ties closer than
// FP64 rounding, ties going to the lowest center index.
// ------------------------------------------------------------------------------
template <bool F64MODE>
__device__ __forceinline__ void argmin_update(float E, int c, float &E1, float &E2, int &best) {
    if (F64MODE) E2 = fminf(E2, fmaxf(E, E1));
    bool lt = E < E1;
    best = lt ? c : best;
    E1 = lt ? E : E1;
}
// The same for two candidates ca < cb at once: their smaller value and its index (ca on
// ties) do not depend on the running state, which shortens its dependency chain; the
// runner-up is the second smallest of {E1, E2, Ea, Eb}.
template <bool F64MODE>
__device__ __forceinline__ void argmin_update2(float Ea, int ca, float Eb, int cb, float &E1, float &E2,
                                               int &best) {
    const float lo = fminf(Ea, Eb);
    const int cab = lo == Ea ? ca : cb;
    if (F64MODE) E2 = fminf(fminf(fmaxf(E1, lo), E2), fmaxf(Ea, Eb));
    const bool lt = lo < E1;
    best = lt ? cab : best;
    E1 = lt ? lo : E1;
}

// Error-bound terms of the FP64-mode certification (see the comment above): the
// bound on |E_fp32 - E_exact| for a point whose coordinate term is e0, against
// candidates with g <= glv (sgl = sqrt(glv)), at the FP32 value Eref.
__device__ __forceinline__ float cert_bound(float e0, float sgl, float glv, float beta2, float Eref) {
    const float beta1 = 2.0f * sgl * e0;
    const float beta0 = glv * e0 * e0;
    const float Estar = 2.0f * Eref + 2.0f * (beta0 + 2.0f * beta1 * beta1);
    return 2.0f * (beta0 + beta1 * sqrtf(Estar) + beta2 * Estar);
}

// The block ids of a lane's 8 points (16 bits when p.a16).
__device__ __forceinline__ void store_blocks(const Prob &p, long long i0, int nval, const int best[8]) {
    if (p.a16) {
        if (nval == 8) {
            uint4 v;
            v.x = (unsigned)best[0] | ((unsigned)best[1] << 16);
            v.y = (unsigned)best[2] | ((unsigned)best[3] << 16);
            v.z = (unsigned)best[4] | ((unsigned)best[5] << 16);
            v.w = (unsigned)best[6] | ((unsigned)best[7] << 16);
            *reinterpret_cast<uint4 *>(p.A16 + i0) = v;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q < nval) p.A16[i0 + q] = (unsigned short)best[q];
        }
    } else if (nval == 8) {
        int4 *dst = reinterpret_cast<int4 *>(p.A + i0);
        dst[0] = make_int4(best[0], best[1], best[2], best[3]);
        dst[1] = make_int4(best[4], best[5], best[6], best[7]);
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < nval) p.A[i0 + q] = best[q];
    }
}

// The block ids of a tile (called by the whole warp), skipping the stores when every
// point of the tile keeps the block that all its stored ids already hold.  prev is the
// tile's marker as the filter read it this pass: b when every stored 16-bit id of the
// tile is b, -1 otherwise; the marker is updated when that changes.  On curve-sorted
// points most tiles lie inside one block and keep it from pass to pass.
// Returns whether every point of the tile got the same block.
__device__ __forceinline__ bool store_blocks_tile(const Prob &p, int t, long long i0, int nval,
                                                  const int best[8], int prev) {
    const int b0 = __shfl_sync(0xffffffffu, best[0], 0);  // lane 0 holds a point of the tile
    bool same = true;
#pragma unroll
    for (int q = 0; q < 8; ++q) same &= q >= nval || best[q] == b0;
    const bool uni = __all_sync(0xffffffffu, same);
    if (!p.a16) {
        store_blocks(p, i0, nval, best);
        return uni;
    }
    if (uni && prev == b0) return true;  // the stored ids are b0 already
    store_blocks(p, i0, nval, best);
    const int now = uni ? b0 : -1;
    if ((threadIdx.x & 31) == 0 && now != prev) reinterpret_cast<int *>(p.tiles)[8 * t + 7] = now;
    return uni;
}

// Block weights of one tile's assignment: runs inside the lane, then a segmented
// reduction over lanes (unit weights: 64-bit counts; weights: 128-bit fixed point).
__device__ __forceinline__ void tile_histogram(const Prob &p, long long i0, int nval, const int best[8]) {
    int cur = -1;
    unsigned long long acc = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (q < nval) {
            unsigned long long v = 1ull;
            if (p.weighted)
                v = (unsigned long long)(p.dtype == 1 ? fix_f64(((const double *)p.Ws)[i0 + q], p.Fw)
                                                      : fix_f32(((const float *)p.Ws)[i0 + q], p.Fw));
            if (best[q] != cur) {
                if (cur >= 0) {
                    if (p.weighted)
                        red_add_u64(&p.Sfix[2 * cur], acc);
                    else
                        atomicAdd(&p.Sfix[2 * cur], acc);
                }
                cur = best[q];
                acc = 0;
            }
            acc += v;
        }
    }
    seg_flush_u64(cur, acc, p.Sfix, p.weighted != 0);
}

// The per-point bound recorded at an evaluation: rho = (lower bound of every other
// center's E) / (upper bound of the own center's E) -- from the runner-up E2 of the
// tile's list less its error bound B and the filter's bound lamT of the centers left
// out, over E1 plus B (FP32 form: B = 0 and a 2^-20 margin on each side for the rounding
// of E) -- stored as log2(rho) lowered by kLqMargin (the two fast logarithms).  A
// re-decided point (recheck) gets -inf: it is evaluated again in the next pass.
// log2 through the hardware approximation, whose error (at most 2^-22.6 absolute on
// [0.5, 2], 2 ulp elsewhere, i.e. below 2^-15 for finite FP32 inputs) kLqMargin covers.
template <bool F64MODE>
__device__ __forceinline__ float bound_lq(float E1, float E2, float B, float lamT, unsigned recheck) {
    if (recheck) return -INFINITY;
    const float U1 = F64MODE ? __fadd_ru(E1, B) : __fmul_ru(E1, 1.0f + 9.5367431640625e-7f);
    float L1 = F64MODE ? (E2 < INFINITY ? __fsub_rd(E2, B) : INFINITY) : __fmul_rd(E2, 1.0f - 9.5367431640625e-7f);
    L1 = fminf(L1, lamT);
    if (!(L1 > 0.0f)) return -INFINITY;  // also NaN
    const float v = __fsub_rd(__fsub_rd(__log2f(L1), __log2f(U1)), kLqMargin);
    return v == v ? v : -INFINITY;
}

// ------------------------------------------------------------------------------
// Cooperative tile: a tile with more candidates than one warp finishes in the time
// the others take (more than kCoopCands, or all k centers when its list overflowed)
// is taken by all kAWarps warps of a CTA.  Warp w evaluates the w-th contiguous
// range of the candidates (ascending centers) for all points of the tile; the
// per-warp (E1, E2, best) are merged in shared memory in ascending range order,
// which keeps the lowest center index on ties.  Warp 0 then certifies (FP64 mode),
// re-decides the flagged points over all candidates, writes the block ids and adds
// the block weights.  Called by every thread of the CTA; scratch holds at least
// 3 * kAWarps * kTile words.
// ------------------------------------------------------------------------------
template <int D, bool F64MODE, bool BOUNDS>
__device__ __noinline__ void coop_tile(const Prob &p, int t, float *scratch, int nwarps,
                                       unsigned long long *nre, int pp, unsigned long long *nevl) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float4 *grec = p.trec + (size_t)t * kRecF4;
    const float4 hdr = grec[0], ob = grec[1];
    const int cnt = __float_as_int(hdr.x);
    const bool all = cnt < 0;
    const int ncand = all ? p.k : cnt;
    const float o[3] = {ob.x, ob.y, ob.z};
    const float4 *cd = p.cdata2 + (size_t)p.ctl->isel * 2 * p.k;
    const long long i0 = (long long)t * kTile + lane * 8;
    const long long nv = p.n - i0;
    const int nval = nv <= 0 ? 0 : (nv >= 8 ? 8 : (int)nv);
    float2 xp[3][4];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) xp[j][q] = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float4 *src = reinterpret_cast<const float4 *>(p.X32 + (size_t)j * p.n_pad + i0);
        const float4 a = src[0], c4 = src[1];
        xp[j][0] = make_float2(a.x - o[j], a.y - o[j]);
        xp[j][1] = make_float2(a.z - o[j], a.w - o[j]);
        xp[j][2] = make_float2(c4.x - o[j], c4.y - o[j]);
        xp[j][3] = make_float2(c4.z - o[j], c4.w - o[j]);
    }
    auto cand = [&](int jj, float4 &qg, int &c) {  // jj < ncand
        if (!all) {
            qg = grec[2 + 2 * jj];
            c = __float_as_int(grec[3 + 2 * jj].x);
        } else {
            c = jj;
            const float4 ch = cd[2 * c], cl = cd[2 * c + 1];
            qg = make_float4((ch.x - o[0]) + cl.x, (ch.y - o[1]) + cl.y,
                             D == 3 ? (ch.z - o[2]) + cl.z : 0.0f, ch.w);
        }
    };
    float E1[8], E2[8];
    int best[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        E1[q] = INFINITY;
        E2[q] = INFINITY;
        best[q] = 0;
    }
    const int rb = (int)((long long)ncand * w / nwarps), re = (int)((long long)ncand * (w + 1) / nwarps);
    for (int base = rb; base < re; base += 32) {
        float4 mqg = make_float4(0.f, 0.f, 0.f, 0.f);
        int mc = 0;
        if (base + lane < re) cand(base + lane, mqg, mc);
        const int m = min(32, re - base);
        for (int jj = 0; jj < m; ++jj) {
            const float2 g2 = make_float2(__shfl_sync(0xffffffffu, mqg.w, jj), 0.f);
            const float qx = __shfl_sync(0xffffffffu, mqg.x, jj), qy = __shfl_sync(0xffffffffu, mqg.y, jj);
            const float qz = __shfl_sync(0xffffffffu, mqg.z, jj);
            const int c = __shfl_sync(0xffffffffu, mc, jj);
            const float2 gg = make_float2(g2.x, g2.x), nqx = make_float2(-qx, -qx), nqy = make_float2(-qy, -qy),
                         nqz = make_float2(-qz, -qz);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 dx = __fadd2_rn(xp[0][q], nqx);
                const float2 dy = __fadd2_rn(xp[1][q], nqy);
                float2 ss = __fmul2_rn(dx, dx);
                ss = __ffma2_rn(dy, dy, ss);
                if (D == 3) {
                    const float2 dz = __fadd2_rn(xp[2][q], nqz);
                    ss = __ffma2_rn(dz, dz, ss);
                }
                const float2 E = __fmul2_rn(gg, ss);
                argmin_update<true>(E.x, c, E1[2 * q], E2[2 * q], best[2 * q]);
                argmin_update<true>(E.y, c, E1[2 * q + 1], E2[2 * q + 1], best[2 * q + 1]);
            }
        }
    }
    // partials to shared memory: [warp][lane][q] of E1, E2, best
    float *sE1 = scratch, *sE2 = scratch + nwarps * kTile;
    int *sB = reinterpret_cast<int *>(scratch + 2 * nwarps * kTile);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int idx = w * kTile + q * 32 + lane;
        sE1[idx] = E1[q];
        sE2[idx] = E2[q];
        sB[idx] = best[q];
    }
    __syncthreads();
    if (w == 0) {
        for (int w2 = 1; w2 < nwarps; ++w2) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int idx = w2 * kTile + q * 32 + lane;
                const float e1 = sE1[idx], e2 = sE2[idx];
                if (e1 < E1[q]) {  // a later range wins only when strictly smaller
                    E2[q] = fminf(E1[q], e2);
                    E1[q] = e1;
                    best[q] = sB[idx];
                } else {
                    E2[q] = fminf(E2[q], e1);
                }
            }
        }
        float Bq[8];
        unsigned flag = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) Bq[q] = 0.0f;
        if (F64MODE) {
            const float gl = hdr.y, sg = sqrtf(gl);
            const float R = p.R, sd = sqrtf((float)D);
            const float beta2 = ((float)D + 4.0f + 8.0f * sd) * kU;
            float xn2 = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < D; ++j) acc = __ffma2_rn(xp[j][q], xp[j][q], acc);
                xn2 = fmaxf(xn2, fmaxf(acc.x, acc.y));
            }
            const float e0 = sd * kU * (R + 8.0f * __fsqrt_ru(__fmul_ru(xn2, 1.0f + 4.0f * kU)));
            float thr[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float B = cert_bound(e0, sg, gl, beta2, E2[q]);
                const bool single = E2[q] == INFINITY && E1[q] < INFINITY;
                const bool okq = single || (E2[q] - E1[q]) > 2.0f * B;
                thr[q] = E1[q] + 2.0f * B;
                Bq[q] = B;
                if (q < nval && !okq) flag |= 1u << q;
            }
            // FP64 re-decision, one flagged point at a time: lanes take 32 candidates at
            // a time, screen them with the FP32 value (every possible FP64 winner has
            // E_fp32 <= thr) and evaluate the survivors in FP64; the warp keeps the
            // smallest value, the lowest center index on ties.
            const double *g64 = p.g64_2 + (size_t)p.ctl->isel * p.k;
            unsigned lanes = __ballot_sync(0xffffffffu, flag != 0u);
            while (lanes) {
                const int L = __ffs(lanes) - 1;
                lanes &= lanes - 1;
                unsigned fl = __shfl_sync(0xffffffffu, flag, L);
                while (fl) {
                    const int q = __ffs(fl) - 1;
                    fl &= fl - 1;
                    float mx[3] = {0.f, 0.f, 0.f}, mt = 0.f;
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) {
                        if (qq == q) {
#pragma unroll
                            for (int j = 0; j < D; ++j) mx[j] = (qq & 1) ? xp[j][qq >> 1].y : xp[j][qq >> 1].x;
                            mt = thr[qq];
                        }
                    }
#pragma unroll
                    for (int j = 0; j < D; ++j) mx[j] = __shfl_sync(0xffffffffu, mx[j], L);
                    mt = __shfl_sync(0xffffffffu, mt, L);
                    const long long ip = (long long)t * kTile + L * 8 + q;
                    double X[3] = {0.0, 0.0, 0.0};
#pragma unroll
                    for (int j = 0; j < D; ++j)
                        X[j] = p.dtype == 1 ? p.X64[(size_t)j * p.n_pad + ip] : (double)p.X32[(size_t)j * p.n_pad + ip];
                    double bE = INFINITY;
                    int bc = 0x7fffffff;
                    for (int base = 0; base < ncand; base += 32) {
                        float4 qg;
                        int c = 0x7fffffff;
                        double E = INFINITY;
                        if (base + lane < ncand) {
                            cand(base + lane, qg, c);
                            const float d0 = mx[0] - qg.x, d1 = mx[1] - qg.y;
                            const float d2 = D == 3 ? mx[2] - qg.z : 0.0f;
                            const float E32 = qg.w * fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
                            if (E32 <= mt) {
                                double s2 = 0.0;
#pragma unroll
                                for (int j = 0; j < D; ++j) {
                                    const double df = X[j] - p.C[c * D + j];
                                    s2 += df * df;
                                }
                                E = s2 * g64[c];
                            }
                        }
                        if (E < bE || (E == bE && c < bc)) {
                            bE = E;
                            bc = c;
                        }
                    }
                    for (int off = 16; off; off >>= 1) {
                        const double oE = __shfl_xor_sync(0xffffffffu, bE, off);
                        const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
                        if (oE < bE || (oE == bE && oc < bc)) {
                            bE = oE;
                            bc = oc;
                        }
                    }
                    if (lane == L && bc != 0x7fffffff) {
#pragma unroll
                        for (int qq = 0; qq < 8; ++qq)
                            if (qq == q) best[qq] = bc;
                    }
                }
            }
            *nre += __popc(flag);
        }
        if constexpr (BOUNDS) {  // every point of a cooperative tile is evaluated: its bound
            const float lamT = hdr.z;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (q >= nval) continue;
                p.lq[i0 + q] = bound_lq<F64MODE>(E1[q], E2[q], Bq[q], lamT, (flag >> q) & 1u);
                p.t1[i0 + q] = (unsigned char)pp;
            }
        }
        if (lane == 0) *nevl += (unsigned long long)(p.n - (long long)t * kTile < kTile ? p.n - (long long)t * kTile : kTile);
        if (store_blocks_tile(p, t, i0, nval, best, __float_as_int(hdr.w))) {
            if (lane == 0) tile_weight_to(p, t, best[0]);
        } else {
            tile_histogram(p, i0, nval, best);
        }
    }
}

// Persistent warps take tiles from shared queues.  Each warp owns two shared-memory
// stages; one lane issues the bulk copies (tile record with its first kFastCands
// candidates, and the d coordinate planes of the tile) for the tile after next as
// soon as a stage is consumed, so the loads of two tiles are always in flight.
constexpr int kAWarps = 4;
constexpr int kAMinBlocks = 5;     // CTAs per SM of the FP32 form
constexpr int kAMinBlocks64 = 4;   // FP64 mode: more registers for the certification
// A stage: the tile's record head and its coordinate planes and, with per-point bounds,
// the per-point state (block id, bound, pass of the bound), all by bulk copy.
template <int D, bool BOUNDS>
struct AStage {
    float4 rec[2 + 2 * kFastCands];
    float x[D][kTile];
};
template <int D>
struct AStage<D, true> {
    float4 rec[2 + 2 * kFastCands];
    float x[D][kTile];
    int a[kTile];             // block ids: the previous ones, then this pass's
    float lq[kTile];          // log2 of the bound, at t1
    unsigned char t1[kTile];
};
static_assert(sizeof(AStage<2, false>) * 2 * kAWarps >= 3 * kAWarps * kTile * 4,
              "scratch of the cooperative tiles (at least two stages per warp)");
// shared-memory stages per warp: three (a tile evaluated while the next two copies are in
// flight), two with the per-point bounds, whose stages are larger
template <int D, bool BOUNDS>
constexpr size_t assign_smem() { return sizeof(AStage<D, BOUNDS>) * (BOUNDS ? 2 : 3) * kAWarps; }

// BOUNDS: per-point bounds across the passes of a phase (gk_options.bounds); without
// them every point is evaluated every pass.
template <int D, bool F64MODE, bool BOUNDS>
__global__ void __launch_bounds__(kAWarps * 32, F64MODE ? kAMinBlocks64 : kAMinBlocks) assign_kernel(Prob p) {
    count_launch(p.ctl);
    if (blockIdx.x == 0 && threadIdx.x == 0) p.ctl->t_assign0 = globaltimer_ns();
    extern __shared__ __align__(128) unsigned char a_dsm[];
    constexpr int kStg = BOUNDS ? 2 : 3;  // must match assign_smem
    AStage<D, BOUNDS> (*st)[kStg] = reinterpret_cast<AStage<D, BOUNDS> (*)[kStg]>(a_dsm);
    __shared__ __align__(8) unsigned long long bar[kAWarps][3];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        for (int i = 0; i < kStg; ++i) mbar_init(&bar[w][i], 1);
        fence_mbarrier_init();
    }
    __syncwarp();
    const int sel = p.ctl->isel;
    unsigned long long nre = 0, nevl = 0;
    // per-point bounds: this pass's index in the phase; a fresh pass evaluates every point
    const int pp = BOUNDS ? p.ctl->phase_pass : 0;
    const bool fresh = !BOUNDS || pp == 0;
    // bytes of one stage's copies besides the record head: coordinate planes (and state)
    const unsigned bytes_pts = (unsigned)(D * kTile * 4) + (fresh ? 0u : (unsigned)(kTile * 9));
    __shared__ float dm_s[kSkipHist];
    __shared__ unsigned char s_act[kAWarps][kTile];  // the points the warp evaluates
    if (!fresh)
        for (int i = threadIdx.x; i <= pp; i += kAWarps * 32) dm_s[i] = p.dm[i];
    __syncthreads();
    {
        // cooperative tiles first (the stages serve as scratch; no copy is in flight yet)
        const int HC = (int)p.ctl->coop_cnt;
        float *scratch = reinterpret_cast<float *>(&st[0][0]);
        for (int ci = blockIdx.x; ci < HC; ci += gridDim.x) {
            coop_tile<D, F64MODE, BOUNDS>(p, p.coop[ci], scratch, kAWarps, &nre, pp, &nevl);
            fence_proxy_async();  // the scratch writes precede the stages' bulk copies
            __syncthreads();
        }
    }
    // The record head is copied up to the tile's last candidate only: cnt (1 .. kFastCands,
    // read from the record when the queue position was resolved) candidates of 2 float4.
    auto issue = [&](int t, int cnt, int b) {
        if (lane == 0) {
            const unsigned rec_bytes = (unsigned)(2 + 2 * cnt) * 16u;
            fence_proxy_async();
            mbar_expect_tx(&bar[w][b], rec_bytes + bytes_pts);
            bulk_g2s(st[w][b].rec, p.trec + (size_t)t * kRecF4, rec_bytes, &bar[w][b]);
            for (int j = 0; j < D; ++j)
                bulk_g2s(st[w][b].x[j], p.X32 + (size_t)j * p.n_pad + (size_t)t * kTile, kTile * 4,
                         &bar[w][b]);
            if constexpr (BOUNDS) {
                if (!fresh) {
                    bulk_g2s(st[w][b].a, p.A + (size_t)t * kTile, kTile * 4, &bar[w][b]);
                    bulk_g2s(st[w][b].lq, p.lq + (size_t)t * kTile, kTile * 4, &bar[w][b]);
                    bulk_g2s(st[w][b].t1, p.t1 + (size_t)t * kTile, kTile, &bar[w][b]);
                }
            }
        }
    };
    // The tiles come from the filter's work list: (tile, candidate count) of every tile
    // with 2 to kFastCands candidates (with per-point bounds, 1 to kFastCands); a tile
    // with one candidate was finished by the filter, a longer list goes to the
    // cooperative CTAs above.  The list is served as kQueues interleaved queues: queue q
    // serves positions q, q + kQueues, ...  A warp claims qch positions at a time (one
    // atomic per chunk) and reads them in parallel, lane j of a half of the ring below
    // one position.  The ring has two halves of qch entries; a half is claimed and read
    // again as soon as its last entry is taken, so its loads have the other half's tiles
    // of work to arrive.  A warp's positions increase, so the first position past the end
    // means that the warp is done.  The tiles go through the warp's two shared-memory
    // stages in order of arrival: a tile's copy is issued when it is taken from the ring
    // and it is evaluated when a later tile needs its stage (or at the end).
    const int qi = (blockIdx.x * kAWarps + w) & (kQueues - 1);
    unsigned *qctr = &p.ctl->tile_q[qi * kQueueStride];
    const long long mcnt = (long long)p.ctl->multi_cnt;
    auto resolve = [&](unsigned m, int &tile, int &cnt) {
        const long long pos = (long long)qi + (long long)kQueues * m;
        if (pos >= mcnt) {
            tile = p.ntiles;
            cnt = 0;
            return;
        }
        const int2 e = __ldcg(&p.mlist[pos]);
        tile = e.x;
        cnt = e.y;
    };
    // A chunk is at most 8 positions and at most 1/16 of a warp's share of the list, so
    // that a warp with few tiles does not hold work the others could take.
    const int qch = (int)min(8LL, max(1LL, mcnt / ((long long)gridDim.x * kAWarps * 16)));
    int r_tile = p.ntiles, r_cnt = 0;  // this lane's ring entry
    // chunk bases are claimed one chunk ahead of their use (lane 0), so that the atomic's
    // latency is not waited for
    unsigned nb = lane == 0 ? atomicAdd(qctr, (unsigned)qch) : 0u;
    auto resolve_half = [&](int h) {
        const unsigned base = __shfl_sync(0xffffffffu, nb, 0);
        if (lane == 0) nb = atomicAdd(qctr, (unsigned)qch);
        const int j = lane - h * qch;
        if (j >= 0 && j < qch) resolve(base + (unsigned)j, r_tile, r_cnt);
    };
    resolve_half(0);
    resolve_half(1);
    int cc = 0;  // ring entry taken next
    // The stages form a ring used in order: the oldest busy stage is s_head, s_busy are
    // in flight; a tile goes into stage (s_head + s_busy) mod kStg.
    int s_t0 = -1, s_t1 = -1, s_t2 = -1;  // tile in each stage
    auto stile = [&](int b) -> int { return b == 0 ? s_t0 : (b == 1 ? s_t1 : s_t2); };
    auto set_stile = [&](int b, int v) {
        if (b == 0) s_t0 = v;
        else if (b == 1) s_t1 = v;
        else s_t2 = v;
    };
    int s_head = 0, s_busy = 0;
    int pend = -1, pend_cnt = 0;  // the tile to copy into the stage being evaluated
    unsigned phs = 0;             // the stages' mbarrier phases (bit b)
    // once stage b has been read: its next tile's copy (lane 0)
    auto refill = [&](int b) {
        if (pend >= 0) issue(pend, pend_cnt, b);
    };
    // Evaluates the tile of stage b (waits for its copy); false when the copy timed out.
    auto process = [&](int b) -> bool {
        const int t = stile(b);
        const unsigned phb = (phs >> b) & 1u;
        bool ok = mbar_wait_bounded(&bar[w][b], phb);
        if (!__all_sync(0xffffffffu, ok)) {
            // A bulk copy did not arrive in time: record it and stop this warp after a
            // bounded wait for the copies still in flight (this stage and the others).
            if (lane == 0) atomicCAS(&p.ctl->status, kOk, kErrTimeout);
            mbar_wait_bounded(&bar[w][b], phb);
            for (int i = 1; i < s_busy; ++i) {
                const int o = (s_head + i) % kStg;
                mbar_wait_bounded(&bar[w][o], (phs >> o) & 1u);
            }
            return false;
        }
        phs ^= 1u << b;
        AStage<D, BOUNDS> &S = st[w][b];
        const int ncand = __float_as_int(S.rec[0].x);  // 0 < ncand <= kFastCands
        const float gl = S.rec[0].y;    // largest g among the tile's candidates
        const float lamT = S.rec[0].z;  // lower bound of the E of every center left out
        const int prev_id = __float_as_int(S.rec[0].w);  // the tile's stored-id marker
        const float sg = sqrtf(gl);
        const float4 ob = S.rec[1];
        const float o[3] = {ob.x, ob.y, ob.z};
        const long long t0 = (long long)t * kTile;
        const long long i0 = t0 + lane * 8;
        long long nv = p.n - i0;
        const int nval = nv <= 0 ? 0 : (nv >= 8 ? 8 : (int)nv);
        // error-bound constants of the FP64 mode (see the comment above); the coordinate
        // term with the tile's radius (rounded up), which bounds |x'| of all its points
        const float sd = sqrtf((float)D);
        const float beta2 = ((float)D + 4.0f + 8.0f * sd) * kU;
        const float e0 = sd * kU * (p.R + 8.0f * __fmul_ru(ob.w, 1.0f + 9.5367431640625e-7f));
        int best[8];
        bool uni = false;  // every point of the tile in one block
        if (fresh) {
            // every point is evaluated: lane l takes points 8l..8l+7
            nevl += (unsigned long long)(p.n - t0 < kTile ? p.n - t0 : kTile);
            float2 xp[3][4];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const float4 *src = reinterpret_cast<const float4 *>(&S.x[j][lane * 8]);
                float4 a = src[0], c4 = src[1];
                xp[j][0] = make_float2(a.x - o[j], a.y - o[j]);
                xp[j][1] = make_float2(a.z - o[j], a.w - o[j]);
                xp[j][2] = make_float2(c4.x - o[j], c4.y - o[j]);
                xp[j][3] = make_float2(c4.z - o[j], c4.w - o[j]);
            }
            float E1[8], E2[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                E1[q] = INFINITY;
                E2[q] = INFINITY;
                best[q] = 0;
            }
            // candidates from the stage (shared-memory broadcast), two at a time
            auto consume = [&](const float4 &qg, int c) {
                const float2 g2 = make_float2(qg.w, qg.w), nqx = make_float2(-qg.x, -qg.x),
                             nqy = make_float2(-qg.y, -qg.y), nqz = make_float2(-qg.z, -qg.z);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 dx = __fadd2_rn(xp[0][q], nqx);
                    const float2 dy = __fadd2_rn(xp[1][q], nqy);
                    float2 ss = __fmul2_rn(dx, dx);
                    ss = __ffma2_rn(dy, dy, ss);
                    if (D == 3) {
                        const float2 dz = __fadd2_rn(xp[2][q], nqz);
                        ss = __ffma2_rn(dz, dz, ss);
                    }
                    const float2 E = __fmul2_rn(g2, ss);
                    argmin_update<F64MODE || BOUNDS>(E.x, c, E1[2 * q], E2[2 * q], best[2 * q]);
                    argmin_update<F64MODE || BOUNDS>(E.y, c, E1[2 * q + 1], E2[2 * q + 1], best[2 * q + 1]);
                }
            };
            // two candidates at a time (ascending center ids)
            auto dist2 = [&](const float4 &qg, int q) -> float2 {
                const float2 dx = __fadd2_rn(xp[0][q], make_float2(-qg.x, -qg.x));
                const float2 dy = __fadd2_rn(xp[1][q], make_float2(-qg.y, -qg.y));
                float2 ss = __fmul2_rn(dx, dx);
                ss = __ffma2_rn(dy, dy, ss);
                if (D == 3) {
                    const float2 dz = __fadd2_rn(xp[2][q], make_float2(-qg.z, -qg.z));
                    ss = __ffma2_rn(dz, dz, ss);
                }
                return __fmul2_rn(make_float2(qg.w, qg.w), ss);
            };
            int jj = 0;
            for (; jj + 1 < ncand; jj += 2) {
                const float4 qa = S.rec[2 + 2 * jj], qb = S.rec[4 + 2 * jj];
                const int ca = __float_as_int(S.rec[3 + 2 * jj].x), cb = __float_as_int(S.rec[5 + 2 * jj].x);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 Ea = dist2(qa, q), Eb = dist2(qb, q);
                    argmin_update2<F64MODE || BOUNDS>(Ea.x, ca, Eb.x, cb, E1[2 * q], E2[2 * q], best[2 * q]);
                    argmin_update2<F64MODE || BOUNDS>(Ea.y, ca, Eb.y, cb, E1[2 * q + 1], E2[2 * q + 1],
                                                      best[2 * q + 1]);
                }
            }
            if (jj < ncand) {
                const float4 qa = S.rec[2 + 2 * jj];
                consume(qa, __float_as_int(S.rec[3 + 2 * jj].x));
            }
            unsigned flag = 0;
            float Bl = 0.0f;
            if (F64MODE) {
                // error-bound constants; see the comment above
                const float R = p.R;
                const float sd = sqrtf((float)D);
                const float beta2 = ((float)D + 4.0f + 8.0f * sd) * kU;
                // coordinate term with the largest |x'| of the lane's points
                float xn2 = 0.0f;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < D; ++j) acc = __ffma2_rn(xp[j][q], xp[j][q], acc);
                    xn2 = fmaxf(xn2, fmaxf(acc.x, acc.y));
                }
                const float e0 = sd * kU * (R + 8.0f * __fsqrt_ru(__fmul_ru(xn2, 1.0f + 4.0f * kU)));
                // B grows with E: one bound at the lane's largest finite runner-up certifies
                // most points; a point it does not certify gets its own bound
                float e2max = 0.0f;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (E2[q] < INFINITY) e2max = fmaxf(e2max, E2[q]);
                Bl = cert_bound(e0, sg, gl, beta2, e2max);
                float thr[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const bool single = E2[q] == INFINITY && E1[q] < INFINITY;
                    bool okq = single || (E2[q] - E1[q]) > 2.0f * Bl;
                    thr[q] = INFINITY;
                    if (!okq) {
                        const float B = cert_bound(e0, sg, gl, beta2, E2[q]);
                        okq = (E2[q] - E1[q]) > 2.0f * B;
                        thr[q] = E1[q] + 2.0f * B;  // every possible FP64 winner has E_fp32 <= thr
                    }
                    if (q < nval && !okq) flag |= 1u << q;
                }
                // FP64 re-decision, one flagged point at a time: lane j takes candidate j,
                // screens it with the FP32 value (every possible FP64 winner has E_fp32 <=
                // thr) and evaluates a survivor in FP64 from the raw coordinates; the warp
                // keeps the smallest value, the lowest center index on ties.
                const double *g64 = p.g64_2 + (size_t)sel * p.k;
                unsigned lanes = __ballot_sync(0xffffffffu, flag != 0u);
                while (lanes) {
                    const int Lf = __ffs(lanes) - 1;
                    lanes &= lanes - 1;
                    unsigned fl = __shfl_sync(0xffffffffu, flag, Lf);
                    while (fl) {
                        const int q = __ffs(fl) - 1;
                        fl &= fl - 1;
                        float mx[3] = {0.f, 0.f, 0.f}, mt = 0.f;
#pragma unroll
                        for (int qq = 0; qq < 8; ++qq) {
                            if (qq == q) {
#pragma unroll
                                for (int j = 0; j < D; ++j) mx[j] = (qq & 1) ? xp[j][qq >> 1].y : xp[j][qq >> 1].x;
                                mt = thr[qq];
                            }
                        }
#pragma unroll
                        for (int j = 0; j < D; ++j) mx[j] = __shfl_sync(0xffffffffu, mx[j], Lf);
                        mt = __shfl_sync(0xffffffffu, mt, Lf);
                        const long long ip = (long long)t * kTile + Lf * 8 + q;
                        double bE = INFINITY;
                        int bc = 0x7fffffff;
                        if (lane < ncand) {
                            const float4 qg = S.rec[2 + 2 * lane];
                            const int c = __float_as_int(S.rec[3 + 2 * lane].x);
                            const float d0 = mx[0] - qg.x, d1 = mx[1] - qg.y;
                            const float d2 = D == 3 ? mx[2] - qg.z : 0.0f;
                            const float E32 = qg.w * fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
                            if (E32 <= mt) {
                                double s2 = 0.0;
#pragma unroll
                                for (int j = 0; j < D; ++j) {
                                    const double xj = p.dtype == 1 ? p.X64[(size_t)j * p.n_pad + ip]
                                                                   : (double)p.X32[(size_t)j * p.n_pad + ip];
                                    const double df = xj - p.C[c * D + j];
                                    s2 += df * df;
                                }
                                bE = s2 * g64[c];
                                bc = c;
                            }
                        }
                        for (int off = 16; off; off >>= 1) {
                            const double oE = __shfl_xor_sync(0xffffffffu, bE, off);
                            const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
                            if (oE < bE || (oE == bE && oc < bc)) {
                                bE = oE;
                                bc = oc;
                            }
                        }
                        if (lane == Lf && bc != 0x7fffffff) {
#pragma unroll
                            for (int qq = 0; qq < 8; ++qq)
                                if (qq == q) best[qq] = bc;
                        }
                    }
                }
                nre += __popc(flag);
            }
            if constexpr (BOUNDS) {  // each point's bound for the next passes of the phase
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q >= nval) continue;
                    p.lq[i0 + q] = bound_lq<F64MODE>(E1[q], E2[q], Bl, lamT, (flag >> q) & 1u);
                    p.t1[i0 + q] = (unsigned char)pp;
                }
            }
            __syncwarp();  // every lane is done with stage b
            refill(b);
            uni = store_blocks_tile(p, t, i0, nval, best, prev_id);
        } else {
            if constexpr (BOUNDS) {
                int *blk = S.a;  // old block ids (bounds), then this pass's
                unsigned char *alist = s_act[w];
                // 1. the lane's points to evaluate: a point keeps its block when rho exceeds the
                //    largest growth of any center's g since its last evaluation t1 over the smallest
                //    (rho: the ratio of the other centers' smallest E to its own E then, stored as
                //    lq = log2 rho rounded down; dm[t1] = log2 of a lower bound of that smallest
                //    over that largest growth): then its own E stays below every other center's.
                unsigned act = nval >= 8 ? 0xffu : ((1u << nval) - 1u);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q < nval) {
                        const int pi = lane * 8 + q;
                        const int t1q = min((int)S.t1[pi], pp);
                        if (__fadd_rd(S.lq[pi], dm_s[t1q]) > 0.0f) act &= ~(1u << q);
                    }
                }
                // 2. the warp's list of points to evaluate, in tile order
                const unsigned cl = __popc(act);
                unsigned pre = cl;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const unsigned y = __shfl_up_sync(0xffffffffu, pre, off);
                    if (lane >= off) pre += y;
                }
                const int nact = (int)__shfl_sync(0xffffffffu, pre, 31);
                {
                    unsigned pos = pre - cl;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if ((act >> q) & 1u) alist[pos++] = (unsigned char)(lane * 8 + q);
                }
                __syncwarp();
                nevl += (unsigned long long)nact;
                // 3. the points of the list, two per lane and round (packed f32x2)
                for (int r0 = 0; r0 < nact; r0 += 64) {
                    const int a0 = r0 + lane, a1 = r0 + 32 + lane;
                    const bool vq[2] = {a0 < nact, a1 < nact};
                    const int pi[2] = {vq[0] ? (int)alist[a0] : 0, vq[1] ? (int)alist[a1] : 0};
                    float2 xp[3];
#pragma unroll
                    for (int j = 0; j < 3; ++j) xp[j] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < D; ++j) xp[j] = make_float2(S.x[j][pi[0]] - o[j], S.x[j][pi[1]] - o[j]);
                    float E1[2] = {INFINITY, INFINITY}, E2[2] = {INFINITY, INFINITY};
                    int best[2] = {0, 0};
                    auto consume = [&](const float4 &qg, int c) {
                        const float2 g2 = make_float2(qg.w, qg.w);
                        const float2 dx = __fadd2_rn(xp[0], make_float2(-qg.x, -qg.x));
                        const float2 dy = __fadd2_rn(xp[1], make_float2(-qg.y, -qg.y));
                        float2 ss = __fmul2_rn(dx, dx);
                        ss = __ffma2_rn(dy, dy, ss);
                        if (D == 3) {
                            const float2 dz = __fadd2_rn(xp[2], make_float2(-qg.z, -qg.z));
                            ss = __ffma2_rn(dz, dz, ss);
                        }
                        const float2 E = __fmul2_rn(g2, ss);
                        argmin_update<true>(E.x, c, E1[0], E2[0], best[0]);
                        argmin_update<true>(E.y, c, E1[1], E2[1], best[1]);
                    };
                    int jj = 0;
                    for (; jj + 1 < ncand; jj += 2) {
                        const float4 qa = S.rec[2 + 2 * jj], qb = S.rec[4 + 2 * jj];
                        const int ca = __float_as_int(S.rec[3 + 2 * jj].x), cb = __float_as_int(S.rec[5 + 2 * jj].x);
                        consume(qa, ca);
                        consume(qb, cb);
                    }
                    if (jj < ncand) consume(S.rec[2 + 2 * jj], __float_as_int(S.rec[3 + 2 * jj].x));
                    float Bq[2] = {0.0f, 0.0f};
                    unsigned flag = 0;
                    if (F64MODE) {
                        float e2max = 0.0f;
#pragma unroll
                        for (int q = 0; q < 2; ++q)
                            if (E2[q] < INFINITY) e2max = fmaxf(e2max, E2[q]);
                        const float Bl = cert_bound(e0, sg, gl, beta2, e2max);
                        float thr[2];
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const bool single = E2[q] == INFINITY && E1[q] < INFINITY;
                            bool okq = single || (E2[q] - E1[q]) > 2.0f * Bl;
                            Bq[q] = Bl;
                            thr[q] = INFINITY;
                            if (!okq) {
                                const float B = cert_bound(e0, sg, gl, beta2, E2[q]);
                                okq = (E2[q] - E1[q]) > 2.0f * B;
                                thr[q] = E1[q] + 2.0f * B;  // every possible FP64 winner has E_fp32 <= thr
                                Bq[q] = B;
                            }
                            if (vq[q] && !okq) flag |= 1u << q;
                        }
                        // FP64 re-decision, one flagged point at a time: lane j takes candidate j,
                        // screens it with the FP32 value (every possible FP64 winner has E_fp32 <=
                        // thr) and evaluates a survivor in FP64 from the raw coordinates; the warp
                        // keeps the smallest value, the lowest center index on ties.
                        const double *g64 = p.g64_2 + (size_t)sel * p.k;
                        unsigned lanes = __ballot_sync(0xffffffffu, flag != 0u);
                        while (lanes) {
                            const int Lf = __ffs(lanes) - 1;
                            lanes &= lanes - 1;
                            unsigned fl = __shfl_sync(0xffffffffu, flag, Lf);
                            while (fl) {
                                const int q = __ffs(fl) - 1;
                                fl &= fl - 1;
                                float mx[3] = {0.f, 0.f, 0.f};
#pragma unroll
                                for (int j = 0; j < D; ++j) mx[j] = __shfl_sync(0xffffffffu, q ? xp[j].y : xp[j].x, Lf);
                                const float mt = __shfl_sync(0xffffffffu, q ? thr[1] : thr[0], Lf);
                                const int pq = __shfl_sync(0xffffffffu, q ? pi[1] : pi[0], Lf);
                                const long long ip = t0 + pq;
                                double bE = INFINITY;
                                int bc = 0x7fffffff;
                                if (lane < ncand) {
                                    const float4 qg = S.rec[2 + 2 * lane];
                                    const int c = __float_as_int(S.rec[3 + 2 * lane].x);
                                    const float d0 = mx[0] - qg.x, d1 = mx[1] - qg.y;
                                    const float d2 = D == 3 ? mx[2] - qg.z : 0.0f;
                                    const float E32 = qg.w * fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
                                    if (E32 <= mt) {
                                        double s2 = 0.0;
#pragma unroll
                                        for (int j = 0; j < D; ++j) {
                                            const double xj = p.dtype == 1 ? p.X64[(size_t)j * p.n_pad + ip]
                                                                           : (double)p.X32[(size_t)j * p.n_pad + ip];
                                            const double df = xj - p.C[c * D + j];
                                            s2 += df * df;
                                        }
                                        bE = s2 * g64[c];
                                        bc = c;
                                    }
                                }
                                for (int off = 16; off; off >>= 1) {
                                    const double oE = __shfl_xor_sync(0xffffffffu, bE, off);
                                    const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
                                    if (oE < bE || (oE == bE && oc < bc)) {
                                        bE = oE;
                                        bc = oc;
                                    }
                                }
                                if (lane == Lf && bc != 0x7fffffff) {
                                    if (q)
                                        best[1] = bc;
                                    else
                                        best[0] = bc;
                                }
                            }
                        }
                        nre += __popc(flag);
                    }
                    // block ids, and each point's bound for the next passes: rho = (lower bound of
                    // every other center's E) / (upper bound of E_own), rounded down; a re-decided
                    // point gets 0 (it is evaluated again next pass)
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        if (!vq[q]) continue;
                        blk[pi[q]] = best[q];
                        p.A[t0 + pi[q]] = best[q];
                        p.lq[t0 + pi[q]] = bound_lq<F64MODE>(E1[q], E2[q], Bq[q], lamT, (flag >> q) & 1u);
                        p.t1[t0 + pi[q]] = (unsigned char)pp;
                    }
                }
                __syncwarp();  // every lane is done with the list and has written its block ids
                // block ids of the lane's points
#pragma unroll
                for (int q = 0; q < 8; ++q) best[q] = q < nval ? blk[lane * 8 + q] : 0;
                fence_proxy_async();  // the stage's block ids were written: order before its refill
                __syncwarp();         // every lane is done with stage b
                refill(b);
                    }
        }
        if (uni) {
            if (lane == 0) tile_weight_to(p, t, best[0]);
        } else {
            tile_histogram(p, i0, nval, best);
        }
        return true;
    };
    // One call site of process (the evaluation is long: a second inlined copy would only
    // crowd the instruction cache).  Until the ring of entries runs out, a tile goes into
    // a free stage, or the oldest busy stage is evaluated and then takes it; after that the
    // busy stages are evaluated in order of their copies.
    bool done = false;
    for (;;) {
        int tile = -1, cnt = 0;
        if (!done) {
            // the next ring entry (every lane holds the same warp-wide state)
            tile = __shfl_sync(0xffffffffu, r_tile, cc);
            cnt = __shfl_sync(0xffffffffu, r_cnt, cc);
            ++cc;
            if (cc == qch) {
                resolve_half(0);
            } else if (cc == 2 * qch) {
                resolve_half(1);
                cc = 0;
            }
            if (tile >= p.ntiles) done = true;
            else if (cnt < 0 || cnt > kFastCands) continue;  // never on the list: cooperative tiles
        }
        if (!done) {
            if (s_busy < kStg) {  // a free stage: copy the tile in
                const int fb = (s_head + s_busy) % kStg;
                issue(tile, cnt, fb);
                set_stile(fb, tile);
                ++s_busy;
                continue;
            }
            pend = tile;  // all busy: evaluate the oldest and copy this tile into it
            pend_cnt = cnt;
        } else if (s_busy == 0) {
            break;
        }
        const int b = s_head;
        if (!process(b)) return;
        if (pend >= 0) {
            set_stile(b, pend);  // now the newest
        } else {
            set_stile(b, -1);
            --s_busy;
        }
        s_head = (s_head + 1) % kStg;
        pend = -1;
    }
    if (F64MODE) {
        for (int off = 16; off; off >>= 1) nre += __shfl_xor_sync(0xffffffffu, nre, off);
        if (lane == 0 && nre) atomicAdd(&p.ctl->rechecks, nre);
    }
    if (lane == 0 && nevl) atomicAdd(&p.ctl->evaluated, nevl);  // nevl is the same in every lane
}

// ------------------------------------------------------------------------------
// Block weights of a given assignment (standalone movement step).
// ------------------------------------------------------------------------------
__global__ void block_weights_kernel(Prob p) {
    count_launch(p.ctl);
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int b = i < p.n ? p.A[i] : -1;
    bool valid = i < p.n && (unsigned)b < (unsigned)p.k;
    if (i < p.n && !valid) atomicOr(&p.ctl->bad_block, 1);
    unsigned long long v = 1;
    if (valid && p.weighted)
        v = (unsigned long long)(p.dtype == 1 ? fix_f64(((const double *)p.Ws)[i], p.Fw)
                                              : fix_f32(((const float *)p.Ws)[i], p.Fw));
    if (valid) red_add_u64(&p.Sfix[2 * b], v);
}

// ------------------------------------------------------------------------------
// Balance test and influence update (Section 2 bound; Section 4.2 Eq. 1 as read:
// I_c <- I_c * clamp((W/k / S_c)^(1/d), 0.95, 1.05)).  Every CTA converts its block
// weights, resets the accumulators and writes the tentatively updated influence into
// the other buffer; the last CTA takes the decision: balanced keeps the buffer,
// unbalanced flips it.  mode 0: main loop, 1: final passes with the centers fixed,
// 2: block weights only (standalone assignment).
// ------------------------------------------------------------------------------
__global__ void __launch_bounds__(kKThreads) balance_kernel(Prob p, int mode,
                                                            cudaGraphConditionalHandle h) {
    count_launch(p.ctl);
    Ctl *ctl = p.ctl;
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // the assignment kernel ran just before
        ctl->assign_ns += globaltimer_ns() - ctl->t_assign0;
        ctl->assign_cnt += 1;
    }
    const int sel = ctl->isel, nsel = sel ^ 1;
    const int gshift = ctl->gshift;
    const double target = ctl->target;
    // per-point bounds: this pass's index in the phase and the next one's (a wrap starts
    // a fresh pass, with the new g as its reference)
    const bool bnd = p.bounds && mode != 2;
    const int pp = ctl->phase_pass;
    const bool wrap = pp + 1 >= kSkipHist;
    float lr = INFINITY, lrh = -INFINITY;  // log2 of this center's g ratio, rounded down / up
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    double S = 0.0, gnew = 0.0;
    float4 hc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c < p.k) {
        const unsigned long long w0 = p.Sfix[2 * c], w1 = p.Sfix[2 * c + 1];
        S = p.weighted ? split_to_f64(w0, w1, p.Fw) : (double)(w0 + (w1 << 32));  // counts < 2^53
        p.S64[c] = S;
        p.Sfix[2 * c] = 0ull;
        p.Sfix[2 * c + 1] = 0ull;
        if (mode != 2) {
            double I = p.I2[(size_t)sel * p.k + c];
            double f;
            if (S > 0.0) {
                double gamma = target / S;
                f = p.d == 2 ? sqrt(gamma) : cbrt(gamma);
            } else {
                f = INFINITY;
            }
            f = fmin(fmax(f, 0.95), 1.05);
            double In = I * f;
            gnew = 1.0 / (In * In);
            p.I2[(size_t)nsel * p.k + c] = In;
            p.g64_2[(size_t)nsel * p.k + c] = gnew;
            if (bnd) {
                const float lgn = lg_of(gnew);
                p.lg[(size_t)(wrap ? 0 : pp + 1) * p.k + c] = lgn;
                if (!wrap) {
                    const float lgo = p.lg[(size_t)pp * p.k + c];
                    lr = __fsub_rd(lgn, lgo);
                    lrh = __fsub_ru(lgn, lgo);
                    if (lr != lr || lrh != lrh) {  // NaN: no bound
                        lr = -INFINITY;
                        lrh = INFINITY;
                    }
                }
            }
            hc = p.cdata2[(size_t)sel * 2 * p.k + 2 * c];
            hc.w = scaled_g32(gnew, gshift);
            p.cdata2[(size_t)nsel * 2 * p.k + 2 * c] = hc;
        }
    }
    if (mode != 2) {
        const float hi[3] = {hc.x, hc.y, hc.z};
        write_group(p, p.gdata2 + (size_t)nsel * 2 * p.ngroups, c < p.k, hi, hc.w);
    }
    // the CTA is one warp (kKThreads == 32): warp reductions of the two maxima
    double mS = S, mg = gnew;
    for (int off = 16; off; off >>= 1) {
        mS = fmax(mS, __shfl_xor_sync(0xffffffffu, mS, off));
        mg = fmax(mg, __shfl_xor_sync(0xffffffffu, mg, off));
        lr = fminf(lr, __shfl_xor_sync(0xffffffffu, lr, off));
        lrh = fmaxf(lrh, __shfl_xor_sync(0xffffffffu, lrh, off));
    }
    if (threadIdx.x == 0) {
        atomicMax(&ctl->maxS_key, okey_f64(mS));
        if (mode != 2) atomicMax(&ctl->maxg_key, okey_f64(mg));
        if (bnd && !wrap) {
            atomicMin(&ctl->min_lr_key, okey_f32(lr));
            atomicMax(&ctl->max_lr_key, okey_f32(lrh));
        }
    }
    const bool last = last_block(ctl);
    __shared__ int s_newpp;
    if (last && threadIdx.x == 0) s_newpp = -1;
    if (last && threadIdx.x == 0) {
        // the other CTAs' atomics precede the last-block fence: plain L2 loads, in parallel
        double maxS = okey_to_f64(__ldcg(&ctl->maxS_key));
        double maxg = okey_to_f64(__ldcg(&ctl->maxg_key));
        ctl->maxS_key = 0ull;
        ctl->maxg_key = 0ull;
        ctl->coop_cnt = 0u;  // the next filter rebuilds the cooperative list
        ctl->big_cnt = 0u;
        ctl->multi_cnt = 0u;  // and the work list
        ctl->jump_cnt = 0u;
        int bal = maxS <= ctl->bound;
        ctl->max_imbalance = maxS / ctl->ceil_avg - 1.0;
        if (mode == 2) return;
        ctl->balanced = bal;
        ctl->passes += 1;
        ctl->iused_sel = sel;
        if (mode == 0)
            ctl->pass_in_phase += 1;
        else
            ctl->final_passes += 1;
        if (!bal) {
            ctl->isel = nsel;
            ctl->gshift = exponent_above(maxg);
        }
        if (bnd) {
            // the next pass continues the phase: the running sum of the passes' (smallest -
            // largest) log2 g ratio, lowered by the margin for the rounding of the logs
            const float m = okey_to_f32(__ldcg(&ctl->min_lr_key)), M = okey_to_f32(__ldcg(&ctl->max_lr_key));
            ctl->min_lr_key = 0xffffffffu;
            ctl->max_lr_key = 0u;
            if (!bal) {
                const int np = wrap ? 0 : pp + 1;
                p.cumm[np] = wrap ? 0.0 : p.cumm[pp] + ((double)m - (double)M - 2.0 * (double)kLgMargin);
                ctl->phase_pass = np;
                s_newpp = np;
            }
        }
        int cont;
        if (mode == 0)
            cont = !bal && ctl->pass_in_phase < p.max_balance_iter;
        else
            cont = !bal && ctl->final_passes < p.final_balance_iter;
        cont = cont && ctl->status == kOk;
        if (mode == 0)
            ctl->cont_balance = cont;
        else
            ctl->cont_final = cont;
        if (h) cudaGraphSetConditional(h, (unsigned)cont);
    }
    if (last) {
        // dm[t1] = cumm[t] - cumm[t1] rounded down, for every earlier pass t1 of the phase
        __syncwarp();
        const int np = s_newpp;
        if (np >= 0) {
            const double ct = __ldcg(&p.cumm[np]);
            for (int t1 = threadIdx.x; t1 <= np; t1 += blockDim.x)
                p.dm[t1] = __double2float_rd(ct - __ldcg(&p.cumm[t1]));
        }
    }
}

// ------------------------------------------------------------------------------
// Center movement, part 1: exact 128-bit fixed-point sums of w*x per block and axis
// and the block bounding boxes (ordered keys, input precision).  One warp per 256
// curve-consecutive points; runs inside a lane, then a segmented reduction over lanes.
// ------------------------------------------------------------------------------
template <typename T>
struct KeyOf;
template <>
struct KeyOf<float> {
    __device__ static unsigned long long key(float v) { return okey_f32(v); }
};
template <>
struct KeyOf<double> {
    __device__ static unsigned long long key(double v) { return okey_f64(v); }
};

// The lane's 8 consecutive values of a plane starting at i0 (16-byte vector loads when
// all 8 are points; the padding of the planes keeps the loads inside the buffers).
template <typename T>
__device__ __forceinline__ void load8(const T *src, long long i0, int nval, T v[8]) {
    if (nval == 8) {
        if constexpr (sizeof(T) == 4) {
            const float4 a = reinterpret_cast<const float4 *>(src + i0)[0];
            const float4 b = reinterpret_cast<const float4 *>(src + i0)[1];
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const double2 a = reinterpret_cast<const double2 *>(src + i0)[h];
                v[2 * h] = a.x;
                v[2 * h + 1] = a.y;
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = q < nval ? src[i0 + q] : (T)0;
    }
}

// The lane's 8 block ids starting at i0 (one 16-byte load when all 8 are points).
__device__ __forceinline__ void load_ids8(const Prob &p, long long i0, int nval, int ids[8]) {
    if (nval == 8 && p.a16) {
        const uint4 v = *reinterpret_cast<const uint4 *>(p.A16 + i0);
        const unsigned u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            ids[2 * h] = (int)(u[h] & 0xffffu);
            ids[2 * h + 1] = (int)(u[h] >> 16);
        }
    } else if (nval == 8) {
        const int4 a = reinterpret_cast<const int4 *>(p.A + i0)[0];
        const int4 b = reinterpret_cast<const int4 *>(p.A + i0)[1];
        ids[0] = a.x; ids[1] = a.y; ids[2] = a.z; ids[3] = a.w;
        ids[4] = b.x; ids[5] = b.y; ids[6] = b.z; ids[7] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) ids[q] = q < nval ? (p.a16 ? (int)p.A16[i0 + q] : p.A[i0 + q]) : -1;
    }
}

// The fixed-point value of one point's (weighted) coordinate, as every movement path
// forms it (the sums are exact integers, so the path a tile takes does not matter).
template <typename T>
__device__ __forceinline__ long long cent_fix(const Prob &p, T w, T x) {
    if (sizeof(T) == 8)
        return p.weighted ? fix_f64((double)w * (double)x, p.Fx) : fix_f64((double)x, p.Fx);
    return p.weighted ? fix_prod_f32((float)w, (float)x, p.Fx) : fix_f32((float)x, p.Fx);
}

// One tile (called by the whole warp): lane l takes points 8l..8l+7, loaded with vector
// loads (ids, weights and every coordinate plane, one round trip).  A tile all of whose
// points lie in one block takes one warp reduction and one set of atomics.  Otherwise the
// runs of equal block ids inside each lane are added directly, except the lane's last run,
// which goes through a segmented reduction over the lanes (runs continue across lanes).
// Sums are fixed point (the carry-free form), extremes ordered keys.  (Taking the tile's
// points block by block instead, one warp reduction and one set of atomics per distinct
// block, needed more instructions per tile and was slower at 1e9 points: 2.12 against
// 1.90 ms per movement.)
template <typename T, int D>
__device__ __noinline__ void centroid_tile(const Prob &p, const T *X, int t) {
    const int lane = threadIdx.x & 31;
    const long long i0 = (long long)t * kTile + lane * 8;
    long long nv = p.n - i0;
    const int nval = nv <= 0 ? 0 : (nv >= 8 ? 8 : (int)nv);
    int ids[8];
    load_ids8(p, i0, nval, ids);
    T wv[8];
    if (p.weighted) load8<T>((const T *)p.Ws, i0, nval, wv);
    T xv[D][8];  // every plane, loaded with the ids (one round trip)
#pragma unroll
    for (int j = 0; j < D; ++j) load8<T>(X + (size_t)j * p.n_pad, i0, nval, xv[j]);
    const int b0 = __shfl_sync(0xffffffffu, ids[0], 0);  // lane 0 holds a point of the tile
    bool same = true, bad = false;
    int last = -1;  // block of the lane's last run
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (q < nval) {
            same &= ids[q] == b0;
            if ((unsigned)ids[q] >= (unsigned)p.k) bad = true;
            else last = ids[q];
        }
    }
    if (bad) atomicOr(&p.ctl->bad_block, 1);
    if (__all_sync(0xffffffffu, same) && (unsigned)b0 < (unsigned)p.k) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            long long sum = 0;
            unsigned long long kmin = ~0ull, kmax = 0ull;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (q < nval) {
                    sum += cent_fix<T>(p, p.weighted ? wv[q] : (T)1, xv[j][q]);
                    const unsigned long long kk = KeyOf<T>::key(xv[j][q]);
                    kmin = kk < kmin ? kk : kmin;
                    kmax = kk > kmax ? kk : kmax;
                }
            }
            for (int off = 16; off; off >>= 1) {
                sum += __shfl_xor_sync(0xffffffffu, sum, off);
                const unsigned long long a = __shfl_xor_sync(0xffffffffu, kmin, off);
                const unsigned long long b = __shfl_xor_sync(0xffffffffu, kmax, off);
                kmin = a < kmin ? a : kmin;
                kmax = b > kmax ? b : kmax;
            }
            if (lane == 0) {
                red_add_s64(&p.SXfix[2 * (b0 * D + j)], sum);
                atomicMin(&p.BBlo[b0 * D + j], kmin);
                atomicMax(&p.BBhi[b0 * D + j], kmax);
            }
        }
        return;
    }
    // segments of the lanes' last runs (the same for every plane)
    const int prev = __shfl_up_sync(0xffffffffu, last, 1);
    const bool head = lane == 0 || last != prev;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    const bool end = lane == 31 || ((heads >> (lane + 1)) & 1u);
#pragma unroll
    for (int j = 0; j < D; ++j) {
        int cur = -1;
        long long sum = 0;
        unsigned long long kmin = ~0ull, kmax = 0ull;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q < nval && (unsigned)ids[q] < (unsigned)p.k) {
                if (ids[q] != cur) {
                    if (cur >= 0) {  // a run that ends inside the lane
                        red_add_s64(&p.SXfix[2 * (cur * D + j)], sum);
                        atomicMin(&p.BBlo[cur * D + j], kmin);
                        atomicMax(&p.BBhi[cur * D + j], kmax);
                    }
                    cur = ids[q];
                    sum = 0;
                    kmin = ~0ull;
                    kmax = 0ull;
                }
                sum += cent_fix<T>(p, p.weighted ? wv[q] : (T)1, xv[j][q]);
                const unsigned long long kk = KeyOf<T>::key(xv[j][q]);
                kmin = kk < kmin ? kk : kmin;
                kmax = kk > kmax ? kk : kmax;
            }
        }
        // the lanes' last runs: a run covers at most 256 values below 2^54, so 64 bits
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const bool take = lane - off >= start;
            const long long s2 = __shfl_up_sync(0xffffffffu, sum, off);
            const unsigned long long a = __shfl_up_sync(0xffffffffu, kmin, off);
            const unsigned long long b = __shfl_up_sync(0xffffffffu, kmax, off);
            if (take) {
                sum += s2;
                kmin = a < kmin ? a : kmin;
                kmax = b > kmax ? b : kmax;
            }
        }
        if (end && cur >= 0) {
            red_add_s64(&p.SXfix[2 * (cur * D + j)], sum);
            atomicMin(&p.BBlo[cur * D + j], kmin);
            atomicMax(&p.BBhi[cur * D + j], kmax);
        }
    }
}

// Tiles per warp of the marker path of the movement: a power of two up to 32, the
// largest that still gives about two waves of warps over the SMs (a warp takes the tiles
// without a marker one at a time, so with few tiles per SM fewer per warp keep every SM
// busy).
__host__ __device__ __forceinline__ int centroid_tiles_per_warp(int ntiles, int nsm) {
    const long long want = (long long)(nsm > 0 ? nsm : 1) * 128;  // warps
    int tpw = 32;
    while (tpw > 1 && (long long)ntiles < want * tpw) tpw >>= 1;
    return tpw;
}

// Center movement, part 1 (Algorithm 2, the weighted means; the block boxes of the
// erosion's beta): one warp per tpw consecutive tiles, lane = tile.  A tile whose stored
// block ids are all b (its marker, kept by the assignment) adds its coordinate sums and
// box, formed once at the bootstrap with the same conversions, to block b: a segmented
// reduction over the lanes, then one set of atomics per run of equal blocks.  A tile sum
// is below 2^62 in magnitude (256 values below 2^54), so the reduction over up to 32
// tiles carries 128 bits.  The other tiles go to a list (the cooperative-tile list of the
// assignment, free during the movement) that centroid_list_kernel takes point by point,
// one warp per tile.
template <typename T, int D>
__global__ void __launch_bounds__(kAssignWarps * 32) centroid_kernel(Prob p) {
    count_launch(p.ctl);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tpw = centroid_tiles_per_warp(p.ntiles, p.nsm);
    const long long t = ((long long)blockIdx.x * kAssignWarps + w) * tpw + lane;
    const bool has = lane < tpw && t < p.ntiles;
    const int mk = has ? reinterpret_cast<const int *>(p.tiles)[8 * t + 7] : -2;
    const int cur = mk >= 0 && mk < p.k ? mk : -1;
    unsigned long long slo[D], shi[D];  // 128-bit sums (two's complement)
    unsigned long long kmin[D], kmax[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const long long v = cur >= 0 ? p.tsx[t * D + j] : 0;
        slo[j] = (unsigned long long)v;
        shi[j] = v < 0 ? ~0ull : 0ull;
        kmin[j] = cur >= 0 ? p.tlo[t * D + j] : ~0ull;
        kmax[j] = cur >= 0 ? p.thi[t * D + j] : 0ull;
    }
    int prev = __shfl_up_sync(0xffffffffu, cur, 1);
    bool head = lane == 0 || cur != prev;
    unsigned heads = __ballot_sync(0xffffffffu, head);
    int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        bool take = lane - off >= start;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const unsigned long long l2 = __shfl_up_sync(0xffffffffu, slo[j], off);
            const unsigned long long h2 = __shfl_up_sync(0xffffffffu, shi[j], off);
            unsigned long long a = __shfl_up_sync(0xffffffffu, kmin[j], off);
            unsigned long long b = __shfl_up_sync(0xffffffffu, kmax[j], off);
            if (take) {
                const unsigned long long lo = slo[j] + l2;
                shi[j] += h2 + (lo < l2 ? 1ull : 0ull);
                slo[j] = lo;
                kmin[j] = a < kmin[j] ? a : kmin[j];
                kmax[j] = b > kmax[j] ? b : kmax[j];
            }
        }
    }
    bool end = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (end && cur >= 0) {
        for (int j = 0; j < D; ++j) {
            red_add_s128(&p.SXfix[2 * (cur * D + j)], slo[j], shi[j]);
            atomicMin(&p.BBlo[cur * D + j], kmin[j]);
            atomicMax(&p.BBhi[cur * D + j], kmax[j]);
        }
    }
    const bool mixed = has && cur < 0;
    const unsigned rest = __ballot_sync(0xffffffffu, mixed);
    if (rest) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&p.ctl->mixed_cnt, (unsigned)__popc(rest));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (mixed) p.coop[base + __popc(rest & ((1u << lane) - 1u))] = (int)t;
    }
}

// The tiles the marker pass listed, one warp per tile (grid-stride over the list).
template <typename T, int D>
__global__ void __launch_bounds__(kAssignWarps * 32) centroid_list_kernel(Prob p) {
    count_launch(p.ctl);
    const int cnt = (int)p.ctl->mixed_cnt;
    const T *X = sizeof(T) == 8 ? (const T *)p.X64 : (const T *)p.X32;
    const int nw = gridDim.x * kAssignWarps;
    for (int i = blockIdx.x * kAssignWarps + (threadIdx.x >> 5); i < cnt; i += nw)
        centroid_tile<T, D>(p, X, p.coop[i]);
}

// The same without tile markers: one tile per warp, in the assignment's permuted tile
// order (neighbouring warps take tiles of different blocks).
template <typename T, int D>
__global__ void __launch_bounds__(kAssignWarps * 32) centroid_points_kernel(Prob p) {
    count_launch(p.ctl);
    const int pos = blockIdx.x * kAssignWarps + (threadIdx.x >> 5);
    if (pos >= p.ntiles) return;
    const T *X = sizeof(T) == 8 ? (const T *)p.X64 : (const T *)p.X32;
    centroid_tile<T, D>(p, X, tile_of(p, pos));
}

// ------------------------------------------------------------------------------
// Center movement, part 2 (ceil(k/32) CTAs): C' = sum(w x) / sum(w) (empty block:
// C' = C), delta_c = |C'_c - C_c|, and per-CTA partial sums of the block diagonals;
// the last CTA forms beta (the mean diagonal of the non-empty blocks, summed in CTA
// order), the convergence test and the loop decision.  mode 1: standalone; mode 3:
// a sample round of the random initialization (Section 4.5), which always moves the
// centers and ends its loop.
// ------------------------------------------------------------------------------
__device__ __forceinline__ double bb_value(const Prob &p, unsigned long long key) {
    return p.dtype == 1 ? okey_to_f64(key) : (double)okey_to_f32((unsigned)key);
}

__global__ void __launch_bounds__(kKThreads) finalize_a_kernel(Prob p, int mode,
                                                               cudaGraphConditionalHandle h_move,
                                                               cudaGraphConditionalHandle h_bal) {
    count_launch(p.ctl);
    __shared__ double r_sum[32];
    __shared__ double red[32];
    __shared__ int r_cnt[32];
    Ctl *ctl = p.ctl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (blockIdx.x == 0 && tid == 0) ctl->mixed_cnt = 0u;  // the list of this movement is done
    int c = blockIdx.x * blockDim.x + tid;
    double dl = 0.0, sdiag = 0.0;
    int cnt = 0;
    if (c < p.k) {
        double S = p.S64[c];
        double dd = 0.0;
        if (S > 0.0) {
            double diag = 0.0;
            for (int j = 0; j < p.d; ++j) {
                size_t q = 2 * ((size_t)c * p.d + j);
                double cm = split_to_f64(p.SXfix[q], p.SXfix[q + 1], p.Fx) / S;
                double m = cm - p.C[c * p.d + j];
                dd += m * m;
                p.Cm[c * p.d + j] = cm;
                double e = bb_value(p, p.BBhi[c * p.d + j]) - bb_value(p, p.BBlo[c * p.d + j]);
                diag += e * e;
            }
            sdiag = sqrt(diag);
            cnt = 1;
        } else {
            for (int j = 0; j < p.d; ++j) p.Cm[c * p.d + j] = p.C[c * p.d + j];
        }
        dl = sqrt(dd);
        p.delta[c] = dl;
        for (int j = 0; j < p.d; ++j) {
            size_t q = 2 * ((size_t)c * p.d + j);
            p.SXfix[q] = 0ull;
            p.SXfix[q + 1] = 0ull;
            p.BBlo[c * p.d + j] = ~0ull;
            p.BBhi[c * p.d + j] = 0ull;
        }
    }
    for (int off = 16; off; off >>= 1) {
        sdiag += __shfl_xor_sync(0xffffffffu, sdiag, off);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    }
    if (lane == 0) {
        r_sum[warp] = sdiag;
        r_cnt[warp] = cnt;
    }
    double mx = block_reduce_max(dl, red);
    if (tid == 0) {
        double s = 0.0;
        int n = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s += r_sum[w];
            n += r_cnt[w];
        }
        p.part[blockIdx.x] = s;
        if (n) atomicAdd(&ctl->nonempty, n);
        atomicMax(&ctl->maxd_key, okey_f64(mx));
    }
    if (last_block(ctl) && tid == 0) {
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(&p.part[b]);
        int n = __ldcg(&ctl->nonempty);
        double m = okey_to_f64(__ldcg(&ctl->maxd_key));
        ctl->nonempty = 0;
        ctl->maxd_key = 0ull;
        ctl->beta = n > 0 ? s / (double)n : 0.0;
        ctl->max_delta = m;
        if (mode == 1) return;
        ctl->iter += 1;
        int conv = m < ctl->thr;
        ctl->converged = conv;
        int move = (mode == 3 || (!conv && ctl->iter < p.max_iter)) && ctl->status == kOk;
        ctl->cont_move = move;
        if (move && p.bounds) {  // new centers: the next pass is a fresh one
            ctl->phase_pass = 0;
            ctl->min_lr_key = 0xffffffffu;
            ctl->max_lr_key = 0u;
            p.cumm[0] = 0.0;
            p.dm[0] = 0.0f;
        }
        ctl->pass_in_phase = 0;
        ctl->cont_balance = 1;
        if (h_move) cudaGraphSetConditional(h_move, mode == 3 ? 0u : (unsigned)move);
        if (h_bal) cudaGraphSetConditional(h_bal, 1u);
    }
}

// Center movement, part 3: when the loop continues, C <- C' and the erosion
// I <- exp((1 - alpha) log I), alpha = 2 / (1 + exp(min(-delta/beta, 0))) - 1 (Eq. 2-3).
__global__ void __launch_bounds__(kKThreads) finalize_b_kernel(Prob p) {
    count_launch(p.ctl);
    const Ctl *ctl = p.ctl;
    if (!ctl->cont_move) return;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = c < p.k;
    const int sel = ctl->isel;
    const double beta = ctl->beta;
    float hi[3] = {0.f, 0.f, 0.f}, lo[3], g32 = 0.0f;
    if (valid) {
        for (int j = 0; j < p.d; ++j) p.C[c * p.d + j] = p.Cm[c * p.d + j];
        double *Ip = p.I2 + (size_t)sel * p.k;
        double I = Ip[c];
        if (p.erosion) {
            double dl = p.delta[c];
            double alpha;
            if (beta > 0.0) {
                double tt = fmin(-dl / beta, 0.0);
                alpha = 2.0 / (1.0 + exp(tt)) - 1.0;
            } else {
                alpha = dl > 0.0 ? 1.0 : 0.0;
            }
            I = exp((1.0 - alpha) * log(I));
            Ip[c] = I;
        }
        double g = 1.0 / (I * I);
        p.g64_2[(size_t)sel * p.k + c] = g;
        if (p.bounds) p.lg[c] = lg_of(g);
        g32 = scaled_g32(g, ctl->gshift);
        frame_center(p, c, hi, lo);
        for (int b = 0; b < 2; ++b) {
            float4 *cd = p.cdata2 + (size_t)b * 2 * p.k;
            cd[2 * c] = make_float4(hi[0], hi[1], hi[2], b == sel ? g32 : 0.0f);
            cd[2 * c + 1] = make_float4(lo[0], lo[1], lo[2], 0.0f);
        }
    }
    write_group(p, p.gdata2 + (size_t)sel * 2 * p.ngroups, valid, hi, g32);
}

// End of a sample round (Section 4.5): the current influence (after the movement
// and its erosion) becomes the next round's starting influence Iin, and the round's
// counters and status move to the main problem's control block.
__global__ void __launch_bounds__(kKThreads) sample_export_kernel(Prob ps, Ctl *main_ctl) {
    count_launch(ps.ctl);
    Ctl *ctl = ps.ctl;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ps.k) ps.Iin[c] = ps.I2[(size_t)ctl->isel * ps.k + c];
    if (last_block(ctl) && threadIdx.x == 0) {
        main_ctl->sample_iters += ctl->iter;
        main_ctl->sample_passes += ctl->passes;
        main_ctl->launches += ctl->launches;
        main_ctl->rechecks += ctl->rechecks;
        ctl->launches = 0ull;
        ctl->rechecks = 0ull;
        if (ctl->status != kOk) main_ctl->status = ctl->status;
    }
}

// ------------------------------------------------------------------------------
// Host launchers.
// ------------------------------------------------------------------------------
static int kgrid(const Prob &p) { return (p.k + kKThreads - 1) / kKThreads; }

static void *filter_fn(int d) {
    return d == 2 ? (void *)filter_kernel<2> : (void *)filter_kernel<3>;
}
static void *hyper_fn(int d) {
    return d == 2 ? (void *)hyper_kernel<2> : (void *)hyper_kernel<3>;
}
static dim3 hyper_grid(const Prob &p) { return dim3((unsigned)((p.nhypers + kFilterWarps - 1) / kFilterWarps)); }
static void *filter_big_fn(int d) {
    return d == 2 ? (void *)filter_big_kernel<2> : (void *)filter_big_kernel<3>;
}
static void *filter_tile_fn(int d) {
    return d == 2 ? (void *)filter_tile_kernel<2> : (void *)filter_tile_kernel<3>;
}
static dim3 filter_tile_grid(const Prob &p) { return dim3((unsigned)(p.nsm > 0 ? p.nsm : 152) * 2); }
static dim3 filter_big_grid(const Prob &p) {
    const long long need = ((long long)p.nsupers * p.stiles + kFilterWarps - 1) / kFilterWarps;
    const long long cap = (long long)(p.nsm > 0 ? p.nsm : 152) * 8;
    return dim3((unsigned)(need < cap ? need : cap));
}
static void *assign_fn(const Prob &p) {
    if (p.bounds) {
        if (p.d == 2) return p.assign_f64 ? (void *)assign_kernel<2, true, true> : (void *)assign_kernel<2, false, true>;
        return p.assign_f64 ? (void *)assign_kernel<3, true, true> : (void *)assign_kernel<3, false, true>;
    }
    if (p.d == 2) return p.assign_f64 ? (void *)assign_kernel<2, true, false> : (void *)assign_kernel<2, false, false>;
    return p.assign_f64 ? (void *)assign_kernel<3, true, false> : (void *)assign_kernel<3, false, false>;
}
// The movement's accumulation: by tile markers when the assignment keeps them (16-bit
// block ids), else one tile per warp in the assignment's permuted tile order.
static void *centroid_fn(const Prob &p) {
    if (p.a16) {
        if (p.dtype == 1) return p.d == 2 ? (void *)centroid_kernel<double, 2> : (void *)centroid_kernel<double, 3>;
        return p.d == 2 ? (void *)centroid_kernel<float, 2> : (void *)centroid_kernel<float, 3>;
    }
    if (p.dtype == 1)
        return p.d == 2 ? (void *)centroid_points_kernel<double, 2> : (void *)centroid_points_kernel<double, 3>;
    return p.d == 2 ? (void *)centroid_points_kernel<float, 2> : (void *)centroid_points_kernel<float, 3>;
}
// the movement's list of point-by-point tiles (marker path only)
static void *centroid_list_fn(const Prob &p) {
    if (!p.a16) return nullptr;
    if (p.dtype == 1) return p.d == 2 ? (void *)centroid_list_kernel<double, 2> : (void *)centroid_list_kernel<double, 3>;
    return p.d == 2 ? (void *)centroid_list_kernel<float, 2> : (void *)centroid_list_kernel<float, 3>;
}
static int centroid_list_grid(const Prob &p) { return (p.nsm > 0 ? p.nsm : 1) * 8; }
// the movement's accumulation: one warp per tpw consecutive tiles, or per tile
static int tile_warp_grid(const Prob &p) {
    const int per = kAssignWarps * (p.a16 ? centroid_tiles_per_warp(p.ntiles, p.nsm) : 1);
    return (p.ntiles + per - 1) / per;
}

// Supergroup records of the current buffer, after every change of the group records.
static void launch_supergroups(const Prob &p, cudaStream_t s) {
    if (p.nsgroups > 0) supergroup_kernel<<<p.nsgroups, kSuperGroup, 0, s>>>(p);
}

cudaError_t launch_init(const Prob &p, cudaStream_t s) {
    init_a_kernel<<<kgrid(p), kKThreads, 0, s>>>(p, 0, 0);
    init_b_kernel<<<kgrid(p), kKThreads, 0, s>>>(p);
    launch_supergroups(p, s);
    return cudaGetLastError();
}
cudaError_t launch_load_state(const Prob &p, cudaStream_t s) { return launch_init(p, s); }

// Filter launch: one warp per supertile.
static cudaError_t filter_config(const Prob &p, dim3 &grid, size_t &smem) {
    smem = 0;
    grid = dim3((unsigned)((p.nsupers + kFilterWarps - 1) / kFilterWarps));
    return cudaSuccess;
}

cudaError_t launch_filter(const Prob &p, cudaStream_t s) {
    void *args1[] = {(void *)&p};
    dim3 grid;
    size_t smem;
    cudaError_t e = filter_config(p, grid, smem);
    if (e != cudaSuccess) return e;
    if (p.hyper) {
        e = cudaLaunchKernel(hyper_fn(p.d), hyper_grid(p), dim3(kFilterThreads), args1, 0, s);
        if (e != cudaSuccess) return e;
    }
    e = cudaLaunchKernel(filter_fn(p.d), grid, dim3(kFilterThreads), args1, smem, s);
    if (e != cudaSuccess) return e;
    e = cudaLaunchKernel(filter_big_fn(p.d), filter_big_grid(p), dim3(kFilterThreads), args1, 0, s);
    if (e != cudaSuccess || !filter_tile_needed(p)) return e;
    return cudaLaunchKernel(filter_tile_fn(p.d), filter_tile_grid(p), dim3(kFilterThreads), args1, 0, s);
}
// resident CTAs per SM: registers (FP64 mode) or the stages' shared memory (3-D)
int assign_max_ctas(const Prob &p) {
    // 3-D stages (three, or two larger ones with bounds) fit four CTAs in shared memory
    return p.assign_f64 ? kAMinBlocks64 : (p.d == 3 ? 4 : kAMinBlocks);
}
int assign_ctas(const Prob &p) {
    const int m = assign_max_ctas(p);
    return (p.actas > 0 && p.actas < m) ? p.actas : m;
}
static int assign_grid(const Prob &p) {
    int need = (p.ntiles + kAWarps - 1) / kAWarps;
    int cap = (p.nsm > 0 ? p.nsm : 152) * assign_ctas(p);
    return need < cap ? need : cap;
}
static size_t assign_smem_of(const Prob &p) {
    if (p.bounds) return p.d == 2 ? assign_smem<2, true>() : assign_smem<3, true>();
    return p.d == 2 ? assign_smem<2, false>() : assign_smem<3, false>();
}
static cudaError_t prepare_assign(void *fn, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
cudaError_t launch_assign(const Prob &p, cudaStream_t s) {
    void *args1[] = {(void *)&p};
    void *fn = assign_fn(p);
    cudaError_t e = prepare_assign(fn, assign_smem_of(p));
    if (e != cudaSuccess) return e;
    return cudaLaunchKernel(fn, dim3(assign_grid(p)), dim3(kAWarps * 32), args1, assign_smem_of(p), s);
}
// The failure path of the assignment's waits, exercised without a fault: one warp waits,
// bounded, for phase 0 of an mbarrier that expects one arrival and gets none (no copy is
// issued on it, so nothing is in flight when the wait gives up).
__device__ int g_wait_status;
__device__ unsigned long long g_wait_ns;

__global__ void wait_check_kernel(unsigned long long limit_ns) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbarrier_init();
    }
    __syncthreads();
    const unsigned long long t0 = global_ns();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    const bool all = __all_sync(0xffffffffu, ok);
    if (threadIdx.x == 0) {
        g_wait_status = all ? kOk : kErrTimeout;
        g_wait_ns = global_ns() - t0;
    }
}

cudaError_t run_wait_check(unsigned long long limit_ns, int *status,
                           unsigned long long *waited_ns, cudaStream_t s) {
    wait_check_kernel<<<1, 32, 0, s>>>(limit_ns);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(status, g_wait_status, sizeof(int), 0,
                                                         cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyFromSymbolAsync(waited_ns, g_wait_ns, sizeof(unsigned long long), 0,
                                      cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

cudaError_t launch_balance(const Prob &p, int mode, cudaStream_t s) {
    balance_kernel<<<kgrid(p), kKThreads, 0, s>>>(p, mode, 0);
    if (mode != 2) launch_supergroups(p, s);
    return cudaGetLastError();
}
cudaError_t launch_pass(const Prob &p, int mode, cudaStream_t s) {
    cudaError_t e = launch_filter(p, s);
    if (e == cudaSuccess) e = launch_assign(p, s);
    if (e == cudaSuccess) e = launch_balance(p, mode, s);
    return e;
}

cudaError_t launch_block_weights(const Prob &p, cudaStream_t s) {
    block_weights_kernel<<<(int)((p.n + 255) / 256), 256, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    balance_kernel<<<kgrid(p), kKThreads, 0, s>>>(p, 2, 0);
    return cudaGetLastError();
}

cudaError_t launch_centroid(const Prob &p, cudaStream_t s) {
    void *args1[] = {(void *)&p};
    cudaError_t e = cudaLaunchKernel(centroid_fn(p), dim3(tile_warp_grid(p)), dim3(kAssignWarps * 32),
                                     args1, 0, s);
    if (e == cudaSuccess && centroid_list_fn(p))
        e = cudaLaunchKernel(centroid_list_fn(p), dim3(centroid_list_grid(p)), dim3(kAssignWarps * 32),
                             args1, 0, s);
    return e;
}
cudaError_t launch_move_finish(const Prob &p, int mode, cudaStream_t s) {
    finalize_a_kernel<<<kgrid(p), kKThreads, 0, s>>>(p, mode, 0, 0);
    if (mode == 0 || mode == 3) {
        finalize_b_kernel<<<kgrid(p), kKThreads, 0, s>>>(p);
        launch_supergroups(p, s);
    }
    return cudaGetLastError();
}
cudaError_t launch_move(const Prob &p, int mode, cudaStream_t s) {
    cudaError_t e = launch_centroid(p, s);
    if (e != cudaSuccess) return e;
    finalize_a_kernel<<<kgrid(p), kKThreads, 0, s>>>(p, mode, 0, 0);
    if (mode == 0 || mode == 3) {
        finalize_b_kernel<<<kgrid(p), kKThreads, 0, s>>>(p);
        launch_supergroups(p, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_final_begin(const Prob &p, cudaStream_t s) {
    final_begin_kernel<<<1, 32, 0, s>>>(p, 0);
    return cudaGetLastError();
}

cudaError_t launch_export(const Prob &p, cudaStream_t s) {
    export_kernel<<<kgrid(p), kKThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_sample_export(const Prob &ps, Ctl *main_ctl, cudaStream_t s) {
    sample_export_kernel<<<kgrid(ps), kKThreads, 0, s>>>(ps, main_ctl);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------
// The whole loop as one CUDA graph:
//   init_a -> init_b -> while(h_move){ while(h_bal){ filter -> filter_big -> assign ->
//   balance(0) } -> centroid -> finalize_a -> finalize_b } -> final_begin ->
//   while(h_fin){ filter -> filter_big -> assign -> balance(1) }
// A batch of problems is one graph with one such chain per problem, no edges between
// chains, so that the chains of small problems run beside those of large ones.
// ------------------------------------------------------------------------------
namespace {
struct NodeAdder {
    cudaGraph_t g;
    cudaGraphNode_t last = nullptr;
    cudaError_t err = cudaSuccess;
    void kernel(void *fn, dim3 grid, dim3 block, void **args, size_t smem = 0) {
        if (err != cudaSuccess) return;
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeKernel;
        np.kernel.func = fn;
        np.kernel.gridDim = grid;
        np.kernel.blockDim = block;
        np.kernel.sharedMemBytes = (unsigned)smem;
        np.kernel.kernelParams = args;
        cudaGraphNode_t node;
        err = cudaGraphAddNode(&node, g, last ? &last : nullptr, nullptr, last ? 1 : 0, &np);
        last = node;
    }
    cudaGraph_t loop(cudaGraphConditionalHandle h) {
        if (err != cudaSuccess) return nullptr;
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        err = cudaGraphAddNode(&node, g, last ? &last : nullptr, nullptr, last ? 1 : 0, &np);
        last = node;
        return err == cudaSuccess ? np.conditional.phGraph_out[0] : nullptr;
    }
};
}  // namespace

// Adds one problem's loop to graph g (its own conditional handles), after node
// `after` (nullptr: an independent chain).  The kernel parameters are copied when
// the nodes are created.
cudaError_t add_loop_chain(cudaGraph_t g, const Prob &pc, cudaGraphNode_t after = nullptr) {
    Prob p = pc;
    cudaGraphConditionalHandle h_move, h_bal, h_fin;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h_move, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h_bal, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h_fin, g, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    int mode0 = 0, mode1 = 1;
    void *a_init[] = {&p, &h_move, &h_bal};
    void *a_p[] = {&p};
    void *a_bal0[] = {&p, &mode0, &h_bal};
    void *a_bal1[] = {&p, &mode1, &h_fin};
    void *a_fin[] = {&p, &mode0, &h_move, &h_bal};
    void *a_fb[] = {&p, &h_fin};
    const dim3 kg(kgrid(p)), kb(kKThreads), tg(tile_warp_grid(p)), tb(kAssignWarps * 32);
    e = prepare_assign(assign_fn(p), assign_smem_of(p));
    dim3 fgrid;
    size_t fsmem = 0;
    if (e == cudaSuccess) e = filter_config(p, fgrid, fsmem);
    if (e != cudaSuccess) return e;
    NodeAdder top{g};
    top.last = after;
    top.kernel((void *)init_a_kernel, kg, kb, a_init);
    top.kernel((void *)init_b_kernel, kg, kb, a_p);
    const dim3 sgg(p.nsgroups > 0 ? p.nsgroups : 1), sgb(kSuperGroup);
    if (p.nsgroups > 0) top.kernel((void *)supergroup_kernel, sgg, sgb, a_p);
    cudaGraph_t body_move = top.loop(h_move);
    if (body_move) {
        NodeAdder mv{body_move};
        cudaGraph_t body_bal = mv.loop(h_bal);
        if (body_bal) {
            NodeAdder bl{body_bal};
            if (p.hyper) bl.kernel(hyper_fn(p.d), hyper_grid(p), dim3(kFilterThreads), a_p);
            bl.kernel(filter_fn(p.d), fgrid, dim3(kFilterThreads), a_p, fsmem);
            bl.kernel(filter_big_fn(p.d), filter_big_grid(p), dim3(kFilterThreads), a_p);
            if (filter_tile_needed(p)) bl.kernel(filter_tile_fn(p.d), filter_tile_grid(p), dim3(kFilterThreads), a_p);
            bl.kernel(assign_fn(p), dim3(assign_grid(p)), dim3(kAWarps * 32), a_p,
                      assign_smem_of(p));
            bl.kernel((void *)balance_kernel, kg, kb, a_bal0);
            if (p.nsgroups > 0) bl.kernel((void *)supergroup_kernel, sgg, sgb, a_p);
            if (bl.err != cudaSuccess) mv.err = bl.err;
        }
        mv.kernel(centroid_fn(p), tg, tb, a_p);
        if (centroid_list_fn(p)) mv.kernel(centroid_list_fn(p), dim3(centroid_list_grid(p)), tb, a_p);
        mv.kernel((void *)finalize_a_kernel, kg, kb, a_fin);
        mv.kernel((void *)finalize_b_kernel, kg, kb, a_p);
        if (p.nsgroups > 0) mv.kernel((void *)supergroup_kernel, sgg, sgb, a_p);
        if (mv.err != cudaSuccess) top.err = mv.err;
    }
    top.kernel((void *)final_begin_kernel, dim3(1), dim3(32), a_fb);
    cudaGraph_t body_fin = top.loop(h_fin);
    if (body_fin) {
        NodeAdder fl{body_fin};
        if (p.hyper) fl.kernel(hyper_fn(p.d), hyper_grid(p), dim3(kFilterThreads), a_p);
        fl.kernel(filter_fn(p.d), fgrid, dim3(kFilterThreads), a_p, fsmem);
        fl.kernel(filter_big_fn(p.d), filter_big_grid(p), dim3(kFilterThreads), a_p);
        if (filter_tile_needed(p)) fl.kernel(filter_tile_fn(p.d), filter_tile_grid(p), dim3(kFilterThreads), a_p);
        fl.kernel(assign_fn(p), dim3(assign_grid(p)), dim3(kAWarps * 32), a_p,
                  assign_smem_of(p));
        fl.kernel((void *)balance_kernel, kg, kb, a_bal1);
        if (p.nsgroups > 0) fl.kernel((void *)supergroup_kernel, sgg, sgb, a_p);
        if (fl.err != cudaSuccess) top.err = fl.err;
    }
    return top.err;
}

// One sample round: selection and gather of the sample, initial state from Iin and
// C, the balance loop, the forced movement with erosion, the hand-over.
static cudaError_t add_sample_round(NodeAdder &top, const Prob &psc, const SampleSel &selc,
                                    Ctl *main_ctl) {
    Prob ps = psc;
    SampleSel sel = selc;
    cudaGraphConditionalHandle h_bal;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h_bal, top.g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle none = 0;
    int mode0 = 0, mode3 = 3;
    void *a_sel[] = {&ps, &sel};
    void *a_p[] = {&ps};
    void *a_init[] = {&ps, &none, &h_bal};
    void *a_bal0[] = {&ps, &mode0, &h_bal};
    void *a_fin[] = {&ps, &mode3, &none, &none};
    void *a_exp[] = {&ps, &main_ctl};
    KNode nodes[kSampleSelectNodes];
    int q = sample_select_nodes(ps, sel, nodes);
    for (int i = 0; i < q; ++i) top.kernel(nodes[i].fn, nodes[i].grid, nodes[i].block, a_sel);
    const dim3 kg(kgrid(ps)), kb(kKThreads), tg(tile_warp_grid(ps)), tb(kAssignWarps * 32);
    const dim3 sgg(ps.nsgroups > 0 ? ps.nsgroups : 1), sgb(kSuperGroup);
    dim3 fgrid;
    size_t fsmem = 0;
    e = filter_config(ps, fgrid, fsmem);
    if (e != cudaSuccess) return e;
    top.kernel((void *)init_a_kernel, kg, kb, a_init);
    top.kernel((void *)init_b_kernel, kg, kb, a_p);
    if (ps.nsgroups > 0) top.kernel((void *)supergroup_kernel, sgg, sgb, a_p);
    cudaGraph_t body_bal = top.loop(h_bal);
    if (body_bal) {
        NodeAdder bl{body_bal};
        if (ps.hyper) bl.kernel(hyper_fn(ps.d), hyper_grid(ps), dim3(kFilterThreads), a_p);
        bl.kernel(filter_fn(ps.d), fgrid, dim3(kFilterThreads), a_p, fsmem);
        bl.kernel(filter_big_fn(ps.d), filter_big_grid(ps), dim3(kFilterThreads), a_p);
        if (filter_tile_needed(ps)) bl.kernel(filter_tile_fn(ps.d), filter_tile_grid(ps), dim3(kFilterThreads), a_p);
        bl.kernel(assign_fn(ps), dim3(assign_grid(ps)), dim3(kAWarps * 32), a_p,
                  assign_smem_of(ps));
        bl.kernel((void *)balance_kernel, kg, kb, a_bal0);
        if (ps.nsgroups > 0) bl.kernel((void *)supergroup_kernel, sgg, sgb, a_p);
        if (bl.err != cudaSuccess) top.err = bl.err;
    }
    top.kernel(centroid_fn(ps), tg, tb, a_p);
    if (centroid_list_fn(ps)) top.kernel(centroid_list_fn(ps), dim3(centroid_list_grid(ps)), tb, a_p);
    top.kernel((void *)finalize_a_kernel, kg, kb, a_fin);
    top.kernel((void *)finalize_b_kernel, kg, kb, a_p);
    if (ps.nsgroups > 0) top.kernel((void *)supergroup_kernel, sgg, sgb, a_p);
    top.kernel((void *)sample_export_kernel, kg, kb, a_exp);
    return top.err;
}

cudaError_t build_sampled_graph(const Prob &p, const Prob *ps, const SampleSel *sel, int R,
                                cudaGraphExec_t *exec_out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    e = prepare_assign(assign_fn(p), assign_smem_of(p));
    NodeAdder top{g};
    for (int r = 0; r < R && e == cudaSuccess; ++r) e = add_sample_round(top, ps[r], sel[r], p.ctl);
    if (e == cudaSuccess) e = add_loop_chain(g, p, top.last);
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec_out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

cudaError_t build_loop_graph(const Prob *probs, int count, cudaGraphExec_t *exec_out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < count && e == cudaSuccess; ++i) e = add_loop_chain(g, probs[i]);
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec_out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

}  // namespace gk
