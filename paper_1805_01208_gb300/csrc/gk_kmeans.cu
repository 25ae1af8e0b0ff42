// gk_kmeans.cu -- the balanced k-means iteration (Algorithm 1 AssignAndBalance and the
// movement / erosion steps of Algorithm 2; Section 4.2 Eq. 1-3; Section 4.4).
//
//   filter_kernel     per-tile candidate centers from the tile's bounding box
//                     (Section 4.4; lower bound minDist/influence against the
//                     smallest upper bound maxDist/influence over all centers)
//   assign_kernel     effective-distance argmin over the tile's candidates + block
//                     weight histogram (Algorithm 1 inner loop, localBlockSizes)
//   balance_kernel    global block weights, balance test, influence update (Eq. 1)
//   centroid_kernel   weighted coordinate sums and block bounding boxes (Algorithm 2)
//   finalize_kernel   new centers, movement, average block diameter, erosion (Eq. 2-3),
//                     convergence test
//
// Effective distances are compared squared: dist^2 / influence^2 orders the
// centers exactly as dist / influence does.
#include "gk_common.cuh"
#include "gk_internal.h"

namespace gk {

constexpr float kU = 5.9604644775390625e-8f;  // 2^-24, unit roundoff of FP32

// Frame coordinates of center c split into an FP32 pair (hi + lo) and g = 1/I^2.
__device__ __forceinline__ void write_cdata(const Prob &p, int c) {
    double I = p.I[c];
    double g = 1.0 / (I * I);
    p.g64[c] = g;
    float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
    for (int j = 0; j < p.d; ++j) {
        double f = (p.C[c * p.d + j] - p.origin[j]) * p.scale;
        hi[j] = __double2float_rn(f);
        lo[j] = __double2float_rn(f - (double)hi[j]);
    }
    p.cdata[2 * c] = make_float4(hi[0], hi[1], hi[2], __double2float_rn(g));
    p.cdata[2 * c + 1] = make_float4(lo[0], lo[1], lo[2], 0.0f);
}

// ------------------------------------------------------------------------------
// Loop control.
// ------------------------------------------------------------------------------
__global__ void init_kernel(Prob p, cudaGraphConditionalHandle h_move,
                            cudaGraphConditionalHandle h_bal) {
    count_launch(p.ctl);
    for (int c = threadIdx.x; c < p.k; c += blockDim.x) {
        write_cdata(p, c);
        p.Iused[c] = p.I[c];
    }
    if (threadIdx.x == 0) {
        Ctl *ctl = p.ctl;
        if (p.weighted)
            ctl->W = i128_to_f64(ctl->wsum_lo, ctl->wsum_hi, p.Fw);
        else
            ctl->W = (double)p.n;
        ctl->target = ctl->W / (double)p.k;
        ctl->ceil_avg = ceil(ctl->W / (double)p.k);
        ctl->bound = (1.0 + p.eps) * ctl->ceil_avg;
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
        if (h_move) cudaGraphSetConditional(h_move, 1u);
        if (h_bal) cudaGraphSetConditional(h_bal, 1u);
    }
}

__global__ void final_begin_kernel(Prob p, cudaGraphConditionalHandle h_fin) {
    count_launch(p.ctl);
    Ctl *ctl = p.ctl;
    int cont = (!ctl->balanced && p.final_balance_iter > 0 && ctl->status == kOk) ? 1 : 0;
    ctl->cont_final = cont;
    if (h_fin) cudaGraphSetConditional(h_fin, (unsigned)cont);
}

// ------------------------------------------------------------------------------
// Candidate filter (Section 4.4).  One warp per tile; all centers pass through
// shared memory in chunks brought in by bulk copies.  For the tile's box B and
// center c (frame coordinates, relative to the tile origin):
//   UB_c = g_c * maxDist(B, c)^2,  LB_c = g_c * minDist(B, c)^2,  tau = min_c UB_c.
// Every point of B has effective distance <= tau to the best center, so c can
// only win if LB_c <= tau.  The box is widened by 4 u R and tau by 64 u so that
// FP32 rounding of points, centers and this arithmetic never drops the FP64
// winner.  Candidates are written in ascending center order; more than kCap
// marks the tile for a scan over all centers.
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

template <int D>
__global__ void __launch_bounds__(kFilterWarps * 32) filter_kernel(Prob p) {
    count_launch(p.ctl);
    __shared__ __align__(128) float4 sc[2 * kCenterChunk];
    __shared__ __align__(8) unsigned long long bar;
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int t = blockIdx.x * kFilterWarps + warp;
    bool active = t < p.ntiles;
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    float o[3] = {0.f, 0.f, 0.f}, h[3] = {0.f, 0.f, 0.f};
    if (active) {
        float4 a = p.tiles[2 * t], b = p.tiles[2 * t + 1];
        float infl = 4.0f * kU * p.R;
        o[0] = a.x;
        o[1] = a.y;
        o[2] = a.z;
        h[0] = __fadd_ru(b.x, infl);
        h[1] = __fadd_ru(b.y, infl);
        h[2] = __fadd_ru(b.z, infl);
    }
    const int nch = (p.k + kCenterChunk - 1) / kCenterChunk;
    unsigned phase = 0;
    bool failed = false;
    auto stage = [&](int ch) -> bool {
        int cb = ch * kCenterChunk;
        int m = min(kCenterChunk, p.k - cb);
        if (tid == 0) {
            fence_proxy_async();
            mbar_expect_tx(&bar, (unsigned)(m * 32));
            bulk_g2s(sc, p.cdata + 2 * (long long)cb, (unsigned)(m * 32), &bar);
        }
        bool ok = mbar_wait_bounded(&bar, phase);
        phase ^= 1u;
        return !__syncthreads_or(!ok);
    };
    float tau = INFINITY;
    for (int ch = 0; ch < nch && !failed; ++ch) {
        if (!stage(ch)) {
            failed = true;
            break;
        }
        int m = min(kCenterChunk, p.k - ch * kCenterChunk);
        if (active) {
            for (int c = lane; c < m; c += 32) {
                float lb, ub;
                box_bounds<D>(sc[2 * c], sc[2 * c + 1], o, h, lb, ub);
                tau = fminf(tau, ub);
            }
        }
        __syncthreads();
    }
    for (int off = 16; off; off >>= 1) tau = fminf(tau, __shfl_xor_sync(0xffffffffu, tau, off));
    tau = __fmul_ru(tau, 1.0f + 64.0f * kU);
    int cnt = 0;
    unsigned lt = (1u << lane) - 1u;
    for (int ch = 0; ch < nch && !failed; ++ch) {
        if (nch > 1 && !stage(ch)) {
            failed = true;
            break;
        }
        int cb = ch * kCenterChunk;
        int m = min(kCenterChunk, p.k - cb);
        if (active) {
            for (int base = 0; base < m; base += 32) {
                int c = base + lane;
                bool keep = false;
                if (c < m) {
                    float lb, ub;
                    box_bounds<D>(sc[2 * c], sc[2 * c + 1], o, h, lb, ub);
                    keep = lb <= tau;
                }
                unsigned bal = __ballot_sync(0xffffffffu, keep);
                int pos = cnt + __popc(bal & lt);
                if (keep && pos < kCap) p.cand_list[(long long)t * kCap + pos] = cb + c;
                cnt += __popc(bal);
            }
        }
        __syncthreads();
    }
    if (failed) {
        // A bulk copy did not complete in time: record it, let the assignment scan
        // every center for these tiles, and wait (bounded) for the copy in flight.
        if (tid == 0) atomicCAS(&p.ctl->status, kOk, kErrTimeout);
        if (active && lane == 0) p.cand_cnt[t] = -1;
        mbar_wait_bounded(&bar, phase ^ 1u);
        return;
    }
    if (active && lane == 0) {
        p.cand_cnt[t] = cnt > kCap ? -1 : cnt;
        if (cnt > kCap) atomicAdd(&p.ctl->overflow_tiles, 1ull);
    }
}

// ------------------------------------------------------------------------------
// Assignment + block-weight histogram (Section 4.2; Algorithm 1 inner loop).
//
// In tile-local frame coordinates x' = x - o the squared effective distance to a
// candidate with frame center q (relative to o) and g = 1/I^2 is
//     E = g |x'|^2 - 2 g q.x' + g |q|^2 = fma chain over per-candidate coefficients.
// FP64 mode: the FP32 winner b is accepted when the FP32 gap to the runner-up
// exceeds twice a rigorous bound on |E_fp32 - E_exact| (coordinate rounding,
// coefficient rounding, fma-chain rounding; evaluated with the tile radius and the
// largest g among the candidates, doubled for safety).  Other points are decided
// again in FP64 from the raw coordinates over all candidates.  The result is the
// FP64 argmin up to ties closer than FP64 rounding.
// ------------------------------------------------------------------------------
template <int D, bool F64MODE>
__global__ void __launch_bounds__(kTile) assign_kernel(Prob p) {
    count_launch(p.ctl);
    if (blockIdx.x == 0 && threadIdx.x == 0) p.ctl->t_assign0 = globaltimer_ns();
    __shared__ __align__(16) float4 coef[kCap];
    __shared__ float ga[kCap];
    __shared__ int cid[kCap];
    __shared__ float s_gmax[kTile / 32];
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int t = blockIdx.x;
    long long i = (long long)t * kTile + tid;
    bool valid = i < p.n;
    float4 ob = p.tiles[2 * t];
    float o[3] = {ob.x, ob.y, ob.z};
    int cnt = p.cand_cnt[t];
    bool all = cnt < 0;
    int ncand = all ? p.k : cnt;
    float xp[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < D; ++j) xp[j] = valid ? (p.X32[j * p.n_pad + i] - o[j]) : 0.0f;
    float xx = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) xx = fmaf(xp[j], xp[j], xx);
    float E1 = INFINITY, E2 = INFINITY;
    int best = 0;
    float gl = 0.f;
    for (int base = 0; base < ncand; base += kCap) {
        int m = min(kCap, ncand - base);
        __syncthreads();
        if (tid < m) {
            int c = all ? base + tid : p.cand_list[(long long)t * kCap + base + tid];
            float4 ch = p.cdata[2 * c], cl = p.cdata[2 * c + 1];
            float q0 = (ch.x - o[0]) + cl.x;
            float q1 = (ch.y - o[1]) + cl.y;
            float q2 = D == 3 ? (ch.z - o[2]) + cl.z : 0.0f;
            float g = ch.w;
            float qq = fmaf(q2, q2, fmaf(q1, q1, q0 * q0));
            coef[tid] = make_float4(-2.0f * g * q0, -2.0f * g * q1, -2.0f * g * q2, g * qq);
            ga[tid] = g;
            cid[tid] = c;
            gl = fmaxf(gl, g);
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < m; ++jj) {
            float4 cf = coef[jj];
            float acc = D == 3 ? fmaf(cf.z, xp[2], cf.w) : cf.w;
            acc = fmaf(cf.y, xp[1], acc);
            acc = fmaf(cf.x, xp[0], acc);
            float E = fmaf(ga[jj], xx, acc);
            if (E < E1) {
                if (F64MODE) E2 = E1;
                E1 = E;
                best = cid[jj];
            } else if (F64MODE) {
                E2 = fminf(E2, E);
            }
        }
    }
    if (F64MODE) {
        for (int off = 16; off; off >>= 1) gl = fmaxf(gl, __shfl_xor_sync(0xffffffffu, gl, off));
        if (lane == 0) s_gmax[warp] = gl;
        __syncthreads();
        float gmax = s_gmax[0];
        for (int w = 1; w < kTile / 32; ++w) gmax = fmaxf(gmax, s_gmax[w]);
        // error bound B(E) = beta0 + beta1 sqrt(E) + beta2 E (see comment above)
        float R = p.R;
        float rp = ob.w + 2.0f * 1.7320508f * kU * R;
        float ex = sqrtf((float)D) * kU * (R + rp);
        float sg = sqrtf(gmax);
        float c2 = (2.0f * D + 10.0f) * kU;
        float beta2 = c2;
        float beta1 = c2 * 4.0f * sg * rp + 2.0f * sg * ex;
        float beta0 = c2 * 4.0f * gmax * rp * rp + gmax * ex * ex;
        float Estar = 2.0f * E2 + 2.0f * (beta0 + 2.0f * beta1 * beta1);
        float B = 2.0f * (beta0 + beta1 * sqrtf(Estar) + beta2 * Estar);
        bool recheck = valid && !((E2 - E1) > 2.0f * B);  // E2 = inf -> certified
        if (recheck) {
            double x64[3];
            for (int j = 0; j < D; ++j)
                x64[j] = p.dtype == 1 ? p.X64[j * p.n_pad + i] : (double)p.X32[j * p.n_pad + i];
            double bestE = INFINITY;
            int b = 0;
            for (int jj = 0; jj < ncand; ++jj) {
                int c = all ? jj : p.cand_list[(long long)t * kCap + jj];
                double s = 0.0;
                for (int j = 0; j < D; ++j) {
                    double df = x64[j] - p.C[c * D + j];
                    s += df * df;
                }
                double E = s * p.g64[c];
                if (E < bestE) {
                    bestE = E;
                    b = c;
                }
            }
            best = b;
        }
        int nre = __syncthreads_count(recheck);
        if (tid == 0 && nre) atomicAdd(&p.ctl->rechecks, (unsigned long long)nre);
    }
    if (valid) p.A[i] = best;
    // block weights: warp aggregation, then one atomic per distinct block and warp
    if (!p.weighted) {
        int key = valid ? best : -1;
        unsigned peers = __match_any_sync(0xffffffffu, key);
        if (valid && (peers & ((1u << lane) - 1u)) == 0u)
            atomicAdd(&p.Sfix[2 * best], (unsigned long long)__popc(peers));
    } else {
        unsigned long long v = 0;
        if (valid)
            v = (unsigned long long)(p.dtype == 1 ? fix_f64(((const double *)p.Ws)[i], p.Fw)
                                                  : fix_f32(((const float *)p.Ws)[i], p.Fw));
        int b0 = __shfl_sync(0xffffffffu, valid ? best : -1, 0);
        bool uniform = __all_sync(0xffffffffu, valid && best == b0);
        if (uniform) {
            for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) atomic_add_u128(&p.Sfix[2 * b0], v);
        } else if (valid) {
            atomic_add_u128(&p.Sfix[2 * best], v);
        }
    }
    int nvalid = __syncthreads_count(valid);
    if (tid == 0) atomicAdd(&p.ctl->cand_sum, (unsigned long long)ncand * (unsigned long long)nvalid);
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
    if (valid) atomic_add_u128(&p.Sfix[2 * b], v);
}

// ------------------------------------------------------------------------------
// Balance test and influence update (Section 2 bound; Section 4.2 Eq. 1 as read:
// I_c <- I_c * clamp((W/k / S_c)^(1/d), 0.95, 1.05)).  mode 0: main loop, 1: final
// passes with centers fixed, 2: block weights only (standalone assignment).
// One CTA.
// ------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) balance_kernel(Prob p, int mode,
                                                       cudaGraphConditionalHandle h) {
    count_launch(p.ctl);
    __shared__ double red[32];
    __shared__ int s_bal;
    Ctl *ctl = p.ctl;
    int tid = threadIdx.x;
    if (tid == 0) {  // the assignment kernel ran just before on this stream
        ctl->assign_ns += globaltimer_ns() - ctl->t_assign0;
        ctl->assign_cnt += 1;
    }
    double mx = 0.0;
    for (int c = tid; c < p.k; c += blockDim.x) {
        unsigned long long lo = p.Sfix[2 * c], hi = p.Sfix[2 * c + 1];
        double S = p.weighted ? i128_to_f64(lo, hi, p.Fw) : (double)lo;
        p.S64[c] = S;
        p.Sfix[2 * c] = 0ull;
        p.Sfix[2 * c + 1] = 0ull;
        mx = fmax(mx, S);
    }
    for (int off = 16; off; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
        double m = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        int bal = m <= ctl->bound;
        s_bal = bal;
        ctl->max_imbalance = m / ctl->ceil_avg - 1.0;
        if (mode != 2) {
            ctl->balanced = bal;
            ctl->passes += 1;
            if (mode == 0)
                ctl->pass_in_phase += 1;
            else
                ctl->final_passes += 1;
        }
    }
    __syncthreads();
    if (mode == 2) return;
    int bal = s_bal;
    for (int c = tid; c < p.k; c += blockDim.x) {
        double I = p.I[c];
        p.Iused[c] = I;
        if (!bal) {
            double S = p.S64[c];
            double f;
            if (S > 0.0) {
                double gamma = ctl->target / S;
                f = p.d == 2 ? sqrt(gamma) : cbrt(gamma);
            } else {
                f = INFINITY;
            }
            f = fmin(fmax(f, 0.95), 1.05);
            I = I * f;
            p.I[c] = I;
            double g = 1.0 / (I * I);
            p.g64[c] = g;
            p.cdata[2 * c].w = __double2float_rn(g);
        }
    }
    if (tid == 0) {
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
}

// ------------------------------------------------------------------------------
// Center movement, part 1: 128-bit fixed-point sums of w*x per block and axis and
// the block bounding boxes (ordered-key min/max).  Exact and order-independent.
// ------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256) centroid_kernel(Prob p) {
    count_launch(p.ctl);
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int lane = threadIdx.x & 31;
    int b = i < p.n ? p.A[i] : -1;
    bool valid = i < p.n && (unsigned)b < (unsigned)p.k;
    if (!valid) b = -1;
    long long v[D];
    unsigned long long kl[D], kh[D];
    double w = 1.0;
    if (valid && p.weighted)
        w = p.dtype == 1 ? ((const double *)p.Ws)[i] : (double)((const float *)p.Ws)[i];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        double x = 0.0;
        long long fv = 0;
        if (valid) {
            if (p.dtype == 1) {
                x = p.X64[j * p.n_pad + i];
                fv = p.weighted ? fix_f64(w * x, p.Fx) : fix_f64(x, p.Fx);
            } else {
                float xf = p.X32[j * p.n_pad + i];
                x = (double)xf;
                fv = p.weighted ? fix_f64(w * x, p.Fx) : fix_f32(xf, p.Fx);
            }
        }
        v[j] = fv;
        kl[j] = valid ? okey_f64(x) : ~0ull;
        kh[j] = valid ? okey_f64(x) : 0ull;
    }
    int b0 = __shfl_sync(0xffffffffu, b, 0);
    bool uniform = __all_sync(0xffffffffu, valid && b == b0);
    if (uniform) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            for (int off = 16; off; off >>= 1) {
                v[j] += (long long)__shfl_xor_sync(0xffffffffu, (unsigned long long)v[j], off);
                unsigned long long a = __shfl_xor_sync(0xffffffffu, kl[j], off);
                unsigned long long c = __shfl_xor_sync(0xffffffffu, kh[j], off);
                kl[j] = a < kl[j] ? a : kl[j];
                kh[j] = c > kh[j] ? c : kh[j];
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < D; ++j) {
                atomic_add_i128(&p.SXfix[2 * (b0 * D + j)], v[j]);
                atomicMin(&p.BBlo[b0 * D + j], kl[j]);
                atomicMax(&p.BBhi[b0 * D + j], kh[j]);
            }
        }
    } else if (valid) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            atomic_add_i128(&p.SXfix[2 * (b * D + j)], v[j]);
            atomicMin(&p.BBlo[b * D + j], kl[j]);
            atomicMax(&p.BBhi[b * D + j], kh[j]);
        }
    }
}

// ------------------------------------------------------------------------------
// Center movement, part 2 (one CTA): C' = sum(w x) / sum(w) (empty block: C' = C),
// delta_c = |C'_c - C_c|, beta = mean diagonal of the non-empty blocks' boxes,
// convergence test, and -- when the loop continues -- C <- C' and the erosion
// I <- exp((1 - alpha) log I), alpha = 2 / (1 + exp(min(-delta/beta, 0))) - 1
// (Eq. 2-3).  mode 0: inside the loop; 1: standalone (outputs only).
// ------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) finalize_kernel(Prob p, int mode,
                                                        cudaGraphConditionalHandle h_move,
                                                        cudaGraphConditionalHandle h_bal) {
    count_launch(p.ctl);
    __shared__ double r_max[32], r_sum[32];
    __shared__ int r_cnt[32];
    __shared__ int s_move;
    __shared__ double s_beta;
    Ctl *ctl = p.ctl;
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double mx = 0.0, sdiag = 0.0;
    int cnt = 0;
    for (int c = tid; c < p.k; c += blockDim.x) {
        double S = p.S64[c];
        double dd = 0.0;
        if (S > 0.0) {
            double diag = 0.0;
            for (int j = 0; j < p.d; ++j) {
                long long q = 2ll * (c * p.d + j);
                double cm = i128_to_f64(p.SXfix[q], p.SXfix[q + 1], p.Fx) / S;
                double m = cm - p.C[c * p.d + j];
                dd += m * m;
                p.Cm[c * p.d + j] = cm;
                double e = okey_to_f64(p.BBhi[c * p.d + j]) - okey_to_f64(p.BBlo[c * p.d + j]);
                diag += e * e;
            }
            sdiag += sqrt(diag);
            cnt += 1;
        } else {
            for (int j = 0; j < p.d; ++j) p.Cm[c * p.d + j] = p.C[c * p.d + j];
        }
        double dl = sqrt(dd);
        p.delta[c] = dl;
        mx = fmax(mx, dl);
        for (int j = 0; j < p.d; ++j) {
            long long q = 2ll * (c * p.d + j);
            p.SXfix[q] = 0ull;
            p.SXfix[q + 1] = 0ull;
            p.BBlo[c * p.d + j] = ~0ull;
            p.BBhi[c * p.d + j] = 0ull;
        }
    }
    for (int off = 16; off; off >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        sdiag += __shfl_xor_sync(0xffffffffu, sdiag, off);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    }
    if (lane == 0) {
        r_max[warp] = mx;
        r_sum[warp] = sdiag;
        r_cnt[warp] = cnt;
    }
    __syncthreads();
    if (tid == 0) {
        double m = r_max[0], s = r_sum[0];
        int n = r_cnt[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            m = fmax(m, r_max[w]);
            s += r_sum[w];
            n += r_cnt[w];
        }
        double beta = n > 0 ? s / (double)n : 0.0;
        s_beta = beta;
        ctl->beta = beta;
        ctl->max_delta = m;
        int move = 0;
        if (mode == 0) {
            ctl->iter += 1;
            int conv = m < ctl->thr;
            ctl->converged = conv;
            move = !conv && ctl->iter < p.max_iter && ctl->status == kOk;
        }
        s_move = move;
    }
    __syncthreads();
    if (mode != 0) return;
    if (s_move) {
        double beta = s_beta;
        for (int c = tid; c < p.k; c += blockDim.x) {
            for (int j = 0; j < p.d; ++j) p.C[c * p.d + j] = p.Cm[c * p.d + j];
            if (p.erosion) {
                double dl = p.delta[c];
                double alpha;
                if (beta > 0.0) {
                    double tt = fmin(-dl / beta, 0.0);
                    alpha = 2.0 / (1.0 + exp(tt)) - 1.0;
                } else {
                    alpha = dl > 0.0 ? 1.0 : 0.0;
                }
                p.I[c] = exp((1.0 - alpha) * log(p.I[c]));
            }
            write_cdata(p, c);
        }
    }
    if (tid == 0) {
        ctl->cont_move = s_move;
        ctl->pass_in_phase = 0;
        ctl->cont_balance = 1;
        if (h_move) cudaGraphSetConditional(h_move, (unsigned)s_move);
        if (h_bal) cudaGraphSetConditional(h_bal, 1u);
    }
}

// Copies C and I into the workspace state and prepares the center data (standalone
// assignment / movement steps).
__global__ void load_state_kernel(Prob p) {
    count_launch(p.ctl);
    for (int c = threadIdx.x; c < p.k; c += blockDim.x) {
        write_cdata(p, c);
        p.Iused[c] = p.I[c];
    }
}

// ------------------------------------------------------------------------------
// Host launchers.
// ------------------------------------------------------------------------------
cudaError_t launch_init(const Prob &p, cudaStream_t s) {
    init_kernel<<<1, 1024, 0, s>>>(p, 0, 0);
    return cudaGetLastError();
}
cudaError_t launch_load_state(const Prob &p, cudaStream_t s) {
    load_state_kernel<<<1, 1024, 0, s>>>(p);
    return cudaGetLastError();
}

static void *filter_fn(int d) {
    return d == 2 ? (void *)filter_kernel<2> : (void *)filter_kernel<3>;
}
static void *assign_fn(int d, int f64) {
    if (d == 2) return f64 ? (void *)assign_kernel<2, true> : (void *)assign_kernel<2, false>;
    return f64 ? (void *)assign_kernel<3, true> : (void *)assign_kernel<3, false>;
}
static void *centroid_fn(int d) {
    return d == 2 ? (void *)centroid_kernel<2> : (void *)centroid_kernel<3>;
}

cudaError_t launch_filter(const Prob &p, cudaStream_t s) {
    void *args1[] = {(void *)&p};
    int fgrid = (p.ntiles + kFilterWarps - 1) / kFilterWarps;
    return cudaLaunchKernel(filter_fn(p.d), dim3(fgrid), dim3(kFilterWarps * 32), args1, 0, s);
}
cudaError_t launch_assign(const Prob &p, cudaStream_t s) {
    void *args1[] = {(void *)&p};
    return cudaLaunchKernel(assign_fn(p.d, p.assign_f64), dim3(p.ntiles), dim3(kTile), args1, 0, s);
}
cudaError_t launch_balance(const Prob &p, int mode, cudaStream_t s) {
    balance_kernel<<<1, 1024, 0, s>>>(p, mode, 0);
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
    balance_kernel<<<1, 1024, 0, s>>>(p, 2, 0);
    return cudaGetLastError();
}

cudaError_t launch_move(const Prob &p, int mode, cudaStream_t s) {
    void *args1[] = {(void *)&p};
    cudaError_t e = cudaLaunchKernel(centroid_fn(p.d), dim3((unsigned)((p.n + 255) / 256)),
                                     dim3(256), args1, 0, s);
    if (e != cudaSuccess) return e;
    finalize_kernel<<<1, 1024, 0, s>>>(p, mode, 0, 0);
    return cudaGetLastError();
}

cudaError_t launch_final_begin(const Prob &p, cudaStream_t s) {
    final_begin_kernel<<<1, 32, 0, s>>>(p, 0);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------
// The whole loop as one CUDA graph:
//   init -> while(h_move){ while(h_bal){ filter -> assign -> balance(0) } ->
//           centroid -> finalize } -> final_begin -> while(h_fin){ filter -> assign ->
//           balance(1) }
// ------------------------------------------------------------------------------
namespace {
struct NodeAdder {
    cudaGraph_t g;
    cudaGraphNode_t last = nullptr;
    cudaError_t err = cudaSuccess;
    void kernel(void *fn, dim3 grid, dim3 block, void **args) {
        if (err != cudaSuccess) return;
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeKernel;
        np.kernel.func = fn;
        np.kernel.gridDim = grid;
        np.kernel.blockDim = block;
        np.kernel.sharedMemBytes = 0;
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

cudaError_t build_loop_graph(const Prob &pc, cudaGraphExec_t *exec_out, int *nodes_per_pass) {
    Prob p = pc;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h_move, h_bal, h_fin;
    e = cudaGraphConditionalHandleCreate(&h_move, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h_bal, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h_fin, g, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    int fgrid = (p.ntiles + kFilterWarps - 1) / kFilterWarps;
    int mode0 = 0, mode1 = 1;
    void *a_init[] = {&p, &h_move, &h_bal};
    void *a_p[] = {&p};
    void *a_bal0[] = {&p, &mode0, &h_bal};
    void *a_bal1[] = {&p, &mode1, &h_fin};
    void *a_fin[] = {&p, &mode0, &h_move, &h_bal};
    void *a_fb[] = {&p, &h_fin};

    NodeAdder top{g};
    top.kernel((void *)init_kernel, dim3(1), dim3(1024), a_init);
    cudaGraph_t body_move = top.loop(h_move);
    if (body_move) {
        NodeAdder mv{body_move};
        cudaGraph_t body_bal = mv.loop(h_bal);
        if (body_bal) {
            NodeAdder bl{body_bal};
            bl.kernel(filter_fn(p.d), dim3(fgrid), dim3(kFilterWarps * 32), a_p);
            bl.kernel(assign_fn(p.d, p.assign_f64), dim3(p.ntiles), dim3(kTile), a_p);
            bl.kernel((void *)balance_kernel, dim3(1), dim3(1024), a_bal0);
            if (bl.err != cudaSuccess) mv.err = bl.err;
        }
        mv.kernel(centroid_fn(p.d), dim3((unsigned)((p.n + 255) / 256)), dim3(256), a_p);
        mv.kernel((void *)finalize_kernel, dim3(1), dim3(1024), a_fin);
        if (mv.err != cudaSuccess) top.err = mv.err;
    }
    top.kernel((void *)final_begin_kernel, dim3(1), dim3(32), a_fb);
    cudaGraph_t body_fin = top.loop(h_fin);
    if (body_fin) {
        NodeAdder fl{body_fin};
        fl.kernel(filter_fn(p.d), dim3(fgrid), dim3(kFilterWarps * 32), a_p);
        fl.kernel(assign_fn(p.d, p.assign_f64), dim3(p.ntiles), dim3(kTile), a_p);
        fl.kernel((void *)balance_kernel, dim3(1), dim3(1024), a_bal1);
        if (fl.err != cudaSuccess) top.err = fl.err;
    }
    e = top.err;
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec_out, g, 0);
    cudaGraphDestroy(g);
    if (nodes_per_pass) *nodes_per_pass = 3;
    return e;
}

}  // namespace gk
