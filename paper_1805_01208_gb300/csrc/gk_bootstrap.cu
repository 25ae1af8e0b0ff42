// gk_bootstrap.cu -- space-filling-curve bootstrap (Algorithm 2: sfcIndex, sortGlobal,
// redistribution, initial centers) and the final scatter to input order.
//
//   bbox_kernel        bounding box, weight range, finiteness (Section 4.4 "bb")
//   keys_kernel        grid quantisation + Hilbert index (Algorithm 2 sfcIndex)
//   radix_*            stable LSD radix sort of (key, index) (Algorithm 2 sortGlobal)
//   gather_kernel      curve-sorted SoA copies + total weight (Algorithm 2 redistribution)
//   tile_box_kernel    per-tile bounding boxes for the candidate filter (Section 4.4)
//   centers_kernel     C[i] = sorted point i*n/k + n/(2k), influence 1 (Algorithm 2)
//   scatter_kernel     block ids back to input order
#include <type_traits>

#include "gk_common.cuh"
#include "gk_internal.h"

namespace gk {

// ------------------------------------------------------------------------------
// Bounding box.  Per-thread extremes in the input precision, CTA reduction, then
// one ordered-key atomic per CTA and axis.
// ------------------------------------------------------------------------------
// The extremes are taken on ordered keys (integer min / max: no FP64 pipe work, which
// is scarce on this GPU); a NaN or infinity sets nonfinite, a weight <= 0 nonpositive_w.
template <typename T>
struct KeyBits;
template <>
struct KeyBits<float> {
    using K = unsigned;
    __device__ static K bits(float v) { return __float_as_uint(v); }
    __device__ static bool nonfinite(K b) { return (b & 0x7f800000u) == 0x7f800000u; }
    __device__ static bool nonpositive(K b) { return (b >> 31) || b == 0u; }
    __device__ static K key(K b) { return (b >> 31) ? ~b : (b | 0x80000000u); }
    __device__ static unsigned long long key64(K k) { return okey_f64((double)okey_to_f32(k)); }
};
template <>
struct KeyBits<double> {
    using K = unsigned long long;
    __device__ static K bits(double v) { return (K)__double_as_longlong(v); }
    __device__ static bool nonfinite(K b) { return ((b >> 52) & 0x7ff) == 0x7ff; }
    __device__ static bool nonpositive(K b) { return (b >> 63) || b == 0ull; }
    __device__ static K key(K b) { return (b >> 63) ? ~b : (b | 0x8000000000000000ull); }
    __device__ static unsigned long long key64(K k) { return k; }
};

template <typename T>
__global__ void bbox_kernel(Prob p) {
    count_launch(p.ctl);
    using KB = KeyBits<T>;
    using K = typename KB::K;
    const K kmin0 = ~(K)0, kmax0 = (K)0;
    const K *x = (const K *)p.coords;
    const K *w = (const K *)p.weights;
    K lo[3] = {kmin0, kmin0, kmin0}, hi[3] = {kmax0, kmax0, kmax0};
    K wlo = kmin0, whi = kmax0;
    int bad = 0, nonpos = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    constexpr int kPts = 4;  // points per thread and step: their loads are in flight together
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < p.n; i0 += kPts * stride) {
        K v[kPts][3], wv[kPts];
#pragma unroll
        for (int u = 0; u < kPts; ++u) {
            const long long i = i0 + u * stride;
            const bool ok = i < p.n;
#pragma unroll
            for (int j = 0; j < 3; ++j) v[u][j] = (ok && j < p.d) ? x[i * p.d + j] : (K)0;
            wv[u] = (ok && w) ? w[i] : (K)0;
        }
#pragma unroll
        for (int u = 0; u < kPts; ++u) {
            if (i0 + u * stride >= p.n) break;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (j >= p.d) break;
                const K b = v[u][j];
                bad |= KB::nonfinite(b);
                const K key = KB::key(b);
                lo[j] = min(lo[j], key);
                hi[j] = max(hi[j], key);
            }
            if (w) {
                const K b = wv[u];
                bad |= KB::nonfinite(b);
                nonpos |= KB::nonpositive(b);
                const K key = KB::key(b);
                wlo = min(wlo, key);
                whi = max(whi, key);
            }
        }
    }
    __shared__ K s_lo[3][32], s_hi[3][32], s_wlo[32], s_whi[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < 3; ++j) {
        K a = lo[j], b = hi[j];
        for (int o = 16; o; o >>= 1) {
            a = min(a, (K)__shfl_xor_sync(0xffffffffu, a, o));
            b = max(b, (K)__shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0) {
            s_lo[j][warp] = a;
            s_hi[j][warp] = b;
        }
    }
    K a = wlo, b = whi;
    for (int o = 16; o; o >>= 1) {
        a = min(a, (K)__shfl_xor_sync(0xffffffffu, a, o));
        b = max(b, (K)__shfl_xor_sync(0xffffffffu, b, o));
    }
    if (lane == 0) {
        s_wlo[warp] = a;
        s_whi[warp] = b;
    }
    bad = __syncthreads_or(bad);
    nonpos = __syncthreads_or(nonpos);
    if (threadIdx.x == 0) {
        for (int j = 0; j < p.d; ++j) {
            K l = s_lo[j][0], h = s_hi[j][0];
            for (int q = 1; q < nw; ++q) {
                l = min(l, s_lo[j][q]);
                h = max(h, s_hi[j][q]);
            }
            if (l != kmin0) atomicMin(&p.ctl->bb_lo[j], KB::key64(l));
            if (h != kmax0) atomicMax(&p.ctl->bb_hi[j], KB::key64(h));
        }
        if (w) {
            K l = s_wlo[0], h = s_whi[0];
            for (int q = 1; q < nw; ++q) {
                l = min(l, s_wlo[q]);
                h = max(h, s_whi[q]);
            }
            if (l != kmin0) atomicMin(&p.ctl->w_lo, KB::key64(l));
            if (h != kmax0) atomicMax(&p.ctl->w_hi, KB::key64(h));
        }
        if (bad) atomicOr(&p.ctl->nonfinite, 1);
        if (nonpos) atomicOr(&p.ctl->nonpositive_w, 1);
    }
}

// ------------------------------------------------------------------------------
// Hilbert keys.  Cell = floor(fl(x - lo) * 2^m) clamped to 2^b - 1, computed from
// the bits of the (non-negative) difference; then J. Skilling's transform
// ("Programming the Hilbert curve", 2004): undo the excess work level by level,
// Gray-encode, and interleave the transposed bits (axis 0 most significant).
// ------------------------------------------------------------------------------
__device__ __forceinline__ unsigned quant_bits_f64(double v, int m, int b) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    int ex = (int)((bits >> 52) & 0x7ff);
    unsigned long long top = (1ull << b) - 1ull;
    if (ex == 0) return 0u;  // zero (v >= 0; subnormals floor to 0 for b <= 32)
    unsigned long long mant = (bits & 0xfffffffffffffull) | 0x10000000000000ull;
    int sh = ex - 1075 + m;  // v * 2^m = mant * 2^sh
    unsigned long long q;
    if (sh >= 0)
        q = sh > 11 ? ~0ull : (mant << sh);
    else
        q = sh > -64 ? (mant >> (-sh)) : 0ull;
    return (unsigned)(q > top ? top : q);
}
__device__ __forceinline__ unsigned quant_bits_f32(float v, int m, int b) {
    unsigned bits = __float_as_uint(v);
    int ex = (int)((bits >> 23) & 0xff);
    unsigned long long top = (1ull << b) - 1ull;
    if (ex == 0) return 0u;
    unsigned long long mant = (unsigned long long)((bits & 0x7fffffu) | 0x800000u);
    int sh = ex - 150 + m;
    unsigned long long q;
    if (sh >= 0)
        q = sh > 40 ? ~0ull : (mant << sh);
    else
        q = sh > -64 ? (mant >> (-sh)) : 0ull;
    return (unsigned)(q > top ? top : q);
}

__host__ __device__ __forceinline__ unsigned long long spread2(unsigned v) {
    unsigned long long x = v;
    x = (x | (x << 16)) & 0x0000ffff0000ffffull;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}
__host__ __device__ __forceinline__ unsigned long long spread3(unsigned v) {
    unsigned long long x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// B bits per axis (32 in 2-D, 21 in 3-D); the levels are unrolled, and each level's
// "exchange the low bits of X[0] and X[i], or invert those of X[0]" is branch-free.
template <int D, int B>
__host__ __device__ __forceinline__ unsigned long long skilling_key(unsigned X[D]) {
    // inverse undo, coarse level first
#pragma unroll
    for (int lev = B - 1; lev >= 1; --lev) {
        const unsigned P = (1u << lev) - 1u;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const unsigned set = 0u - ((X[i] >> lev) & 1u);  // all ones if bit lev of X[i] is set
            const unsigned t = (X[0] ^ X[i]) & P & ~set;       // low bits to exchange (clear bit)
            X[0] ^= (P & set) | t;
            if (i > 0) X[i] ^= t;
        }
    }
    // Gray encode
#pragma unroll
    for (int i = 1; i < D; ++i) X[i] ^= X[i - 1];
    unsigned y = X[D - 1] >> 1;  // bit l of t = xor of the bits of X[D-1] above l
    y ^= y >> 1;
    y ^= y >> 2;
    y ^= y >> 4;
    y ^= y >> 8;
    y ^= y >> 16;
#pragma unroll
    for (int i = 0; i < D; ++i) X[i] ^= y;
    if (D == 2) return (spread2(X[0]) << 1) | spread2(X[1]);
    return (spread3(X[0]) << 2) | (spread3(X[1]) << 1) | spread3(X[2]);
}

// The 2-D curve of skilling_key<2, 32> as a four-state machine, one level (two key bits)
// per step: entry 4 s + 2 xbit + ybit holds the level's digit and, shifted by two, the
// next state; the walk starts in state 0 at the top level.  The states were read off
// skilling_key level by level, and the walk gives its key for every input (the key tests
// compare the keys of both dimensions with the oracle's independent level descent).  Four
// levels per step come from a 1024-entry table each CTA builds from this one.
__constant__ unsigned char kHilbertStep2[16] = {4, 1, 11, 2, 0, 15, 5, 6, 10, 9, 3, 12, 14, 7, 13, 8};

template <typename T, int D>
__global__ void __launch_bounds__(256) keys_kernel(Prob p, unsigned long long *keys_out, unsigned *perm_out) {
    count_launch(p.ctl);
    __shared__ unsigned short step4[D == 2 ? 1024 : 1];  // 2-D: state, x and y nibbles
    if constexpr (D == 2) {
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
            const int xn = (e >> 4) & 15, yn = e & 15;
            int st = e >> 8, out = 0;
            for (int l = 3; l >= 0; --l) {
                const int v = kHilbertStep2[st * 4 + ((((xn >> l) & 1) << 1) | ((yn >> l) & 1))];
                out = (out << 2) | (v & 3);
                st = v >> 2;
            }
            step4[e] = (unsigned short)(out | (st << 8));
        }
        __syncthreads();
    }
    const T *x = (const T *)p.coords;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) {
        unsigned q[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            if (sizeof(T) == 8) {
                double v = __dsub_rn((double)x[i * D + j], p.origin[j]);
                q[j] = quant_bits_f64(v, p.grid_m, p.bits);
            } else {
                float v = __fsub_rn((float)x[i * D + j], (float)p.origin[j]);
                q[j] = quant_bits_f32(v, p.grid_m, p.bits);
            }
        }
        unsigned long long key;
        if constexpr (D == 2) {
            key = 0ull;
            unsigned st = 0u;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const unsigned e = (((q[0] >> (28 - 4 * c)) & 15u) << 4) | ((q[1] >> (28 - 4 * c)) & 15u);
                const unsigned v = step4[(st << 8) | e];
                key = (key << 8) | (v & 255u);
                st = v >> 8;
            }
        } else {
            key = skilling_key<D, 21>(q);
        }
        keys_out[i] = key;
        if (perm_out) perm_out[i] = (unsigned)i;
    }
}

// ------------------------------------------------------------------------------
// LSD radix sort of (uint64 key, uint32 value), 8-bit digits, stable.
// The array is cut into G contiguous segments of whole tiles (2048 items); each
// CTA owns one segment.  Per pass: upsweep (segment digit counts), a scan of each
// digit's row of the count table (one CTA per digit), downsweep (digit starts from
// the digit totals and the row prefixes; tiles of a segment in order; stable ranks
// inside a tile from per-warp match_any counting).
// ------------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortWarps = kSortThreads / 32;

__global__ void __launch_bounds__(kSortThreads)
radix_upsweep(const unsigned long long *keys, long long n, int shift, int tiles_per_seg, int G,
              unsigned *hist, Ctl *ctl) {
    count_launch(ctl);
    __shared__ unsigned cnt[kSortWarps][256];  // per-warp counts (a shared atomic per key)
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int w = 0; w < kSortWarps; ++w) cnt[w][tid] = 0;
    __syncthreads();
    const long long beg = (long long)blockIdx.x * tiles_per_seg * kSortTile;  // even
    long long end = beg + (long long)tiles_per_seg * kSortTile;
    if (end > n) end = n;
    auto count = [&](unsigned d) {
        if (d < 256u) atomicAdd(&cnt[warp][d], 1u);
    };
    // pairs of keys (16-byte loads), kLoads pairs in flight per thread
    constexpr int kLoads = 4;
    const ulonglong2 *k2 = reinterpret_cast<const ulonglong2 *>(keys);
    const long long pend = beg + ((end - beg) & ~1ll);  // end of the whole pairs
    for (long long i0 = beg; i0 < pend; i0 += 2ll * kSortThreads * kLoads) {
        ulonglong2 v[kLoads];
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
            const long long i = i0 + 2ll * (u * kSortThreads + tid);
            v[u] = i < pend ? k2[i >> 1] : make_ulonglong2(~0ull, ~0ull);
        }
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
            const long long i = i0 + 2ll * (u * kSortThreads + tid);
            count(i < pend ? ((unsigned)(v[u].x >> shift) & 255u) : 256u);
            count(i < pend ? ((unsigned)(v[u].y >> shift) & 255u) : 256u);
        }
    }
    if (pend < end) count(tid == 0 ? ((unsigned)(keys[pend] >> shift) & 255u) : 256u);
    __syncthreads();
    unsigned c = 0;
    for (int w = 0; w < kSortWarps; ++w) c += cnt[w][tid];
    hist[(long long)tid * G + blockIdx.x] = c;
}

// Row scan of the digit-major count table: CTA d turns hist[d][0..G) into exclusive
// prefixes over the segments and writes the digit's total to totals[d].
__global__ void __launch_bounds__(256) radix_scan(unsigned *hist, int G, unsigned *totals, Ctl *ctl) {
    count_launch(ctl);
    __shared__ unsigned wsum[8];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    unsigned *row = hist + (long long)blockIdx.x * G;
    const int per = (G + 255) / 256;
    const int b = t * per, e = min(G, b + per);
    unsigned s = 0;
    for (int i = b; i < e; ++i) s += row[i];
    // exclusive scan of the 256 thread sums
    unsigned x = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    unsigned before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        before += w < warp ? wsum[w] : 0u;
        total += wsum[w];
    }
    unsigned run = before + x - s;
    for (int i = b; i < e; ++i) {
        const unsigned c = row[i];
        row[i] = run;
        run += c;
    }
    if (t == 0) totals[blockIdx.x] = total;
}

// Dynamic shared memory of the downsweep: the current tile in digit order.  The tile
// comes into registers straight from global memory (coalesced 8-byte loads); with no
// staging copy in shared memory four CTAs fit an SM, whose other warps hide the loads.
constexpr size_t kDownsweepSmem = (size_t)kSortTile * (8 + 4);

__global__ void __launch_bounds__(kSortThreads, 4)
radix_downsweep(const unsigned long long *keys_in, const unsigned *vals_in,
                unsigned long long *keys_out, unsigned *vals_out, long long n, int shift,
                int tiles_per_seg, int G, const unsigned *offs, const unsigned *totals, Ctl *ctl) {
    count_launch(ctl);
    extern __shared__ __align__(16) unsigned char dsm[];
    unsigned long long *skey = reinterpret_cast<unsigned long long *>(dsm);  // digit order
    unsigned *sval = reinterpret_cast<unsigned *>(dsm + (size_t)kSortTile * 8);
    __shared__ unsigned run_off[256];               // output position of the digit's next item
    __shared__ unsigned whist[kSortWarps][256];     // per-warp counts, then per-warp offsets
    __shared__ unsigned tstart[256];                // start of each digit in the tile's order
    __shared__ unsigned wsum[kSortWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    static_assert(kSortThreads == 256, "one thread per digit below");
    // exclusive scan over the 256 digits of v (thread tid holds digit tid's value)
    auto digit_scan = [&](unsigned v) -> unsigned {
        unsigned x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        unsigned before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        __syncthreads();
        return before + x - v;
    };
    const long long seg_beg = (long long)blockIdx.x * tiles_per_seg * kSortTile;
    // start of each digit: exclusive scan of the digit totals, plus this segment's prefix
    // within the digit
    run_off[tid] = digit_scan(totals[tid]) + offs[(long long)tid * G + blockIdx.x];
    for (int w = 0; w < kSortWarps; ++w) whist[w][tid] = 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int t = 0; t < tiles_per_seg; ++t) {
        const long long tile_beg = seg_beg + (long long)t * kSortTile;
        if (tile_beg >= n) break;
        const int nt = (int)(n - tile_beg < kSortTile ? n - tile_beg : kSortTile);
        unsigned long long k[kSortItems];
        unsigned v[kSortItems], dig[kSortItems], loc[kSortItems];
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const int li = warp * (32 * kSortItems) + r * 32 + lane;
            k[r] = li < nt ? __ldcs(keys_in + tile_beg + li) : 0ull;  // read once: streaming
            v[r] = li < nt ? __ldcs(vals_in + tile_beg + li) : 0u;
        }
        // the per-warp counts were cleared by other threads (thread d clears digit d of every
        // warp's row): they must be zero before any warp ranks
        __syncthreads();
        // ranks inside the warp: items of a warp in order, equal digits counted with match_any
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const int li = warp * (32 * kSortItems) + r * 32 + lane;
            const bool ok = li < nt;
            dig[r] = ok ? ((unsigned)(k[r] >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, dig[r]);
            const unsigned base = ok ? whist[warp][dig[r]] : 0u;
            loc[r] = base + __popc(peers & lt_mask);
            __syncwarp();
            if (ok && (peers & lt_mask) == 0u) whist[warp][dig[r]] = base + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // thread = digit: per-warp offsets (in place), the tile's count and its start
        unsigned tc = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            const unsigned c = whist[w][tid];
            whist[w][tid] = tc;
            tc += c;
        }
        tstart[tid] = digit_scan(tc);
        __syncthreads();
        // the tile in digit order in shared memory
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            if (dig[r] < 256u) {
                const unsigned pos = tstart[dig[r]] + whist[warp][dig[r]] + loc[r];
                if (pos < (unsigned)kSortTile) {  // always true when the counts are consistent
                    skey[pos] = k[r];
                    sval[pos] = v[r];
                }
            }
        }
        __syncthreads();
        // write-out in tile order: runs of equal digits go to consecutive addresses
        for (int i = tid; i < nt; i += kSortThreads) {
            const unsigned long long kk = skey[i];
            const unsigned d = (unsigned)(kk >> shift) & 255u;
            const unsigned dst = run_off[d] + (unsigned)i - tstart[d];
            if (dst < (unsigned long long)n) {  // always true when counts are consistent
                keys_out[dst] = kk;
                vals_out[dst] = sval[i];
            }
        }
        __syncthreads();
        run_off[tid] += tc;
        for (int w = 0; w < kSortWarps; ++w) whist[w][tid] = 0;
    }
}

// ------------------------------------------------------------------------------
// Gather into curve order: SoA frame coordinates (FP32), raw FP64 coordinates,
// sorted weights, and the total weight as a 128-bit fixed-point sum.
// ------------------------------------------------------------------------------
// perm: destination index -> input index (nullptr: identity); nsrc: input points.
template <typename T>
__device__ __forceinline__ void gather_body(const Prob &p, const unsigned *perm, long long nsrc) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const T *x = (const T *)p.coords;
    const T *w = (const T *)p.weights;
    unsigned long long wfix = 0;
    if (i < p.n_pad) {
        long long src = i < p.n ? (perm ? (long long)perm[i] : i) : 0;
        bool ok = i < p.n && src < nsrc;  // a permutation entry is always < nsrc
        T xv[3] = {(T)0, (T)0, (T)0};
        if (ok) {
            if (p.d == 2 && ((uintptr_t)x % (2 * sizeof(T))) == 0) {  // one 2-element load
                using V2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
                const V2 q = reinterpret_cast<const V2 *>(x)[src];
                xv[0] = q.x;
                xv[1] = q.y;
            } else {
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (j < p.d) xv[j] = x[src * p.d + j];
            }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (j >= p.d) break;
            T v = xv[j];
            if (sizeof(T) == 8) {
                double dv = (double)v;
                p.X64[j * p.n_pad + i] = dv;
                double f = ok ? __dmul_rn(__dsub_rn(dv, p.origin[j]), p.scale) : 0.0;
                p.X32[j * p.n_pad + i] = __double2float_rn(f);
            } else {
                p.X32[j * p.n_pad + i] = (float)v;
            }
        }
        if (p.weighted) {
            T wv = ok ? w[src] : (T)0;
            ((T *)p.Ws)[i] = wv;
            if (ok) wfix = (unsigned long long)(sizeof(T) == 8 ? fix_f64((double)wv, p.Fw)
                                                                : fix_f32((float)wv, p.Fw));
        }
    }
    if (p.weighted) {
        for (int o = 16; o; o >>= 1) wfix += __shfl_xor_sync(0xffffffffu, wfix, o);
        if ((threadIdx.x & 31) == 0 && wfix) atomic_add_u128(&p.ctl->wsum_lo, wfix);
    }
}

template <typename T>
__global__ void gather_kernel(Prob p, const unsigned *perm) {
    count_launch(p.ctl);
    gather_body<T>(p, perm, p.n);
}

// Per tile: origin = centre of the bounding box of its frame coordinates, half
// extents and radius rounded upwards so that every point of the tile lies inside.
// One warp per tile (lane l: points 8l..8l+7), kTileBoxWarps tiles per CTA.
constexpr int kTileBoxWarps = 8;
__global__ void __launch_bounds__(kTileBoxWarps * 32) tile_box_kernel(Prob p) {
    count_launch(p.ctl);
    const int lane = threadIdx.x & 31;
    const long long t = (long long)blockIdx.x * kTileBoxWarps + (threadIdx.x >> 5);
    if (t >= p.ntiles) return;
    const long long i0 = t * kTile + lane * 8;
    float lo[3], hi[3];
    for (int j = 0; j < 3; ++j) {
        lo[j] = INFINITY;
        hi[j] = -INFINITY;
    }
    for (int j = 0; j < p.d; ++j) {
        const float4 *src = reinterpret_cast<const float4 *>(p.X32 + (size_t)j * p.n_pad + i0);
        const float4 a = src[0], b = src[1];  // inside the padded plane
        const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (i0 + q < p.n) {
                lo[j] = fminf(lo[j], v[q]);
                hi[j] = fmaxf(hi[j], v[q]);
            }
        }
        for (int o = 16; o; o >>= 1) {
            lo[j] = fminf(lo[j], __shfl_xor_sync(0xffffffffu, lo[j], o));
            hi[j] = fmaxf(hi[j], __shfl_xor_sync(0xffffffffu, hi[j], o));
        }
    }
    // the tile's fixed-point coordinate sums (w x) and the ordered keys of its smallest and
    // largest coordinates, as the movement converts them (its points never move)
    for (int j = 0; j < p.d; ++j) {
        long long sum = 0;
        unsigned long long kmin = ~0ull, kmax = 0ull;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (i0 + q < p.n) {
                long long v;
                unsigned long long kk;
                if (p.dtype == 1) {
                    const double x = p.X64[(size_t)j * p.n_pad + i0 + q];
                    v = p.weighted ? fix_f64(((const double *)p.Ws)[i0 + q] * x, p.Fx) : fix_f64(x, p.Fx);
                    kk = okey_f64(x);
                } else {
                    const float x = p.X32[(size_t)j * p.n_pad + i0 + q];
                    v = p.weighted ? fix_prod_f32(((const float *)p.Ws)[i0 + q], x, p.Fx) : fix_f32(x, p.Fx);
                    kk = okey_f32(x);
                }
                sum += v;
                kmin = kk < kmin ? kk : kmin;
                kmax = kk > kmax ? kk : kmax;
            }
        }
        for (int o = 16; o; o >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, kmin, o);
            const unsigned long long b = __shfl_xor_sync(0xffffffffu, kmax, o);
            kmin = a < kmin ? a : kmin;
            kmax = b > kmax ? b : kmax;
        }
        if (lane == 0) {
            p.tsx[t * p.d + j] = sum;
            p.tlo[t * p.d + j] = kmin;
            p.thi[t * p.d + j] = kmax;
        }
    }
    if (p.weighted) {  // the tile's weight sum, as the assignment's histogram converts weights
        unsigned long long ws = 0ull;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (i0 + q < p.n)
                ws += (unsigned long long)(p.dtype == 1 ? fix_f64(((const double *)p.Ws)[i0 + q], p.Fw)
                                                        : fix_f32(((const float *)p.Ws)[i0 + q], p.Fw));
        for (int o = 16; o; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
        if (lane == 0) p.tws[t] = ws;
    }
    if (lane == 0) {
        float o[3] = {0.f, 0.f, 0.f}, h[3] = {0.f, 0.f, 0.f};
        float r2 = 0.0f;
        for (int j = 0; j < p.d; ++j) {
            o[j] = 0.5f * lo[j] + 0.5f * hi[j];
            h[j] = fmaxf(__fsub_ru(hi[j], o[j]), __fsub_ru(o[j], lo[j]));
            r2 = __fadd_ru(r2, __fmul_ru(h[j], h[j]));
        }
        p.tiles[2 * t] = make_float4(o[0], o[1], o[2], __fsqrt_ru(r2));
        // w: the block id that every stored 16-bit id of the tile holds, -1 for none yet
        // (kept up to date by the assignment, forwarded to it by the filter)
        p.tiles[2 * t + 1] = make_float4(h[0], h[1], h[2], __int_as_float(-1));
    }
}
static int tile_box_grid(int ntiles) { return (ntiles + kTileBoxWarps - 1) / kTileBoxWarps; }

// Initial centers on the curve (raw coordinates, FP64) and influence 1.
__global__ void centers_kernel(Prob p) {
    count_launch(p.ctl);
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.k) return;
    long long idx = (long long)c * p.n / p.k + p.n / (2ll * p.k);
    for (int j = 0; j < p.d; ++j)
        p.C[c * p.d + j] = p.dtype == 1 ? p.X64[j * p.n_pad + idx] : (double)p.X32[j * p.n_pad + idx];
    p.Iin[c] = 1.0;
}

// Supertile boxes from the boxes of their tiles (rounded outwards).
__global__ void super_box_kernel(Prob p) {
    count_launch(p.ctl);
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.nsupers) return;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int t0 = s * p.stiles, t1 = min(p.ntiles, t0 + p.stiles);
    for (int t = t0; t < t1; ++t) {
        float4 a = p.tiles[2 * t], b = p.tiles[2 * t + 1];
        float o[3] = {a.x, a.y, a.z}, h[3] = {b.x, b.y, b.z};
        for (int j = 0; j < 3; ++j) {
            lo[j] = fminf(lo[j], __fsub_rd(o[j], h[j]));
            hi[j] = fmaxf(hi[j], __fadd_ru(o[j], h[j]));
        }
    }
    float o[3] = {0.f, 0.f, 0.f}, h[3] = {0.f, 0.f, 0.f};
    float r2 = 0.0f;
    for (int j = 0; j < p.d; ++j) {
        o[j] = 0.5f * lo[j] + 0.5f * hi[j];
        h[j] = fmaxf(__fsub_ru(hi[j], o[j]), __fsub_ru(o[j], lo[j]));
        r2 = __fadd_ru(r2, __fmul_ru(h[j], h[j]));
    }
    p.supers[2 * s] = make_float4(o[0], o[1], o[2], __fsqrt_ru(r2));
    p.supers[2 * s + 1] = make_float4(h[0], h[1], h[2], 0.0f);
}

// Hypertile boxes from the boxes of their supertiles (rounded outwards).
__global__ void hyper_box_kernel(Prob p) {
    count_launch(p.ctl);
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= p.nhypers) return;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int s0 = h * kHyperSupers, s1 = min(p.nsupers, s0 + kHyperSupers);
    for (int s = s0; s < s1; ++s) {
        float4 a = p.supers[2 * s], b = p.supers[2 * s + 1];
        float o[3] = {a.x, a.y, a.z}, hh[3] = {b.x, b.y, b.z};
        for (int j = 0; j < 3; ++j) {
            lo[j] = fminf(lo[j], __fsub_rd(o[j], hh[j]));
            hi[j] = fmaxf(hi[j], __fadd_ru(o[j], hh[j]));
        }
    }
    float o[3] = {0.f, 0.f, 0.f}, hh[3] = {0.f, 0.f, 0.f};
    float r2 = 0.0f;
    for (int j = 0; j < p.d; ++j) {
        o[j] = 0.5f * lo[j] + 0.5f * hi[j];
        hh[j] = fmaxf(__fsub_ru(hi[j], o[j]), __fsub_ru(o[j], lo[j]));
        r2 = __fadd_ru(r2, __fmul_ru(hh[j], hh[j]));
    }
    p.hypers[2 * h] = make_float4(o[0], o[1], o[2], __fsqrt_ru(r2));
    p.hypers[2 * h + 1] = make_float4(hh[0], hh[1], hh[2], 0.0f);
}


__global__ void scatter_kernel(const int *A_sorted, const unsigned short *A16_sorted, const unsigned *perm,
                               long long n, int *out, Ctl *ctl) {
    count_launch(ctl);
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        long long j = perm ? (long long)perm[i] : i;
        if (j < n) out[j] = A16_sorted ? (int)A16_sorted[i] : A_sorted[i];
    }
}

__global__ void perm_to_i64_kernel(const unsigned *perm, long long n, long long *out, Ctl *ctl) {
    count_launch(ctl);
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = perm[i];
}

// ------------------------------------------------------------------------------
// Random initialization (Section 4.5).  The random order of the points is an
// input: order[r] = input index of the point of rank r.  Round byte of rank r:
// the first round whose sample (the m0 * 2^j lowest ranks) holds it.  A sample
// round then selects the curve positions with round byte <= j, in curve order.
// ------------------------------------------------------------------------------
__device__ __forceinline__ unsigned char sample_round_of(long long rank, long long m0) {
    int r = 0;
    while (r < 254 && (m0 << r) <= rank) ++r;  // m0 >= 1 and rank < 2^32: r <= 32
    return (unsigned char)r;
}

// rho_in[order[r]] = round byte of rank r (rho_in preset to 0xff); entries of
// order outside [0, n) set bad_order.
__global__ void order_round_kernel(const long long *order, long long n, long long m0,
                                   unsigned char *rho_in, Ctl *ctl) {
    count_launch(ctl);
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    long long o = order[r];
    if (o < 0 || o >= n)
        atomicOr(&ctl->bad_order, 1);
    else
        rho_in[o] = sample_round_of(r, m0);
}

// rho[pos] = round byte of the point at curve position pos, 0xff beyond n; an
// input index that order never named (order is not a permutation) sets bad_order.
__global__ void rho_kernel(const unsigned char *rho_in, const unsigned *perm, long long n,
                           long long nrho, unsigned char *rho, Ctl *ctl) {
    count_launch(ctl);
    long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= nrho) return;
    unsigned char v = 0xff;
    if (pos < n) {
        v = rho_in[perm[pos]];
        if (v == 0xff) atomicOr(&ctl->bad_order, 1);
    }
    rho[pos] = v;
}

constexpr int kSelThreads = kSampleChunk / 16;  // 16 round bytes per thread (one uint4)

// Selected positions among the 16 bytes of v: bytes <= round.
__device__ __forceinline__ unsigned sel_mask16(uint4 v, unsigned rr) {
    unsigned a = __vcmpleu4(v.x, rr), b = __vcmpleu4(v.y, rr), c = __vcmpleu4(v.z, rr),
             d = __vcmpleu4(v.w, rr);
    unsigned m = 0;
    const unsigned w[4] = {a, b, c, d};
    for (int q = 0; q < 4; ++q)
        for (int j = 0; j < 4; ++j) m |= ((w[q] >> (8 * j + 7)) & 1u) << (4 * q + j);
    return m;
}

// Selection, part 1: selected positions per chunk; resets the sample's weight sum.
__global__ void __launch_bounds__(kSelThreads) sample_count_kernel(Prob ps, SampleSel sel) {
    count_launch(ps.ctl);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ps.ctl->wsum_lo = 0ull;
        ps.ctl->wsum_hi = 0ull;
    }
    const unsigned rr = 0x01010101u * (unsigned)sel.round;
    const uint4 v = ((const uint4 *)(sel.rho + (size_t)blockIdx.x * kSampleChunk))[threadIdx.x];
    unsigned c = __popc(sel_mask16(v, rr));
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ unsigned red[kSelThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int w = 0; w < kSelThreads / 32; ++w) t += red[w];
        sel.counts[blockIdx.x] = t;
    }
}

// Selection, part 2 (one CTA): exclusive prefix sums of the chunk counts, in place.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) sample_scan_kernel(Prob ps, SampleSel sel) {
    count_launch(ps.ctl);
    __shared__ unsigned wsum[kScanThreads / 32];
    const int per = (sel.nchunks + kScanThreads - 1) / kScanThreads;
    const int b0 = threadIdx.x * per, b1 = min(sel.nchunks, b0 + per);
    unsigned t = 0;
    for (int b = b0; b < b1; ++b) t += sel.counts[b];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = t;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    unsigned before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    unsigned run = before + x - t;
    for (int b = b0; b < b1; ++b) {
        unsigned c = sel.counts[b];
        sel.counts[b] = run;
        run += c;
    }
}

// Selection, part 3: sp[offset of the position among the selected] = input index.
__global__ void __launch_bounds__(kSelThreads) sample_write_kernel(Prob ps, SampleSel sel) {
    count_launch(ps.ctl);
    const unsigned rr = 0x01010101u * (unsigned)sel.round;
    const uint4 v = ((const uint4 *)(sel.rho + (size_t)blockIdx.x * kSampleChunk))[threadIdx.x];
    unsigned m = sel_mask16(v, rr);
    const unsigned c = __popc(m);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = c;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __shared__ unsigned wsum[kSelThreads / 32];
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    unsigned off = sel.counts[blockIdx.x] + x - c;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    const long long pos0 = (long long)blockIdx.x * kSampleChunk + 16 * threadIdx.x;
    while (m) {
        int j = __ffs(m) - 1;
        m &= m - 1;
        sel.sp[off++] = sel.perm[pos0 + j];  // a selected position is < n
    }
}

// Selection, part 4: the sample's sorted arrays (its own frame is the problem's).
template <typename T>
__global__ void sample_gather_kernel(Prob ps, SampleSel sel) {
    count_launch(ps.ctl);
    gather_body<T>(ps, sel.sp, sel.n);
}

// ------------------------------------------------------------------------------
// Host launchers.
// ------------------------------------------------------------------------------
static int blocks_for(long long n, int threads) { return (int)((n + threads - 1) / threads); }

cudaError_t launch_bbox(const Prob &p, cudaStream_t s) {
    int grid = 152 * 4;
    long long need = (p.n + 255) / 256;
    if (need < grid) grid = (int)need;
    if (grid < 1) grid = 1;
    if (p.dtype == 1)
        bbox_kernel<double><<<grid, 256, 0, s>>>(p);
    else
        bbox_kernel<float><<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_keys(const Prob &p, unsigned long long *keys, unsigned *perm, cudaStream_t s) {
    int grid = blocks_for(p.n, 256);
    const int cap = (p.nsm > 0 ? p.nsm : 152) * 16;  // grid-stride: each CTA builds its table once
    if (grid > cap) grid = cap;
    if (p.dtype == 1) {
        if (p.d == 2)
            keys_kernel<double, 2><<<grid, 256, 0, s>>>(p, keys, perm);
        else
            keys_kernel<double, 3><<<grid, 256, 0, s>>>(p, keys, perm);
    } else {
        if (p.d == 2)
            keys_kernel<float, 2><<<grid, 256, 0, s>>>(p, keys, perm);
        else
            keys_kernel<float, 3><<<grid, 256, 0, s>>>(p, keys, perm);
    }
    return cudaGetLastError();
}

size_t radix_hist_entries(long long n) {
    long long ntiles = (n + kSortTile - 1) / kSortTile;
    long long tps = (ntiles + 1215) / 1216;
    if (tps < 1) tps = 1;
    long long G = (ntiles + tps - 1) / tps;
    if (G < 1) G = 1;
    return (size_t)(256 * G + 256);  // count table, then the digit totals
}

// Sorts keys[0]/perm[0] (n items) in place through the alternate buffers; returns
// in *sel the index of the buffer pair holding the result.
cudaError_t launch_radix_sort(const Prob &p, int key_bits, unsigned *hist, int *sel,
                              cudaStream_t s) {
    long long n = p.n;
    long long ntiles = (n + kSortTile - 1) / kSortTile;
    int tps = (int)((ntiles + 1215) / 1216);
    if (tps < 1) tps = 1;
    int G = (int)((ntiles + tps - 1) / tps);
    if (G < 1) G = 1;
    // static + dynamic shared memory of the downsweep exceeds the default 48 KB
    cudaError_t e = cudaFuncSetAttribute(radix_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kDownsweepSmem);
    if (e != cudaSuccess) return e;
    int cur = 0;
    for (int shift = 0; shift < key_bits; shift += 8) {
        radix_upsweep<<<G, 256, 0, s>>>(p.keys[cur], n, shift, tps, G, hist, p.ctl);
        unsigned *totals = hist + (size_t)256 * G;
        radix_scan<<<256, 256, 0, s>>>(hist, G, totals, p.ctl);
        radix_downsweep<<<G, kSortThreads, kDownsweepSmem, s>>>(p.keys[cur], p.perm[cur], p.keys[cur ^ 1],
                                                    p.perm[cur ^ 1], n, shift, tps, G, hist, totals,
                                                    p.ctl);
        cur ^= 1;
    }
    *sel = cur;
    return cudaGetLastError();
}

cudaError_t launch_gather(const Prob &p, const unsigned *perm, cudaStream_t s) {
    int grid = blocks_for(p.n_pad, 256);
    if (p.dtype == 1)
        gather_kernel<double><<<grid, 256, 0, s>>>(p, perm);
    else
        gather_kernel<float><<<grid, 256, 0, s>>>(p, perm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tile_box_kernel<<<tile_box_grid(p.ntiles), kTileBoxWarps * 32, 0, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    super_box_kernel<<<blocks_for(p.nsupers, 128), 128, 0, s>>>(p);
    hyper_box_kernel<<<blocks_for(p.nhypers, 128), 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_super_boxes(const Prob &p, cudaStream_t s) {
    super_box_kernel<<<blocks_for(p.nsupers, 128), 128, 0, s>>>(p);
    hyper_box_kernel<<<blocks_for(p.nhypers, 128), 128, 0, s>>>(p);
    return cudaGetLastError();
}

long long sample_rho_entries(long long n) {
    return (n + kSampleChunk - 1) / kSampleChunk * kSampleChunk;
}

cudaError_t launch_sample_rho(const Prob &p, const long long *order, long long m0,
                              const unsigned *perm, unsigned char *rho_in, unsigned char *rho,
                              cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(rho_in, 0xff, (size_t)p.n, s);
    if (e != cudaSuccess) return e;
    order_round_kernel<<<blocks_for(p.n, 256), 256, 0, s>>>(order, p.n, m0, rho_in, p.ctl);
    const long long nrho = sample_rho_entries(p.n);
    rho_kernel<<<blocks_for(nrho, 256), 256, 0, s>>>(rho_in, perm, p.n, nrho, rho, p.ctl);
    return cudaGetLastError();
}

int sample_select_nodes(const Prob &ps, const SampleSel &sel, KNode *out) {
    int q = 0;
    const dim3 cg((unsigned)sel.nchunks), cb(kSelThreads);
    out[q++] = {(void *)sample_count_kernel, cg, cb};
    out[q++] = {(void *)sample_scan_kernel, dim3(1), dim3(kScanThreads)};
    out[q++] = {(void *)sample_write_kernel, cg, cb};
    out[q++] = {ps.dtype == 1 ? (void *)sample_gather_kernel<double> : (void *)sample_gather_kernel<float>,
                dim3((unsigned)blocks_for(ps.n_pad, 256)), dim3(256)};
    out[q++] = {(void *)tile_box_kernel, dim3((unsigned)tile_box_grid(ps.ntiles)), dim3(kTileBoxWarps * 32)};
    out[q++] = {(void *)super_box_kernel, dim3((unsigned)blocks_for(ps.nsupers, 128)), dim3(128)};
    out[q++] = {(void *)hyper_box_kernel, dim3((unsigned)blocks_for(ps.nhypers, 128)), dim3(128)};
    return q;
}

cudaError_t launch_sample_select(const Prob &ps, const SampleSel &sel, cudaStream_t s) {
    KNode nodes[kSampleSelectNodes];
    int q = sample_select_nodes(ps, sel, nodes);
    Prob pa = ps;
    SampleSel sa = sel;
    void *args[] = {(void *)&pa, (void *)&sa};
    for (int i = 0; i < q; ++i) {
        cudaError_t e = cudaLaunchKernel(nodes[i].fn, nodes[i].grid, nodes[i].block, args, 0, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

__global__ void iota_kernel(unsigned *perm, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = (unsigned)i;
}
cudaError_t launch_iota(unsigned *perm, long long n, cudaStream_t s) {
    iota_kernel<<<blocks_for(n, 256), 256, 0, s>>>(perm, n);
    return cudaGetLastError();
}

cudaError_t launch_centers(const Prob &p, cudaStream_t s) {
    centers_kernel<<<blocks_for(p.k, 256), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const Prob &p, const unsigned *perm, int *out, cudaStream_t s) {
    scatter_kernel<<<blocks_for(p.n, 256), 256, 0, s>>>(p.A, p.a16 ? p.A16 : nullptr, perm, p.n, out, p.ctl);
    return cudaGetLastError();
}

cudaError_t launch_perm_out(const Prob &p, const unsigned *perm, long long *out, cudaStream_t s) {
    perm_to_i64_kernel<<<blocks_for(p.n, 256), 256, 0, s>>>(perm, p.n, out, p.ctl);
    return cudaGetLastError();
}

}  // namespace gk
