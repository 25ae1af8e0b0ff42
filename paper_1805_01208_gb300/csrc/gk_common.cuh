// gk_common.cuh -- shared device-side definitions of the balanced k-means library.
//
// Data layout in device memory (one problem at a time, inside the workspace):
//   X32    d planes of n_pad FP32: curve-sorted coordinates in the assignment frame
//          (FP64 inputs: (x - lo) * 2^-E rounded to FP32, E = grid exponent of the
//          bounding box; FP32 inputs: the raw coordinates).  Padding entries are 0.
//   X64    d planes of n_pad FP64: curve-sorted raw coordinates (FP64 inputs only).
//   Ws     n_pad sorted weights in the input dtype (weighted problems only).
//   A      n_pad int32 block ids in sorted order (A16: the same as 16 bits, which the
//          k-means loop uses instead when k <= 65535: 2 B per point written per pass).
//   tiles  2 float4 per tile of kTile points: {origin xyz, radius}, {half extents xyz, -};
//   supers the same per supertile of stiles tiles.
//   per tile record (written by the filter every pass, kRecF4 float4): header
//          {count (int32; -1 = overflow: scan all centers), largest g of the tile's
//          candidates, lower bound of the E of every center left out of the list, 0},
//          {tile origin xyz, tile radius}, then up to kCap candidates
//          of 2 float4: {q xyz, g}, {center id (int32 bits), 0, 0, 0}; q = frame center
//          relative to the tile origin, g = scaled 1/I^2, ascending center order.
//   coop   the tiles with more than kFastCands candidates (or an overflowed list), taken
//          by a whole CTA of the assignment.
//   per center: C, Cm (k x d FP64, input units), delta, S64, Iin (k FP64), influence and
//          1/I^2 double-buffered (I2, g64_2: 2 x k FP64), cdata2 (2 x 2 float4 per center:
//          {frame center hi xyz, g32}, {frame center lo xyz, 0}), 128-bit fixed-point
//          block weights and coordinate sums, ordered-key bounding boxes.
//   per group of 32 consecutive centers, double-buffered like cdata2 (gdata2, 2 float4):
//          {box mid xyz, smallest g32}, {box half extents xyz, largest g32}; the same per
//          supergroup of 32 groups (sgdata, rebuilt from the current buffer's groups).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gk {

constexpr int kTile = 256;          // points per tile (one warp of the assign kernel)
constexpr int kSuperTiles = 16;     // tiles per supertile (one warp of the filter), default and
                                    // the smallest choice (it sizes the per-supertile arrays)
constexpr int kMaxSuperTiles = 32;  // the largest choice (one lane per tile in the filter)
constexpr int kHyperSupers = 16;    // supertiles per hypertile (the filter's first level)
constexpr int kHyperList = 128;     // longest hypertile list a supertile builds its own from
constexpr int kCap = 128;           // candidate centers stored per tile
constexpr int kFastCands = 32;      // candidates brought in with the tile's bulk copy
constexpr int kCoopCands = kFastCands;  // tiles with more candidates are taken by a whole CTA
constexpr int kRecF4 = 2 + 2 * kCap;  // float4 per tile record (header + candidates)
constexpr unsigned kRecFastBytes = (2 + 2 * kFastCands) * 16;  // largest record copy of a tile
constexpr int kKThreads = 32;       // threads per CTA of the k-sized kernels
constexpr int kSuperCap = 1024;     // candidate centers kept per supertile
constexpr int kGroup = 32;          // centers per group record (one CTA of the k-sized kernels)
constexpr int kSuperGroup = 32;     // groups per supergroup record (used when ngroups > 64)
constexpr int kWarpSG = 8;          // kept supergroups per supertile (more: sweep every group)
constexpr int kQueues = 8;          // interleaved tile queues of the assignment
constexpr int kWarpList = 512;      // level-1 candidate list kept per supertile by the filter
constexpr int kWarpGroups = 64;     // kept center groups per supertile
constexpr int kLaneMax = 64;        // longer lists: level 2 with a warp per tile
constexpr int kQueueStride = 32;    // one 128-byte line per queue counter
static_assert(kGroup == kKThreads, "a group record is written by one CTA of the k-sized kernels");
constexpr int kFixBits = 54;        // |fixed-point value| < 2^54 per point
constexpr int kStripes = 64;        // striped counters for per-pass statistics
constexpr int kStripeStride = 16;   // 64-bit words per stripe: each in its own 128-byte line
constexpr long long kSpinLimit = 1ll << 26;  // bounded waits on mbarriers: most polls,
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // and most device time (2 s)
constexpr int kSkipHist = 64;       // passes of a phase with per-point bounds (then a fresh pass)

// Error codes mirrored from gk.h (device code does not include the C header).
constexpr int kOk = 0;
constexpr int kErrTimeout = 5;

// Device-resident control block: geometry found by the bounding-box kernel, loop
// state and counters.  Written by kernels, read back by the host.
struct Ctl {
    unsigned long long bb_lo[3], bb_hi[3];  // ordered keys of the coordinate extremes
    unsigned long long w_lo, w_hi;          // ordered keys of the weight extremes
    int nonfinite;                          // a coordinate or weight is NaN/Inf
    int nonpositive_w;                      // a weight is <= 0
    int bad_block;                          // a given block id is outside [0, k)
    int bad_order;                          // the sample order is not a permutation
    int sample_iters;                       // movement phases of the sample rounds
    int sample_passes;                      // assignment passes of the sample rounds
    int phase_pass;                         // passes since the centers last moved (bounds)
    unsigned int min_lr_key;                // ordered keys of the pass's smallest and largest
    unsigned int max_lr_key;                //   log2 g ratio over the centers (bounds)
    unsigned long long evaluated;           // points whose assignment was evaluated (bounds)
    int status;                             // kOk or an error code
    int balanced;                           // last pass met the bound
    int converged;                          // movement below threshold
    int pass_in_phase;                      // passes in the current balance loop
    int iter;                               // movement phases done
    int passes;                             // total assignment passes
    int cont_balance;                       // inner while-loop condition
    int cont_move;                          // outer while-loop condition
    int cont_final;                         // final balance loop condition
    int final_passes;
    int isel;                               // current buffer of I2 / g64_2 / cdata2
    int iused_sel;                          // buffer the last assignment was computed with
    int gshift;                             // g32 = g * 2^-gshift
    unsigned int done_count;                // last-block-done counter (reset by the last block)
    unsigned int coop_cnt;                  // tiles in the cooperative list (reset before each filter)
    unsigned int big_cnt;                   // supertiles with long candidate lists (same)
    unsigned int multi_cnt;                 // tiles in the assignment's work list (same)
    unsigned int jump_cnt;                  // tiles for a level 1 on their own box (same)
    unsigned int mixed_cnt;                 // tiles the movement takes point by point (reset
                                            //   by the movement's finalize kernel)
    int nonempty;                           // non-empty blocks of the last movement
    double max_imbalance;
    double max_delta;
    double thr;                             // absolute movement threshold
    double W, target, ceil_avg, bound;      // total weight, W/k, ceil(W/k), (1+eps)ceil(W/k)
    double beta;
    unsigned long long maxS_key, maxg_key, maxd_key;  // ordered keys of per-pass maxima
    unsigned long long rechecks;            // FP64 re-decisions
    unsigned long long overflow_tiles;      // tiles whose candidate list overflowed
    unsigned long long wsum_lo, wsum_hi;    // total weight, 128-bit fixed point
    unsigned long long launches;            // kernel executions counted on the device
    unsigned long long t_assign0;           // globaltimer at the start of the last assign launch
    unsigned long long assign_ns;           // sum of assign launch durations (globaltimer)
    unsigned long long assign_cnt;          // assign launches measured
    // sum over tiles and passes of candidates x points (stripe i at i * kStripeStride)
    unsigned long long cand_stripes[kStripes * kStripeStride];
    alignas(128) unsigned int tile_q[kQueues * kQueueStride];  // assignment queues (reset by the filter)
};

// Problem descriptor passed by value to every kernel.
struct Prob {
    long long n;
    long long n_pad;
    long long n_global;         // points of the whole problem (n, unless the call is one shard)
    int d, k, dtype, weighted, assign_f64;
    int ntiles, nsupers;
    int stiles;                 // tiles per supertile (kSuperTiles or kMaxSuperTiles)
    int hyper;                  // 1: supertile lists from hypertile lists (a level above them)
    int nhypers;                // hypertiles of kHyperSupers supertiles
    float4 *hypers;             // per hypertile: 2 float4 box, as the supertiles
    int *hlists;                // per hypertile: its candidate list, kWarpList entries
    int *hlen;                  // per hypertile: list length (-1: longer than kWarpList)
    float *hlam;                // per hypertile: lower bound of the E of every center left out
    int actas;                  // resident CTAs per SM of the assignment (0: the default)
    int qmul;                   // tile order of the assignment: t = pos * qmul mod ntiles
    unsigned long long tile_magic;  // floor((2^64 - 1) / ntiles), for that reduction
    int bits, grid_m;           // Hilbert bits per axis and the scaling exponent b - E
    int Fw, Fx;                 // fixed-point exponents of weights and coordinate sums
    double origin[3];           // frame: (x - origin) * scale
    double scale;
    float R;                    // bound on |frame coordinate|
    double eps;
    int max_iter, max_balance_iter, final_balance_iter, erosion;
    // inputs (device)
    const void *coords;
    const void *weights;
    // bootstrap buffers
    unsigned long long *keys[2];
    unsigned int *perm[2];
    // sorted data
    float *X32;
    double *X64;
    void *Ws;
    int *A;
    unsigned short *A16;        // the block ids as 16 bits (a16: k <= 65535, no bounds)
    int a16;
    float4 *tiles, *supers;
    unsigned long long *tws;    // per tile: sum of its points' fixed-point weights (weighted)
    long long *tsx;             // per tile and axis: sum of the points' fixed-point w x
    unsigned long long *tlo, *thi;  // per tile and axis: ordered keys of the smallest / largest x
    // per-tile candidate records; tiles that need more than the inline candidates
    float4 *trec;
    int *coop;                  // tiles of the cooperative path (ntiles entries)
    int2 *mlist;                // the assignment's work list: (tile, candidate count) of
                                // every tile it evaluates per warp (ntiles entries)
    int *tlist;                 // tiles whose record comes from a level 1 on their own box
                                // (ntiles entries)
    int *bigs;                  // per long-list supertile: index, list length, largest g, smallest
                                // dropped lower bound (bits)
    int *blists;                // their candidate lists, kWarpList entries each
    int nsm;                    // streaming multiprocessors of the device
    // per-center state
    double *C, *Cm, *delta, *S64, *Iin, *I2, *g64_2, *part;
    unsigned long long *Sfix;   // 2 per block, the carry-free form (red_add_*)
    unsigned long long *SXfix;  // 2 per (block, axis), the carry-free form
    unsigned long long *BBlo, *BBhi;  // per (block, axis) ordered keys (input precision)
    float4 *cdata2;             // 2 buffers x 2 float4 per block
    float4 *gdata2;             // 2 buffers x 2 float4 per group of kGroup blocks
    int ngroups;
    float4 *sgdata;             // 2 float4 per supergroup of kSuperGroup groups (current buffer)
    int nsgroups;               // 0: no supergroup level
    // per-point bounds across the passes of a phase (centers fixed, influences change)
    int bounds;                 // 1: skip points whose assignment provably holds
    float *lg;                  // kSkipHist x k: log2 of each center's g at each pass of the phase
    double *cumm;               // kSkipHist: running sum over the passes of (smallest - largest)
                                // log2 g ratio, each lowered by the rounding margin
    float *dm;                  // kSkipHist: for the current pass t, cumm[t] - cumm[t1] rounded down
    float *lq;                  // n_pad: per point, log2 of a lower bound of E_other / E_own at its
                                // last evaluation, plus log2 g of its own center then (rounded down)
    unsigned char *t1;          // n_pad: phase pass of that evaluation
    Ctl *ctl;
};

// Tile at position pos of the permuted tile order: pos * qmul mod ntiles by a Barrett
// reduction with m = floor((2^64 - 1) / ntiles) (integer pipe only).  pos, qmul < ntiles
// < 2^24, so the product is below 2^48 and the quotient estimate floor(prod m / 2^64) is
// low by at most one: one conditional subtraction completes the remainder.
__device__ __forceinline__ int tile_of(const Prob &p, long long pos) {
    const unsigned long long prod = (unsigned long long)pos * (unsigned long long)p.qmul;
    const unsigned long long q = __umul64hi(prod, p.tile_magic);
    unsigned long long r = prod - q * (unsigned long long)p.ntiles;
    if (r >= (unsigned long long)p.ntiles) r -= (unsigned long long)p.ntiles;
    return (int)r;
}

// Selection of one sample round of the random initialization (Section 4.5): the
// curve positions whose round byte rho is <= round, in ascending position order.
// rho has nchunks * kSampleChunk entries (0xff beyond n); counts has nchunks entries.
constexpr int kSampleChunk = 4096;  // positions per CTA of the selection kernels
struct SampleSel {
    const unsigned char *rho;   // per curve position: first sample round holding it
    const unsigned *perm;       // curve position -> input index
    unsigned *counts;           // per chunk: selected positions, then their offsets
    unsigned *sp;               // sample index -> input index
    long long n;                // points of the whole problem
    int nchunks;
    int round;
};

// ------------------------------------------------------------------------------
// Ordered keys: unsigned integers whose order is the numeric order of the value.
// ------------------------------------------------------------------------------
__host__ __device__ inline unsigned long long okey_f64(double v) {
#ifdef __CUDA_ARCH__
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
#else
    unsigned long long b;
    __builtin_memcpy(&b, &v, 8);
#endif
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double okey_to_f64(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double v;
    __builtin_memcpy(&v, &b, 8);
    return v;
#endif
}
__device__ __forceinline__ unsigned okey_f32(float v) {
    unsigned b = __float_as_uint(v);
    return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float okey_to_f32(unsigned k) {
    unsigned b = (k >> 31) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(b);
}

// ------------------------------------------------------------------------------
// Fixed point: trunc(v * 2^F) as a signed 64-bit integer, from the bits of v.
// Valid when |v| * 2^F < 2^62; subnormals map to 0 (contribution below 2^-1022+F).
// ------------------------------------------------------------------------------
__device__ __forceinline__ long long fix_f64(double v, int F) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return 0;
    unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;
    int sh = ex - 1075 + F;
    unsigned long long mag = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
    return (b >> 63) ? -(long long)mag : (long long)mag;
}
__device__ __forceinline__ long long fix_f32(float v, int F) {
    unsigned int b = __float_as_uint(v);
    int ex = (int)((b >> 23) & 0xff);
    if (ex == 0) return 0;
    unsigned long long m = (unsigned long long)((b & 0x7fffffu) | 0x800000u);
    int sh = ex - 150 + F;
    unsigned long long mag = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
    return (b >> 31) ? -(long long)mag : (long long)mag;
}
// trunc(w * x * 2^F) for FP32 w > 0 and x, from the exact 48-bit product of the
// mantissas (integer arithmetic only).
__device__ __forceinline__ long long fix_prod_f32(float w, float x, int F) {
    unsigned bw = __float_as_uint(w), bx = __float_as_uint(x);
    int ew = (int)((bw >> 23) & 0xff), ex = (int)((bx >> 23) & 0xff);
    if (ew == 0 || ex == 0) return 0;
    unsigned long long m = (unsigned long long)((bw & 0x7fffffu) | 0x800000u) *
                           (unsigned long long)((bx & 0x7fffffu) | 0x800000u);
    int sh = ew + ex - 300 + F;
    unsigned long long mag = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
    return (bx >> 31) ? -(long long)mag : (long long)mag;
}

// 128-bit two's-complement accumulation of a signed 64-bit value into (lo, hi).
__device__ __forceinline__ void atomic_add_i128(unsigned long long *lohi, long long v) {
    unsigned long long uv = (unsigned long long)v;
    unsigned long long old = atomicAdd(lohi, uv);
    unsigned long long carry = (old + uv < old) ? 1ull : 0ull;
    unsigned long long hinc = (v < 0 ? ~0ull : 0ull) + carry;
    if (hinc) atomicAdd(lohi + 1, hinc);
}
// A full 128-bit addend (two's complement, low word lo, high word hi).
__device__ __forceinline__ void atomic_add_i128_full(unsigned long long *lohi, unsigned long long lo,
                                                     unsigned long long hi) {
    const unsigned long long old = atomicAdd(lohi, lo);
    const unsigned long long hinc = hi + ((old + lo < old) ? 1ull : 0ull);
    if (hinc) atomicAdd(lohi + 1, hinc);
}
__device__ __forceinline__ void atomic_add_u128(unsigned long long *lohi, unsigned long long v) {
    unsigned long long old = atomicAdd(lohi, v);
    if (old + v < old) atomicAdd(lohi + 1, 1ull);
}
// Value of a 128-bit two's-complement integer times 2^-F, as FP64.
// Exact sums without carries (the loop's block weights and coordinate sums): word 0
// gathers the low 32 bits of every addend, word 1 the rest (an arithmetic shift by 32,
// wrapping in 64 bits), so every update is a plain add whose result is not waited for.
// The sum is word1 * 2^32 + word0 while fewer than 2^32 values are added and the high
// parts total below 2^63 in magnitude.
__device__ __forceinline__ void red_add_s64(unsigned long long *w, long long v) {
    atomicAdd(w, (unsigned long long)v & 0xffffffffull);
    const long long h = v >> 32;
    if (h) atomicAdd(w + 1, (unsigned long long)h);
}
__device__ __forceinline__ void red_add_u64(unsigned long long *w, unsigned long long v) {
    atomicAdd(w, v & 0xffffffffull);
    if (v >> 32) atomicAdd(w + 1, v >> 32);
}
// a 128-bit two's-complement addend (lo, hi) of magnitude below 2^95
__device__ __forceinline__ void red_add_s128(unsigned long long *w, unsigned long long lo, unsigned long long hi) {
    atomicAdd(w, lo & 0xffffffffull);
    const unsigned long long h = (hi << 32) | (lo >> 32);
    if (h) atomicAdd(w + 1, h);
}
// (word0, word1) of the carry-free form -> 128-bit two's complement (lo, hi)
__host__ __device__ __forceinline__ void split_to_i128(unsigned long long w0, unsigned long long w1,
                                                       unsigned long long &lo, unsigned long long &hi) {
    const unsigned long long a = w1 << 32;
    const unsigned long long b = (unsigned long long)((long long)w1 >> 32);
    lo = a + w0;
    hi = b + (lo < a ? 1ull : 0ull);
}
// 128-bit two's complement (lo, hi) of magnitude below 2^95 -> the carry-free form
__host__ __device__ __forceinline__ void i128_to_split(unsigned long long lo, unsigned long long hi,
                                                       unsigned long long &w0, unsigned long long &w1) {
    w0 = lo & 0xffffffffull;
    w1 = (hi << 32) | (lo >> 32);
}
__device__ __forceinline__ double split_to_f64(unsigned long long w0, unsigned long long w1, int F) {
    unsigned long long lo, hi;
    split_to_i128(w0, w1, lo, hi);
    return ldexp((double)(long long)hi * 18446744073709551616.0 + (double)lo, -F);
}
__device__ __forceinline__ double i128_to_f64(unsigned long long lo, unsigned long long hi, int F) {
    double v = (double)(long long)hi * 18446744073709551616.0 + (double)lo;
    return ldexp(v, -F);
}

// ------------------------------------------------------------------------------
// mbarrier + bulk-copy (TMA, non-tensor) helpers.  Waits are bounded: on timeout
// the caller records kErrTimeout and skips its work.
// ------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Device time in nanoseconds (the global timer).
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Returns false if the phase did not complete within limit_ns of device time (a try_wait
// may suspend the thread for a time of the hardware's choosing, so a count of polls alone
// does not bound the wait in seconds) or kSpinLimit polls, whichever comes first.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < kSpinLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}
__device__ __forceinline__ void fence_mbarrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One bulk copy global -> shared, completion signalled on bar (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void count_launch(Ctl *ctl) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctl->launches, 1ull);
}

// Last-block-done: every thread of every CTA calls this once; it returns true (in
// all threads) in the CTA that finished last, to which the global writes of all
// CTAs are then visible.  That CTA resets the counter.
__device__ __forceinline__ bool last_block(Ctl *ctl) {
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(&ctl->done_count, 1u);
        s_last = prev == gridDim.x - 1;
        if (s_last) ctl->done_count = 0u;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

}  // namespace gk
