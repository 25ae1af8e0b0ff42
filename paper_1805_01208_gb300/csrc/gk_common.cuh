// gk_common.cuh -- shared device-side definitions of the balanced k-means library.
//
// Data layout in device memory (one problem at a time, inside the workspace):
//   X32   d planes of n_pad FP32: curve-sorted coordinates in the assignment frame
//         (FP64 inputs: (x - lo) * 2^-E rounded to FP32, E = grid exponent of the
//         bounding box; FP32 inputs: the raw coordinates).
//   X64   d planes of n_pad FP64: curve-sorted raw coordinates (FP64 inputs only).
//   Ws    n_pad sorted weights in the input dtype (weighted problems only).
//   A     n_pad int32 block ids in sorted order.
//   tiles 2 float4 per tile of kTile points: {origin xyz, radius}, {half extents xyz, -}.
//   cands per tile: count (int32; -1 = overflow, scan all centers) + kCap ids.
//   per center: C (k x d FP64, input units), I, I_used, g64 = 1/I^2, moved centers,
//         delta, 128-bit fixed-point block weights, 128-bit fixed-point coordinate
//         sums, ordered-key bounding boxes, and cdata = 2 float4 per center
//         {frame center hi xyz, g = 1/I^2 as FP32}, {frame center lo xyz, 0}.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gk {

constexpr int kTile = 256;          // points per tile (one CTA of the assign kernel)
constexpr int kCap = 256;           // candidate centers stored per tile
constexpr int kFilterWarps = 8;     // tiles per CTA of the filter kernel
constexpr int kCenterChunk = 1024;  // centers staged in shared memory per bulk copy
constexpr int kFixBits = 55;        // |fixed-point value| < 2^55 per point
constexpr long long kSpinLimit = 1ll << 26;  // bounded waits on mbarriers

// Error codes mirrored from gk.h (device code does not include the C header).
constexpr int kOk = 0;
constexpr int kErrTimeout = 5;

// Device-resident control block: geometry found by the bounding-box kernel,
// loop state and counters.  Written by kernels, read back by the host.
struct Ctl {
    unsigned long long bb_lo[3], bb_hi[3];  // ordered keys of the coordinate extremes
    unsigned long long w_lo, w_hi;          // ordered keys of the weight extremes
    int nonfinite;                          // a coordinate or weight is NaN/Inf
    int nonpositive_w;                      // a weight is <= 0
    int bad_block;                          // a given block id is outside [0, k)
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
    double max_imbalance;
    double max_delta;
    double thr;                             // absolute movement threshold
    double W, target, ceil_avg, bound;      // total weight, W/k, ceil(W/k), (1+eps)ceil(W/k)
    double beta;
    unsigned long long cand_sum;            // sum over points and passes of candidates
    unsigned long long rechecks;            // FP64 re-decisions
    unsigned long long overflow_tiles;      // tiles whose candidate list overflowed
    unsigned long long wsum_lo, wsum_hi;    // total weight, 128-bit fixed point
    unsigned long long launches;            // kernel executions counted on the device
    unsigned long long t_assign0;           // globaltimer at the start of the last assign launch
    unsigned long long assign_ns;           // sum of assign launch durations (globaltimer)
    unsigned long long assign_cnt;          // assign launches measured
};

// Problem descriptor passed by value to every kernel.
struct Prob {
    long long n;
    long long n_pad;
    int d, k, dtype, weighted, assign_f64;
    int ntiles;
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
    float4 *tiles;
    int *cand_cnt;
    int *cand_list;
    // per-center state
    double *C, *I, *Iused, *g64, *Cm, *delta, *S64;
    unsigned long long *Sfix;   // 2 per block (lo, hi)
    unsigned long long *SXfix;  // 2 per (block, axis)
    unsigned long long *BBlo, *BBhi;  // per (block, axis) ordered keys
    float4 *cdata;              // 2 per block
    Ctl *ctl;
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

// 128-bit two's-complement accumulation of a signed 64-bit value into (lo, hi).
__device__ __forceinline__ void atomic_add_i128(unsigned long long *lohi, long long v) {
    unsigned long long uv = (unsigned long long)v;
    unsigned long long old = atomicAdd(lohi, uv);
    unsigned long long carry = (old + uv < old) ? 1ull : 0ull;
    unsigned long long hinc = (v < 0 ? ~0ull : 0ull) + carry;
    if (hinc) atomicAdd(lohi + 1, hinc);
}
__device__ __forceinline__ void atomic_add_u128(unsigned long long *lohi, unsigned long long v) {
    unsigned long long old = atomicAdd(lohi, v);
    if (old + v < old) atomicAdd(lohi + 1, 1ull);
}
// Value of a 128-bit two's-complement integer times 2^-F, as FP64.
__device__ __forceinline__ double i128_to_f64(unsigned long long lo, unsigned long long hi, int F) {
    double v = (double)(long long)hi * 18446744073709551616.0 + (double)lo;
    return ldexp(v, -F);
}

__device__ __forceinline__ unsigned long long shfl_u64(unsigned long long v, int src) {
    return __shfl_sync(0xffffffffu, v, src);
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
// Returns false if the phase did not complete within kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity) {
    for (long long it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
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

}  // namespace gk
