// gk_noalloc.cu -- gk_move_centers_noalloc: the center-movement step with no memory
// allocation at all, for callers that must not (or cannot) allocate device memory
// while they run: processes whose device memory is owned by their own pool or
// allocator (so that a library cudaMalloc could fail or fragment it), and latency-
// critical loops where a cudaMalloc/cudaFree (which may synchronise the device) is
// not acceptable.
//
// All scratch (per-block 128-bit fixed-point sums, block bounding boxes, the
// coordinate and weight maxima, per-CTA partial sums and counters) lives in one
// file-scope static __device__ array of fixed size, so every GPU that loads this
// library holds it (about 450 KB) until the process exits.  The caller passes its
// inputs and outputs in device memory.  Limits: k <= kNoAllocMaxK (4096), d in {2,3}.
//
// Every call uses the same array and leaves its contents behind; each call clears
// what must start at zero before it accumulates.  Calls whose work overlaps on the
// GPU (on different streams, or from different host threads) race on the array and
// must not be issued.
#include <cuda_runtime.h>
#include <string.h>

#include <atomic>

#include "../../include/gk.h"
#include "gk_common.cuh"

namespace gk {
namespace {

constexpr int kNoAllocMaxK = GK_NOALLOC_MAX_K;
constexpr int kNAThreads = 256;   // accumulation CTAs
constexpr int kNAKThreads = kKThreads;  // per-center CTAs (same as the allocating path)

struct NAScratch {
    unsigned long long xabs_key;  // ordered key of max |x| (FP64 value)
    unsigned long long wmax_key;  // ordered key of max w (FP64 value)
    unsigned long long maxd_key;  // ordered key of the largest movement
    unsigned int done;            // last-block-done counter
    int nonempty;
    int bad;      // bit 0: a block id outside [0, k); bit 1: a non-finite coordinate or a
                  // weight that is not finite and > 0
    int pad;
    double beta;
    double part[(kNoAllocMaxK + kNAKThreads - 1) / kNAKThreads];
    unsigned long long Sfix[2 * kNoAllocMaxK];
    unsigned long long SXfix[2 * 3 * kNoAllocMaxK];
    unsigned long long BBlo[3 * kNoAllocMaxK];
    unsigned long long BBhi[3 * kNoAllocMaxK];
};

// The scratch.  Host code must not use this name as an address: it is a host-side
// stand-in; the device address comes from cudaGetSymbolAddress (na_scratch_ptr).
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NAScratch)];

__device__ __forceinline__ int exp_above(double v) {  // smallest e with |v| < 2^e
    if (v == 0.0) return 0;
    int e;
    frexp(fabs(v), &e);
    return e;
}

// Fixed-point exponents, derived on the device from the maxima (as the allocating
// path derives them on the host).
__device__ __forceinline__ void na_scales(const NAScratch *s, int weighted, int &Fw, int &Fx) {
    double xmax = okey_to_f64(s->xabs_key);
    if (weighted) {
        double wmax = okey_to_f64(s->wmax_key);
        Fw = kFixBits - exp_above(wmax);
        Fx = kFixBits - exp_above(wmax * xmax * (1.0 + 1e-12));
    } else {
        Fw = 0;
        Fx = kFixBits - exp_above(xmax);
    }
}

__global__ void na_clear_kernel(NAScratch *s, int k, int d) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        s->xabs_key = 0ull;
        s->wmax_key = 0ull;
        s->maxd_key = 0ull;
        s->done = 0u;
        s->nonempty = 0;
        s->bad = 0;
        s->beta = 0.0;
    }
    if (i < 2 * k) s->Sfix[i] = 0ull;
    if (i < 2 * k * d) s->SXfix[i] = 0ull;
    if (i < k * d) {
        s->BBlo[i] = ~0ull;
        s->BBhi[i] = 0ull;
    }
}

// Largest |x| and largest w, and a check of the input: every coordinate finite, every
// weight finite and > 0 (as the allocating path requires).  A bad value sets bit 1 of
// s->bad; the accumulation then does nothing and the call reports GK_ERR_INVALID_ARG.
template <typename T>
__global__ void na_range_kernel(const T *x, const T *w, long long n, int d, NAScratch *s) {
    double xm = 0.0, wm = 0.0;
    bool badv = false;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        for (int j = 0; j < d; ++j) {
            const double v = (double)x[i * d + j];
            badv |= !isfinite(v);
            xm = fmax(xm, fabs(v));
        }
        if (w) {
            const double v = (double)w[i];
            badv |= !(v > 0.0 && isfinite(v));
            wm = fmax(wm, v);
        }
    }
    if (__any_sync(0xffffffffu, badv) && (threadIdx.x & 31) == 0) atomicOr(&s->bad, 2);
    for (int off = 16; off; off >>= 1) {
        xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, off));
        wm = fmax(wm, __shfl_xor_sync(0xffffffffu, wm, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&s->xabs_key, okey_f64(xm));
        if (w) atomicMax(&s->wmax_key, okey_f64(wm));
    }
}

template <typename T>
__device__ __forceinline__ unsigned long long na_key(T v);
template <>
__device__ __forceinline__ unsigned long long na_key<float>(float v) { return okey_f32(v); }
template <>
__device__ __forceinline__ unsigned long long na_key<double>(double v) { return okey_f64(v); }

// One point per thread, points in input order; block weights, coordinate sums and
// block boxes are combined over equal-id runs of a warp before the atomics.
template <typename T, int D>
__global__ void __launch_bounds__(kNAThreads) na_accum_kernel(const T *x, const T *w,
                                                              const int *block, long long n, int k,
                                                              NAScratch *s) {
    const int lane = threadIdx.x & 31;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s->bad & 2) return;  // rejected input (the range kernel ran before on this stream)
    int Fw, Fx;
    na_scales(s, w != nullptr, Fw, Fx);
    int b = i < n ? block[i] : -1;
    if (i < n && (unsigned)b >= (unsigned)k) {
        atomicOr(&s->bad, 1);
        b = -1;
    }
    unsigned long long wv = 0ull;
    long long sum[D];
    unsigned long long kmin[D], kmax[D];
    T wt = (T)1;
    if (b >= 0) {
        if (w) {
            wt = w[i];
            wv = (unsigned long long)(sizeof(T) == 8 ? fix_f64((double)wt, Fw) : fix_f32((float)wt, Fw));
        } else {
            wv = 1ull;
        }
    }
#pragma unroll
    for (int j = 0; j < D; ++j) {
        sum[j] = 0;
        kmin[j] = ~0ull;
        kmax[j] = 0ull;
        if (b >= 0) {
            T xv = x[i * D + j];
            if (sizeof(T) == 8)
                sum[j] = w ? fix_f64((double)wt * (double)xv, Fx) : fix_f64((double)xv, Fx);
            else
                sum[j] = w ? fix_prod_f32((float)wt, (float)xv, Fx) : fix_f32((float)xv, Fx);
            kmin[j] = kmax[j] = na_key<T>(xv);
        }
    }
    int prev = __shfl_up_sync(0xffffffffu, b, 1);
    bool head = lane == 0 || b != prev;
    unsigned heads = __ballot_sync(0xffffffffu, head);
    int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        bool take = lane - off >= start;
        unsigned long long y = __shfl_up_sync(0xffffffffu, wv, off);
        if (take) wv += y;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            long long s2 = __shfl_up_sync(0xffffffffu, sum[j], off);
            unsigned long long lo = __shfl_up_sync(0xffffffffu, kmin[j], off);
            unsigned long long hi = __shfl_up_sync(0xffffffffu, kmax[j], off);
            if (take) {
                sum[j] += s2;
                kmin[j] = lo < kmin[j] ? lo : kmin[j];
                kmax[j] = hi > kmax[j] ? hi : kmax[j];
            }
        }
    }
    bool end = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (end && b >= 0) {
        atomic_add_u128(&s->Sfix[2 * b], wv);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            atomic_add_i128(&s->SXfix[2 * (b * D + j)], sum[j]);
            atomicMin(&s->BBlo[b * D + j], kmin[j]);
            atomicMax(&s->BBhi[b * D + j], kmax[j]);
        }
    }
}

// New centers, movement and the mean block diagonal (summed over CTAs in order by
// the last CTA).  An empty block keeps its center.
__global__ void __launch_bounds__(kNAKThreads) na_finalize_kernel(NAScratch *s, int k, int d, int dtype,
                                                                 int weighted, const double *C,
                                                                 double *Cout, double *delta) {
    __shared__ double r_sum[(kNAKThreads + 31) / 32];
    __shared__ int r_cnt[(kNAKThreads + 31) / 32];
    __shared__ double r_max[(kNAKThreads + 31) / 32];
    __shared__ bool s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int Fw, Fx;
    na_scales(s, weighted, Fw, Fx);
    int c = blockIdx.x * blockDim.x + tid;
    double dl = 0.0, sdiag = 0.0;
    int cnt = 0;
    if (c < k) {
        double S = weighted ? i128_to_f64(s->Sfix[2 * c], s->Sfix[2 * c + 1], Fw) : (double)s->Sfix[2 * c];
        double dd = 0.0;
        if (S > 0.0) {
            double diag = 0.0;
            for (int j = 0; j < d; ++j) {
                size_t q = 2 * ((size_t)c * d + j);
                double cm = i128_to_f64(s->SXfix[q], s->SXfix[q + 1], Fx) / S;
                double m = cm - C[c * d + j];
                dd += m * m;
                Cout[c * d + j] = cm;
                unsigned long long khi = s->BBhi[c * d + j], klo = s->BBlo[c * d + j];
                double e = dtype == GK_F64 ? okey_to_f64(khi) - okey_to_f64(klo)
                                           : (double)okey_to_f32((unsigned)khi) - (double)okey_to_f32((unsigned)klo);
                diag += e * e;
            }
            sdiag = sqrt(diag);
            cnt = 1;
        } else {
            for (int j = 0; j < d; ++j) Cout[c * d + j] = C[c * d + j];
        }
        dl = sqrt(dd);
        if (delta) delta[c] = dl;
    }
    double mx = dl;
    for (int off = 16; off; off >>= 1) {
        sdiag += __shfl_xor_sync(0xffffffffu, sdiag, off);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    if (lane == 0) {
        r_sum[warp] = sdiag;
        r_cnt[warp] = cnt;
        r_max[warp] = mx;
    }
    __syncthreads();
    if (tid == 0) {
        double sm = 0.0, m = 0.0;
        int nn = 0;
        for (int w = 0; w < (kNAKThreads + 31) / 32; ++w) {
            sm += r_sum[w];
            nn += r_cnt[w];
            m = fmax(m, r_max[w]);
        }
        s->part[blockIdx.x] = sm;
        if (nn) atomicAdd(&s->nonempty, nn);
        atomicMax(&s->maxd_key, okey_f64(m));
        __threadfence();
        unsigned prev = atomicAdd(&s->done, 1u);
        s_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && tid == 0) {
        __threadfence();
        double sm = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) sm += __ldcg(&s->part[b]);
        int nn = atomicAdd(&s->nonempty, 0);
        s->beta = nn > 0 ? sm / (double)nn : 0.0;
        s->done = 0u;
    }
}

// Device address of the scratch, looked up once per device (set-up on first use).  The
// entries are atomic: host threads may look them up concurrently (they all store the
// same value).
constexpr int kMaxDevices = 64;
std::atomic<void *> g_na_ptr[kMaxDevices];

gk_status na_scratch_ptr(NAScratch **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GK_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return GK_ERR_CUDA;
    void *ptr = g_na_ptr[dev].load(std::memory_order_acquire);
    if (!ptr) {
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return GK_ERR_CUDA;
        }
        g_na_ptr[dev].store(ptr, std::memory_order_release);
    }
    *out = (NAScratch *)ptr;
    return GK_OK;
}

bool on_device(const void *p, int dev) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace
}  // namespace gk

using namespace gk;

extern "C" gk_status gk_move_centers_noalloc(const void *coords, int32_t dtype, const void *weights,
                                             int64_t n, int32_t d, int32_t k, const int32_t *block,
                                             const double *centers, double *centers_out,
                                             double *delta_out, double *beta_out, void *stream) {
    if (!coords || (dtype != GK_F32 && dtype != GK_F64) || (d != 2 && d != 3) || n < 1 ||
        n >= (1ll << 40) || k < 1 || k > kNoAllocMaxK || !block || !centers || !centers_out)
        return GK_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GK_ERR_CUDA;
    }
    size_t es = dtype == GK_F64 ? 8 : 4;
    if (!on_device(coords, dev) || !on_device(block, dev) || !on_device(centers, dev) ||
        !on_device(centers_out, dev) || (weights && !on_device(weights, dev)) ||
        (delta_out && !on_device(delta_out, dev)) || ((uintptr_t)coords % es) ||
        (weights && ((uintptr_t)weights % es)))
        return GK_ERR_INVALID_ARG;
    NAScratch *s = nullptr;
    gk_status st = na_scratch_ptr(&s);
    if (st != GK_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    int clear_n = 2 * k * d > 2 * k ? 2 * k * d : 2 * k;
    na_clear_kernel<<<(clear_n + 255) / 256, 256, 0, cs>>>(s, k, d);
    unsigned agrid = (unsigned)((n + kNAThreads - 1) / kNAThreads);
    int rgrid = (int)((n + 255) / 256);
    if (rgrid > 1216) rgrid = 1216;
    if (dtype == GK_F64) {
        const double *x = (const double *)coords, *w = (const double *)weights;
        na_range_kernel<double><<<rgrid, 256, 0, cs>>>(x, w, n, d, s);
        if (d == 2)
            na_accum_kernel<double, 2><<<agrid, kNAThreads, 0, cs>>>(x, w, block, n, k, s);
        else
            na_accum_kernel<double, 3><<<agrid, kNAThreads, 0, cs>>>(x, w, block, n, k, s);
    } else {
        const float *x = (const float *)coords, *w = (const float *)weights;
        na_range_kernel<float><<<rgrid, 256, 0, cs>>>(x, w, n, d, s);
        if (d == 2)
            na_accum_kernel<float, 2><<<agrid, kNAThreads, 0, cs>>>(x, w, block, n, k, s);
        else
            na_accum_kernel<float, 3><<<agrid, kNAThreads, 0, cs>>>(x, w, block, n, k, s);
    }
    na_finalize_kernel<<<(k + kNAKThreads - 1) / kNAKThreads, kNAKThreads, 0, cs>>>(
        s, k, d, dtype, weights != nullptr, centers, centers_out, delta_out);
    if (cudaGetLastError() != cudaSuccess) return GK_ERR_CUDA;
    int bad = 0;
    double beta = 0.0;
    if (cudaMemcpyAsync(&bad, &s->bad, sizeof(int), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaMemcpyAsync(&beta, &s->beta, sizeof(double), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess) {
        cudaGetLastError();
        return GK_ERR_CUDA;
    }
    if (bad) return GK_ERR_INVALID_ARG;
    if (beta_out) {
        if (on_device(beta_out, dev)) {  // device memory: a copy on the stream
            if (cudaMemcpyAsync(beta_out, &s->beta, sizeof(double), cudaMemcpyDeviceToDevice, cs) !=
                    cudaSuccess ||
                cudaStreamSynchronize(cs) != cudaSuccess) {
                cudaGetLastError();
                return GK_ERR_CUDA;
            }
        } else {
            *beta_out = beta;
        }
    }
    return GK_OK;
}
