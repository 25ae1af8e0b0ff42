// gk_api.cu -- the C ABI declared in include/gk.h: argument checks, host/device
// pointer staging, the device workspace, and the order of kernel launches for the
// space-filling-curve bootstrap and the balanced k-means loop (Algorithms 1 and 2).
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gk.h"
#include "gk_common.cuh"
#include "gk_internal.h"

namespace gk {
namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// One device workspace per process (grown on demand, reused across calls) plus a
// pinned host mirror of the control block and a cached loop graph.
struct Workspace {
    int device = -1;
    char *dev = nullptr;
    size_t dev_bytes = 0;
    Ctl *host_ctl = nullptr;
    cudaGraphExec_t exec = nullptr;
    Prob graph_key;
    bool has_graph = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t kev[4] = {nullptr, nullptr, nullptr, nullptr};
    // batches: pinned control blocks and the cached graph of the last batch
    Ctl *batch_ctl = nullptr;
    int batch_cap = 0;
    cudaGraphExec_t batch_exec = nullptr;
    std::vector<Prob> batch_key;
    // the cached graph of the last call with random initialization
    cudaGraphExec_t sample_exec = nullptr;
    std::vector<unsigned char> sample_key;
};
Workspace g_ws;

// Where the workspace comes from: cudaMalloc, or the caller's allocator
// (gk_set_allocator).  The memory is returned to whoever provided it.
struct Allocator {
    gk_alloc_fn alloc = nullptr;
    gk_free_fn free = nullptr;
    void *ctx = nullptr;
};
Allocator g_alloc;

bool dev_alloc(char **ptr, size_t bytes) {
    if (g_alloc.alloc) {
        void *q = g_alloc.alloc(bytes, g_alloc.ctx);
        if (q && ((uintptr_t)q % 256) != 0) {  // the layout needs 256-byte alignment
            g_alloc.free(q, bytes, g_alloc.ctx);
            q = nullptr;
        }
        *ptr = (char *)q;
        return q != nullptr;
    }
    if (cudaMalloc((void **)ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return false;
    }
    return true;
}

void dev_free(char *ptr, size_t bytes) {
    if (!ptr) return;
    if (g_alloc.free) {
        cudaDeviceSynchronize();  // no kernel of this library may still use the memory
        g_alloc.free(ptr, bytes, g_alloc.ctx);
    } else {
        cudaFree(ptr);
    }
}

void drop_graph() {
    if (g_ws.exec) cudaGraphExecDestroy(g_ws.exec);
    g_ws.exec = nullptr;
    g_ws.has_graph = false;
    if (g_ws.batch_exec) cudaGraphExecDestroy(g_ws.batch_exec);
    g_ws.batch_exec = nullptr;
    g_ws.batch_key.clear();
    if (g_ws.sample_exec) cudaGraphExecDestroy(g_ws.sample_exec);
    g_ws.sample_exec = nullptr;
    g_ws.sample_key.clear();
}

void release_all() {
    drop_graph();
    dev_free(g_ws.dev, g_ws.dev_bytes);
    if (g_ws.host_ctl) cudaFreeHost(g_ws.host_ctl);
    if (g_ws.batch_ctl) cudaFreeHost(g_ws.batch_ctl);
    for (auto &e : g_ws.ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : g_ws.kev)
        if (e) cudaEventDestroy(e);
    g_ws = Workspace();
}

// The exchange of a sharded call (gk_balanced_kmeans_sharded): the caller's reduction
// over all shards of a host vector of int64.  The global sums of the method (block
// weights, coordinate sums: 128-bit fixed point, so exact in any order) travel as four
// 32-bit limbs per value, each in an int64, so that a plain int64 sum over fewer than 2^31
// shards cannot overflow; ordered keys (bounding boxes: unsigned) travel with their top
// bit flipped, so that a signed minimum or maximum orders them as unsigned.
struct Exchange {
    gk_reduce_fn fn = nullptr;
    void *ctx = nullptr;
    std::vector<int64_t> buf;
    bool on() const { return fn != nullptr; }
    // count 128-bit values as (lo, hi) word pairs, summed over the shards in place
    gk_status sum128(unsigned long long *w, size_t count) {
        buf.resize(4 * count);
        for (size_t i = 0; i < count; ++i)
            for (int j = 0; j < 4; ++j)
                buf[4 * i + j] = (int64_t)((w[2 * i + (j >> 1)] >> (32 * (j & 1))) & 0xffffffffull);
        if (fn(buf.data(), (int64_t)buf.size(), GK_REDUCE_SUM, ctx) != 0) return GK_ERR_CUDA;
        for (size_t i = 0; i < count; ++i) {
            unsigned long long limb[4], carry = 0;
            for (int j = 0; j < 4; ++j) {
                const unsigned long long v = (unsigned long long)buf[4 * i + j] + carry;
                limb[j] = v & 0xffffffffull;
                carry = v >> 32;
            }
            w[2 * i] = limb[0] | (limb[1] << 32);
            w[2 * i + 1] = limb[2] | (limb[3] << 32);
        }
        return GK_OK;
    }
    // count ordered keys, their minimum (or maximum) over the shards in place
    gk_status keys(unsigned long long *k, size_t count, bool max) {
        buf.resize(count);
        for (size_t i = 0; i < count; ++i) buf[i] = (int64_t)(k[i] ^ 0x8000000000000000ull);
        if (fn(buf.data(), (int64_t)count, max ? GK_REDUCE_MAX : GK_REDUCE_MIN, ctx) != 0)
            return GK_ERR_CUDA;
        for (size_t i = 0; i < count; ++i) k[i] = (unsigned long long)buf[i] ^ 0x8000000000000000ull;
        return GK_OK;
    }
    gk_status imax(int *v, size_t count) {
        buf.resize(count);
        for (size_t i = 0; i < count; ++i) buf[i] = v[i];
        if (fn(buf.data(), (int64_t)count, GK_REDUCE_MAX, ctx) != 0) return GK_ERR_CUDA;
        for (size_t i = 0; i < count; ++i) v[i] = (int)buf[i];
        return GK_OK;
    }
};

// Pointer kinds.
enum PtrKind { kHost = 0, kDevice = 1, kForeign = 2 };
PtrKind ptr_kind(const void *p, int device) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return kHost;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        return a.device == device ? kDevice : kForeign;
    return kHost;
}

struct Bufs {
    // staging of host inputs / outputs
    void *coords_stage = nullptr, *weights_stage = nullptr;
    int *block_stage = nullptr;
    long long *perm_stage = nullptr;
    unsigned *hist = nullptr;
};

// Sizes of everything a problem needs; with base != nullptr also assigns pointers.
size_t layout(Prob &p, Bufs &b, char *base, bool sort, bool stage_coords, bool stage_weights,
              bool stage_block, bool perm_out) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *ptr = base ? base + off : nullptr;
        off += align_up(bytes);
        return ptr;
    };
    size_t es = p.dtype == 1 ? 8 : 4;
    long long n = p.n, np = p.n_pad, k = p.k, d = p.d;
    p.ctl = (Ctl *)take(sizeof(Ctl));
    b.coords_stage = stage_coords ? take((size_t)n * d * es) : nullptr;
    b.weights_stage = stage_weights ? take((size_t)n * es) : nullptr;
    if (sort) {
        p.keys[0] = (unsigned long long *)take((size_t)n * 8);
        p.keys[1] = (unsigned long long *)take((size_t)n * 8);
        p.perm[0] = (unsigned *)take((size_t)n * 4);
        p.perm[1] = (unsigned *)take((size_t)n * 4);
        b.hist = (unsigned *)take(radix_hist_entries(n) * 4);
    } else {
        p.keys[0] = p.keys[1] = nullptr;
        p.perm[0] = p.perm[1] = nullptr;
        b.hist = nullptr;
    }
    p.X32 = (float *)take((size_t)d * np * 4);
    p.X64 = p.dtype == 1 ? (double *)take((size_t)d * np * 8) : nullptr;
    p.Ws = p.weighted ? (void *)take((size_t)np * es) : nullptr;
    p.A = (int *)take((size_t)np * 4);
    p.A16 = (unsigned short *)take((size_t)np * 2);
    p.tiles = (float4 *)take((size_t)p.ntiles * 32);
    p.tws = (unsigned long long *)take((size_t)p.ntiles * 8);
    p.tsx = (long long *)take((size_t)p.ntiles * d * 8);
    p.tlo = (unsigned long long *)take((size_t)p.ntiles * d * 8);
    p.thi = (unsigned long long *)take((size_t)p.ntiles * d * 8);
    p.supers = (float4 *)take((size_t)p.nsupers * 32);
    p.trec = (float4 *)take((size_t)p.ntiles * kRecF4 * 16);
    p.coop = (int *)take((size_t)p.ntiles * 4);
    p.mlist = (int2 *)take((size_t)p.ntiles * 8);
    p.tlist = (int *)take((size_t)p.ntiles * 4);
    p.bigs = (int *)take((size_t)p.nsupers * 16);
    p.blists = (int *)take((size_t)p.nsupers * kWarpList * 4);
    {
        const long long nh = (p.nsupers + kHyperSupers - 1) / kHyperSupers;
        p.hypers = (float4 *)take((size_t)nh * 32);
        p.hlists = (int *)take((size_t)nh * kWarpList * 4);
        p.hlen = (int *)take((size_t)nh * 4);
        p.hlam = (float *)take((size_t)nh * 4);
    }
    p.C = (double *)take((size_t)k * d * 8);
    p.Cm = (double *)take((size_t)k * d * 8);
    p.delta = (double *)take((size_t)k * 8);
    p.S64 = (double *)take((size_t)k * 8);
    p.Iin = (double *)take((size_t)k * 8);
    p.I2 = (double *)take((size_t)2 * k * 8);
    p.g64_2 = (double *)take((size_t)2 * k * 8);
    p.part = (double *)take((size_t)(k + kKThreads - 1) / kKThreads * 8);
    p.Sfix = (unsigned long long *)take((size_t)k * 16);
    p.SXfix = (unsigned long long *)take((size_t)k * d * 16);
    p.BBlo = (unsigned long long *)take((size_t)k * d * 8);
    p.BBhi = (unsigned long long *)take((size_t)k * d * 8);
    p.lg = (float *)take((size_t)kSkipHist * k * 4);
    p.cumm = (double *)take((size_t)kSkipHist * 8);
    p.dm = (float *)take((size_t)kSkipHist * 4);
    p.lq = (float *)take((size_t)np * 4);
    p.t1 = (unsigned char *)take((size_t)np);
    p.cdata2 = (float4 *)take((size_t)2 * k * 32);
    p.ngroups = (int)((k + kGroup - 1) / kGroup);
    p.gdata2 = (float4 *)take((size_t)2 * p.ngroups * 32);
    p.nsgroups = p.ngroups > 2 * kSuperGroup ? (p.ngroups + kSuperGroup - 1) / kSuperGroup : 0;
    p.sgdata = (float4 *)take((size_t)(p.nsgroups > 0 ? p.nsgroups : 1) * 32);
    b.block_stage = stage_block ? (int *)take((size_t)n * 4) : nullptr;
    b.perm_stage = perm_out ? (long long *)take((size_t)n * 8) : nullptr;
    return off;
}

// Random initialization (Section 4.5): the round bytes, the selection scratch and
// the point-side arrays of the largest sample (its center-side state is the main
// problem's); the sample's own control block.
struct SampleBufs {
    long long m0 = 0, m_max = 0, nrho = 0;
    int rounds = 0;
    long long *order_stage = nullptr;
    unsigned char *rho_in = nullptr, *rho = nullptr;
    unsigned *counts = nullptr, *sp = nullptr;
    Ctl *ctl = nullptr;
    float *X32 = nullptr;
    double *X64 = nullptr;
    void *Ws = nullptr;
    int *A = nullptr;
    unsigned short *A16 = nullptr;
    float4 *tiles = nullptr, *supers = nullptr, *trec = nullptr;
    unsigned long long *tws = nullptr;
    long long *tsx = nullptr;
    unsigned long long *tlo = nullptr, *thi = nullptr;
    int *coop = nullptr, *bigs = nullptr, *blists = nullptr;
    int2 *mlist = nullptr;
    int *tlist = nullptr;
    float4 *hypers = nullptr;
    int *hlists = nullptr, *hlen = nullptr;
    float *hlam = nullptr;
    float *prho = nullptr;            // per-point bounds of the sample
    unsigned char *pt1 = nullptr;
};

size_t layout_sample(const Prob &p, SampleBufs &sb, char *base, bool stage_order) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *ptr = base ? base + off : nullptr;
        off += align_up(bytes);
        return ptr;
    };
    const size_t es = p.dtype == 1 ? 8 : 4;
    const long long np = (sb.m_max + kTile - 1) / kTile * kTile;
    const long long nt = np / kTile, ns = (nt + kSuperTiles - 1) / kSuperTiles;
    sb.nrho = sample_rho_entries(p.n);
    sb.order_stage = stage_order ? (long long *)take((size_t)p.n * 8) : nullptr;
    sb.rho_in = (unsigned char *)take((size_t)p.n);
    sb.rho = (unsigned char *)take((size_t)sb.nrho);
    sb.counts = (unsigned *)take((size_t)(sb.nrho / kSampleChunk + 1) * 4);
    sb.sp = (unsigned *)take((size_t)sb.m_max * 4);
    sb.ctl = (Ctl *)take(sizeof(Ctl));
    sb.X32 = (float *)take((size_t)p.d * np * 4);
    sb.X64 = p.dtype == 1 ? (double *)take((size_t)p.d * np * 8) : nullptr;
    sb.Ws = p.weighted ? (void *)take((size_t)np * es) : nullptr;
    sb.A = (int *)take((size_t)np * 4);
    sb.A16 = (unsigned short *)take((size_t)np * 2);
    sb.tiles = (float4 *)take((size_t)nt * 32);
    sb.tws = (unsigned long long *)take((size_t)nt * 8);
    sb.tsx = (long long *)take((size_t)nt * p.d * 8);
    sb.tlo = (unsigned long long *)take((size_t)nt * p.d * 8);
    sb.thi = (unsigned long long *)take((size_t)nt * p.d * 8);
    sb.supers = (float4 *)take((size_t)ns * 32);
    sb.trec = (float4 *)take((size_t)nt * kRecF4 * 16);
    sb.coop = (int *)take((size_t)nt * 4);
    sb.mlist = (int2 *)take((size_t)nt * 8);
    sb.tlist = (int *)take((size_t)nt * 4);
    sb.bigs = (int *)take((size_t)ns * 16);
    sb.blists = (int *)take((size_t)ns * kWarpList * 4);
    {
        const long long nh = (ns + kHyperSupers - 1) / kHyperSupers;
        sb.hypers = (float4 *)take((size_t)nh * 32);
        sb.hlists = (int *)take((size_t)nh * kWarpList * 4);
        sb.hlen = (int *)take((size_t)nh * 4);
        sb.hlam = (float *)take((size_t)nh * 4);
    }
    sb.prho = (float *)take((size_t)np * 4);
    sb.pt1 = (unsigned char *)take((size_t)np);
    return off;
}

gk_status ensure_workspace(size_t bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GK_ERR_CUDA;
    if (g_ws.device != dev && g_ws.device != -1) release_all();
    g_ws.device = dev;
    if (!g_ws.host_ctl) {
        if (cudaMallocHost((void **)&g_ws.host_ctl, sizeof(Ctl)) != cudaSuccess) {
            cudaGetLastError();
            return GK_ERR_OOM;
        }
        for (auto &e : g_ws.ev)
            if (cudaEventCreate(&e) != cudaSuccess) return GK_ERR_CUDA;
        for (auto &e : g_ws.kev)
            if (cudaEventCreate(&e) != cudaSuccess) return GK_ERR_CUDA;
    }
    if (g_ws.dev_bytes >= bytes) return GK_OK;
    drop_graph();
    dev_free(g_ws.dev, g_ws.dev_bytes);
    g_ws.dev = nullptr;
    g_ws.dev_bytes = 0;
    size_t want = bytes + bytes / 8;
    if (!dev_alloc(&g_ws.dev, want)) {
        if (!dev_alloc(&g_ws.dev, bytes)) return GK_ERR_OOM;
        want = bytes;
    }
    g_ws.dev_bytes = want;
    return GK_OK;
}

#define GK_CUDA(x)                        \
    do {                                  \
        if ((x) != cudaSuccess) {         \
            cudaGetLastError();           \
            return GK_ERR_CUDA;           \
        }                                 \
    } while (0)

long long gcd_ll(long long a, long long b) {
    while (b) {
        long long t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Multiplier of the assignment's tile order (see assign_kernel): coprime to ntiles,
// near 0.618 ntiles, so that consecutive positions land far apart on the curve.
int tile_order_multiplier(int ntiles) {
    if (ntiles <= 2) return 1;
    long long m = (long long)(0.6180339887498949 * ntiles);
    if (m < 1) m = 1;
    while (gcd_ll(m, ntiles) != 1) ++m;
    return (int)(m % ntiles == 0 ? 1 : m);
}

int exponent_above(double v) {  // smallest e with |v| < 2^e (v finite)
    if (v == 0.0) return 0;
    int e;
    frexp(fabs(v), &e);
    return e;
}

int grid_exponent(double s) {  // smallest E with 2^E >= s
    if (!(s > 0.0)) return 0;
    int e;
    double f = frexp(s, &e);
    return f == 0.5 ? e - 1 : e;
}

void options_or_default(const gk_options *opt, gk_options *o) {
    if (opt)
        *o = *opt;
    else
        gk_default_options(o);
}

gk_status check_common(const void *coords, int32_t dtype, int64_t n, int32_t d) {
    if (!coords || (dtype != GK_F32 && dtype != GK_F64) || (d != 2 && d != 3) || n < 1 ||
        n >= (1ll << 32) - 1024)
        return GK_ERR_INVALID_ARG;
    return GK_OK;
}

// Launch-shape tuner cache: the shapes measured fastest per kind of problem.
// d, dtype, f64, w, bounds, log2 n, log2 k, and the shapes the caller fixed (0: free):
// supertile tiles, hypertiles, CTAs per SM
using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int, int>;
struct TuneChoice {
    int stiles, hyper, actas;
};
std::map<TuneKey, TuneChoice> g_tune;
std::mutex g_tune_mu;

int ilog2(long long v) {
    int e = 0;
    while (v > 1) {
        v >>= 1;
        ++e;
    }
    return e;
}

// The loop's sums are kept in the carry-free form (two words per value, see
// red_add_s64); the exchange between shards sums them as 128-bit integers.
static void splits_to_i128(std::vector<unsigned long long> &v) {
    for (size_t i = 0; i + 1 < v.size(); i += 2) split_to_i128(v[i], v[i + 1], v[i], v[i + 1]);
}
static void i128s_to_split(std::vector<unsigned long long> &v) {
    for (size_t i = 0; i + 1 < v.size(); i += 2) i128_to_split(v[i], v[i + 1], v[i], v[i + 1]);
}

// State shared by the entry points of one call.
struct Call {
    cudaStream_t s;
    Prob p;
    Bufs b;
    bool coords_host, weights_host;
    gk_status setup(const void *weights, int64_t n, int32_t d, int32_t k, int32_t dtype) {
        memset(&p, 0, sizeof(p));
        p.n = n;
        p.n_global = n;
        p.n_pad = (n + kTile - 1) / kTile * kTile;
        p.d = d;
        p.k = k;
        p.dtype = dtype;
        p.weighted = weights != nullptr;
        p.ntiles = (int)(p.n_pad / kTile);
        p.stiles = kSuperTiles;
        p.nsupers = (p.ntiles + kSuperTiles - 1) / kSuperTiles;
        p.nhypers = (p.nsupers + kHyperSupers - 1) / kHyperSupers;
        p.qmul = tile_order_multiplier(p.ntiles);
        p.tile_magic = ~0ull / (unsigned long long)p.ntiles;
        p.bits = d == 2 ? 32 : 21;
        int dev = 0;
        GK_CUDA(cudaGetDevice(&dev));
        GK_CUDA(cudaDeviceGetAttribute(&p.nsm, cudaDevAttrMultiProcessorCount, dev));
        return GK_OK;
    }
    // Control block (from the pinned host slot hc) and accumulators of the problem.
    gk_status upload_state(Ctl *hc) {
        Ctl c0;
        memset(&c0, 0, sizeof(c0));
        for (int j = 0; j < 3; ++j) {
            c0.bb_lo[j] = ~0ull;
            c0.bb_hi[j] = 0ull;
        }
        c0.w_lo = ~0ull;
        c0.w_hi = 0ull;
        *hc = c0;
        GK_CUDA(cudaMemcpyAsync(p.ctl, hc, sizeof(Ctl), cudaMemcpyHostToDevice, s));
        GK_CUDA(cudaMemsetAsync(p.Sfix, 0, (size_t)p.k * 16, s));
        GK_CUDA(cudaMemsetAsync(p.SXfix, 0, (size_t)p.k * p.d * 16, s));
        GK_CUDA(cudaMemsetAsync(p.BBlo, 0xff, (size_t)p.k * p.d * 8, s));
        GK_CUDA(cudaMemsetAsync(p.BBhi, 0, (size_t)p.k * p.d * 8, s));
        return GK_OK;
    }
    size_t main_bytes = 0;  // the problem's part of the workspace; `extra` bytes follow it
    gk_status init(const void *coords, int32_t dtype, const void *weights, int64_t n, int32_t d,
                   int32_t k, bool sort, bool block_host, bool perm_out,
                   SampleBufs *sb = nullptr, bool stage_order = false) {
        gk_status st0 = setup(weights, n, d, k, dtype);
        if (st0 != GK_OK) return st0;
        int dev = 0;
        GK_CUDA(cudaGetDevice(&dev));
        PtrKind kc = ptr_kind(coords, dev);
        PtrKind kw = weights ? ptr_kind(weights, dev) : kHost;
        if (kc == kForeign || kw == kForeign) return GK_ERR_INVALID_ARG;
        size_t es = dtype == GK_F64 ? 8 : 4;
        if (kc == kDevice && ((uintptr_t)coords % es)) return GK_ERR_INVALID_ARG;
        if (weights && kw == kDevice && ((uintptr_t)weights % es)) return GK_ERR_INVALID_ARG;
        coords_host = kc == kHost;
        weights_host = weights && kw == kHost;
        main_bytes = align_up(layout(p, b, nullptr, sort, coords_host, weights_host, block_host, perm_out));
        size_t need = main_bytes + (sb ? layout_sample(p, *sb, nullptr, stage_order) : 0);
        gk_status st = ensure_workspace(need);
        if (st != GK_OK) return st;
        layout(p, b, g_ws.dev, sort, coords_host, weights_host, block_host, perm_out);
        if (sb) layout_sample(p, *sb, g_ws.dev + main_bytes, stage_order);
        p.coords = coords_host ? b.coords_stage : coords;
        p.weights = weights ? (weights_host ? b.weights_stage : weights) : nullptr;
        GK_CUDA(cudaEventRecord(g_ws.ev[0], s));
        if (coords_host)
            GK_CUDA(cudaMemcpyAsync(b.coords_stage, coords, (size_t)n * d * es,
                                    cudaMemcpyHostToDevice, s));
        if (weights_host)
            GK_CUDA(cudaMemcpyAsync(b.weights_stage, weights, (size_t)n * es,
                                    cudaMemcpyHostToDevice, s));
        return upload_state(g_ws.host_ctl);
    }
    gk_status read_ctl() {
        GK_CUDA(cudaMemcpyAsync(g_ws.host_ctl, p.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaStreamSynchronize(s));
        return GK_OK;
    }
    // Bounding box -> frame, grid and fixed-point parameters (one readback).  A shard
    // takes the box, weight range and input flags of all shards.
    gk_status geometry(double delta_threshold) {
        GK_CUDA(launch_bbox(p, s));
        gk_status st = read_ctl();
        if (st != GK_OK) return st;
        if (ex && ex->on()) {
            Ctl &c = *g_ws.host_ctl;
            int flags[2] = {c.nonfinite, c.nonpositive_w};
            if ((st = ex->keys(c.bb_lo, 3, false)) != GK_OK || (st = ex->keys(c.bb_hi, 3, true)) != GK_OK ||
                (st = ex->keys(&c.w_lo, 1, false)) != GK_OK || (st = ex->keys(&c.w_hi, 1, true)) != GK_OK ||
                (st = ex->imax(flags, 2)) != GK_OK)
                return st;
            c.nonfinite = flags[0];
            c.nonpositive_w = flags[1];
        }
        return frame(*g_ws.host_ctl, delta_threshold);
    }
    // A shard: the total weight of all shards (after the gather formed the local one).
    gk_status exchange_weight() {
        if (!(ex && ex->on()) || !p.weighted) return GK_OK;
        gk_status st = read_ctl();
        if (st != GK_OK) return st;
        unsigned long long w[2] = {g_ws.host_ctl->wsum_lo, g_ws.host_ctl->wsum_hi};
        if ((st = ex->sum128(w, 1)) != GK_OK) return st;
        GK_CUDA(cudaMemcpy(&p.ctl->wsum_lo, w, 16, cudaMemcpyHostToDevice));
        return GK_OK;
    }
    // A shard: the block weights of the pass summed over all shards.
    gk_status exchange_pass() {
        if (!(ex && ex->on())) return GK_OK;
        std::vector<unsigned long long> w(2 * (size_t)p.k);
        GK_CUDA(cudaMemcpyAsync(w.data(), p.Sfix, w.size() * 8, cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaStreamSynchronize(s));
        splits_to_i128(w);
        gk_status st = ex->sum128(w.data(), p.k);
        if (st != GK_OK) return st;
        i128s_to_split(w);
        GK_CUDA(cudaMemcpyAsync(p.Sfix, w.data(), w.size() * 8, cudaMemcpyHostToDevice, s));
        GK_CUDA(cudaStreamSynchronize(s));
        return GK_OK;
    }
    // A shard: the coordinate sums and block boxes of the movement over all shards.
    gk_status exchange_move() {
        if (!(ex && ex->on())) return GK_OK;
        const size_t kd = (size_t)p.k * p.d;
        std::vector<unsigned long long> sx(2 * kd), lo(kd), hi(kd);
        GK_CUDA(cudaMemcpyAsync(sx.data(), p.SXfix, sx.size() * 8, cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaMemcpyAsync(lo.data(), p.BBlo, kd * 8, cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaMemcpyAsync(hi.data(), p.BBhi, kd * 8, cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaStreamSynchronize(s));
        gk_status st;
        splits_to_i128(sx);
        if ((st = ex->sum128(sx.data(), kd)) != GK_OK || (st = ex->keys(lo.data(), kd, false)) != GK_OK ||
            (st = ex->keys(hi.data(), kd, true)) != GK_OK)
            return st;
        i128s_to_split(sx);
        GK_CUDA(cudaMemcpyAsync(p.SXfix, sx.data(), sx.size() * 8, cudaMemcpyHostToDevice, s));
        GK_CUDA(cudaMemcpyAsync(p.BBlo, lo.data(), kd * 8, cudaMemcpyHostToDevice, s));
        GK_CUDA(cudaMemcpyAsync(p.BBhi, hi.data(), kd * 8, cudaMemcpyHostToDevice, s));
        GK_CUDA(cudaStreamSynchronize(s));
        return GK_OK;
    }
    Exchange *ex = nullptr;
    float tune_ms = 0.f;

    void apply_shape(int stiles, int hyper, int actas) {
        p.stiles = stiles;
        p.hyper = hyper;
        p.nsupers = (p.ntiles + stiles - 1) / stiles;
        p.nhypers = (p.nsupers + kHyperSupers - 1) / kHyperSupers;
        p.actas = actas;
    }
    // The launch shapes (gk_options supertile_tiles, assign_ctas_per_sm; 0: tuned).  Runs
    // after the bootstrap: measures the first pass's filter and assignment for every
    // candidate shape, keeps the fastest and restores the state (control block, block
    // weights; the stored block ids and tile markers the trials wrote are those of the
    // first pass, consistent with each other).
    gk_status tune(const gk_options &o) {
        std::vector<int> sts, hys, cts;
        if (o.supertile_tiles)
            sts.push_back(o.supertile_tiles);
        else
            sts = {kSuperTiles, kMaxSuperTiles};
        if (o.hypertiles)
            hys.push_back(o.hypertiles == 2 ? 1 : 0);
        else
            hys = {0, 1};
        const int mc = assign_max_ctas(p);
        if (o.assign_ctas_per_sm)
            cts.push_back(o.assign_ctas_per_sm < mc ? o.assign_ctas_per_sm : mc);
        else
            for (int c = mc; c >= 1 && c >= mc - 1; --c) cts.push_back(c);
        TuneChoice best{sts[0], hys[0], cts[0]};
        const size_t ncand = sts.size() * hys.size() * cts.size();
        const TuneKey key{p.d, p.dtype, p.assign_f64, p.weighted, p.bounds, ilog2(p.n), ilog2(p.k),
                          o.supertile_tiles, o.hypertiles, o.assign_ctas_per_sm};
        bool cached = false;
        if (ncand > 1) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) {
                best = it->second;
                cached = true;
            }
        }
        if (ncand > 1 && !cached) {
            gk_status st = read_ctl();
            if (st != GK_OK) return st;
            const Ctl saved = *g_ws.host_ctl;
            GK_CUDA(launch_init(p, s));
            float best_ms = INFINITY;
            cudaEvent_t e0 = g_ws.kev[0], e1 = g_ws.kev[1];
            for (int stl : sts) {
                apply_shape(stl, 0, cts[0]);
                GK_CUDA(launch_super_boxes(p, s));
                for (int hy : hys)
                for (int c : cts) {
                    apply_shape(stl, hy, c);
                    float ms_min = INFINITY;
                    for (int rep = 0; rep < 4; ++rep) {
                        GK_CUDA(cudaEventRecord(e0, s));
                        GK_CUDA(launch_filter(p, s));
                        GK_CUDA(launch_assign(p, s));
                        GK_CUDA(cudaEventRecord(e1, s));
                        GK_CUDA(cudaMemsetAsync(p.Sfix, 0, (size_t)p.k * 16, s));
                        GK_CUDA(cudaMemsetAsync(&p.ctl->coop_cnt, 0, 4 * sizeof(unsigned), s));
                        GK_CUDA(cudaEventSynchronize(e1));
                        float ms = 0.f;
                        GK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                        tune_ms += ms;
                        if (rep > 0 && ms < ms_min) ms_min = ms;  // the first run warms up
                    }
                    // the hypertile level is taken within 2 %: the trial is the first pass
                    // (initial centers, all influences 1), where the level saves less than in
                    // the passes after the centers have spread; without the bias the choice
                    // flipped between runs at 1e9 points
                    const float score = hy ? ms_min * 0.98f : ms_min;
                    if (score < best_ms) {
                        best_ms = score;
                        best = {stl, hy, c};
                    }
                }
            }
            GK_CUDA(cudaMemcpyAsync(p.ctl, &saved, sizeof(Ctl), cudaMemcpyHostToDevice, s));
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[key] = best;
        }
        apply_shape(best.stiles, best.hyper, best.actas);
        GK_CUDA(launch_super_boxes(p, s));
        return GK_OK;
    }
    gk_status frame(const Ctl &c, double delta_threshold) {
        if (c.nonfinite || c.nonpositive_w) return GK_ERR_INVALID_ARG;
        double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, ext = 0.0, xmax = 0.0;
        for (int j = 0; j < p.d; ++j) {
            lo[j] = okey_to_f64(c.bb_lo[j]);
            hi[j] = okey_to_f64(c.bb_hi[j]);
            ext = fmax(ext, hi[j] - lo[j]);
            xmax = fmax(xmax, fmax(fabs(lo[j]), fabs(hi[j])));
        }
        int E = grid_exponent(ext);
        p.grid_m = p.bits - E;
        for (int j = 0; j < 3; ++j) p.origin[j] = lo[j];
        if (p.dtype == GK_F64) {
            p.scale = ldexp(1.0, -E);
            p.R = 1.0f;
        } else {  // FP32 inputs: the assignment frame is the raw coordinates
            p.scale = 1.0;
            for (int j = 0; j < 3; ++j) p.origin[j] = 0.0;
            p.R = (float)xmax * (1.0f + 1e-6f);
        }
        // keep the quantisation origin (lo) separately: keys use lo in both cases
        for (int j = 0; j < 3; ++j) key_origin[j] = lo[j];
        double wmax = p.weighted ? okey_to_f64(c.w_hi) : 1.0;
        p.Fw = p.weighted ? kFixBits - exponent_above(wmax) : 0;
        p.Fx = kFixBits - exponent_above(p.weighted ? wmax * xmax * (1.0 + 1e-12) : xmax);
        extent = ext;
        thr = delta_threshold >= 0.0 ? delta_threshold : 1e-4 * ext;
        return GK_OK;
    }
    double key_origin[3] = {0, 0, 0};
    double extent = 0.0, thr = 0.0;
    double t_filter = 0, t_assign = 0, t_balance = 0, t_move = 0;
    long long n_pass = 0, n_move = 0;

    Prob key_prob() const {  // frame for the Hilbert quantisation: origin = lo
        Prob q = p;
        for (int j = 0; j < 3; ++j) q.origin[j] = key_origin[j];
        return q;
    }
};

void fill_result(gk_result *r, const Ctl &c, gk_status st, double t_boot, double t_loop,
                 double t_tot, long long n, const Call &cl) {
    if (!r) return;
    memset(r, 0, sizeof(*r));
    r->status = st;
    r->iterations = c.iter + c.sample_iters;
    r->balance_passes = c.passes + c.sample_passes;
    r->converged = c.converged;
    r->balanced = c.balanced;
    r->max_imbalance = c.max_imbalance;
    r->max_delta = c.max_delta;
    r->delta_threshold = c.thr;
    unsigned long long cand = 0;
    for (int i = 0; i < kStripes; ++i) cand += c.cand_stripes[i * kStripeStride];
    r->avg_candidates = c.passes > 0 ? (double)cand / ((double)c.passes * (double)n) : 0.0;
    r->rechecked_points = (int64_t)c.rechecks;
    r->kernel_launches = (int64_t)c.launches;
    r->time_bootstrap_ms = t_boot;
    r->time_kmeans_ms = t_loop;
    r->time_total_ms = t_tot;
    r->time_filter_ms = cl.t_filter;
    r->time_assign_ms = cl.t_assign;
    r->time_balance_ms = cl.t_balance;
    r->time_move_ms = cl.t_move;
    r->filter_launches = cl.n_pass;
    r->assign_launches = cl.n_pass;
    r->balance_launches = cl.n_pass;
    r->move_launches = cl.n_move;
    r->assign_live_ms = (double)c.assign_ns * 1e-6;
    r->assign_live_launches = (int64_t)c.assign_cnt;
    r->evaluated_points = (int64_t)c.evaluated;
    r->supertile_tiles = cl.p.stiles;
    r->assign_ctas_per_sm = assign_ctas(cl.p);
    r->hypertiles = cl.p.hyper ? 2 : 1;
    r->tune_ms = cl.tune_ms;
}

gk_status copy_out(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (!dst) return GK_OK;
    GK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
    return GK_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

// Runs the k-means loop on the prepared problem (C, I in the workspace).
gk_status run_loop(Call &cl, const gk_options &o) {
    Prob &p = cl.p;
    cudaStream_t s = cl.s;
    const bool sharded = cl.ex && cl.ex->on();  // host-driven: the exchanges sit between kernels
    if (o.use_graph && !sharded) {
        Prob key = p;
        key.coords = nullptr;
        key.weights = nullptr;
        if (!(g_ws.has_graph && memcmp(&key, &g_ws.graph_key, sizeof(Prob)) == 0)) {
            drop_graph();
            cudaGraphExec_t ex = nullptr;
            if (build_loop_graph(&key, 1, &ex) != cudaSuccess) {
                cudaGetLastError();
                return GK_ERR_CUDA;
            }
            g_ws.exec = ex;
            g_ws.graph_key = key;
            g_ws.has_graph = true;
        }
        GK_CUDA(cudaGraphLaunch(g_ws.exec, s));
        return GK_OK;
    }
    // host-driven loop: one readback of the loop condition per pass; with
    // o.timing, CUDA events around every kernel (read after that readback)
    cudaEvent_t *ev = g_ws.kev;
    auto pass = [&](int mode) -> gk_status {
        if (o.timing) GK_CUDA(cudaEventRecord(ev[0], s));
        GK_CUDA(launch_filter(p, s));
        if (o.timing) GK_CUDA(cudaEventRecord(ev[1], s));
        GK_CUDA(launch_assign(p, s));
        if (o.timing) GK_CUDA(cudaEventRecord(ev[2], s));
        if (sharded) {
            gk_status xs = cl.exchange_pass();
            if (xs != GK_OK) return xs;
        }
        GK_CUDA(launch_balance(p, mode, s));
        if (o.timing) GK_CUDA(cudaEventRecord(ev[3], s));
        gk_status st = cl.read_ctl();
        if (st == GK_OK && o.timing) {
            cl.t_filter += elapsed(ev[0], ev[1]);
            cl.t_assign += elapsed(ev[1], ev[2]);
            cl.t_balance += elapsed(ev[2], ev[3]);
            cl.n_pass += 1;
        }
        return st;
    };
    GK_CUDA(launch_init(p, s));
    for (int it = 0; it < o.max_iter; ++it) {
        for (int bp = 0; bp < o.max_balance_iter; ++bp) {
            gk_status st = pass(0);
            if (st != GK_OK) return st;
            if (!g_ws.host_ctl->cont_balance) break;
        }
        if (o.timing) GK_CUDA(cudaEventRecord(ev[0], s));
        if (sharded) {
            GK_CUDA(launch_centroid(p, s));
            gk_status xs = cl.exchange_move();
            if (xs != GK_OK) return xs;
            GK_CUDA(launch_move_finish(p, 0, s));
        } else {
            GK_CUDA(launch_move(p, 0, s));
        }
        if (o.timing) GK_CUDA(cudaEventRecord(ev[1], s));
        gk_status st = cl.read_ctl();
        if (st != GK_OK) return st;
        if (o.timing) {
            cl.t_move += elapsed(ev[0], ev[1]);
            cl.n_move += 1;
        }
        if (!g_ws.host_ctl->cont_move) break;
    }
    GK_CUDA(launch_final_begin(p, s));
    gk_status st = cl.read_ctl();
    if (st != GK_OK) return st;
    while (g_ws.host_ctl->cont_final) {
        st = pass(1);
        if (st != GK_OK) return st;
    }
    return GK_OK;
}

// Random initialization: the Prob of sample round r (m points) and its selection.
Prob sample_prob(const Prob &p, const SampleBufs &sb, long long m) {
    Prob ps = p;
    ps.n = m;
    ps.n_global = m;
    ps.n_pad = (m + kTile - 1) / kTile * kTile;
    ps.ntiles = (int)(ps.n_pad / kTile);
    ps.nsupers = (ps.ntiles + ps.stiles - 1) / ps.stiles;
    ps.qmul = tile_order_multiplier(ps.ntiles);
    ps.tile_magic = ~0ull / (unsigned long long)ps.ntiles;
    ps.keys[0] = ps.keys[1] = nullptr;
    ps.perm[0] = ps.perm[1] = nullptr;
    ps.X32 = sb.X32;
    ps.X64 = sb.X64;
    ps.Ws = sb.Ws;
    ps.A = sb.A;
    ps.A16 = sb.A16;
    ps.tiles = sb.tiles;
    ps.tws = sb.tws;
    ps.tsx = sb.tsx;
    ps.tlo = sb.tlo;
    ps.thi = sb.thi;
    ps.supers = sb.supers;
    ps.trec = sb.trec;
    ps.coop = sb.coop;
    ps.mlist = sb.mlist;
    ps.tlist = sb.tlist;
    ps.bigs = sb.bigs;
    ps.blists = sb.blists;
    ps.hypers = sb.hypers;
    ps.hlists = sb.hlists;
    ps.hlen = sb.hlen;
    ps.hlam = sb.hlam;
    ps.nhypers = (ps.nsupers + kHyperSupers - 1) / kHyperSupers;
    ps.lq = sb.prho;
    ps.t1 = sb.pt1;
    ps.ctl = sb.ctl;
    ps.max_iter = 1;
    ps.final_balance_iter = 0;
    return ps;
}

// Runs the sample rounds and then the main loop (p.max_iter already reduced by the
// rounds): one cached graph, or host-driven with a readback per pass.
gk_status run_sampled(Call &cl, const gk_options &o, const SampleBufs &sb, const unsigned *perm) {
    Prob &p = cl.p;
    cudaStream_t s = cl.s;
    const int R = sb.rounds;
    std::vector<Prob> ps(R);
    std::vector<SampleSel> sel(R);
    for (int r = 0; r < R; ++r) {
        ps[r] = sample_prob(p, sb, sb.m0 << r);
        memset(&sel[r], 0, sizeof(SampleSel));
        sel[r].rho = sb.rho;
        sel[r].perm = perm;
        sel[r].counts = sb.counts;
        sel[r].sp = sb.sp;
        sel[r].n = p.n;
        sel[r].nchunks = (int)(sb.nrho / kSampleChunk);
        sel[r].round = r;
    }
    if (o.use_graph) {
        std::vector<unsigned char> key(sizeof(Prob) * (1 + R) + sizeof(SampleSel) * R);
        memcpy(key.data(), &p, sizeof(Prob));
        if (R) {
            memcpy(key.data() + sizeof(Prob), ps.data(), sizeof(Prob) * R);
            memcpy(key.data() + sizeof(Prob) * (1 + R), sel.data(), sizeof(SampleSel) * R);
        }
        if (!(g_ws.sample_exec && g_ws.sample_key == key)) {
            if (g_ws.sample_exec) cudaGraphExecDestroy(g_ws.sample_exec);
            g_ws.sample_exec = nullptr;
            g_ws.sample_key.clear();
            cudaGraphExec_t ex = nullptr;
            if (build_sampled_graph(p, ps.data(), sel.data(), R, &ex) != cudaSuccess) {
                cudaGetLastError();
                return GK_ERR_CUDA;
            }
            g_ws.sample_exec = ex;
            g_ws.sample_key = key;
        }
        GK_CUDA(cudaGraphLaunch(g_ws.sample_exec, s));
        return GK_OK;
    }
    Ctl *hc = g_ws.host_ctl;
    for (int r = 0; r < R; ++r) {
        GK_CUDA(launch_sample_select(ps[r], sel[r], s));
        GK_CUDA(launch_init(ps[r], s));
        for (int bp = 0; bp < o.max_balance_iter; ++bp) {
            GK_CUDA(launch_pass(ps[r], 0, s));
            GK_CUDA(cudaMemcpyAsync(hc, ps[r].ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            GK_CUDA(cudaStreamSynchronize(s));
            if (!hc->cont_balance) break;
        }
        GK_CUDA(launch_move(ps[r], 3, s));
        GK_CUDA(launch_sample_export(ps[r], p.ctl, s));
    }
    gk_options rest = o;
    rest.max_iter = p.max_iter;
    return run_loop(cl, rest);
}

gk_status check_options(const gk_options &o) {
    if (o.max_iter < 1 || o.max_balance_iter < 1 || o.final_balance_iter < 0 ||
        (o.assign_dtype != GK_F32 && o.assign_dtype != GK_F64) || !(o.delta_threshold == o.delta_threshold))
        return GK_ERR_INVALID_ARG;
    if (o.bounds != 0 && o.bounds != 1) return GK_ERR_INVALID_ARG;
    if (o.supertile_tiles != 0 && o.supertile_tiles != kSuperTiles && o.supertile_tiles != kMaxSuperTiles)
        return GK_ERR_INVALID_ARG;
    if (o.assign_ctas_per_sm < 0 || o.assign_ctas_per_sm > 64) return GK_ERR_INVALID_ARG;
    if (o.hypertiles < 0 || o.hypertiles > 2) return GK_ERR_INVALID_ARG;
    if (o.reserved[0] != 0) return GK_ERR_INVALID_ARG;
    return GK_OK;
}

// Shared body of gk_partition (sort = true) and gk_balanced_kmeans (sort = false).
// order != nullptr: random initialization (Section 4.5) with that order and first
// sample size sample0 (<= 0: 100 k).
gk_status kmeans_common(const void *coords, int32_t dtype, const void *weights, int64_t n,
                        int32_t d, int32_t k, double eps, const gk_options *opt, bool sort,
                        double *centers_io, double *influence_io, int32_t *block_out,
                        double *centers_out, double *influence_out, gk_result *result,
                        void *stream, const int64_t *order = nullptr, int64_t sample0 = 0,
                        Exchange *ex = nullptr, int64_t n_global = 0) {
    gk_status st = check_common(coords, dtype, n, d);
    if (st != GK_OK) return st;
    const int64_t n_all = ex ? n_global : n;  // a shard: k is bounded by all shards' points
    if (k < 1 || k > n_all || !(eps >= 0.0) || !block_out) return GK_ERR_INVALID_ARG;
    if (!sort && (!centers_io || !influence_io)) return GK_ERR_INVALID_ARG;
    gk_options o;
    options_or_default(opt, &o);
    if ((st = check_options(o)) != GK_OK) return st;
    int dev = 0;
    GK_CUDA(cudaGetDevice(&dev));
    if (ptr_kind(block_out, dev) == kForeign) return GK_ERR_INVALID_ARG;
    bool block_host = ptr_kind(block_out, dev) == kHost;
    SampleBufs sb;
    bool order_host = false;
    if (order) {
        PtrKind ko = ptr_kind(order, dev);
        if (ko == kForeign || (ko == kDevice && ((uintptr_t)order % 8))) return GK_ERR_INVALID_ARG;
        order_host = ko == kHost;
        // first sample: 100 points per block (the paper's 100 per process, k = p), at
        // least k, at most n; rounds until the sample would reach n, at most max_iter - 1
        sb.m0 = sample0 > 0 ? sample0 : 100ll * k;
        if (sb.m0 < k) sb.m0 = k;
        if (sb.m0 > n) sb.m0 = n;
        while (sb.rounds < 62 && (sb.m0 << sb.rounds) < n) ++sb.rounds;
        if (sb.rounds > o.max_iter - 1) sb.rounds = o.max_iter - 1;
        sb.m_max = sb.rounds > 0 ? sb.m0 << (sb.rounds - 1) : 1;
    }
    Call cl;
    cl.s = (cudaStream_t)stream;
    cl.ex = ex;
    st = cl.init(coords, dtype, weights, n, d, k, sort, block_host, false, order ? &sb : nullptr,
                 order_host);
    if (st != GK_OK) return st;
    Prob &p = cl.p;
    p.n_global = n_all;
    p.eps = eps;
    p.assign_f64 = o.assign_dtype == GK_F64;
    p.max_iter = o.max_iter - sb.rounds;
    p.max_balance_iter = o.max_balance_iter;
    p.final_balance_iter = o.final_balance_iter;
    p.erosion = o.erosion;
    p.bounds = o.bounds;
    p.a16 = k <= 65535 && !o.bounds;
    if ((st = cl.geometry(o.delta_threshold)) != GK_OK) return st;
    GK_CUDA(cudaMemcpyAsync(&p.ctl->thr, &cl.thr, sizeof(double), cudaMemcpyHostToDevice, cl.s));
    const unsigned *perm = nullptr;
    if (sort) {
        Prob kp = cl.key_prob();
        GK_CUDA(launch_keys(kp, p.keys[0], p.perm[0], cl.s));
        int sel = 0;
        GK_CUDA(launch_radix_sort(p, d == 2 ? 64 : 63, cl.b.hist, &sel, cl.s));
        perm = p.perm[sel];
    }
    GK_CUDA(launch_gather(p, perm, cl.s));
    if ((st = cl.exchange_weight()) != GK_OK) return st;
    if (sort) {
        GK_CUDA(launch_centers(p, cl.s));
    } else {
        GK_CUDA(cudaMemcpyAsync(p.C, centers_io, (size_t)k * d * 8, cudaMemcpyDefault, cl.s));
        GK_CUDA(cudaMemcpyAsync(p.Iin, influence_io, (size_t)k * 8, cudaMemcpyDefault, cl.s));
    }
    if ((st = cl.tune(o)) != GK_OK) return st;
    if (order) {
        const long long *ord = (const long long *)order;
        if (order_host) {
            GK_CUDA(cudaMemcpyAsync(sb.order_stage, order, (size_t)n * 8, cudaMemcpyHostToDevice, cl.s));
            ord = sb.order_stage;
        }
        GK_CUDA(cudaMemsetAsync(sb.ctl, 0, sizeof(Ctl), cl.s));
        GK_CUDA(launch_sample_rho(p, ord, sb.m0, perm, sb.rho_in, sb.rho, cl.s));
        if ((st = cl.read_ctl()) != GK_OK) return st;
        if (g_ws.host_ctl->bad_order) return GK_ERR_INVALID_ARG;
    }
    GK_CUDA(cudaEventRecord(g_ws.ev[1], cl.s));
    if ((st = order ? run_sampled(cl, o, sb, perm) : run_loop(cl, o)) != GK_OK) return st;
    GK_CUDA(cudaEventRecord(g_ws.ev[2], cl.s));
    int *out = block_host ? cl.b.block_stage : block_out;
    GK_CUDA(launch_scatter(p, perm, out, cl.s));
    if (block_host) st = copy_out(block_out, out, (size_t)n * 4, cl.s);
    if (st == GK_OK) st = copy_out(sort ? centers_out : centers_io, p.C, (size_t)k * d * 8, cl.s);
    GK_CUDA(launch_export(p, cl.s));
    if (st == GK_OK) st = copy_out(sort ? influence_out : influence_io, p.Iin, (size_t)k * 8, cl.s);
    if (st != GK_OK) return st;
    GK_CUDA(cudaEventRecord(g_ws.ev[3], cl.s));
    if ((st = cl.read_ctl()) != GK_OK) return st;
    const Ctl &c = *g_ws.host_ctl;
    gk_status res = GK_OK;
    if (c.status != kOk)
        res = GK_ERR_TIMEOUT;
    else if (!c.balanced)
        res = GK_ERR_NOT_BALANCED;
    fill_result(result, c, res, elapsed(g_ws.ev[0], g_ws.ev[1]), elapsed(g_ws.ev[1], g_ws.ev[2]),
                elapsed(g_ws.ev[0], g_ws.ev[3]), n, cl);
    return res;
}

// gk_partition_batched: every instance in its own slice of the workspace; bounding
// boxes of all instances and one readback; the bootstraps in turn; the loops of all
// instances as one graph (independent chains); scatter and export per instance.
gk_status partition_batched(const gk_instance *inst, int32_t count, const gk_options *opt,
                            gk_result *results, void *stream) {
    if (!inst || count < 1) return GK_ERR_INVALID_ARG;
    gk_options o;
    options_or_default(opt, &o);
    gk_status st = check_options(o);
    if (st != GK_OK) return st;
    int dev = 0;
    GK_CUDA(cudaGetDevice(&dev));
    for (int i = 0; i < count; ++i) {
        const gk_instance &q = inst[i];
        if ((st = check_common(q.coords, q.dtype, q.n, q.d)) != GK_OK) return st;
        if (q.k < 1 || q.k > q.n || !(q.eps >= 0.0) || !q.block_out || q.reserved != 0)
            return GK_ERR_INVALID_ARG;
        const size_t es = q.dtype == GK_F64 ? 8 : 4;
        if (ptr_kind(q.coords, dev) != kDevice || ((uintptr_t)q.coords % es)) return GK_ERR_INVALID_ARG;
        if (q.weights && (ptr_kind(q.weights, dev) != kDevice || ((uintptr_t)q.weights % es)))
            return GK_ERR_INVALID_ARG;
        if (ptr_kind(q.block_out, dev) != kDevice || ((uintptr_t)q.block_out % 4)) return GK_ERR_INVALID_ARG;
        if ((q.centers_out && ptr_kind(q.centers_out, dev) == kForeign) ||
            (q.influence_out && ptr_kind(q.influence_out, dev) == kForeign))
            return GK_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Call> cl(count);
    std::vector<size_t> off(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        cl[i].s = s;
        if ((st = cl[i].setup(inst[i].weights, inst[i].n, inst[i].d, inst[i].k, inst[i].dtype)) != GK_OK)
            return st;
        off[i + 1] = off[i] + align_up(layout(cl[i].p, cl[i].b, nullptr, true, false, false, false, false));
    }
    if ((st = ensure_workspace(off[count])) != GK_OK) return st;
    if (g_ws.batch_cap < count) {
        if (g_ws.batch_ctl) cudaFreeHost(g_ws.batch_ctl);
        g_ws.batch_ctl = nullptr;
        g_ws.batch_cap = 0;
        if (cudaMallocHost((void **)&g_ws.batch_ctl, sizeof(Ctl) * (size_t)count) != cudaSuccess) {
            cudaGetLastError();
            return GK_ERR_OOM;
        }
        g_ws.batch_cap = count;
    }
    Ctl *hc = g_ws.batch_ctl;
    GK_CUDA(cudaEventRecord(g_ws.ev[0], s));
    for (int i = 0; i < count; ++i) {
        Prob &p = cl[i].p;
        layout(p, cl[i].b, g_ws.dev + off[i], true, false, false, false, false);
        p.coords = inst[i].coords;
        p.weights = inst[i].weights;
        p.eps = inst[i].eps;
        p.assign_f64 = o.assign_dtype == GK_F64;
        p.max_iter = o.max_iter;
        p.max_balance_iter = o.max_balance_iter;
        p.final_balance_iter = o.final_balance_iter;
        p.erosion = o.erosion;
        p.bounds = o.bounds;
        p.a16 = p.k <= 65535 && !o.bounds;
        if ((st = cl[i].upload_state(&hc[i])) != GK_OK) return st;
        GK_CUDA(launch_bbox(p, s));
    }
    for (int i = 0; i < count; ++i)
        GK_CUDA(cudaMemcpyAsync(&hc[i], cl[i].p.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    std::vector<const unsigned *> perm(count);
    for (int i = 0; i < count; ++i) {
        Prob &p = cl[i].p;
        if ((st = cl[i].frame(hc[i], o.delta_threshold)) != GK_OK) return st;
        GK_CUDA(cudaMemcpyAsync(&p.ctl->thr, &cl[i].thr, sizeof(double), cudaMemcpyHostToDevice, s));
        Prob kp = cl[i].key_prob();
        GK_CUDA(launch_keys(kp, p.keys[0], p.perm[0], s));
        int sel = 0;
        GK_CUDA(launch_radix_sort(p, p.d == 2 ? 64 : 63, cl[i].b.hist, &sel, s));
        perm[i] = p.perm[sel];
        GK_CUDA(launch_gather(p, perm[i], s));
        GK_CUDA(launch_centers(p, s));
        if ((st = cl[i].tune(o)) != GK_OK) return st;  // the instance's launch shapes
    }
    GK_CUDA(cudaEventRecord(g_ws.ev[1], s));
    std::vector<Prob> key(count);
    for (int i = 0; i < count; ++i) {
        key[i] = cl[i].p;
        key[i].coords = nullptr;
        key[i].weights = nullptr;
    }
    bool same = g_ws.batch_exec && g_ws.batch_key.size() == key.size() &&
                memcmp(g_ws.batch_key.data(), key.data(), sizeof(Prob) * key.size()) == 0;
    if (!same) {
        if (g_ws.batch_exec) cudaGraphExecDestroy(g_ws.batch_exec);
        g_ws.batch_exec = nullptr;
        g_ws.batch_key.clear();
        cudaGraphExec_t ex = nullptr;
        if (build_loop_graph(key.data(), count, &ex) != cudaSuccess) {
            cudaGetLastError();
            return GK_ERR_CUDA;
        }
        g_ws.batch_exec = ex;
        g_ws.batch_key = key;
    }
    GK_CUDA(cudaGraphLaunch(g_ws.batch_exec, s));
    GK_CUDA(cudaEventRecord(g_ws.ev[2], s));
    for (int i = 0; i < count; ++i) {
        Prob &p = cl[i].p;
        GK_CUDA(launch_scatter(p, perm[i], inst[i].block_out, s));
        if ((st = copy_out(inst[i].centers_out, p.C, (size_t)p.k * p.d * 8, s)) != GK_OK) return st;
        GK_CUDA(launch_export(p, s));
        if ((st = copy_out(inst[i].influence_out, p.Iin, (size_t)p.k * 8, s)) != GK_OK) return st;
        GK_CUDA(cudaMemcpyAsync(&hc[i], p.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    }
    GK_CUDA(cudaEventRecord(g_ws.ev[3], s));
    GK_CUDA(cudaStreamSynchronize(s));
    const double t_boot = elapsed(g_ws.ev[0], g_ws.ev[1]), t_loop = elapsed(g_ws.ev[1], g_ws.ev[2]),
                 t_tot = elapsed(g_ws.ev[0], g_ws.ev[3]);
    bool any_timeout = false, any_unbalanced = false;
    for (int i = 0; i < count; ++i) {
        const Ctl &c = hc[i];
        gk_status r = GK_OK;
        if (c.status != kOk) {
            r = GK_ERR_TIMEOUT;
            any_timeout = true;
        } else if (!c.balanced) {
            r = GK_ERR_NOT_BALANCED;
            any_unbalanced = true;
        }
        if (results) fill_result(&results[i], c, r, t_boot, t_loop, t_tot, inst[i].n, cl[i]);
    }
    return any_timeout ? GK_ERR_TIMEOUT : (any_unbalanced ? GK_ERR_NOT_BALANCED : GK_OK);
}

}  // namespace
}  // namespace gk

using namespace gk;

extern "C" {

void gk_default_options(gk_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->max_iter = 50;
    opt->max_balance_iter = 50;
    opt->final_balance_iter = 500;
    opt->erosion = 1;
    opt->delta_threshold = -1.0;
    opt->assign_dtype = GK_F64;
    opt->use_graph = 1;
    opt->bounds = 0;
}

const char *gk_status_string(int32_t status) {
    switch (status) {
        case GK_OK: return "GK_OK";
        case GK_ERR_INVALID_ARG: return "GK_ERR_INVALID_ARG";
        case GK_ERR_CUDA: return "GK_ERR_CUDA";
        case GK_ERR_OOM: return "GK_ERR_OOM";
        case GK_ERR_NOT_BALANCED: return "GK_ERR_NOT_BALANCED";
        case GK_ERR_TIMEOUT: return "GK_ERR_TIMEOUT";
        default: return "GK_UNKNOWN_STATUS";
    }
}

int32_t gk_abi_version(void) { return GK_ABI_VERSION; }

gk_status gk_check_wait_timeout(int64_t limit_us, int64_t *waited_us, void *stream) {
    if (limit_us < 1 || limit_us > 10000000) return GK_ERR_INVALID_ARG;
    int st = kOk;
    unsigned long long ns = 0;
    GK_CUDA(run_wait_check((unsigned long long)limit_us * 1000ull, &st, &ns, (cudaStream_t)stream));
    if (waited_us) *waited_us = (int64_t)(ns / 1000ull);
    return st == kOk ? GK_OK : GK_ERR_TIMEOUT;
}

gk_status gk_partition_batched(const gk_instance *inst, int32_t count, const gk_options *opt,
                               gk_result *results, void *stream) {
    return partition_batched(inst, count, opt, results, stream);
}

gk_status gk_hilbert_keys(const void *coords, int32_t dtype, int64_t n, int32_t d,
                          uint64_t *keys_out, void *stream) {
    gk_status st = check_common(coords, dtype, n, d);
    if (st != GK_OK) return st;
    if (!keys_out) return GK_ERR_INVALID_ARG;
    int dev = 0;
    GK_CUDA(cudaGetDevice(&dev));
    PtrKind kk = ptr_kind(keys_out, dev);
    if (kk == kForeign || (kk == kDevice && ((uintptr_t)keys_out % 8))) return GK_ERR_INVALID_ARG;
    Call cl;
    cl.s = (cudaStream_t)stream;
    // sort buffers are used as the key staging area
    st = cl.init(coords, dtype, nullptr, n, d, 1, true, false, false);
    if (st != GK_OK) return st;
    if ((st = cl.geometry(-1.0)) != GK_OK) return st;
    Prob kp = cl.key_prob();
    unsigned long long *dst = kk == kDevice ? (unsigned long long *)keys_out : cl.p.keys[0];
    GK_CUDA(launch_keys(kp, dst, nullptr, cl.s));
    if (kk != kDevice) st = copy_out(keys_out, dst, (size_t)n * 8, cl.s);
    if (st != GK_OK) return st;
    GK_CUDA(cudaStreamSynchronize(cl.s));
    return GK_OK;
}

gk_status gk_bounding_box(const void *coords, int32_t dtype, int64_t n, int32_t d, double *lo_out,
                          double *hi_out, void *stream) {
    gk_status st = check_common(coords, dtype, n, d);
    if (st != GK_OK) return st;
    if (!lo_out || !hi_out) return GK_ERR_INVALID_ARG;
    Call cl;
    cl.s = (cudaStream_t)stream;
    if ((st = cl.init(coords, dtype, nullptr, n, d, 1, false, false, false)) != GK_OK) return st;
    GK_CUDA(launch_bbox(cl.p, cl.s));
    if ((st = cl.read_ctl()) != GK_OK) return st;
    const Ctl &c = *g_ws.host_ctl;
    if (c.nonfinite) return GK_ERR_INVALID_ARG;
    for (int j = 0; j < d; ++j) {
        lo_out[j] = okey_to_f64(c.bb_lo[j]);
        hi_out[j] = okey_to_f64(c.bb_hi[j]);
    }
    return GK_OK;
}

gk_status gk_hilbert_keys_in_box(const void *coords, int32_t dtype, int64_t n, int32_t d,
                                 const double *lo, const double *hi, uint64_t *keys_out,
                                 void *stream) {
    gk_status st = check_common(coords, dtype, n, d);
    if (st != GK_OK) return st;
    if (!keys_out || !lo || !hi) return GK_ERR_INVALID_ARG;
    for (int j = 0; j < d; ++j)
        if (!(lo[j] <= hi[j]) || !isfinite(lo[j]) || !isfinite(hi[j])) return GK_ERR_INVALID_ARG;
    int dev = 0;
    GK_CUDA(cudaGetDevice(&dev));
    PtrKind kk = ptr_kind(keys_out, dev);
    if (kk == kForeign || (kk == kDevice && ((uintptr_t)keys_out % 8))) return GK_ERR_INVALID_ARG;
    Call cl;
    cl.s = (cudaStream_t)stream;
    if ((st = cl.init(coords, dtype, nullptr, n, d, 1, true, false, false)) != GK_OK) return st;
    GK_CUDA(launch_bbox(cl.p, cl.s));
    if ((st = cl.read_ctl()) != GK_OK) return st;
    Ctl c = *g_ws.host_ctl;
    if (c.nonfinite) return GK_ERR_INVALID_ARG;
    for (int j = 0; j < d; ++j) {  // the points must lie in the given box
        if (okey_to_f64(c.bb_lo[j]) < lo[j] || okey_to_f64(c.bb_hi[j]) > hi[j]) return GK_ERR_INVALID_ARG;
        c.bb_lo[j] = okey_f64(lo[j]);
        c.bb_hi[j] = okey_f64(hi[j]);
    }
    if ((st = cl.frame(c, -1.0)) != GK_OK) return st;
    Prob kp = cl.key_prob();
    unsigned long long *dst = kk == kDevice ? (unsigned long long *)keys_out : cl.p.keys[0];
    GK_CUDA(launch_keys(kp, dst, nullptr, cl.s));
    if (kk != kDevice) st = copy_out(keys_out, dst, (size_t)n * 8, cl.s);
    if (st != GK_OK) return st;
    GK_CUDA(cudaStreamSynchronize(cl.s));
    return GK_OK;
}

gk_status gk_sort_keys(const uint64_t *keys, int64_t n, int32_t d, int64_t *perm_out, void *stream) {
    if (!keys || !perm_out || n < 1 || n >= 0xffffffffll || (d != 2 && d != 3)) return GK_ERR_INVALID_ARG;
    int dev = 0;
    GK_CUDA(cudaGetDevice(&dev));
    const PtrKind kk = ptr_kind(keys, dev), kp = ptr_kind(perm_out, dev);
    if (kk == kForeign || kp == kForeign || (kk == kDevice && ((uintptr_t)keys % 8)) ||
        (kp == kDevice && ((uintptr_t)perm_out % 8)))
        return GK_ERR_INVALID_ARG;
    Prob p;
    memset(&p, 0, sizeof(p));
    p.n = n;
    p.n_global = n;
    p.n_pad = (n + kTile - 1) / kTile * kTile;
    p.d = d;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes);
        return o;
    };
    const size_t o_ctl = take(sizeof(Ctl)), o_k0 = take((size_t)n * 8), o_k1 = take((size_t)n * 8),
                 o_p0 = take((size_t)n * 4), o_p1 = take((size_t)n * 4),
                 o_h = take(radix_hist_entries(n) * 4), o_out = take((size_t)n * 8);
    gk_status st = ensure_workspace(off);
    if (st != GK_OK) return st;
    char *base = g_ws.dev;
    p.ctl = (Ctl *)(base + o_ctl);
    p.keys[0] = (unsigned long long *)(base + o_k0);
    p.keys[1] = (unsigned long long *)(base + o_k1);
    p.perm[0] = (unsigned *)(base + o_p0);
    p.perm[1] = (unsigned *)(base + o_p1);
    long long *out = kp == kDevice ? (long long *)perm_out : (long long *)(base + o_out);
    cudaStream_t s = (cudaStream_t)stream;
    GK_CUDA(cudaMemsetAsync(p.ctl, 0, sizeof(Ctl), s));
    GK_CUDA(cudaMemcpyAsync(p.keys[0], keys, (size_t)n * 8, cudaMemcpyDefault, s));
    GK_CUDA(launch_iota(p.perm[0], n, s));
    int sel = 0;
    GK_CUDA(launch_radix_sort(p, d == 2 ? 64 : 63, (unsigned *)(base + o_h), &sel, s));
    GK_CUDA(launch_perm_out(p, p.perm[sel], out, s));
    if (kp != kDevice) GK_CUDA(cudaMemcpyAsync(perm_out, out, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    return GK_OK;
}

gk_status gk_sfc_init(const void *coords, int32_t dtype, int64_t n, int32_t d, int32_t k,
                      int64_t *perm_out, double *centers_out, void *stream) {
    gk_status st = check_common(coords, dtype, n, d);
    if (st != GK_OK) return st;
    if (k < 1 || k > n) return GK_ERR_INVALID_ARG;
    int dev = 0;
    GK_CUDA(cudaGetDevice(&dev));
    if ((perm_out && ptr_kind(perm_out, dev) == kForeign) ||
        (centers_out && ptr_kind(centers_out, dev) == kForeign))
        return GK_ERR_INVALID_ARG;
    Call cl;
    cl.s = (cudaStream_t)stream;
    st = cl.init(coords, dtype, nullptr, n, d, k, true, false, perm_out != nullptr);
    if (st != GK_OK) return st;
    if ((st = cl.geometry(-1.0)) != GK_OK) return st;
    Prob &p = cl.p;
    Prob kp = cl.key_prob();
    GK_CUDA(launch_keys(kp, p.keys[0], p.perm[0], cl.s));
    int sel = 0;
    GK_CUDA(launch_radix_sort(p, d == 2 ? 64 : 63, cl.b.hist, &sel, cl.s));
    GK_CUDA(launch_gather(p, p.perm[sel], cl.s));
    GK_CUDA(launch_centers(p, cl.s));
    if (perm_out) {
        GK_CUDA(launch_perm_out(p, p.perm[sel], cl.b.perm_stage, cl.s));
        st = copy_out(perm_out, cl.b.perm_stage, (size_t)n * 8, cl.s);
    }
    if (st == GK_OK) st = copy_out(centers_out, p.C, (size_t)k * d * 8, cl.s);
    if (st != GK_OK) return st;
    GK_CUDA(cudaStreamSynchronize(cl.s));
    return GK_OK;
}

gk_status gk_assign(const void *coords, int32_t dtype, const void *weights, int64_t n, int32_t d,
                    int32_t k, const double *centers, const double *influence,
                    int32_t assign_dtype, int32_t *block_out, double *block_weights_out,
                    void *stream) {
    gk_status st = check_common(coords, dtype, n, d);
    if (st != GK_OK) return st;
    if (k < 1 || !centers || !influence || !block_out ||
        (assign_dtype != GK_F32 && assign_dtype != GK_F64))
        return GK_ERR_INVALID_ARG;
    int dev = 0;
    GK_CUDA(cudaGetDevice(&dev));
    if (ptr_kind(block_out, dev) == kForeign || ptr_kind(centers, dev) == kForeign ||
        ptr_kind(influence, dev) == kForeign ||
        (block_weights_out && ptr_kind(block_weights_out, dev) == kForeign))
        return GK_ERR_INVALID_ARG;
    bool block_host = ptr_kind(block_out, dev) == kHost;
    Call cl;
    cl.s = (cudaStream_t)stream;
    st = cl.init(coords, dtype, weights, n, d, k, false, block_host, false);
    if (st != GK_OK) return st;
    Prob &p = cl.p;
    p.assign_f64 = assign_dtype == GK_F64;
    if ((st = cl.geometry(-1.0)) != GK_OK) return st;
    GK_CUDA(launch_gather(p, nullptr, cl.s));
    GK_CUDA(cudaMemcpyAsync(p.C, centers, (size_t)k * d * 8, cudaMemcpyDefault, cl.s));
    GK_CUDA(cudaMemcpyAsync(p.Iin, influence, (size_t)k * 8, cudaMemcpyDefault, cl.s));
    GK_CUDA(launch_load_state(p, cl.s));
    GK_CUDA(launch_pass(p, 2, cl.s));
    int *out = block_host ? cl.b.block_stage : block_out;
    GK_CUDA(launch_scatter(p, nullptr, out, cl.s));
    if (block_host) st = copy_out(block_out, out, (size_t)n * 4, cl.s);
    if (st == GK_OK) st = copy_out(block_weights_out, p.S64, (size_t)k * 8, cl.s);
    if (st != GK_OK) return st;
    if ((st = cl.read_ctl()) != GK_OK) return st;
    if (g_ws.host_ctl->status != kOk) return GK_ERR_TIMEOUT;
    return GK_OK;
}

gk_status gk_move_centers(const void *coords, int32_t dtype, const void *weights, int64_t n,
                          int32_t d, int32_t k, const int32_t *block, const double *centers,
                          double *centers_out, double *delta_out, double *beta_out,
                          void *stream) {
    gk_status st = check_common(coords, dtype, n, d);
    if (st != GK_OK) return st;
    if (k < 1 || !block || !centers || !centers_out) return GK_ERR_INVALID_ARG;
    int dev = 0;
    GK_CUDA(cudaGetDevice(&dev));
    if (ptr_kind(block, dev) == kForeign || ptr_kind(centers, dev) == kForeign ||
        ptr_kind(centers_out, dev) == kForeign || (delta_out && ptr_kind(delta_out, dev) == kForeign))
        return GK_ERR_INVALID_ARG;
    Call cl;
    cl.s = (cudaStream_t)stream;
    st = cl.init(coords, dtype, weights, n, d, k, false, false, false);
    if (st != GK_OK) return st;
    Prob &p = cl.p;
    if ((st = cl.geometry(-1.0)) != GK_OK) return st;
    GK_CUDA(launch_gather(p, nullptr, cl.s));
    GK_CUDA(cudaMemcpyAsync(p.A, block, (size_t)n * 4, cudaMemcpyDefault, cl.s));
    GK_CUDA(cudaMemcpyAsync(p.C, centers, (size_t)k * d * 8, cudaMemcpyDefault, cl.s));
    GK_CUDA(launch_block_weights(p, cl.s));
    GK_CUDA(launch_move(p, 1, cl.s));
    st = copy_out(centers_out, p.Cm, (size_t)k * d * 8, cl.s);
    if (st == GK_OK) st = copy_out(delta_out, p.delta, (size_t)k * 8, cl.s);
    if (st != GK_OK) return st;
    if ((st = cl.read_ctl()) != GK_OK) return st;
    if (g_ws.host_ctl->bad_block) return GK_ERR_INVALID_ARG;
    if (beta_out) *beta_out = g_ws.host_ctl->beta;
    return GK_OK;
}

gk_status gk_balanced_kmeans(const void *coords, int32_t dtype, const void *weights, int64_t n,
                             int32_t d, int32_t k, double eps, double *centers_inout,
                             double *influence_inout, int32_t *block_out, const gk_options *opt,
                             gk_result *result, void *stream) {
    return kmeans_common(coords, dtype, weights, n, d, k, eps, opt, false, centers_inout,
                         influence_inout, block_out, nullptr, nullptr, result, stream);
}

gk_status gk_balanced_kmeans_sharded(const void *coords, int32_t dtype, const void *weights,
                                     int64_t n_local, int64_t n_global, int32_t d, int32_t k,
                                     double eps, double *centers_inout, double *influence_inout,
                                     int32_t *block_out, const gk_options *opt, gk_result *result,
                                     gk_reduce_fn reduce, void *reduce_ctx, void *stream) {
    if (!reduce || n_global < n_local) return GK_ERR_INVALID_ARG;
    Exchange ex;
    ex.fn = reduce;
    ex.ctx = reduce_ctx;
    return kmeans_common(coords, dtype, weights, n_local, d, k, eps, opt, false, centers_inout,
                         influence_inout, block_out, nullptr, nullptr, result, stream, nullptr, 0,
                         &ex, n_global);
}

gk_status gk_partition(const void *coords, int32_t dtype, const void *weights, int64_t n,
                       int32_t d, int32_t k, double eps, const gk_options *opt,
                       int32_t *block_out, double *centers_out, double *influence_out,
                       gk_result *result, void *stream) {
    return kmeans_common(coords, dtype, weights, n, d, k, eps, opt, true, nullptr, nullptr,
                         block_out, centers_out, influence_out, result, stream);
}

gk_status gk_partition_sampled(const void *coords, int32_t dtype, const void *weights, int64_t n,
                               int32_t d, int32_t k, double eps, const int64_t *order,
                               int64_t sample0, const gk_options *opt, int32_t *block_out,
                               double *centers_out, double *influence_out, gk_result *result,
                               void *stream) {
    if (!order) return GK_ERR_INVALID_ARG;
    return kmeans_common(coords, dtype, weights, n, d, k, eps, opt, true, nullptr, nullptr,
                         block_out, centers_out, influence_out, result, stream, order, sample0);
}

gk_status gk_partition_quality(const int64_t *row_ptr, const int32_t *col, int64_t n, int64_t nnz,
                               const int32_t *block, int32_t k, int64_t *ext_out,
                               int64_t *comm_out, gk_quality *quality, void *stream) {
    if (!row_ptr || (!col && nnz > 0) || !block || n < 1 || n >= (1ll << 31) || nnz < 0 || k < 1)
        return GK_ERR_INVALID_ARG;
    int dev = 0;
    GK_CUDA(cudaGetDevice(&dev));
    const void *in[3] = {row_ptr, col, block};
    const size_t in_bytes[3] = {(size_t)(n + 1) * 8, (size_t)nnz * 4, (size_t)n * 4};
    const size_t align[3] = {8, 4, 4};
    PtrKind kind[3];
    size_t need = 0;
    for (int i = 0; i < 3; ++i) {
        kind[i] = in[i] ? ptr_kind(in[i], dev) : kDevice;
        if (kind[i] == kForeign || (kind[i] == kDevice && ((uintptr_t)in[i] % align[i])))
            return GK_ERR_INVALID_ARG;
        if (kind[i] == kHost) need += align_up(in_bytes[i]);
    }
    if ((ext_out && ptr_kind(ext_out, dev) == kForeign) || (comm_out && ptr_kind(comm_out, dev) == kForeign))
        return GK_ERR_INVALID_ARG;
    need += 2 * align_up((size_t)k * 8) + align_up(5 * 8) + align_up(sizeof(int));
    gk_status st = ensure_workspace(need);
    if (st != GK_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = g_ws.dev;
    const void *dptr[3];
    for (int i = 0; i < 3; ++i) {
        if (kind[i] == kHost) {
            GK_CUDA(cudaMemcpyAsync(ws, in[i], in_bytes[i], cudaMemcpyHostToDevice, s));
            dptr[i] = ws;
            ws += align_up(in_bytes[i]);
        } else {
            dptr[i] = in[i];
        }
    }
    unsigned long long *ext = (unsigned long long *)ws;
    ws += align_up((size_t)k * 8);
    unsigned long long *comm = (unsigned long long *)ws;
    ws += align_up((size_t)k * 8);
    unsigned long long *out = (unsigned long long *)ws;
    ws += align_up(5 * 8);
    int *bad = (int *)ws;
    GK_CUDA(launch_quality((const long long *)dptr[0], (const int *)dptr[1], n, nnz,
                           (const int *)dptr[2], k, ext, comm, out, bad, s));
    if (ext_out) GK_CUDA(cudaMemcpyAsync(ext_out, ext, (size_t)k * 8, cudaMemcpyDefault, s));
    if (comm_out) GK_CUDA(cudaMemcpyAsync(comm_out, comm, (size_t)k * 8, cudaMemcpyDefault, s));
    unsigned long long h[5];
    int hbad = 0;
    GK_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    if (hbad) return GK_ERR_INVALID_ARG;
    if (quality) {
        quality->edge_cut = (int64_t)h[0];
        quality->total_comm_volume = (int64_t)h[1];
        quality->max_comm_volume = (int64_t)h[2];
        quality->max_ext = (int64_t)h[3];
        quality->boundary_vertices = (int64_t)h[4];
    }
    return GK_OK;
}

gk_status gk_block_diameter(const int64_t *row_ptr, const int32_t *col, int64_t n, int64_t nnz,
                            const int32_t *block, int32_t k, int32_t sweeps, int32_t *diam_out,
                            gk_diameter *summary, void *stream) {
    if (!row_ptr || (!col && nnz > 0) || !block || n < 1 || n >= (1ll << 31) || nnz < 0 || k < 1 ||
        sweeps < 1 || sweeps > GK_MAX_SWEEPS)
        return GK_ERR_INVALID_ARG;
    int dev = 0;
    GK_CUDA(cudaGetDevice(&dev));
    const void *in[3] = {row_ptr, col, block};
    const size_t in_bytes[3] = {(size_t)(n + 1) * 8, (size_t)nnz * 4, (size_t)n * 4};
    const size_t align[3] = {8, 4, 4};
    PtrKind kind[3];
    size_t need = 0;
    for (int i = 0; i < 3; ++i) {
        kind[i] = in[i] ? ptr_kind(in[i], dev) : kDevice;
        if (kind[i] == kForeign || (kind[i] == kDevice && ((uintptr_t)in[i] % align[i])))
            return GK_ERR_INVALID_ARG;
        if (kind[i] == kHost) need += align_up(in_bytes[i]);
    }
    if (diam_out && ptr_kind(diam_out, dev) == kForeign) return GK_ERR_INVALID_ARG;
    need += align_up(diameter_work_bytes(n, k)) + align_up((size_t)k * 4) + align_up(16) +
            align_up(8);
    gk_status st = ensure_workspace(need);
    if (st != GK_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = g_ws.dev;
    const void *dptr[3];
    for (int i = 0; i < 3; ++i) {
        if (kind[i] == kHost) {
            GK_CUDA(cudaMemcpyAsync(ws, in[i], in_bytes[i], cudaMemcpyHostToDevice, s));
            dptr[i] = ws;
            ws += align_up(in_bytes[i]);
        } else {
            dptr[i] = in[i];
        }
    }
    void *work = ws;
    ws += align_up(diameter_work_bytes(n, k));
    int *diam = (int *)ws;
    ws += align_up((size_t)k * 4);
    long long *out_i = (long long *)ws;
    ws += align_up(16);
    double *out_d = (double *)ws;
    int hbad = 0;
    long long levels = 0;
    GK_CUDA(run_diameter((const long long *)dptr[0], (const int *)dptr[1], n, nnz,
                         (const int *)dptr[2], k, sweeps, work, diam, out_i, out_d, &hbad, &levels,
                         s));
    if (hbad) return GK_ERR_INVALID_ARG;
    if (diam_out) GK_CUDA(cudaMemcpyAsync(diam_out, diam, (size_t)k * 4, cudaMemcpyDefault, s));
    long long hi[2];
    double hd = 0.0;
    GK_CUDA(cudaMemcpyAsync(hi, out_i, sizeof(hi), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaMemcpyAsync(&hd, out_d, sizeof(hd), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    if (summary) {
        summary->max_diameter = hi[0];
        summary->disconnected_blocks = hi[1];
        summary->bfs_levels = levels;
        summary->harmonic_mean = hd;
    }
    return GK_OK;
}

void gk_release(void) { release_all(); }

gk_status gk_set_allocator(gk_alloc_fn alloc, gk_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) return GK_ERR_INVALID_ARG;
    release_all();  // the current workspace goes back to whoever provided it
    g_alloc.alloc = alloc;
    g_alloc.free = free_fn;
    g_alloc.ctx = ctx;
    return GK_OK;
}

}  // extern "C"
