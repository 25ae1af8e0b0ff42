// gk_quality.cu -- partition quality measures of Section 5 on a graph given as a
// symmetric CSR adjacency: per block ext(V_i) (edges leaving the block) and comm(V_i)
// (for every vertex of the block, the number of other blocks holding a neighbour),
// then edge cut = sum ext / 2, total and maximum communication volume; and per block a
// lower bound of diam(V_i), the largest distance between two vertices of V_i inside the
// subgraph V_i induces, from breadth-first sweeps.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <climits>

#include "gk_common.cuh"
#include "gk_internal.h"

namespace gk {

// Foreign neighbours (nf) and distinct foreign blocks (nd) of vertex v of block b, one
// thread alone: each foreign neighbour is checked against the neighbours stored before it
// (quadratic in the degree).  Entries that are out of range set *bad and are skipped.
__device__ void vertex_counts(const long long *row_ptr, const int *col, long long n,
                              const int *block, int k, long long v, int b, long long e0,
                              long long e1, unsigned &nf, unsigned &nd, int *bad) {
    nf = 0;
    nd = 0;
    for (long long e = e0; e < e1; ++e) {
        const int u = col[e];
        if ((unsigned long long)(long long)u >= (unsigned long long)n) {
            atomicOr(bad, 1);
            continue;
        }
        if (u == v) continue;  // self-loop
        const int bu = block[u];
        if ((unsigned)bu >= (unsigned)k) {
            atomicOr(bad, 1);
            continue;
        }
        if (bu == b) continue;
        ++nf;
        bool seen = false;
        for (long long f = e0; f < e && !seen; ++f) {
            const int w = col[f];
            if ((unsigned long long)(long long)w < (unsigned long long)n && w != v) seen = block[w] == bu;
        }
        if (!seen) ++nd;
    }
}

constexpr int kQWarps = 8;    // warps per CTA of the quality kernel
constexpr int kQCap = 512;    // adjacency entries of a warp's 32 vertices staged in shared memory

// One warp per 32 consecutive vertices.  Their rows are one contiguous range of col; the
// lanes walk it together (coalesced neighbour loads, independent block-id gathers), store
// each entry's foreign block (-1: own block or self-loop) in shared memory, then count per
// row the foreign entries and the first occurrences of each foreign block (the check
// against the earlier entries of the row reads shared memory).  A warp whose rows hold
// more than kQCap entries counts each vertex in its own thread instead.  Malformed input
// (a row range outside [0, nnz], a neighbour outside [0, n), a block id outside [0, k))
// sets *bad; a warp with a malformed row skips its counts (the call then fails).
__global__ void __launch_bounds__(kQWarps * 32) quality_vertex_kernel(
    const long long *row_ptr, const int *col, long long n, long long nnz, const int *block, int k,
    unsigned long long *ext, unsigned long long *comm, unsigned long long *boundary, int *bad) {
    __shared__ long long s_rp[kQWarps][33];
    __shared__ int s_fb[kQWarps][kQCap];
    __shared__ int s_b[kQWarps][32];
    __shared__ unsigned s_nf[kQWarps][32], s_nd[kQWarps][32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long v0 = ((long long)blockIdx.x * kQWarps + w) * 32;
    if (v0 >= n) return;  // the whole warp
    const long long v = v0 + lane;
    const bool has = v < n;
    const int cnt = (int)min(32ll, n - v0);
    int b = 0;
    long long e0 = 0, e1 = 0;
    bool ok = true;
    if (has) {
        b = block[v];
        e0 = row_ptr[v];
        e1 = row_ptr[v + 1];
        if ((unsigned)b >= (unsigned)k || e0 < 0 || e1 < e0 || e1 > nnz) {
            atomicOr(bad, 1);
            ok = false;
        }
    }
    if (!__all_sync(full, ok)) return;  // the whole warp
    const long long Eend = __shfl_sync(full, e1, cnt - 1);
    s_rp[w][lane] = has ? e0 : Eend;
    if (lane == 0) s_rp[w][32] = Eend;
    s_b[w][lane] = b;
    s_nf[w][lane] = 0;
    s_nd[w][lane] = 0;
    __syncwarp();
    const long long E0 = s_rp[w][0];
    const long long m = Eend - E0;
    unsigned nf = 0, nd = 0;
    if (m > kQCap) {
        if (has) vertex_counts(row_ptr, col, n, block, k, v, b, e0, e1, nf, nd, bad);
    } else {
        int *fb = s_fb[w];
        const long long *rp = s_rp[w];
        for (int i = lane; i < (int)m; i += 32) {
            const long long e = E0 + i;
            int lo = 0, hi = 32;  // the row of entry e: rp[lo] <= e < rp[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (rp[mid] <= e) lo = mid;
                else hi = mid;
            }
            const int u = col[e];
            int f = -1;
            if ((unsigned long long)(long long)u >= (unsigned long long)n) {
                atomicOr(bad, 1);
            } else if (u != v0 + lo) {
                const int bu = block[u];
                if ((unsigned)bu >= (unsigned)k) atomicOr(bad, 1);
                else if (bu != s_b[w][lo]) f = bu;
            }
            fb[i] = f;
        }
        __syncwarp();
        for (int i = lane; i < (int)m; i += 32) {
            const int f = fb[i];
            if (f < 0) continue;
            const long long e = E0 + i;
            int lo = 0, hi = 32;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (rp[mid] <= e) lo = mid;
                else hi = mid;
            }
            bool seen = false;
            for (int j = (int)(rp[lo] - E0); j < i && !seen; ++j) seen = fb[j] == f;
            atomicAdd(&s_nf[w][lo], 1u);
            if (!seen) atomicAdd(&s_nd[w][lo], 1u);
        }
        __syncwarp();
        nf = s_nf[w][lane];
        nd = s_nd[w][lane];
    }
    if (has && nf) {
        atomicAdd(&ext[b], (unsigned long long)nf);
        atomicAdd(&comm[b], (unsigned long long)nd);
    }
    const unsigned bm = __ballot_sync(full, has && nf != 0);  // boundary vertices of the warp
    if (lane == 0 && bm) atomicAdd(boundary, (unsigned long long)__popc(bm));
}

// One CTA: sums and maxima over the k blocks -> out[0..3] = edge cut, total comm,
// max comm, max ext (ext summed over blocks is even for a symmetric graph).
__global__ void __launch_bounds__(256) quality_final_kernel(const unsigned long long *ext,
                                                            const unsigned long long *comm, int k,
                                                            unsigned long long *out) {
    __shared__ unsigned long long s[4][8];
    unsigned long long se = 0, sc = 0, mc = 0, me = 0;
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        se += ext[c];
        sc += comm[c];
        mc = max(mc, comm[c]);
        me = max(me, ext[c]);
    }
    for (int o = 16; o; o >>= 1) {
        se += __shfl_xor_sync(0xffffffffu, se, o);
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
        mc = max(mc, __shfl_xor_sync(0xffffffffu, mc, o));
        me = max(me, __shfl_xor_sync(0xffffffffu, me, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        s[0][w] = se;
        s[1][w] = sc;
        s[2][w] = mc;
        s[3][w] = me;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            se += s[0][q];
            sc += s[1][q];
            mc = max(mc, s[2][q]);
            me = max(me, s[3][q]);
        }
        out[0] = se / 2;
        out[1] = sc;
        out[2] = mc;
        out[3] = me;
    }
}

cudaError_t launch_quality(const long long *row_ptr, const int *col, long long n, long long nnz,
                           const int *block, int k, unsigned long long *ext,
                           unsigned long long *comm, unsigned long long *out, int *bad,
                           cudaStream_t s) {
    // out[4] = boundary vertices, accumulated by the vertex kernel
    cudaError_t e = cudaMemsetAsync(ext, 0, (size_t)k * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(comm, 0, (size_t)k * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, 5 * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (n > 0)
        quality_vertex_kernel<<<(unsigned)((n + kQWarps * 32 - 1) / (kQWarps * 32)), kQWarps * 32, 0,
                                s>>>(row_ptr, col, n, nnz, block, k, ext, comm, out + 4, bad);
    quality_final_kernel<<<1, 256, 0, s>>>(ext, comm, k, out);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------
// Block diameters.  The paper evaluates a lower bound from the first rounds of iFUB; here
// the bound of every block comes from `sweeps` breadth-first sweeps inside the block, the
// first from its smallest vertex index, each later one from the vertex the previous sweep
// reached last (smallest index among those at the largest distance).  Each sweep's
// eccentricity lies in [diam / 2, diam].  A block the first sweep does not cover is not
// connected (infinite diameter, reported as -1).
//
// The sweeps of all blocks run together: an edge between two blocks is never followed, so
// one search seeded with one vertex per block is k separate searches.  Each level expands
// a frontier list; a vertex joins the next list when its distance moves from -1 to the
// next level (compare-and-swap, so once per sweep), and the host reads the length of the
// next list to stop when it is empty.  A level's new vertices are gathered per CTA in
// shared memory and appended with one global atomic per CTA and round: one counter that
// every new vertex incremented took about one L2 atomic per vertex on a single address.
// ----------------------------------------------------------------------------------------
__global__ void diam_fill_kernel(int *a, long long m, int v) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) a[i] = v;
}

// Block sizes, smallest vertex of every block, and the checks of the input (row ranges,
// neighbours, block ids): the searches run only on input that passed.
__global__ void diam_init_kernel(const long long *row_ptr, const int *col, long long n,
                                 long long nnz, const int *block, int k, int *size, int *start,
                                 int *bad) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int b = block[v];
    const long long e0 = row_ptr[v], e1 = row_ptr[v + 1];
    if ((unsigned)b >= (unsigned)k || e0 < 0 || e1 < e0 || e1 > nnz) {
        atomicOr(bad, 1);
        return;
    }
    for (long long e = e0; e < e1; ++e)
        if ((unsigned long long)(long long)col[e] >= (unsigned long long)n) atomicOr(bad, 1);
    atomicAdd(&size[b], 1);
    atomicMin(&start[b], (int)v);
}

// One thread per block: its start vertex (if any) opens the sweep at distance 0.
__global__ void diam_seed_kernel(int k, const int *start, int *dist, int *front, unsigned *cnt,
                                 int *ecc, int *reached) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= k) return;
    const int s = start[b];
    ecc[b] = 0;
    reached[b] = s != INT_MAX;
    if (s != INT_MAX) {
        dist[s] = 0;
        front[atomicAdd(cnt, 1u)] = s;
    }
}

// One breadth-first level over the frontier list of distance `level` (its length read on
// the device, so that the host can enqueue several levels without waiting; an empty
// frontier does nothing).  The CTA takes kExpandThreads entries per round, one per thread;
// the vertices a round finds go to a shared buffer (a warp-aggregated shared counter), which
// one atomic on cnt_out places in the next list; a round that finds more than the buffer
// holds appends the rest one by one.  levels counts the non-empty levels.
constexpr int kExpandThreads = 256;
constexpr unsigned kExpandBuf = 2048;

__global__ void __launch_bounds__(kExpandThreads) diam_expand_kernel(
    const int *front, const unsigned *cnt_in, int level, const long long *row_ptr,
    const int *col, const int *block, int *dist, int *next, unsigned *cnt_out, int *ecc,
    int *reached, unsigned long long *levels) {
    namespace cg = cooperative_groups;
    __shared__ int sbuf[kExpandBuf];
    __shared__ unsigned scnt, sbase;
    const unsigned m = *cnt_in;
    if (m == 0) return;  // the same for every thread of the grid
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(levels, 1ull);
    if (threadIdx.x == 0) scnt = 0;
    __syncthreads();
    const unsigned stride = gridDim.x * kExpandThreads;
    for (unsigned i0 = blockIdx.x * kExpandThreads; i0 < m; i0 += stride) {  // CTA-uniform
        const unsigned i = i0 + threadIdx.x;
        if (i < m) {
            const int v = front[i];
            const int b = block[v];
            const long long e1 = row_ptr[v + 1];
            for (long long e = row_ptr[v]; e < e1; ++e) {
                const int u = col[e];
                if (u == v || block[u] != b) continue;
                if (atomicCAS(&dist[u], -1, level + 1) == -1) {
                    cg::coalesced_group g = cg::coalesced_threads();
                    unsigned pos = 0;
                    if (g.thread_rank() == 0) pos = atomicAdd(&scnt, g.size());
                    pos = g.shfl(pos, 0) + g.thread_rank();
                    if (pos < kExpandBuf)
                        sbuf[pos] = u;
                    else
                        next[atomicAdd(cnt_out, 1u)] = u;
                    atomicAdd(&reached[b], 1);
                    atomicMax(&ecc[b], level + 1);
                }
            }
        }
        __syncthreads();
        const unsigned c = min(scnt, kExpandBuf);
        if (threadIdx.x == 0 && c > 0) sbase = atomicAdd(cnt_out, c);
        __syncthreads();
        for (unsigned j = threadIdx.x; j < c; j += kExpandThreads) next[sbase + j] = sbuf[j];
        __syncthreads();  // every thread has read scnt and sbuf
        if (threadIdx.x == 0) scnt = 0;
        __syncthreads();
    }
}

// The next start of every block: its smallest vertex at the largest distance.
__global__ void diam_far_kernel(long long n, const int *block, const int *dist, const int *ecc,
                                int *start) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int dv = dist[v];
    const int b = block[v];
    if (dv >= 0 && dv == ecc[b]) atomicMin(&start[b], (int)v);
}

// Bound and connectivity per block after a sweep.
__global__ void diam_record_kernel(int k, int sweep, const int *size, const int *reached,
                                   const int *ecc, int *bound, int *conn) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= k) return;
    if (sweep == 0) {
        conn[b] = reached[b] == size[b];
        bound[b] = ecc[b];
    } else {
        bound[b] = max(bound[b], ecc[b]);
    }
}

// One CTA: per-block results (bound, -1 when not connected, 0 when empty) and the summary
// out_i[0..1] = largest bound over the connected blocks, disconnected blocks;
// out_d[0] = harmonic mean over the blocks of at least two vertices (1/inf = 0 for a
// disconnected block; +inf when the sum of reciprocals is 0, 0 when there is no such
// block).  Every thread sums a fixed stride of blocks, then a fixed tree: the same sum
// on every run.
__global__ void __launch_bounds__(256) diam_final_kernel(int k, const int *size, const int *bound,
                                                         const int *conn, int *diam,
                                                         long long *out_i, double *out_d) {
    __shared__ double sr[256];
    __shared__ long long sm[256], sd[256], sb[256];
    long long mx = 0, nd = 0, nb = 0;
    double r = 0.0;
    for (int b = threadIdx.x; b < k; b += blockDim.x) {
        const int sz = size[b];
        const int val = sz == 0 ? 0 : (conn[b] ? bound[b] : -1);
        diam[b] = val;
        if (val >= 0) mx = max(mx, (long long)val);
        if (val < 0) ++nd;
        if (sz >= 2) {
            ++nb;
            if (val > 0) r += 1.0 / (double)val;
        }
    }
    sr[threadIdx.x] = r;
    sm[threadIdx.x] = mx;
    sd[threadIdx.x] = nd;
    sb[threadIdx.x] = nb;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sr[threadIdx.x] += sr[threadIdx.x + o];
            sm[threadIdx.x] = max(sm[threadIdx.x], sm[threadIdx.x + o]);
            sd[threadIdx.x] += sd[threadIdx.x + o];
            sb[threadIdx.x] += sb[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out_i[0] = sm[0];
        out_i[1] = sd[0];
        const double sum = sr[0];
        out_d[0] = sb[0] == 0 ? 0.0 : (sum == 0.0 ? __longlong_as_double(0x7ff0000000000000ll)
                                                  : (double)sb[0] / sum);
    }
}

size_t diameter_work_bytes(long long n, int k) {
    return (size_t)n * 4 * 3 + (size_t)k * 4 * 6 + 64;
}

static unsigned blocks_of(long long m) { return (unsigned)((m + 255) / 256); }

cudaError_t run_diameter(const long long *row_ptr, const int *col, long long n, long long nnz,
                         const int *block, int k, int sweeps, void *work, int *diam,
                         long long *out_i, double *out_d, int *hbad, long long *hlevels,
                         cudaStream_t s) {
    // work: dist, two frontier lists (n each), six k-vectors, two counters and the flag
    int *dist = (int *)work;
    int *front[2] = {dist + n, dist + 2 * n};
    int *size = dist + 3 * n, *start = size + k, *ecc = start + k, *reached = ecc + k;
    int *bound = reached + k, *conn = bound + k;
    unsigned *cnt = (unsigned *)(conn + k);
    int *bad = (int *)(cnt + 2);
    unsigned long long *levels = (unsigned long long *)(((uintptr_t)(bad + 1) + 7) & ~(uintptr_t)7);
    *hbad = 0;
    *hlevels = 0;
    cudaError_t e = cudaMemsetAsync(size, 0, (size_t)k * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(levels, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    diam_fill_kernel<<<blocks_of(k), 256, 0, s>>>(start, k, INT_MAX);
    diam_init_kernel<<<blocks_of(n), 256, 0, s>>>(row_ptr, col, n, nnz, block, k, size, start, bad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (*hbad) return cudaSuccess;
    for (int sweep = 0; sweep < sweeps; ++sweep) {
        if ((e = cudaMemsetAsync(dist, 0xff, (size_t)n * 4, s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(cnt, 0, 4, s)) != cudaSuccess) return e;
        diam_seed_kernel<<<blocks_of(k), 256, 0, s>>>(k, start, dist, front[0], cnt, ecc, reached);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // kLevelsPerWait levels are enqueued between two reads of the frontier length;
        // the search ends with an empty frontier (at most n levels: every vertex joins one
        // list once)
        constexpr int kLevelsPerWait = 16;
        const int grid = (int)(blocks_of(n) < 1216 ? blocks_of(n) : 1216);
        int cur = 0, level = 0;
        for (;;) {
            for (int g = 0; g < kLevelsPerWait; ++g, ++level) {
                if ((e = cudaMemsetAsync(cnt + (cur ^ 1), 0, 4, s)) != cudaSuccess) return e;
                diam_expand_kernel<<<grid, kExpandThreads, 0, s>>>(front[cur], cnt + cur, level, row_ptr, col, block,
                                                        dist, front[cur ^ 1], cnt + (cur ^ 1), ecc,
                                                        reached, levels);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                cur ^= 1;
            }
            unsigned h = 0;
            if ((e = cudaMemcpyAsync(&h, cnt + cur, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                return e;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            if (h == 0) break;
        }
        diam_record_kernel<<<blocks_of(k), 256, 0, s>>>(k, sweep, size, reached, ecc, bound, conn);
        if (sweep + 1 < sweeps) {
            diam_fill_kernel<<<blocks_of(k), 256, 0, s>>>(start, k, INT_MAX);
            diam_far_kernel<<<blocks_of(n), 256, 0, s>>>(n, block, dist, ecc, start);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    diam_final_kernel<<<1, 256, 0, s>>>(k, size, bound, conn, diam, out_i, out_d);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    unsigned long long lv = 0;
    if ((e = cudaMemcpyAsync(&lv, levels, sizeof(lv), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *hlevels = (long long)lv;
    return cudaSuccess;
}

}  // namespace gk
