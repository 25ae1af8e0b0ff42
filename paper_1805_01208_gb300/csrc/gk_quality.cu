// gk_quality.cu -- partition quality measures of Section 5 on a graph given as a
// symmetric CSR adjacency: per block ext(V_i) (edges leaving the block) and comm(V_i)
// (for every vertex of the block, the number of other blocks holding a neighbour),
// then edge cut = sum ext / 2, total and maximum communication volume.
#include <cuda_runtime.h>

#include "gk_common.cuh"
#include "gk_internal.h"

namespace gk {

// One thread per vertex.  The distinct foreign blocks among a vertex's neighbours are
// counted by checking, for each foreign neighbour, the neighbours stored before it
// (quadratic in the degree; mesh degrees are small).  Malformed input (a row range
// outside [0, nnz], a neighbour outside [0, n), a block id outside [0, k)) sets *bad and
// the offending entries are skipped.
__global__ void quality_vertex_kernel(const long long *row_ptr, const int *col, long long n,
                                      long long nnz, const int *block, int k,
                                      unsigned long long *ext, unsigned long long *comm,
                                      unsigned long long *boundary, int *bad) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = v < n;  // every lane stays to the warp vote at the end
    int b = 0;
    long long e0 = 0, e1 = 0;
    if (ok) {
        b = block[v];
        e0 = row_ptr[v];
        e1 = row_ptr[v + 1];
        if ((unsigned)b >= (unsigned)k || e0 < 0 || e1 < e0 || e1 > nnz) {
            atomicOr(bad, 1);
            ok = false;
        }
    }
    unsigned nf = 0, nd = 0;
    for (long long e = e0; ok && e < e1; ++e) {
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
    if (nf) {
        atomicAdd(&ext[b], (unsigned long long)nf);
        atomicAdd(&comm[b], (unsigned long long)nd);
    }
    const unsigned m = __ballot_sync(0xffffffffu, nf != 0);  // boundary vertices of the warp
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(boundary, (unsigned long long)__popc(m));
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
        quality_vertex_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(row_ptr, col, n, nnz, block, k,
                                                                          ext, comm, out + 4, bad);
    quality_final_kernel<<<1, 256, 0, s>>>(ext, comm, k, out);
    return cudaGetLastError();
}

}  // namespace gk
