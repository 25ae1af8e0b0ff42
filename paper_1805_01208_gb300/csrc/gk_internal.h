// gk_internal.h -- host-side launchers shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include "gk_common.cuh"

namespace gk {

// bootstrap (gk_bootstrap.cu)
cudaError_t launch_bbox(const Prob &p, cudaStream_t s);
cudaError_t launch_keys(const Prob &p, unsigned long long *keys, unsigned *perm, cudaStream_t s);
size_t radix_hist_entries(long long n);
cudaError_t launch_radix_sort(const Prob &p, int key_bits, unsigned *hist, int *sel,
                              cudaStream_t s);
cudaError_t launch_gather(const Prob &p, const unsigned *perm, cudaStream_t s);
cudaError_t launch_centers(const Prob &p, cudaStream_t s);
// supertile boxes for p.stiles tiles per supertile (p.nsupers of them)
cudaError_t launch_super_boxes(const Prob &p, cudaStream_t s);
cudaError_t launch_scatter(const Prob &p, const unsigned *perm, int *out, cudaStream_t s);
cudaError_t launch_perm_out(const Prob &p, const unsigned *perm, long long *out, cudaStream_t s);

// A kernel of a fixed launch sequence, for direct launches and graph nodes alike.
struct KNode {
    void *fn;
    dim3 grid, block;
};
// Random initialization (Section 4.5): round bytes of the curve positions from the
// caller's order (sets ctl->bad_order unless order is a permutation of [0, n)), and
// the kernels that select and gather one sample round (arguments: {&ps, &sel}).
long long sample_rho_entries(long long n);
cudaError_t launch_sample_rho(const Prob &p, const long long *order, long long m0,
                              const unsigned *perm, unsigned char *rho_in, unsigned char *rho,
                              cudaStream_t s);
constexpr int kSampleSelectNodes = 7;
int sample_select_nodes(const Prob &ps, const SampleSel &sel, KNode *out);
cudaError_t launch_sample_select(const Prob &ps, const SampleSel &sel, cudaStream_t s);

// partition quality (gk_quality.cu): ext and comm per block (k entries each), out[0..4] =
// edge cut, total comm, max comm, max ext, boundary vertices; *bad set on malformed input
cudaError_t launch_quality(const long long *row_ptr, const int *col, long long n, long long nnz,
                           const int *block, int k, unsigned long long *ext,
                           unsigned long long *comm, unsigned long long *out, int *bad,
                           cudaStream_t s);
// Block diameter lower bounds from `sweeps` breadth-first sweeps (gk_quality.cu).  work:
// diameter_work_bytes(n, k) bytes of device memory, 4-byte aligned; diam: k int32 (device);
// out_i[0..1] = largest bound, disconnected blocks; out_d[0] = harmonic mean (device).
// Synchronises the stream once per level; on malformed input sets *hbad and returns
// before any search.
size_t diameter_work_bytes(long long n, int k);
cudaError_t run_diameter(const long long *row_ptr, const int *col, long long n, long long nnz,
                         const int *block, int k, int sweeps, void *work, int *diam,
                         long long *out_i, double *out_d, int *hbad, long long *hlevels,
                         cudaStream_t s);

// One bounded wait, with limit_ns of device time, on an mbarrier that nothing completes
// (gk_kmeans.cu); *status = kErrTimeout when it gave up, *waited_ns its device time.
// Synchronises the stream.
cudaError_t run_wait_check(unsigned long long limit_ns, int *status,
                           unsigned long long *waited_ns, cudaStream_t s);

// iteration (gk_kmeans.cu)
cudaError_t launch_init(const Prob &p, cudaStream_t s);
cudaError_t launch_load_state(const Prob &p, cudaStream_t s);
cudaError_t launch_pass(const Prob &p, int mode, cudaStream_t s);
cudaError_t launch_filter(const Prob &p, cudaStream_t s);
cudaError_t launch_assign(const Prob &p, cudaStream_t s);
// resident CTAs per SM of the assignment: its largest count, and the count p launches with
int assign_max_ctas(const Prob &p);
int assign_ctas(const Prob &p);
cudaError_t launch_balance(const Prob &p, int mode, cudaStream_t s);
cudaError_t launch_block_weights(const Prob &p, cudaStream_t s);
cudaError_t launch_move(const Prob &p, int mode, cudaStream_t s);
// launch_move in two parts (a sharded run exchanges the block sums in between)
cudaError_t launch_centroid(const Prob &p, cudaStream_t s);
cudaError_t launch_move_finish(const Prob &p, int mode, cudaStream_t s);
// identity permutation 0..n-1 (the values of a standalone key sort)
cudaError_t launch_iota(unsigned *perm, long long n, cudaStream_t s);
cudaError_t launch_final_begin(const Prob &p, cudaStream_t s);
cudaError_t launch_export(const Prob &p, cudaStream_t s);
// The whole loop of each of count problems as one graph (independent chains).
cudaError_t build_loop_graph(const Prob *probs, int count, cudaGraphExec_t *exec_out);
// Random initialization: forced movement closing a sample round (mode 3 of the
// movement) and the hand-over of its influence and counters to the main problem.
cudaError_t launch_sample_export(const Prob &ps, Ctl *main_ctl, cudaStream_t s);
// Sample rounds ps[0..R) (each selected, run and handed over in turn), then the
// loop of the main problem p, as one graph.
cudaError_t build_sampled_graph(const Prob &p, const Prob *ps, const SampleSel *sel, int R,
                                cudaGraphExec_t *exec_out);

}  // namespace gk
