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
cudaError_t launch_scatter(const Prob &p, const unsigned *perm, int *out, cudaStream_t s);
cudaError_t launch_perm_out(const Prob &p, const unsigned *perm, long long *out, cudaStream_t s);

// iteration (gk_kmeans.cu)
cudaError_t launch_init(const Prob &p, cudaStream_t s);
cudaError_t launch_load_state(const Prob &p, cudaStream_t s);
cudaError_t launch_pass(const Prob &p, int mode, cudaStream_t s);
cudaError_t launch_filter(const Prob &p, cudaStream_t s);
cudaError_t launch_assign(const Prob &p, cudaStream_t s);
cudaError_t launch_balance(const Prob &p, int mode, cudaStream_t s);
cudaError_t launch_block_weights(const Prob &p, cudaStream_t s);
cudaError_t launch_move(const Prob &p, int mode, cudaStream_t s);
cudaError_t launch_final_begin(const Prob &p, cudaStream_t s);
cudaError_t launch_export(const Prob &p, cudaStream_t s);
// The whole loop of each of count problems as one graph (independent chains).
cudaError_t build_loop_graph(const Prob *probs, int count, cudaGraphExec_t *exec_out);

}  // namespace gk
