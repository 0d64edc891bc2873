// Host-side launchers of the chain kernel, one translation unit per
// working precision (compiled in parallel).
#pragma once

#include <cuda_runtime.h>

#include "skr_common.h"

namespace skr {

// Launch chain_kernel<T> with nclusters clusters of cs CTAs (threads each)
// and dynamic shared memory smem.  Sets the kernel attributes it needs.
cudaError_t launch_chain_f32(const ChainArgs &a, int nclusters, int cs, int threads, size_t smem,
                             cudaStream_t st);
cudaError_t launch_chain_f64(const ChainArgs &a, int nclusters, int cs, int threads, size_t smem,
                             cudaStream_t st);
// Clusters of cs CTAs that can be resident at once (0 on error).
int max_active_clusters_f32(int cs, int threads, size_t smem);
int max_active_clusters_f64(int cs, int threads, size_t smem);
// Threads per CTA the chain kernel is compiled for.
int chain_threads();
// Dynamic shared memory of the chain kernel for (m, k, threads, element size).
size_t chain_smem_bytes(int m, int k, int threads, int esz);

}  // namespace skr
