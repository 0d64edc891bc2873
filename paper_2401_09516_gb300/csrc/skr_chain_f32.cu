// Mixed form: FP32 Krylov vectors and reductions; FP64 solution, true
// residual, right-hand side and small dense step.
#include "skr_chain_launch.cuh"
#include "skr_launch.h"

namespace skr {

cudaError_t launch_chain_f32(const ChainArgs &a, int nclusters, int cs, int threads, size_t smem,
                             cudaStream_t st) {
    return chain_launch<float>(a, nclusters, cs, threads, smem, st);
}

int max_active_clusters_f32(int cs, int threads, size_t smem) {
    return chain_max_clusters<float>(cs, threads, smem);
}

size_t chain_smem_bytes(int m, int k, int threads, int esz) { return plan_bytes(make_plan(m, k, threads, esz)); }

int chain_threads() { return CHAIN_THREADS; }

}  // namespace skr
