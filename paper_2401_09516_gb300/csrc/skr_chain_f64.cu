// FP64 form: every Krylov vector and reduction in FP64.
#include "skr_chain_launch.cuh"
#include "skr_launch.h"

namespace skr {

cudaError_t launch_chain_f64(const ChainArgs &a, int nclusters, int cs, int threads, size_t smem,
                             cudaStream_t st) {
    return chain_launch<double>(a, nclusters, cs, threads, smem, st);
}

int max_active_clusters_f64(int cs, int threads, size_t smem) {
    return chain_max_clusters<double>(cs, threads, smem);
}

}  // namespace skr
