// Launch helpers for chain_kernel<T> (cluster launch, attributes, occupancy).
#pragma once

#include "skr_chain.cuh"

namespace skr {

template <typename T>
static cudaError_t chain_set_attributes(int cs, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(chain_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    if (cs > 8) e = cudaFuncSetAttribute(chain_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

static inline void chain_config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *at, int nclusters, int cs,
                                int threads, size_t smem, cudaStream_t st) {
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3(nclusters * cs);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
}

template <typename T>
static cudaError_t chain_launch(const ChainArgs &a, int nclusters, int cs, int threads, size_t smem,
                                cudaStream_t st) {
    cudaError_t e = chain_set_attributes<T>(cs, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    chain_config(cfg, at, nclusters, cs, threads, smem, st);
    return cudaLaunchKernelEx(&cfg, chain_kernel<T>, a);
}

template <typename T>
static int chain_max_clusters(int cs, int threads, size_t smem) {
    if (chain_set_attributes<T>(cs, smem) != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    chain_config(cfg, at, 1, cs, threads, smem, 0);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void *)chain_kernel<T>, &cfg) != cudaSuccess) return 0;
    return n;
}

}  // namespace skr
