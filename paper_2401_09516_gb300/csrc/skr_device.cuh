// Device utilities shared by the SKR kernels: 16-byte vector types, warp /
// CTA / cluster reductions with a fixed summation order, and the cluster
// primitives (barrier, distributed shared memory).
//
// Every reduction sums in an order that depends only on the data layout
// (lane butterfly, then warps in index order, then cluster ranks in index
// order), never on timing, so that all CTAs of a cluster obtain bit-identical
// results and runs are reproducible.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace skr {

namespace cg = cooperative_groups;

// ---------------------------------------------------------------- vectors
template <typename T> struct Vec;
template <> struct Vec<float> {
    typedef float4 type;
    static constexpr int N = 4;
};
template <> struct Vec<double> {
    typedef double2 type;
    static constexpr int N = 2;
};

__device__ __forceinline__ float vdot(const float4 a, const float4 b) {
    return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
__device__ __forceinline__ double vdot(const double2 a, const double2 b) {
    return a.x * b.x + a.y * b.y;
}
// a - s * b
__device__ __forceinline__ float4 vaxmy(const float4 a, float s, const float4 b) {
    return make_float4(a.x - s * b.x, a.y - s * b.y, a.z - s * b.z, a.w - s * b.w);
}
__device__ __forceinline__ double2 vaxmy(const double2 a, double s, const double2 b) {
    return make_double2(a.x - s * b.x, a.y - s * b.y);
}
// a + s * b
__device__ __forceinline__ float4 vaxpy(const float4 a, float s, const float4 b) {
    return make_float4(a.x + s * b.x, a.y + s * b.y, a.z + s * b.z, a.w + s * b.w);
}
__device__ __forceinline__ double2 vaxpy(const double2 a, double s, const double2 b) {
    return make_double2(a.x + s * b.x, a.y + s * b.y);
}
__device__ __forceinline__ float4 vscale(const float4 a, float s) {
    return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}
__device__ __forceinline__ double2 vscale(const double2 a, double s) {
    return make_double2(a.x * s, a.y * s);
}
__device__ __forceinline__ float4 vzero(float) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ double2 vzero(double) { return make_double2(0.0, 0.0); }

// ---------------------------------------------------------------- reductions
template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
__device__ __forceinline__ int num_warps() { return blockDim.x >> 5; }

// Sum acc[0..nv) over the CTA.  wsum: scratch of num_warps()*NV values.
// Result: out[i] for i < nv (visible to all threads on return).
template <int NV, typename R>
__device__ __forceinline__ void block_sum(const R (&acc)[NV], int nv, R *wsum, R *out) {
    const int lane = lane_id(), w = warp_id(), nw = num_warps();
#pragma unroll
    for (int i = 0; i < NV; i++) {
        if (i < nv) {
            R v = warp_sum(acc[i]);
            if (lane == 0) wsum[w * NV + i] = v;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        R s = R(0);
        for (int q = 0; q < nw; q++) s += wsum[q * NV + i];
        out[i] = s;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- cluster
__device__ __forceinline__ unsigned cl_rank() { return cg::this_cluster().block_rank(); }
__device__ __forceinline__ unsigned cl_size() { return cg::this_cluster().num_blocks(); }
__device__ __forceinline__ void cl_sync() { cg::this_cluster().sync(); }
template <typename P>
__device__ __forceinline__ P *cl_map(P *p, unsigned rank) {
    return cg::this_cluster().map_shared_rank(p, rank);
}

// ---------------------------------------------------------------- TMA
// Tiled bulk copies global -> shared through the tensor memory accelerator,
// completing on an mbarrier with a transaction count.
__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// make barrier initialisation visible to the async proxy
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// arrive once and announce `bytes` of incoming transactions for this phase
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// TMA load of the box at (x, y) of a 2D tensor map (param-space address of
// a __grid_constant__ descriptor) into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *map, int x, int y, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Hint: fetch `bytes` (a multiple of 16) of global memory from the 16-byte
// aligned address p into L2 ahead of use; nothing waits for it.
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(bytes)
                 : "memory");
}
// Order this thread's earlier generic-proxy global writes before later
// async-proxy (bulk copy) reads of the same addresses.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Device clock in nanoseconds.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of an mbarrier, for at most limit_ns; false when
// the limit ran out (the caller records the stall and carries on).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

}  // namespace skr
