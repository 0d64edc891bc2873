// Greedy nearest-neighbour sort (Algorithm 1, Sec. 4.1) on the device.
//
// Phase 1 computes every pairwise squared distance ||P(i) - P(j)||_F^2 in
// one fixed summation order, so the result is bit-identical to any other
// implementation of the same order: element t of the flattened parameter
// array goes to lane t mod 256; each lane adds its squares left to right
// with separately rounded multiply and add (no fused multiply-add); the 256
// lane sums are then combined pairwise, lane l with lane l + half for
// half = 128, 64, ..., 1.  A CTA handles a 4 x 4 tile of pairs, reusing
// each loaded row for four pairs.
//
// Phase 2 runs the greedy chain in one CTA: N-1 rounds of "argmin over the
// systems not yet placed", keeping the first strictly smaller distance in
// ascending index order (ties go to the lowest index), as Algorithm 1 does.
#pragma once

#include "skr_device.cuh"

namespace skr {

constexpr int SORT_LANES = 256;
constexpr int SORT_TILE = 4;

// dist: N x N, row-major; only tiles with bi <= bj are computed, both
// (i, j) and (j, i) are written (the order makes them bit-identical).
// err: set to 1 if a distance is not finite.
__global__ void __launch_bounds__(SORT_LANES) sort_dist_kernel(const double *__restrict__ P, long long N,
                                                                long long p, double *__restrict__ dist,
                                                                int *err) {
    __shared__ double part[SORT_TILE * SORT_TILE][SORT_LANES];
    const long long ntile = (N + SORT_TILE - 1) / SORT_TILE;
    // map blockIdx.x to (bi, bj) with bi <= bj
    long long t = blockIdx.x, bi = 0;
    while (t >= ntile - bi) {
        t -= ntile - bi;
        bi++;
    }
    const long long bj = bi + t;
    const int lane = threadIdx.x;
    double acc[SORT_TILE][SORT_TILE];
#pragma unroll
    for (int a = 0; a < SORT_TILE; a++)
#pragma unroll
        for (int b = 0; b < SORT_TILE; b++) acc[a][b] = 0.0;
    long long ri[SORT_TILE], rj[SORT_TILE];
#pragma unroll
    for (int a = 0; a < SORT_TILE; a++) {
        ri[a] = min(bi * SORT_TILE + a, N - 1);
        rj[a] = min(bj * SORT_TILE + a, N - 1);
    }
    for (long long e = lane; e < p; e += SORT_LANES) {
        double xi[SORT_TILE], xj[SORT_TILE];
#pragma unroll
        for (int a = 0; a < SORT_TILE; a++) {
            xi[a] = P[ri[a] * p + e];
            xj[a] = P[rj[a] * p + e];
        }
#pragma unroll
        for (int a = 0; a < SORT_TILE; a++)
#pragma unroll
            for (int b = 0; b < SORT_TILE; b++) {
                const double d = __dsub_rn(xi[a], xj[b]);
                acc[a][b] = __dadd_rn(acc[a][b], __dmul_rn(d, d));
            }
    }
#pragma unroll
    for (int a = 0; a < SORT_TILE; a++)
#pragma unroll
        for (int b = 0; b < SORT_TILE; b++) part[a * SORT_TILE + b][lane] = acc[a][b];
    __syncthreads();
    for (int half = SORT_LANES / 2; half >= 1; half >>= 1) {
        if (lane < half) {
#pragma unroll
            for (int e = 0; e < SORT_TILE * SORT_TILE; e++)
                part[e][lane] = __dadd_rn(part[e][lane], part[e][lane + half]);
        }
        __syncthreads();
    }
    if (lane < SORT_TILE * SORT_TILE) {
        const int a = lane / SORT_TILE, b = lane % SORT_TILE;
        const long long i = bi * SORT_TILE + a, j = bj * SORT_TILE + b;
        if (i < N && j < N) {
            const double v = part[lane][0];
            if (!isfinite(v)) atomicExch(err, 1);
            dist[i * N + j] = v;
            dist[j * N + i] = v;
        }
    }
}

// Greedy chain over the distance matrix.  One CTA; taken: N bytes scratch.
__global__ void __launch_bounds__(1024) sort_chain_kernel(const double *__restrict__ dist, long long N,
                                                          long long start, int *perm, unsigned char *taken) {
    __shared__ double bv[32];
    __shared__ long long bi[32];
    __shared__ long long cur;
    for (long long j = threadIdx.x; j < N; j += blockDim.x) taken[j] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        perm[0] = (int)start;
        taken[start] = 1;
        cur = start;
    }
    __syncthreads();
    for (long long step = 1; step < N; step++) {
        const long long i0 = cur;
        double best = INFINITY;
        long long bidx = N;
        for (long long j = threadIdx.x; j < N; j += blockDim.x) {
            if (!taken[j]) {
                const double d = dist[i0 * N + j];
                if (d < best || (d == best && j < bidx)) {
                    best = d;
                    bidx = j;
                }
            }
        }
        // lexicographic (value, index) minimum: warp, then CTA
        for (int off = 16; off >= 1; off >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, off);
            const long long oi = __shfl_xor_sync(0xffffffffu, bidx, off);
            if (ov < best || (ov == best && oi < bidx)) {
                best = ov;
                bidx = oi;
            }
        }
        if (lane_id() == 0) {
            bv[warp_id()] = best;
            bi[warp_id()] = bidx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = INFINITY;
            long long ix = N;
            for (int w = 0; w < num_warps(); w++)
                if (bv[w] < b || (bv[w] == b && bi[w] < ix)) {
                    b = bv[w];
                    ix = bi[w];
                }
            if (ix >= N) {
                // only infinite distances remain: take the lowest untaken index
                for (long long j = 0; j < N; j++)
                    if (!taken[j]) {
                        ix = j;
                        break;
                    }
            }
            perm[step] = (int)ix;
            taken[ix] = 1;
            cur = ix;
        }
        __syncthreads();
    }
}

}  // namespace skr
