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

// Squared distances of a 4 x 4 tile of pairs (rows ri[a], rj[b] of P) in
// the fixed order above.  Called by all SORT_LANES threads of a CTA; part is
// SORT_TILE^2 x SORT_LANES shared doubles.  On return part[a * 4 + b][0]
// holds ||P(ri[a]) - P(rj[b])||^2 on every thread.
__device__ __forceinline__ void tile_sqdist(const double *__restrict__ P, long long p, const long long *ri,
                                            const long long *rj, double (*part)[SORT_LANES]) {
    const int lane = threadIdx.x;
    double acc[SORT_TILE][SORT_TILE];
#pragma unroll
    for (int a = 0; a < SORT_TILE; a++)
#pragma unroll
        for (int b = 0; b < SORT_TILE; b++) acc[a][b] = 0.0;
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
}

// Tile (bi, bj), bi <= bj, of a triangle of ntile x ntile tiles numbered row
// by row: tile t of row bi is (bi, bi + t).
__device__ __forceinline__ void triangle_tile(long long t, long long ntile, long long &bi, long long &bj) {
    // rows before row b hold b * ntile - b (b - 1) / 2 tiles; start from the
    // real root and correct by whole rows
    const double nt = (double)ntile;
    long long b = (long long)floor(nt + 0.5 - sqrt((nt + 0.5) * (nt + 0.5) - 2.0 * (double)t));
    b = max(0LL, min(b, ntile - 1));
    auto before = [ntile](long long r) { return r * ntile - r * (r - 1) / 2; };
    while (b > 0 && before(b) > t) b--;
    while (b + 1 < ntile && before(b + 1) <= t) b++;
    bi = b;
    bj = b + (t - before(b));
}

// dist: N x N, row-major; only tiles with bi <= bj are computed, both
// (i, j) and (j, i) are written (the order makes them bit-identical).
// err: set to 1 if a distance is not finite.
__global__ void __launch_bounds__(SORT_LANES) sort_dist_kernel(const double *__restrict__ P, long long N,
                                                                long long p, double *__restrict__ dist,
                                                                int *err) {
    __shared__ double part[SORT_TILE * SORT_TILE][SORT_LANES];
    const long long ntile = (N + SORT_TILE - 1) / SORT_TILE;
    long long bi, bj;
    triangle_tile(blockIdx.x, ntile, bi, bj);
    long long ri[SORT_TILE], rj[SORT_TILE];
#pragma unroll
    for (int a = 0; a < SORT_TILE; a++) {
        ri[a] = min(bi * SORT_TILE + a, N - 1);
        rj[a] = min(bj * SORT_TILE + a, N - 1);
    }
    tile_sqdist(P, p, ri, rj, part);
    const int lane = threadIdx.x;
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

// Greedy chain over an N x N distance matrix, run by one CTA (any multiple
// of 32 threads up to 1024): N-1 rounds of "argmin over the systems not yet
// placed", the first strictly smaller distance in ascending index order.
// perm[step] = map[chosen] (or the chosen index when map is NULL);
// taken: N bytes of scratch.
__device__ void greedy_chain(const double *__restrict__ dist, long long N, long long start,
                             const int *__restrict__ map, int *perm, unsigned char *taken) {
    __shared__ double bv[32];
    __shared__ long long bi[32];
    __shared__ long long cur;
    for (long long j = threadIdx.x; j < N; j += blockDim.x) taken[j] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        perm[0] = map ? map[start] : (int)start;
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
            perm[step] = map ? map[ix] : (int)ix;
            taken[ix] = 1;
            cur = ix;
        }
        __syncthreads();
    }
}

// Greedy chain over the whole distance matrix.  One CTA; taken: N bytes.
__global__ void __launch_bounds__(1024) sort_chain_kernel(const double *__restrict__ dist, long long N,
                                                          long long start, int *perm, unsigned char *taken) {
    greedy_chain(dist, N, start, nullptr, perm, taken);
}

// ------------------------------------------------------------------ large-N grouped sort
//
// For N in the thousands and beyond (Sec. 4.1, after Algorithm 1): the
// systems are divided into groups of at most G by recursive coordinate
// bisection, Algorithm 1 runs inside every group, and the groups' orders
// are concatenated.  A set of s > G systems is split along the coordinate
// (entry of the flattened parameter array) of largest spread max - min over
// the set, lowest coordinate on ties; with the set ordered by (value,
// index), the first floor(s/2) systems form the first half.  Inside a group
// the scan order is ascending index and the chain starts at the group's
// lowest index.  The sizes of all sets follow from N and G alone, so the
// host knows every set's offset in the working index array; only which
// systems land in a set depends on the data.

// err = 1 if any of the n values is not finite.
__global__ void finite_kernel(const double *__restrict__ P, long long n, int *err) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        if (!isfinite(P[e])) atomicExch(err, 1);
}

__global__ void iota_kernel(int *idx, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) idx[i] = (int)i;
}

// Order-preserving map of a double onto an unsigned integer (for atomic
// min / max); -0.0 maps below +0.0, which leaves max - min unchanged.
__device__ __forceinline__ unsigned long long ordered_key(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ULL);
}
__device__ __forceinline__ double ordered_value(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffULL) : ~k));
}

__global__ void spread_init_kernel(unsigned long long *mn, unsigned long long *mx, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) {
        mn[i] = ~0ULL;
        mx[i] = 0ULL;
    }
}

constexpr int SPREAD_THREADS = 256;
constexpr int SPREAD_CHUNK = 64;   // systems per block

// Per-coordinate min and max over the systems of nn sets.  Set q holds
// idx[off[q] .. off[q] + size[q]); blockIdx.x = q * cps + chunk (cps chunks
// of SPREAD_CHUNK systems per set), blockIdx.y = coordinate tile.  mn, mx:
// nn x p ordered keys.
__global__ void __launch_bounds__(SPREAD_THREADS) spread_kernel(const double *__restrict__ P, long long p,
                                                                const int *__restrict__ idx,
                                                                const long long *__restrict__ off,
                                                                const long long *__restrict__ size, long long cps,
                                                                unsigned long long *mn, unsigned long long *mx) {
    const long long q = blockIdx.x / cps, ch = blockIdx.x % cps;
    const long long t = (long long)blockIdx.y * SPREAD_THREADS + threadIdx.x;
    const long long i0 = ch * SPREAD_CHUNK, i1 = min(size[q], i0 + SPREAD_CHUNK);
    if (t >= p || i0 >= i1) return;
    unsigned long long lo = ~0ULL, hi = 0ULL;
    for (long long i = i0; i < i1; i++) {
        const unsigned long long k = ordered_key(P[(long long)idx[off[q] + i] * p + t]);
        lo = min(lo, k);
        hi = max(hi, k);
    }
    atomicMin(&mn[q * p + t], lo);
    atomicMax(&mx[q * p + t], hi);
}

// coord[slot[q]] = the coordinate of largest spread of set q (lowest on
// ties).  One CTA per set.
__global__ void __launch_bounds__(SPREAD_THREADS) spread_argmax_kernel(const unsigned long long *mn,
                                                                       const unsigned long long *mx, long long p,
                                                                       const long long *__restrict__ slot,
                                                                       int *coord) {
    __shared__ double sv[SPREAD_THREADS / 32];
    __shared__ long long st[SPREAD_THREADS / 32];
    const long long q = blockIdx.x;
    double best = -INFINITY;
    long long bt = p;
    for (long long t = threadIdx.x; t < p; t += SPREAD_THREADS) {
        const double s = ordered_value(mx[q * p + t]) - ordered_value(mn[q * p + t]);
        if (s > best) {   // t ascends per thread: the first maximum is kept
            best = s;
            bt = t;
        }
    }
    for (int o = 16; o >= 1; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const long long ot = __shfl_xor_sync(0xffffffffu, bt, o);
        if (ov > best || (ov == best && ot < bt)) {
            best = ov;
            bt = ot;
        }
    }
    if (lane_id() == 0) {
        sv[warp_id()] = best;
        st[warp_id()] = bt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = -INFINITY;
        long long x = p;
        for (int w = 0; w < SPREAD_THREADS / 32; w++)
            if (sv[w] > b || (sv[w] == b && st[w] < x)) {
                b = sv[w];
                x = st[w];
            }
        coord[slot[q]] = (int)(x < p ? x : 0);
    }
}

// Sort key of one working position: its set, the value of the set's split
// coordinate (0 for a set that is not split), the system index.
struct GroupKey {
    double v;
    int set;
    int idx;
};

__device__ __forceinline__ bool key_less(const GroupKey &a, const GroupKey &b) {
    if (a.set != b.set) return a.set < b.set;
    if (a.v < b.v) return true;
    if (b.v < a.v) return false;
    return a.idx < b.idx;
}

// keys[i] for positions i < M; positions >= N are padding that sorts last.
// off: nn + 1 set offsets; coord[q] < 0: set q is not split.
__global__ void group_keys_kernel(const double *__restrict__ P, long long p, const int *__restrict__ idx,
                                  long long N, long long M, const long long *__restrict__ off, int nn,
                                  const int *__restrict__ coord, GroupKey *keys) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= M) return;
    GroupKey k;
    if (i < N) {
        int lo = 0, hi = nn - 1;   // the set q with off[q] <= i < off[q + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const int c = coord[lo];
        k.set = lo;
        k.idx = idx[i];
        k.v = (c >= 0) ? P[(long long)k.idx * p + c] : 0.0;
    } else {
        k.set = 0x7fffffff;
        k.idx = 0x7fffffff;
        k.v = 0.0;
    }
    keys[i] = k;
}

constexpr int BITONIC_LOCAL = 1024;   // keys per CTA in the shared-memory stages

__device__ __forceinline__ void bitonic_pair(GroupKey *a, long long base, int q, long long k, long long j) {
    const long long i = 2 * j * (q / j) + (q % j), l = i + j;
    const bool up = ((base + i) & k) == 0;
    const GroupKey x = a[i], y = a[l];
    if (up ? key_less(y, x) : key_less(x, y)) {
        a[i] = y;
        a[l] = x;
    }
}

// Stages with partner distance j < BITONIC_LOCAL in shared memory: kfix = 0
// runs every stage k <= BITONIC_LOCAL; otherwise the steps j = 512 .. 1 of
// stage kfix.  BITONIC_LOCAL / 2 threads.
__global__ void __launch_bounds__(BITONIC_LOCAL / 2) bitonic_local_kernel(GroupKey *keys, long long kfix) {
    __shared__ GroupKey s[BITONIC_LOCAL];
    const long long base = (long long)blockIdx.x * BITONIC_LOCAL;
    const int t = threadIdx.x;
    s[t] = keys[base + t];
    s[t + BITONIC_LOCAL / 2] = keys[base + t + BITONIC_LOCAL / 2];
    __syncthreads();
    if (kfix == 0) {
        for (long long k = 2; k <= BITONIC_LOCAL; k <<= 1)
            for (long long j = k >> 1; j > 0; j >>= 1) {
                bitonic_pair(s, base, t, k, j);
                __syncthreads();
            }
    } else {
        for (long long j = BITONIC_LOCAL / 2; j > 0; j >>= 1) {
            bitonic_pair(s, base, t, kfix, j);
            __syncthreads();
        }
    }
    keys[base + t] = s[t];
    keys[base + t + BITONIC_LOCAL / 2] = s[t + BITONIC_LOCAL / 2];
}

// One step (k, j), j >= BITONIC_LOCAL, over all M / 2 pairs.
__global__ void bitonic_global_kernel(GroupKey *keys, long long M, long long k, long long j) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= M / 2) return;
    const long long i = 2 * j * (q / j) + (q % j), l = i + j;
    const bool up = (i & k) == 0;
    const GroupKey x = keys[i], y = keys[l];
    if (up ? key_less(y, x) : key_less(x, y)) {
        keys[i] = y;
        keys[l] = x;
    }
}

__global__ void keys_to_idx_kernel(const GroupKey *keys, long long N, int *idx) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < N) idx[i] = keys[i].idx;
}

// Pairwise squared distances inside every group.  Group g holds
// idx[goff[g] .. goff[g + 1]) (ascending system index); its s x s matrix
// (row-major, local indices) starts at dist + doff[g]; its tiles are blocks
// boff[g] .. boff[g + 1) of the grid.
__global__ void __launch_bounds__(SORT_LANES) group_dist_kernel(const double *__restrict__ P, long long p,
                                                                const int *__restrict__ idx,
                                                                const long long *__restrict__ goff,
                                                                const long long *__restrict__ boff,
                                                                const long long *__restrict__ doff, int ng,
                                                                double *__restrict__ dist, int *err) {
    __shared__ double part[SORT_TILE * SORT_TILE][SORT_LANES];
    const long long blk = blockIdx.x;
    int lo = 0, hi = ng - 1;   // the group g with boff[g] <= blk < boff[g + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (boff[mid] <= blk) lo = mid;
        else hi = mid - 1;
    }
    const int g = lo;
    const long long s = goff[g + 1] - goff[g];
    const long long ntile = (s + SORT_TILE - 1) / SORT_TILE;
    long long bi, bj;
    triangle_tile(blk - boff[g], ntile, bi, bj);
    long long ri[SORT_TILE], rj[SORT_TILE];
#pragma unroll
    for (int a = 0; a < SORT_TILE; a++) {
        ri[a] = idx[goff[g] + min(bi * SORT_TILE + a, s - 1)];
        rj[a] = idx[goff[g] + min(bj * SORT_TILE + a, s - 1)];
    }
    tile_sqdist(P, p, ri, rj, part);
    const int lane = threadIdx.x;
    if (lane < SORT_TILE * SORT_TILE) {
        const int a = lane / SORT_TILE, b = lane % SORT_TILE;
        const long long i = bi * SORT_TILE + a, j = bj * SORT_TILE + b;
        if (i < s && j < s) {
            const double v = part[lane][0];
            if (!isfinite(v)) atomicExch(err, 1);
            dist[doff[g] + i * s + j] = v;
            dist[doff[g] + j * s + i] = v;
        }
    }
}

// Short parameter vectors (p <= SORT_SMALL_P): every lane of the fixed
// order holds at most one term, lanes p .. 255 hold +0, and the rounds of
// the lane tree with half >= P2 (the power of two >= p) add exact zeros.
// One thread then reproduces the order for one pair in registers: the p
// terms, then the rounds P2/2 .. 1.  FP64 issue, not memory, bounds this
// work on this GPU, and a thread per pair shares each FP64 instruction among
// 32 pairs.  One CTA per row a of a group, its threads over the rows
// b >= a of the group; writes both (a, b) and (b, a).  Groups: rows
// goff[g] .. goff[g + 1) of idx (system indices), matrix at dist + doff[g];
// ng = 0: one group, rows 0 .. nrows of the identity, matrix at dist.
constexpr int SORT_SMALL_P = 32;
template <int P2>
__global__ void __launch_bounds__(256) pair_dist_small_kernel(const double *__restrict__ P, long long p,
                                                              const int *__restrict__ idx,
                                                              const long long *__restrict__ goff,
                                                              const long long *__restrict__ doff, int ng,
                                                              long long nrows, double *__restrict__ dist,
                                                              int *err) {
    const long long row = blockIdx.x;
    if (row >= nrows) return;
    long long base = 0, s = nrows, dof = 0;
    if (ng > 0) {
        int lo = 0, hi = ng - 1;   // the group g with goff[g] <= row < goff[g + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (goff[mid] <= row) lo = mid;
            else hi = mid - 1;
        }
        base = goff[lo];
        s = goff[lo + 1] - base;
        dof = doff[lo];
    }
    const long long a = row - base;
    const long long ri = idx ? idx[row] : row;
    double xi[P2];
#pragma unroll
    for (int t = 0; t < P2; t++) xi[t] = (t < p) ? P[ri * p + t] : 0.0;
    for (long long b = a + threadIdx.x; b < s; b += blockDim.x) {
        const long long rj = idx ? idx[base + b] : base + b;
        double v[P2];
#pragma unroll
        for (int t = 0; t < P2; t++) {
            double acc = 0.0;
            if (t < p) {
                const double d = __dsub_rn(xi[t], P[rj * p + t]);
                acc = __dadd_rn(acc, __dmul_rn(d, d));
            }
            v[t] = acc;
        }
#pragma unroll
        for (int half = P2 / 2; half >= 1; half >>= 1)
#pragma unroll
            for (int l = 0; l < half; l++) v[l] = __dadd_rn(v[l], v[l + half]);
        if (!isfinite(v[0])) atomicExch(err, 1);
        dist[dof + a * s + b] = v[0];
        dist[dof + b * s + a] = v[0];
    }
}

// Launch of the kernel above for p <= SORT_SMALL_P.
inline void launch_pair_dist_small(const double *P, long long p, const int *idx, const long long *goff,
                                   const long long *doff, int ng, long long nrows, double *dist, int *err,
                                   cudaStream_t st) {
    const unsigned grid = (unsigned)nrows;
    if (p <= 1) pair_dist_small_kernel<1><<<grid, 256, 0, st>>>(P, p, idx, goff, doff, ng, nrows, dist, err);
    else if (p <= 2) pair_dist_small_kernel<2><<<grid, 256, 0, st>>>(P, p, idx, goff, doff, ng, nrows, dist, err);
    else if (p <= 4) pair_dist_small_kernel<4><<<grid, 256, 0, st>>>(P, p, idx, goff, doff, ng, nrows, dist, err);
    else if (p <= 8) pair_dist_small_kernel<8><<<grid, 256, 0, st>>>(P, p, idx, goff, doff, ng, nrows, dist, err);
    else if (p <= 16) pair_dist_small_kernel<16><<<grid, 256, 0, st>>>(P, p, idx, goff, doff, ng, nrows, dist, err);
    else pair_dist_small_kernel<32><<<grid, 256, 0, st>>>(P, p, idx, goff, doff, ng, nrows, dist, err);
}

// Algorithm 1 inside every group (one CTA per group), from the group's
// lowest index; writes perm[goff[g] ..) as system indices.
__global__ void __launch_bounds__(256) group_chain_kernel(const double *__restrict__ dist,
                                                          const long long *__restrict__ doff,
                                                          const long long *__restrict__ goff,
                                                          const int *__restrict__ idx, int *perm,
                                                          unsigned char *taken) {
    const int g = blockIdx.x;
    const long long o = goff[g], s = goff[g + 1] - o;
    greedy_chain(dist + doff[g], s, 0, idx + o, perm + o, taken + o);
}

}  // namespace skr
