// The chain kernel: one thread-block cluster solves one chain of systems,
// in order, with GCRO-DR (Algorithm 2) and residual refinement, carrying
// U_k, C_k from each system to the next (App. B).
//
// Work split.  Every vector of a system (x, r, b, the Krylov basis, U_k,
// C_k) is cut into cs contiguous row ranges, one per CTA of the cluster;
// every streaming pass touches only the CTA's own rows.  The only data that
// crosses CTAs are (a) the stencil halo of the operator's input vector,
// read through L2 (ld.global.cg) after a cluster barrier, and (b) partial
// sums, combined through distributed shared memory.  Every CTA then holds
// the same reduced values and runs the small dense step itself, so all
// control decisions are taken identically by every CTA without a broadcast.
//
// Precision: T is the working precision of the Krylov vectors and of their
// reductions (float for the mixed form, double for the FP64 form).  The
// solution, the true residual, the right-hand side and the small dense step
// are always FP64.
#pragma once

#include "skr_common.h"
#include "skr_dense.cuh"
#include "skr_device.cuh"
#include "skr_stencil.cuh"

namespace skr {

template <typename T> struct Tiles;
// Threads per CTA of the chain kernel: 16 warps, one CTA per SM.  The
// streaming passes issue 16-byte loads of up to 32 basis columns per row
// group; measured on GB300 this keeps more bytes in flight than 8 warps
// with more registers, or than register-resident one-element passes.
constexpr int CHAIN_THREADS = 512;
constexpr int CHAIN_MIN_BLOCKS = 1;

template <> struct Tiles<float> {
    static constexpr int TA = 8;   // Gram tile rows (recycle refresh)
    static constexpr int TB = 8;   // Gram tile cols
};
template <> struct Tiles<double> {
    static constexpr int TA = 4;
    static constexpr int TB = 8;
};


template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };

// four consecutive coefficients from shared memory (16-byte aligned)
__device__ __forceinline__ void ld4(const float *p, float &a, float &b, float &c, float &d) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void ld4(const double *p, double &a, double &b, double &c, double &d) {
    const double2 v0 = *reinterpret_cast<const double2 *>(p);
    const double2 v1 = *reinterpret_cast<const double2 *>(p + 2);
    a = v0.x; b = v0.y; c = v1.x; d = v1.y;
}

// Shared-memory layout, computed identically on host and device.
//
// The regions that live through the Arnoldi steps (reductions, H, B, the
// coefficient vectors, the monitor, control ints, mbarriers) come first.
// Behind them one region holds, at different times, either the small dense
// scratch of a cycle end and of a recycle refresh (R_H, the Givens data, F/M,
// the Schur vectors, P_k, the QR factors) or the staging ring of the
// streaming passes; no streaming pass runs while that scratch is live.
struct SmemPlan {
    int m, k, nwarps;
    int ldh, redcap, redsz;   // redsz: one reduction buffer, in doubles
    // offsets in doubles
    int o_red, o_vals, o_wsum, o_H, o_B, o_Rw, o_gvec, o_y2, o_gam, o_avec, o_gc, o_gs, o_dscr, o_F,
        o_Z, o_wr, o_wi, o_xr, o_xi, o_vscr, o_P, o_GP, o_Qc, o_Rc, o_tau, o_D, o_sc, o_Tco, o_mon,
        o_int, o_bar, o_req, o_ring, total;
    // staging ring: ring_cap doubles; a pass with s segments per block of
    // ring_rows rows uses min(RING_MAX_NS, ring_cap / (s segments)) stages
    int ring_cap, ring_rows;
    // offsets inside the T coefficient region (in T elements)
    int t_h, t_cC, t_cU, t_cr, t_cd, t_s, t_al, t_total;
};

__host__ __device__ inline int align2(int x) { return (x + 1) & ~1; }

// Shared memory of one CTA on sm_103 (opt-in maximum) and the staging
// ring's largest depth (one mbarrier per stage; a segment is
// RING_SEG_BYTES, one row of a TMA box).
constexpr int SMEM_LIMIT_BYTES = 227 * 1024;
constexpr int RING_MAX_NS = 8;
// TMA requests per staged block: at most 4 runs of at most MMAX + 1 columns,
// each cut into boxes of 16 columns and a binary remainder.
constexpr int RING_MAX_REQ = 32;
// A staged copy that has not landed after this long is recorded as a stall;
// after a stall, the launch waits this long for copies in flight before it ends.
constexpr unsigned long long RING_WAIT_NS = 2000000000ull;
constexpr unsigned long long RING_DRAIN_NS = 20000000ull;

__host__ __device__ inline SmemPlan make_plan(int m, int k, int nthreads, int esz) {
    SmemPlan P;
    P.m = m;
    P.k = k;
    P.nwarps = nthreads / 32;
    P.ldh = m + 1;
    int rc = 2 * m + 8;   // the Arnoldi step reduces 2 q + 3 <= 2 m + 3 values
    if ((m + 1) * k + 2 * k + 8 > rc) rc = (m + 1) * k + 2 * k + 8;
    if (k * k + 8 > rc) rc = k * k + 8;
    P.redcap = align2(rc);
    P.redsz = align2((P.redcap * esz + 7) / 8);   // reductions are in the working precision
    const int kk = k + 1;
    int o = 0;
    // ---- live through the Arnoldi steps
    P.o_red = o;   o += 2 * P.redsz;
    P.o_vals = o;  o += P.redsz;
    P.o_wsum = o;  o += align2(P.nwarps * 32);
    P.o_H = o;     o += align2(P.ldh * m);
    P.o_B = o;     o += align2(k * m);
    P.o_dscr = o;  o += align2(2 * m + 4);
    // T coefficient region (sized in doubles: T is at most 8 bytes)
    P.t_h = 0;
    P.t_cC = P.t_h + ((m + 4 + 3) & ~3);   // multiple of 4 elements: float4 loads
    const int ks = ((k > 0 ? k : 1) + 3) & ~3;   // padded coefficient row stride
    P.t_cU = P.t_cC + align2((m + 1) * ks);
    P.t_cr = P.t_cU + align2(m * ks);
    P.t_cd = P.t_cr + align2(m + 2);
    P.t_s = (P.t_cd + m + k + 2 + 3) & ~3;   // 16-byte aligned
    P.t_al = P.t_s + ((m + 4 + 3) & ~3);
    P.t_total = P.t_al + ((m + 4 + 3) & ~3);
    // the eigenvector workspace (xr, xi, in the eigen-solve precision: FP64,
    // or FP32 on request in the mixed form, so room for FP64) and the Gram
    // tile buffer live in the coefficient region: it is written only after
    // the eigen-solve
    const int xsz = align2(kk * m);
    int tco = align2(P.t_total);
    if (2 * xsz > tco) tco = 2 * xsz;
    if (tco < 32) tco = 32;
    P.o_Tco = o;   o += tco;
    P.o_xr = P.o_Tco;
    P.o_xi = P.o_Tco + xsz;
    P.o_mon = o;   o += align2(3 * m + 4);             // FP32 Givens monitor (as floats, room to spare)
    P.o_int = o;   o += align2(64 + 8 + 3 * MMAX);      // control ints
    P.o_bar = o;   o += 8;                              // one mbarrier per stage (<= 8)
    P.o_req = o;   o += RING_MAX_REQ * 3 / 2;           // TMA requests of the current pass (3 ints each)
    // ---- shared region, 1024-byte aligned: dense scratch or staging ring
    o = (o + 127) & ~127;
    const int u0 = o;
    P.o_Rw = o;    o += align2(P.ldh * m);
    P.o_gvec = o;  o += align2(m + 2);
    P.o_y2 = o;    o += align2(m + 2);
    P.o_gam = o;   o += align2(m + 2);
    P.o_avec = o;  o += align2(k + 2);
    P.o_gc = o;    o += align2(m + 2);
    P.o_gs = o;    o += align2(m + 2);
    P.o_F = o;     o += align2(P.ldh * (m > k ? m : k));   // F / M; also the refresh Gram
    // Schur vectors (and, in the mixed form, the FP32 eigen-matrix with an
    // odd leading dimension beside them); also R, R^-1 of the refresh
    P.o_Z = o;     o += align2(m * m + m > 2 * k * k ? m * m + m : 2 * k * k);
    P.o_wr = o;    o += align2(m);
    P.o_wi = o;    o += align2(m);
    P.o_vscr = o;  o += align2(m + 2);
    P.o_P = o;     o += align2(m * kk);
    // G P_k and its Q factor are formed after the eigen-solve, when the F/M
    // and R_H regions are free again
    P.o_GP = P.o_F;
    P.o_Qc = P.o_Rw;
    P.o_Rc = o;    o += align2(kk * kk);
    P.o_tau = o;   o += align2(kk + 1);
    P.o_D = o;     o += align2(k + 2);
    P.o_sc = o;    o += 16;
    const int dense_end = o;
    // the ring: at least two stages of the widest pass (m + 2 segments)
    P.o_ring = u0;
    P.ring_rows = RING_SEG_BYTES / esz;
    const int seg = RING_SEG_BYTES / 8;
    // three stages of the widest pass: a larger ring takes L1 capacity from the
    // register-streamed passes and measured slower
    int cap = (SMEM_LIMIT_BYTES / 8 - u0) / seg * seg;
    if (cap > 3 * (m + 2) * seg) cap = 3 * (m + 2) * seg;
    if (cap < 2 * (m + 2) * seg) cap = 2 * (m + 2) * seg;   // the plan then exceeds the limit: refused
    P.ring_cap = cap;
    const int ring_end = u0 + cap;
    P.total = dense_end > ring_end ? dense_end : ring_end;
    return P;
}

__host__ __device__ inline size_t plan_bytes(const SmemPlan &P) { return (size_t)P.total * 8; }

template <typename T>
struct Ctx {
    // cluster and rows
    unsigned rank, cs;
    long long lo, cnt;
    Geom g;
    long long ld;
    // slot buffers
    T *basis;
    double *A64;
    T *Aw;
    double *dinv, *x, *r, *b, *anode;
    int *cols;   // CSR input: the slot's column indices (nullptr without that room)
    // parameters
    int m, k, maxit, precond, pc_blocks;
    int eig32;         // mixed form: harmonic-Ritz eigen-solve in FP32 (opt-in)
    int symc;          // operator kept in the compact symmetric form (sym_compact_form)
    long long pc_bs;   // rows per block of the colour sweeps (n unless block-Jacobi)
    // shared memory
    SmemPlan P;
    double *sm;
    int parity;
    // recycle dimension carried by this chain
    int kc;
    // per-system statistics
    int steps, cycles, matvecs, refinements;
    int updates_since_refresh;   // recycle updates since C = A U was last recomputed
    bool breakdown;
    unsigned long long bytes;
    // optional per-phase device time (rank 0, thread 0)
    unsigned long long *prof;
    unsigned long long tmark;
    // staging ring: stage buffers and one mbarrier per stage
    T *ring;
    unsigned long long *bars;
    unsigned phase;   // bit i: parity of the next phase of mbarrier i
    const CUtensorMap *tmap;        // basis boxes of 16 >> i columns, i < NBOX
    int ybase;                      // first column of this slot in the tensor maps

    // the Hessenberg, Schur form and eigenvector parts of a harmonic-Ritz
    // solve, from the device clock marks it wrote (mk[2] after the Hessenberg
    // reduction, mk[0] after the Schur form, mk[1] after the eigenvectors);
    // call after a tick that closed the phase before it
    __device__ __forceinline__ void tick_eigen(const unsigned long long *mk) {
        if (prof != nullptr && rank == 0 && threadIdx.x == 0) {
            const unsigned long long mh = mk[2] > tmark ? mk[2] : tmark;
            const unsigned long long m0 = mk[0] > mh ? mk[0] : mh;
            const unsigned long long m1 = mk[1] > m0 ? mk[1] : m0;
            atomicAdd(prof + PH_HESS, mh - tmark);
            atomicAdd(prof + PH_SCHUR, m0 - mh);
            atomicAdd(prof + PH_EIGVEC, m1 - m0);
            tmark = m1;
        }
    }

    __device__ __forceinline__ void tick(int ph) {
        if (prof != nullptr && rank == 0 && threadIdx.x == 0) {
            const unsigned long long t = global_ns();
            atomicAdd(prof + ph, t - tmark);
            tmark = t;
        }
    }

    __device__ T *col(int c) const { return basis + (long long)c * ld; }
    __device__ double *D(int off) const { return sm + off; }
    template <typename R>
    __device__ R *red() const { return reinterpret_cast<R *>(sm + P.o_red + parity * P.redsz); }
    template <typename R>
    __device__ R *vals() const { return reinterpret_cast<R *>(sm + P.o_vals); }
    __device__ T *tco(int off) const { return reinterpret_cast<T *>(sm + P.o_Tco) + off; }
    __device__ int *ints() const { return reinterpret_cast<int *>(sm + P.o_int); }
    __device__ float *mon() const { return reinterpret_cast<float *>(sm + P.o_mon); }
};

// Bytes of the column indices one pass over a CSR operator reads (0 for grids).
template <typename T>
__device__ __forceinline__ unsigned long long csr_index_bytes(const Ctx<T> &c) {
    return c.g.cols ? (unsigned long long)c.g.nst * c.g.n * 4 : 0ull;
}

// Arrays of the working-precision operator one pass over it reads.
template <typename T>
__device__ __forceinline__ int op_slots(const Ctx<T> &c) {
    return c.symc ? sym_compact_slots(c.g) : c.g.nst;
}

// Sum the CTA partials red<R>()[0..nv) over the cluster into vals<R>().
// One cluster barrier; the reduction buffers alternate so that the next
// call never overwrites a buffer that another CTA may still be reading.
template <typename T, typename R>
__device__ __forceinline__ void allreduce(Ctx<T> &c, int nv) {
    cl_sync();
    R *src = c.template red<R>();
    R *dst = c.template vals<R>();
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        R s = R(0);
        for (unsigned q = 0; q < c.cs; q++) s += *cl_map(src + i, q);
        dst[i] = s;
    }
    c.parity ^= 1;
    __syncthreads();
}

// ------------------------------------------------------------------ streaming passes

// ------------------------------------------------------------------ staged streaming

// Control int set when a staged copy did not land within RING_WAIT_NS.
constexpr int INT_STALL = 6;

// A pass that streams the CTA's own rows of up to four runs of contiguous
// basis columns through the shared-memory ring.  For every block of
// R = RING_SEG_BYTES / sizeof(T) rows, warp 0 issues TMA boxes of {R rows x
// 16 columns} and a binary remainder of narrower boxes (one box per lane)
// onto the stage's mbarrier, ns - 1 blocks ahead of the block being
// consumed, so the bytes in flight do not depend on registers; ns is as
// large as the ring allows for this pass's stage size.  In a stage, the runs' columns follow
// each other, one segment (R elements) per column.  Use:
//   RingPass rp = ring_begin(c, ...);
//   for (b = 0; b < rp.nblk; b++) { sb = ring_acquire(c, rp, b); ...; __syncthreads(); }
//   ring_end(c, rp);
// Each pass starts at stage 0 and consumes every block it issues, so the
// ring is empty between passes.
struct RingPass {
    int nseg, nreq, nblk, ns, stage_elems;
};

// Request i of the current pass: ints (segment, column, box index) at
// ints + 3 i of the plan's request table.
template <typename T>
__device__ __forceinline__ int *ring_reqs(Ctx<T> &c) {
    return reinterpret_cast<int *>(c.sm + c.P.o_req);
}

template <typename T>
__device__ __forceinline__ void ring_issue(Ctx<T> &c, const RingPass &rp, int blk) {
    constexpr int R = RING_SEG_BYTES / (int)sizeof(T);
    const int lane = lane_id();
    if (c.ints()[INT_STALL]) return;   // after a stall nothing more is staged
    const int st = blk % rp.ns;
    T *dst = c.ring + (long long)st * rp.stage_elems;
    const int x = (int)(c.lo + (long long)blk * R);
    if (lane == 0) mbar_arrive_expect(c.bars + st, (unsigned)(rp.nseg * R * (int)sizeof(T)));
    __syncwarp();
    if (lane < rp.nreq) {   // one request per lane
        const int *rq = ring_reqs(c) + 3 * lane;
        tma_load_2d(dst + rq[0] * R, c.tmap + rq[2], x, c.ybase + rq[1], c.bars + st);
    }
}

// Start a pass over the runs (start, length) given in rs/rl (length 0: skipped).
template <typename T>
__device__ __forceinline__ RingPass ring_begin_runs(Ctx<T> &c, const int *rs, const int *rl, int nr) {
    constexpr int R = RING_SEG_BYTES / (int)sizeof(T);
    RingPass rp;
    int nseg = 0, nreq = 0;
    int *rq = ring_reqs(c);
    // boxes of 16 columns, then a binary remainder (the same on every thread)
    auto add = [&](int seg, int col, int w) {
        if (threadIdx.x == 0 && nreq < RING_MAX_REQ) {
            rq[3 * nreq] = seg;
            rq[3 * nreq + 1] = col;
            rq[3 * nreq + 2] = w;
        }
        nreq++;
    };
    for (int i = 0; i < nr; i++) {
        if (rl[i] <= 0) continue;
        int off = 0;
        for (; rl[i] - off >= 16; off += 16) add(nseg + off, rs[i] + off, 0);
        for (int w = 1; w < NBOX; w++) {   // remainder < 16: each narrower width at most once
            const int width = 16 >> w;
            if (rl[i] - off >= width) {
                add(nseg + off, rs[i] + off, w);
                off += width;
            }
        }
        nseg += rl[i];
    }
    rp.nseg = nseg;
    rp.nreq = nreq;
    rp.nblk = (int)((c.cnt + R - 1) / R);
    rp.stage_elems = rp.nseg * R;
    // as many stages of exactly this pass's segments as the ring holds
    const int cap_elems = (int)((long long)c.P.ring_cap * 8 / (long long)sizeof(T));
    rp.ns = min(RING_MAX_NS, cap_elems / max(rp.stage_elems, 1));
    // the columns were written by generic stores of this CTA's threads; the
    // barrier also publishes the request table
    fence_proxy_async_global();
    __syncthreads();
    if (warp_id() == 0)
        for (int b0 = 0; b0 < rp.ns - 1 && b0 < rp.nblk; b0++) ring_issue(c, rp, b0);
    return rp;
}

// q columns from c0, then the single columns xc0 and xc1 (-1: none).
template <typename T>
__device__ __forceinline__ RingPass ring_begin(Ctx<T> &c, int c0, int q, int xc0, int xc1) {
    const int rs[3] = {c0, xc0, xc1};
    const int rl[3] = {q, xc0 >= 0 ? 1 : 0, xc1 >= 0 ? 1 : 0};
    return ring_begin_runs(c, rs, rl, 3);
}

// Issue the block ns - 1 ahead, wait for block b0; returns its stage.  The
// caller ends its use of the stage with a CTA barrier.
template <typename T>
__device__ __forceinline__ const T *ring_acquire(Ctx<T> &c, const RingPass &rp, int b0) {
    if (warp_id() == 0 && b0 + rp.ns - 1 < rp.nblk) ring_issue(c, rp, b0 + rp.ns - 1);
    const int st = b0 % rp.ns;
    // after a stall the waits are skipped: the launch finishes quickly and
    // every later system of this CTA is flagged
    if (c.ints()[INT_STALL] == 0 && !mbar_wait_bounded(c.bars + st, (c.phase >> st) & 1u, RING_WAIT_NS))
        c.ints()[INT_STALL] = 1;
    c.phase ^= 1u << st;
    return c.ring + (long long)st * rp.stage_elems;
}

template <typename T>
__device__ __forceinline__ void ring_end(Ctx<T> &c, const RingPass &rp) {
    c.bytes += (unsigned long long)rp.nseg * c.g.n * sizeof(T);
}

// CTA partials of the dots of one Arnoldi step with delayed
// re-orthogonalisation, over own rows, for the q basis columns Z from c0:
//   out[0..q) = Z^T u (if DU), out[q..2q) = Z^T w (if DW),
//   out[2q] = u.u (if DU), out[2q+1] = u.w (if DW), out[2q+2] = w.w (if DW).
// u (column ucol) is the not yet re-orthogonalised candidate, w (column
// wcol) = A M^-1 u.  The rows stream through the ring.  A staged block holds
// 64 16-byte vectors per column; thread t owns vector t % 64 of every block
// and the columns j = t / 64 (mod 8), so each shared-memory load feeds
// 2 x E multiply-adds.  Each column's partial is then the sum over its
// group's two warps.
template <typename T, bool DU, bool DW>
__device__ void staged_dual_dots(Ctx<T> &c, int c0, int q, int ucol, int wcol, T *out) {
    typedef typename Vec<T>::type VT;
    constexpr int E = Vec<T>::N;
    constexpr int R = RING_SEG_BYTES / (int)sizeof(T);
    constexpr int RV = R / E;                       // vectors per segment
    constexpr int NGRP = CHAIN_THREADS / RV;        // column groups
    constexpr int WPG = RV / 32;                    // warps per group
    constexpr int CM = (MMAX + NGRP - 1) / NGRP;    // columns per thread
    constexpr int NVW = 2 * CM + 3;
    static_assert(RV % 32 == 0 && NGRP >= 1, "ring geometry");
    const int lane = lane_id(), wp = warp_id();
    const int gi = threadIdx.x / RV, vi = threadIdx.x % RV;
    T acc[NVW];
#pragma unroll
    for (int e = 0; e < NVW; e++) acc[e] = T(0);
    const RingPass rp = ring_begin(c, c0, q, ucol, DW ? wcol : -1);
    for (int b0 = 0; b0 < rp.nblk; b0++) {
        const VT *sb = reinterpret_cast<const VT *>(ring_acquire(c, rp, b0));
        // rows of the chunk are a multiple of 8, so whole vectors are valid
        const int nv = (int)(min((long long)R, c.cnt - (long long)b0 * R) / E);
        if (vi < nv) {
            const VT uu = sb[q * RV + vi];
            const VT ww = DW ? sb[(q + 1) * RV + vi] : uu;
#pragma unroll
            for (int jj = 0; jj < CM; jj++) {
                const int j = jj * NGRP + gi;
                if (j < q) {
                    const VT z = sb[j * RV + vi];
                    if (DU) acc[2 * jj] += vdot(z, uu);
                    if (DW) acc[2 * jj + 1] += vdot(z, ww);
                }
            }
            if (gi == 0) {
                if (DU) acc[2 * CM] += vdot(uu, uu);
                if (DW) {
                    acc[2 * CM + 1] += vdot(uu, ww);
                    acc[2 * CM + 2] += vdot(ww, ww);
                }
            }
        }
        __syncthreads();   // the stage may be refilled
    }
    ring_end(c, rp);
    // warp sums, then the warps of each column group in index order
    T *wsum = reinterpret_cast<T *>(c.D(c.P.o_wsum));
#pragma unroll
    for (int e = 0; e < NVW; e++) {
        const T v = warp_sum(acc[e]);
        if (lane == 0) wsum[wp * NVW + e] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * q + 3; e += blockDim.x) {
        int g, slot;
        bool want;
        if (e < 2 * q) {
            const int j = (e < q) ? e : e - q;
            g = j % NGRP;
            slot = 2 * (j / NGRP) + ((e < q) ? 0 : 1);
            want = (e < q) ? DU : DW;
        } else {
            g = 0;   // u.u, u.w, w.w are accumulated by group 0
            slot = 2 * CM + (e - 2 * q);
            want = (e == 2 * q) ? DU : DW;
        }
        if (want) {
            T sacc = T(0);
            for (int r = 0; r < WPG; r++) sacc += wsum[(g * WPG + r) * NVW + slot];
            out[e] = sacc;
        }
    }
    __syncthreads();
}

// The update of one Arnoldi step with delayed re-orthogonalisation, over own
// rows (registers, 16-byte loads): V_j = (u - Z sv) * rinv into column vcol
// and, if NEXT, the next candidate ((w - bet u) - Z al) * rinv into column
// wcol, in place over w.
template <typename T, bool NEXT>
__device__ void dual_update(Ctx<T> &c, int c0, int q, const T *sv, const T *al, T bet, T rinv, int ucol,
                                   int wcol, int vcol) {
    typedef typename Vec<T>::type VT;
    constexpr int E = Vec<T>::N;
    const int nvec = (int)(c.cnt / E);
    const VT *uv = reinterpret_cast<const VT *>(c.col(ucol) + c.lo);
    VT *wv = reinterpret_cast<VT *>(c.col(wcol) + c.lo);
    VT *ov = reinterpret_cast<VT *>(c.col(vcol) + c.lo);
    // the loads of one block of rows per thread are few (one vector per
    // column, eight columns in flight): warp 0 asks L2 for the block two
    // ahead of every column the pass reads, so that the loads find it there
    const int bv = blockDim.x;   // vectors per block of rows
    auto prefetch = [&](int blk) {
        const long long v0 = (long long)blk * bv;
        if (warp_id() != 0 || v0 >= nvec) return;
        const unsigned bytes = (unsigned)(min((long long)bv, (long long)nvec - v0) * sizeof(VT));
        for (int j = lane_id(); j < q + 2; j += 32) {
            const int col = (j < q) ? c0 + j : (j == q ? ucol : wcol);
            if (j == q + 1 && !NEXT) continue;
            prefetch_l2(c.col(col) + c.lo + v0 * E, bytes);
        }
    };
    prefetch(0);
    prefetch(1);
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
        prefetch(i / bv + 2);
        VT vv = uv[i];
        VT nx = vv;
        if (NEXT) nx = vaxmy(wv[i], bet, vv);
#pragma unroll 8
        for (int j = 0; j < q; j++) {
            const VT xv = reinterpret_cast<const VT *>(c.col(c0 + j) + c.lo)[i];
            vv = vaxmy(vv, sv[j], xv);
            if (NEXT) nx = vaxmy(nx, al[j], xv);
        }
        ov[i] = vscale(vv, rinv);
        if (NEXT) wv[i] = vscale(nx, rinv);
    }
    __syncthreads();
    c.bytes += (unsigned long long)(q + 2 + (NEXT ? 2 : 0)) * c.g.n * sizeof(T);
}

// CTA partials of the Gram matrix of a cycle end, over own rows:
//   out[a * nb + b] = Z_a . U_b  (a < na columns Z from a0, b < nb columns U from b0),
//   out[na * nb + b] = U_b . U_b.
// One staged pass per chunk of up to 4 BW columns of U (and of up to 4 AW
// columns of Z).  The warps form a 4 x 4 grid: warp (ag, bg) owns the Z
// columns a = ag (mod 4) and the U columns b = bg (mod 4) of the chunk, and
// its lanes consecutive 16-byte row vectors, so shared-memory loads are
// conflict free, every lane loads AW + BW vectors per row for AW x BW
// products, and every output is one warp sum.
template <typename T>
__device__ __noinline__ void staged_gram(Ctx<T> &c, int a0, int na, int b0, int nb, T *out) {
    typedef typename Vec<T>::type VT;
    constexpr int E = Vec<T>::N;
    constexpr int R = RING_SEG_BYTES / (int)sizeof(T);
    constexpr int RV = R / E;   // vectors per segment
    constexpr int AW = 12;      // Z columns per warp and chunk
    constexpr int BW = (sizeof(T) == 4) ? 5 : 2;   // U columns per warp and chunk (registers)
    static_assert(RV % 32 == 0 && CHAIN_THREADS == 512, "ring geometry");
    const int lane = lane_id(), wp = warp_id();
    const int ag = wp & 3, bg = wp >> 2;
    const int cap_segs = (int)((long long)c.P.ring_cap * 8 / RING_SEG_BYTES);
    for (int ac = 0; ac < na; ac += 4 * AW) {
        const int nac = min(4 * AW, na - ac);
        // two stages of nac + nbc segments fit: the ring holds >= 2 (m + 2)
        const int gbmax = min(4 * BW, cap_segs / 2 - nac);
        for (int bc = 0; bc < nb; bc += gbmax) {
            const int nbc = min(gbmax, nb - bc);
            const bool norms = (ac == 0) && (ag == 0);
            T acc[AW][BW];
            T nrm[BW];
#pragma unroll
            for (int bb = 0; bb < BW; bb++) {
                nrm[bb] = T(0);
#pragma unroll
                for (int aa = 0; aa < AW; aa++) acc[aa][bb] = T(0);
            }
            const int rs[2] = {a0 + ac, b0 + bc};
            const int rl[2] = {nac, nbc};
            const RingPass rp = ring_begin_runs(c, rs, rl, 2);
            for (int blk = 0; blk < rp.nblk; blk++) {
                const VT *sb = reinterpret_cast<const VT *>(ring_acquire(c, rp, blk));
                const int nv = (int)(min((long long)R, c.cnt - (long long)blk * R) / E);
#pragma unroll
                for (int h = 0; h < RV / 32; h++) {
                    const int vi = lane + 32 * h;
                    if (vi < nv) {
                        VT u[BW];
#pragma unroll
                        for (int bb = 0; bb < BW; bb++) {
                            const int bidx = bg + 4 * bb;
                            u[bb] = (bidx < nbc) ? sb[(nac + bidx) * RV + vi] : vzero(T(0));
                            if (norms) nrm[bb] += vdot(u[bb], u[bb]);
                        }
#pragma unroll
                        for (int aa = 0; aa < AW; aa++) {
                            const int aidx = ag + 4 * aa;
                            if (aidx < nac) {
                                const VT z = sb[aidx * RV + vi];
#pragma unroll
                                for (int bb = 0; bb < BW; bb++) acc[aa][bb] += vdot(z, u[bb]);
                            }
                        }
                    }
                }
                __syncthreads();   // the stage may be refilled
            }
            ring_end(c, rp);
#pragma unroll
            for (int aa = 0; aa < AW; aa++) {
                const int aidx = ag + 4 * aa;
#pragma unroll
                for (int bb = 0; bb < BW; bb++) {
                    const int bidx = bg + 4 * bb;
                    const T v = warp_sum(acc[aa][bb]);
                    if (lane == 0 && aidx < nac && bidx < nbc) out[(ac + aidx) * nb + bc + bidx] = v;
                }
            }
            if (norms) {
#pragma unroll
                for (int bb = 0; bb < BW; bb++) {
                    const int bidx = bg + 4 * bb;
                    const T v = warp_sum(nrm[bb]);
                    if (lane == 0 && bidx < nbc) out[na * nb + bc + bidx] = v;
                }
            }
        }
    }
    __syncthreads();
}

// Own rows of an operator pass in the compact symmetric form (FP32 only;
// see sym_compact_form): E consecutive rows per thread, the fastest grid
// index along the vector.  Row p gets
//   y_p = s (u_p + f_p d_{p+1} u_{p+1} + f_{p-1} d_{p-1} u_{p-1}
//            + sum over the other axis pairs t of the same two terms at +-o_t),
// with d = D^-1 and f the plus-side couplings of the pair.  The rows of this
// CTA were written by it (read through L1); neighbour rows through L2.
template <typename T>
__device__ __forceinline__ void spmv_sym_rows(Ctx<T> &c, const T *src, T s, T *vout, T *y) {
    typedef typename Vec<T>::type VT;
    constexpr int E = Vec<T>::N;
    const long long n = c.g.n, hi = c.lo + c.cnt;
    const int tf = (c.g.nst - 1) >> 1;            // the pair of the fastest axis
    const T *dv = c.Aw;                            // D^-1
    const T *ff = c.Aw + (long long)tf * c.ld;     // couplings to p + 1
    const long long brows = (long long)E * blockDim.x;
    auto prefetch = [&](long long blk) {
        const long long r0 = c.lo + blk * brows;
        if (warp_id() != 0 || r0 >= hi) return;
        const unsigned bytes = (unsigned)(min(brows, hi - r0) * sizeof(T));
        for (int t = lane_id(); t <= tf + 1; t += 32)
            prefetch_l2((t <= tf ? c.Aw + (long long)t * c.ld : src) + r0, bytes);
    };
    prefetch(0);
    prefetch(1);
    for (long long p = c.lo + (long long)E * threadIdx.x; p < hi; p += (long long)E * blockDim.x) {
        prefetch((p - c.lo) / brows + 2);
        if (p >= n) {
            if (vout) *reinterpret_cast<VT *>(vout + p) = vzero(T(0));
            *reinterpret_cast<VT *>(y + p) = vzero(T(0));
            continue;
        }
        const VT xc = __ldcg(reinterpret_cast<const VT *>(src + p));
        const VT dc = *reinterpret_cast<const VT *>(dv + p);
        const VT fc = *reinterpret_cast<const VT *>(ff + p);
        const bool hl = p > 0, hr = p + E < n;
        const T xlf = hl ? __ldcg(src + p - 1) : T(0), dlf = hl ? __ldcg(dv + p - 1) : T(0);
        const T flf = hl ? __ldcg(ff + p - 1) : T(0);
        const T xrg = hr ? __ldcg(src + p + E) : T(0), drg = hr ? __ldcg(dv + p + E) : T(0);
        const T *xa = reinterpret_cast<const T *>(&xc);
        const T *da = reinterpret_cast<const T *>(&dc);
        const T *fa = reinterpret_cast<const T *>(&fc);
        T acc[E];
#pragma unroll
        for (int e = 0; e < E; e++) {
            const T xr = (e == E - 1) ? xrg : xa[e + 1], dr = (e == E - 1) ? drg : da[e + 1];
            const T xl = (e == 0) ? xlf : xa[e - 1], dl = (e == 0) ? dlf : da[e - 1];
            const T fl = (e == 0) ? flf : fa[e - 1];
            acc[e] = xa[e] + fa[e] * (dr * xr) + fl * (dl * xl);
        }
        for (int t = 1; t < tf; t++) {
            const long long o = c.g.off[2 * t];   // > 0, a multiple of E
            const T *ft = c.Aw + (long long)t * c.ld;
            if (p + o < n) {
                const VT fp = *reinterpret_cast<const VT *>(ft + p);
                const VT xq = __ldcg(reinterpret_cast<const VT *>(src + p + o));
                const VT dq = __ldcg(reinterpret_cast<const VT *>(dv + p + o));
                const T *f1 = reinterpret_cast<const T *>(&fp);
                const T *x1 = reinterpret_cast<const T *>(&xq);
                const T *d1 = reinterpret_cast<const T *>(&dq);
#pragma unroll
                for (int e = 0; e < E; e++) acc[e] += f1[e] * (d1[e] * x1[e]);
            }
            if (p - o >= 0) {
                const VT fm = __ldcg(reinterpret_cast<const VT *>(ft + p - o));
                const VT xq = __ldcg(reinterpret_cast<const VT *>(src + p - o));
                const VT dq = __ldcg(reinterpret_cast<const VT *>(dv + p - o));
                const T *f1 = reinterpret_cast<const T *>(&fm);
                const T *x1 = reinterpret_cast<const T *>(&xq);
                const T *d1 = reinterpret_cast<const T *>(&dq);
#pragma unroll
                for (int e = 0; e < E; e++) acc[e] += f1[e] * (d1[e] * x1[e]);
            }
        }
        VT out, vv;
        T *oa = reinterpret_cast<T *>(&out);
        T *va = reinterpret_cast<T *>(&vv);
#pragma unroll
        for (int e = 0; e < E; e++) {
            oa[e] = s * acc[e];
            va[e] = s * xa[e];
        }
        if (vout) *reinterpret_cast<VT *>(vout + p) = vv;
        *reinterpret_cast<VT *>(y + p) = out;
    }
}

// Operator pass of an Arnoldi step: for own rows, vout = s * src (the new
// basis vector, if vout) and y = A M^-1 (s * src); padded rows get zeros.
template <typename T>
__device__ void spmv_pass(Ctx<T> &c, const T *src, T s, T *vout, T *y) {
    typedef typename Vec<T>::type VT;
    constexpr int E = Vec<T>::N;
    const long long hi = c.lo + c.cnt;
    // the fastest grid index runs along the vector when its extent is a
    // multiple of E: then the two neighbours along it come from the vector
    // itself (plus one value at each end) and every other neighbour offset
    // is a multiple of E, so all loads are 16-byte vectors
    const int last = (c.g.nst == 5) ? c.g.ny : c.g.nz;
    const int sL = (c.g.nst == 5) ? 3 : 5;   // slots of the -1 / +1 neighbours
    if (sizeof(T) == 4 && c.symc) {
        spmv_sym_rows(c, src, s, vout, y);
    } else if (!c.g.cols && last % E == 0) {
        const long long n = c.g.n;
        // warp 0 asks L2 for the coefficient rows and the source rows two
        // blocks ahead (a block = E rows per thread)
        const long long brows = (long long)E * blockDim.x;
        auto prefetch = [&](long long blk) {
            const long long r0 = c.lo + blk * brows;
            if (warp_id() != 0 || r0 >= hi) return;
            const unsigned bytes = (unsigned)(min(brows, hi - r0) * sizeof(T));
            for (int s = lane_id(); s <= c.g.nst; s += 32)
                prefetch_l2((s < c.g.nst ? c.Aw + (long long)s * c.ld : src) + r0, bytes);
        };
        prefetch(0);
        prefetch(1);
        for (long long p = c.lo + (long long)E * threadIdx.x; p < hi; p += (long long)E * blockDim.x) {
            prefetch((p - c.lo) / brows + 2);
            if (p >= n) {
                if (vout) *reinterpret_cast<VT *>(vout + p) = vzero(T(0));
                *reinterpret_cast<VT *>(y + p) = vzero(T(0));
                continue;
            }
            const VT xc = __ldcg(reinterpret_cast<const VT *>(src + p));
            const T left = (p > 0) ? __ldcg(src + p - 1) : T(0);
            const T right = (p + E < n) ? __ldcg(src + p + E) : T(0);
            T xl[E], xr[E], xm[E];
            {
                const T *xa = reinterpret_cast<const T *>(&xc);
#pragma unroll
                for (int e = 0; e < E; e++) {
                    xm[e] = xa[e];
                    xl[e] = (e == 0) ? left : xa[e - 1];
                    xr[e] = (e == E - 1) ? right : xa[e + 1];
                }
            }
            T acc[E];
            {
                const VT a0 = *reinterpret_cast<const VT *>(c.Aw + p);
                const T *aa = reinterpret_cast<const T *>(&a0);
#pragma unroll
                for (int e = 0; e < E; e++) acc[e] = aa[e] * xm[e];
            }
            {
                const VT am = *reinterpret_cast<const VT *>(c.Aw + (long long)sL * c.ld + p);
                const VT ap = *reinterpret_cast<const VT *>(c.Aw + (long long)(sL + 1) * c.ld + p);
                const T *a1 = reinterpret_cast<const T *>(&am);
                const T *a2 = reinterpret_cast<const T *>(&ap);
#pragma unroll
                for (int e = 0; e < E; e++) acc[e] += a1[e] * xl[e] + a2[e] * xr[e];
            }
            for (int sl = 1; sl < c.g.nst; sl++) {
                if (sl == sL || sl == sL + 1) continue;
                const long long q = p + c.g.off[sl];
                const VT xv = (q >= 0 && q < n) ? __ldcg(reinterpret_cast<const VT *>(src + q)) : xc;
                const VT av = *reinterpret_cast<const VT *>(c.Aw + (long long)sl * c.ld + p);
                const T *xa = reinterpret_cast<const T *>(&xv);
                const T *aa = reinterpret_cast<const T *>(&av);
#pragma unroll
                for (int e = 0; e < E; e++) acc[e] += aa[e] * xa[e];
            }
            VT out, vv;
            T *oa = reinterpret_cast<T *>(&out);
            T *va = reinterpret_cast<T *>(&vv);
#pragma unroll
            for (int e = 0; e < E; e++) {
                oa[e] = s * acc[e];
                va[e] = s * xm[e];
            }
            if (vout) *reinterpret_cast<VT *>(vout + p) = vv;
            *reinterpret_cast<VT *>(y + p) = out;
        }
    } else {
        for (long long p = c.lo + threadIdx.x; p < hi; p += blockDim.x) {
            if (p < c.g.n) {
                if (vout) vout[p] = s * __ldcg(src + p);
                y[p] = stencil_apply_row(c.g, c.Aw, c.ld, src, s, p);
            } else {
                if (vout) vout[p] = T(0);
                y[p] = T(0);
            }
        }
    }
    __syncthreads();
    c.bytes += (unsigned long long)(3 + (vout ? 1 : 0) + op_slots(c)) * c.g.n * sizeof(T) -
               (unsigned long long)(vout ? 0 : 1) * c.g.n * sizeof(T) + csr_index_bytes(c);
}

// Operator pass with the red-black ILU(0) right preconditioner:
// vout = s * src (if vout), z = M^-1 (s * src) in two colour sweeps, then
// y = A z (= s * src on red rows).  Two extra cluster barriers: the second
// sweep reads the neighbours' black z, the last one their red z.
template <typename T>
__device__ void ilu_spmv_pass(Ctx<T> &c, const T *src, T s, T *vout, T *y) {
    const T *inv = c.Aw + (long long)7 * c.ld;
    T *z = c.col(COL_Z);
    const long long hi = c.lo + c.cnt, n = c.g.n;
    const bool blocks = c.pc_bs < c.g.n;
    // two consecutive rows per thread: along a grid line the first rows of
    // all lanes share a colour, so each colour sweep runs without divergence
    // and every thread has two rows' loads in flight (chunks hold an even
    // number of rows)
    const long long step = 2LL * blockDim.x;
    for (long long p0 = c.lo + 2LL * threadIdx.x; p0 < hi; p0 += step) {
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const long long p = p0 + e;
            if (p < n) {
                if (vout) vout[p] = s * src[p];
                if (grid_color(c.g, p) == 1) {
                    long long blo, bhi;
                    pc_block(p, c.pc_bs, n, blo, bhi);
                    z[p] = ilu_sweep1_row<T, T>(c.g, c.Aw, c.ld, inv, src, s, p, blo, bhi, c.lo, hi);
                }
            } else {
                if (vout) vout[p] = T(0);
                z[p] = T(0);
                y[p] = T(0);
            }
        }
    }
    cl_sync();
    for (long long p0 = c.lo + 2LL * threadIdx.x; p0 < hi; p0 += step) {
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const long long p = p0 + e;
            if (p < n && grid_color(c.g, p) == 0) {
                long long blo, bhi;
                pc_block(p, c.pc_bs, n, blo, bhi);
                z[p] = ilu_sweep2_row<T, T>(c.g, c.Aw, c.ld, inv, src, s, z, p, blo, bhi, c.lo, hi);
                // block-Jacobi leaves the couplings to other blocks out of M, so
                // the red rows of A M^-1 keep them
                const T v = s * src[p];
                y[p] = blocks ? v + ilu_red_cross_row(c.g, c.Aw, c.ld, z, p, blo, bhi, c.lo, hi) : v;
            }
        }
    }
    cl_sync();
    for (long long p0 = c.lo + 2LL * threadIdx.x; p0 < hi; p0 += step) {
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const long long p = p0 + e;
            if (p < n && grid_color(c.g, p) == 1) y[p] = ilu_black_apply_row(c.g, c.Aw, c.ld, z, p, c.lo, hi);
        }
    }
    __syncthreads();
    c.bytes += (unsigned long long)(6 + (vout ? 1 : 0) + 2 * c.g.nst) * c.g.n * sizeof(T);
}

template <typename T>
__device__ __forceinline__ void operator_pass(Ctx<T> &c, const T *src, T s, T *vout, T *y) {
    if (colour_sweep_pc(c.precond))
        ilu_spmv_pass(c, src, s, vout, y);
    else
        spmv_pass(c, src, s, vout, y);
}

// Tiled CTA partials of X_a . Y_b (a < na from column xa0, b < nb from
// column yb0), into out[a * nb + b].
template <typename T>
__device__ void part_gram(Ctx<T> &c, int xa0, int na, int yb0, int nb, T *out) {
    typedef typename Vec<T>::type VT;
    constexpr int E = Vec<T>::N, TA = Tiles<T>::TA, TB = Tiles<T>::TB;
    const int nvec = (int)(c.cnt / E);
    T *wsum = reinterpret_cast<T *>(c.D(c.P.o_wsum));
    T *tmp = reinterpret_cast<T *>(c.D(c.P.o_dscr));   // TA*TB <= 64 values needed
    // a symmetric Gram (the same columns on both sides) needs the tiles on
    // and above the diagonal only; the rest are mirrored
    const bool sym = (xa0 == yb0 && na == nb && TA == TB);
    for (int a0 = 0; a0 < na; a0 += TA) {
        const int ta = min(TA, na - a0);
        for (int b0 = 0; b0 < nb; b0 += TB) {
            const int tb = min(TB, nb - b0);
            if (sym && b0 < a0) continue;
            T acc[TA * TB];
#pragma unroll
            for (int e = 0; e < TA * TB; e++) acc[e] = T(0);
            for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
                VT yv[TB];
#pragma unroll
                for (int bb = 0; bb < TB; bb++)
                    yv[bb] = (bb < tb) ? reinterpret_cast<const VT *>(c.col(yb0 + b0 + bb) + c.lo)[i]
                                       : vzero(T(0));
#pragma unroll
                for (int aa = 0; aa < TA; aa++) {
                    if (aa < ta) {
                        const VT xv = reinterpret_cast<const VT *>(c.col(xa0 + a0 + aa) + c.lo)[i];
#pragma unroll
                        for (int bb = 0; bb < TB; bb++) acc[aa * TB + bb] += vdot(xv, yv[bb]);
                    }
                }
            }
            (void)tmp;
            // reduce the whole tile, then scatter the valid entries
            T *tout = reinterpret_cast<T *>(c.D(c.P.o_vscr)) ;
            (void)tout;
            block_sum<TA * TB>(acc, TA * TB, wsum, reinterpret_cast<T *>(c.D(c.P.o_xr)));
            const T *res = reinterpret_cast<const T *>(c.D(c.P.o_xr));
            for (int e = threadIdx.x; e < ta * tb; e += blockDim.x) {
                const int aa = e / tb, bb = e % tb;
                out[(a0 + aa) * nb + (b0 + bb)] = res[aa * TB + bb];
                if (sym && b0 > a0) out[(b0 + bb) * nb + (a0 + aa)] = res[aa * TB + bb];
            }
            __syncthreads();
        }
    }
    c.bytes += (unsigned long long)(sym ? na : na + nb) * c.g.n * sizeof(T);
}

// ------------------------------------------------------------------ assembly

// Build A (FP64), b, M^-1 diag and the working-precision operator A M^-1 for
// system `sys` into the slot.  Three phases separated by cluster barriers:
// node values, rows of A, folded operator (needs the neighbours' diagonal).
template <typename T>
__device__ __noinline__ void assemble_system(Ctx<T> &c, const DevSystem &sys) {
    const long long nn = node_count(sys, c.g);
    if (nn > 0) {
        const long long per = (nn + c.cs - 1) / c.cs;
        const long long a0 = (long long)c.rank * per, a1 = min(nn, a0 + per);
        for (long long q = a0 + threadIdx.x; q < a1; q += blockDim.x) c.anode[q] = exp(sys.coef[q]);
        cl_sync();
    }
    const long long hi = c.lo + c.cnt;
    for (long long p = c.lo + threadIdx.x; p < hi; p += blockDim.x) {
        if (p < c.g.n) {
            double row[7];
            if (sys.fmt == SKR_FMT_CSR) {
                int ci[7];
                csr_row(sys, p, c.g.nst, row, ci);
                for (int s = 0; s < c.g.nst; s++) c.cols[(long long)s * c.ld + p] = ci[s];
            } else {
                system_row(sys, c.g, c.anode, p, row);
            }
            for (int s = 0; s < c.g.nst; s++) c.A64[(long long)s * c.ld + p] = row[s];
            c.b[p] = system_rhs(sys, c.g, p);
            c.dinv[p] = (c.precond == SKR_PC_NONE) ? 1.0 : 1.0 / row[0];
        } else {
            for (int s = 0; s < c.g.nst; s++) c.A64[(long long)s * c.ld + p] = 0.0;
            c.b[p] = 0.0;
            c.dinv[p] = 1.0;
        }
    }
    cl_sync();
    if (colour_sweep_pc(c.precond)) {
        // red-black ILU(0) / SSOR: inverse pivots (ILU's black ones need the
        // neighbours' rows), and the unscaled operator in working precision
        T *inv = c.Aw + (long long)7 * c.ld;
        for (long long p = c.lo + threadIdx.x; p < hi; p += blockDim.x) {
            if (p < c.g.n) {
                const double ip = sweep_inv_pivot(c.g, c.A64, c.ld, p, c.precond, c.pc_bs);
                c.dinv[p] = ip;
                inv[p] = (T)ip;
                for (int s = 0; s < c.g.nst; s++) c.Aw[(long long)s * c.ld + p] = (T)c.A64[(long long)s * c.ld + p];
            } else {
                inv[p] = T(0);
                for (int s = 0; s < c.g.nst; s++) c.Aw[(long long)s * c.ld + p] = T(0);
            }
        }
    } else if (c.symc) {
        // compact symmetric form: D^-1 and the plus-side couplings of own
        // rows; operator passes read the neighbours' rows of it, so the
        // cluster waits for every CTA's part
        const int ns = sym_compact_slots(c.g);
        for (long long p = c.lo + threadIdx.x; p < hi; p += blockDim.x) {
            if (p < c.g.n) {
                sym_compact_fold_row(c.g, c.A64, c.ld, c.dinv, c.Aw, p);
            } else {
                for (int t = 0; t < ns; t++) c.Aw[(long long)t * c.ld + p] = T(0);
            }
        }
        cl_sync();
    } else {
        for (long long p = c.lo + threadIdx.x; p < hi; p += blockDim.x) {
            if (p < c.g.n) {
                for (int s = 0; s < c.g.nst; s++) {
                    const long long q = nb_index(c.g, p, s);
                    const double a = c.A64[(long long)s * c.ld + p];
                    c.Aw[(long long)s * c.ld + p] = (T)(a * __ldcg(c.dinv + q));
                }
            } else {
                for (int s = 0; s < c.g.nst; s++) c.Aw[(long long)s * c.ld + p] = T(0);
            }
        }
    }
    __syncthreads();
    c.bytes += (unsigned long long)c.g.n * (8 * (c.g.nst + 3) + sizeof(T) * op_slots(c)) +
               (unsigned long long)nn * 16 + csr_index_bytes(c) * 2;
}

// True residual r = b - A x (FP64) over own rows; returns ||r|| (cluster-wide).
template <typename T>
__device__ __noinline__ double true_residual(Ctx<T> &c) {
    cl_sync();   // x of the neighbours must be complete
    const long long hi = c.lo + c.cnt;
    double acc[1] = {0.0};
    for (long long p = c.lo + threadIdx.x; p < hi; p += blockDim.x) {
        double rv = 0.0;
        if (p < c.g.n) rv = residual_row(c.g, c.A64, c.ld, c.b, c.x, p);
        c.r[p] = rv;
        acc[0] += rv * rv;
    }
    block_sum<1>(acc, 1, c.D(c.P.o_wsum), c.template red<double>());
    allreduce<T, double>(c, 1);
    c.bytes += (unsigned long long)c.g.n * 8 * (c.g.nst + 3) + csr_index_bytes(c);
    return sqrt(c.template vals<double>()[0]);
}

// ------------------------------------------------------------------ recycle refresh

// App. B.1: [Q, R] = qr(A_new U), C = Q, U = U R^-1, by Cholesky QR applied
// twice (the Gram matrices are reduced over the cluster, the k x k factors
// are FP64).  On a failed Cholesky the recycle space is dropped (kc = 0).
template <typename T>
__device__ __noinline__ void refresh_recycle(Ctx<T> &c) {
    cl_sync();   // U of the neighbours (halo of the operator) must be complete
    c.updates_since_refresh = 0;
    const int kc = c.kc;
    const int cC0 = COL_C_END - kc;
    // W = A M^-1 U into the C columns
    const long long hi = c.lo + c.cnt;
    if (colour_sweep_pc(c.precond)) {
        for (int b = 0; b < kc; b++) ilu_spmv_pass(c, c.col(COL_U0 + b), T(1), (T *)nullptr, c.col(cC0 + b));
    } else
    for (long long p = c.lo + threadIdx.x; p < hi; p += blockDim.x) {
        T acc[KMAX];
#pragma unroll
        for (int b = 0; b < KMAX; b++) acc[b] = T(0);
        if (p < c.g.n) {
            for (int s = 0; s < c.g.nst; s++) {
                const long long q = nb_index(c.g, p, s);
                const T a = c.symc ? sym_folded(c.g, c.Aw, c.ld, p, s) : c.Aw[(long long)s * c.ld + p];
#pragma unroll
                for (int b = 0; b < KMAX; b++)
                    if (b < kc) acc[b] += a * __ldcg(c.col(COL_U0 + b) + q);
            }
        }
#pragma unroll
        for (int b = 0; b < KMAX; b++)
            if (b < kc) c.col(cC0 + b)[p] = acc[b];
    }
    __syncthreads();
    c.matvecs += kc;
    c.bytes += (unsigned long long)c.g.n * sizeof(T) * (op_slots(c) + 2 * kc) + csr_index_bytes(c);
    double *G = c.D(c.P.o_F);
    double *R = c.D(c.P.o_Z);
    double *Ri = c.D(c.P.o_Z) + kc * kc;
    for (int pass = 0; pass < 2; pass++) {
        part_gram(c, cC0, kc, cC0, kc, c.template red<T>());
        allreduce<T, T>(c, kc * kc);
        const T *gv = c.template vals<T>();
        for (int e = threadIdx.x; e < kc * kc; e += blockDim.x) G[e] = (double)gv[e];  // symmetric
        __syncthreads();
        const int bad = cholesky_upper(G, kc, kc, R, kc, c.ints());
        __syncthreads();
        if (bad) {
            c.kc = 0;
            return;
        }
        upper_inverse(R, kc, kc, Ri, kc);
        T *rt = c.tco(c.P.t_cC);
        for (int e = threadIdx.x; e < kc * kc; e += blockDim.x) rt[e] = (T)Ri[e];  // column-major (i + j kc)
        __syncthreads();
        // W <- W R^-1, U <- U R^-1 (row-local, in place)
        for (long long p = c.lo + threadIdx.x; p < hi; p += blockDim.x) {
            for (int which = 0; which < 2; which++) {
                T *base = (which == 0) ? c.col(cC0) : c.col(COL_U0);
                T in[KMAX], out[KMAX];
#pragma unroll
                for (int b = 0; b < KMAX; b++) in[b] = (b < kc) ? base[(long long)b * c.ld + p] : T(0);
#pragma unroll
                for (int j = 0; j < KMAX; j++) {
                    T s = T(0);
#pragma unroll
                    for (int i = 0; i < KMAX; i++)
                        if (i <= j && j < kc) s += in[i] * rt[i + j * kc];
                    out[j] = s;
                }
#pragma unroll
                for (int b = 0; b < KMAX; b++)
                    if (b < kc) base[(long long)b * c.ld + p] = out[b];
            }
        }
        __syncthreads();
        c.bytes += (unsigned long long)c.g.n * sizeof(T) * (2 * kc + 4 * kc);
    }
}

// Projection at the start of a recycled cycle (the first step of
// Algorithm 2): z = C^T r, d += U z, r -= C z.  Returns ||r||.
template <typename T>
__device__ __noinline__ double project_recycle(Ctx<T> &c) {
    const int kc = c.kc;
    const int cC0 = COL_C_END - kc;
    T *rw = c.col(COL_RW), *dh = c.col(COL_DH);
    staged_dual_dots<T, true, false>(c, cC0, kc, COL_RW, -1, c.template red<T>());
    allreduce<T, T>(c, kc);
    T *z = c.tco(c.P.t_h);
    for (int i = threadIdx.x; i < kc; i += blockDim.x) z[i] = c.template vals<T>()[i];
    __syncthreads();
    typedef typename Vec<T>::type VT;
    constexpr int E = Vec<T>::N;
    const int nvec = (int)(c.cnt / E);
    T acc[1] = {T(0)};
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
        VT rr = reinterpret_cast<VT *>(rw + c.lo)[i];
        VT dd = reinterpret_cast<VT *>(dh + c.lo)[i];
        for (int a = 0; a < kc; a++) {
            rr = vaxmy(rr, z[a], reinterpret_cast<const VT *>(c.col(cC0 + a) + c.lo)[i]);
            dd = vaxpy(dd, z[a], reinterpret_cast<const VT *>(c.col(COL_U0 + a) + c.lo)[i]);
        }
        reinterpret_cast<VT *>(rw + c.lo)[i] = rr;
        reinterpret_cast<VT *>(dh + c.lo)[i] = dd;
        acc[0] += vdot(rr, rr);
    }
    block_sum<1>(acc, 1, reinterpret_cast<T *>(c.D(c.P.o_wsum)), c.template red<T>());
    allreduce<T, T>(c, 1);
    c.bytes += (unsigned long long)c.g.n * sizeof(T) * (2 * kc + 4);
    return sqrt((double)c.template vals<T>()[0]);
}

// ------------------------------------------------------------------ one cycle

// FP32 Givens monitor on column j of H: returns the LSQ residual estimate.
template <typename T>
__device__ float monitor_step(Ctx<T> &c, int j, float beta) {
    float *mc = c.mon(), *ms = mc + c.m, *mg = ms + c.m;
    const double *H = c.D(c.P.o_H);
    const int ldh = c.P.ldh;
    if (threadIdx.x == 0) {
        if (j == 0) mg[0] = beta;
        float a = (float)M_(H, ldh, 0, j);
        for (int i = 0; i < j; i++) {
            const float b = (float)M_(H, ldh, i + 1, j);
            const float na = mc[i] * a + ms[i] * b;
            const float nb = -ms[i] * a + mc[i] * b;
            a = nb;
            (void)na;
        }
        // the rotated entry a now sits in row j; rotation j zeroes H(j+1, j)
        const float b = (float)M_(H, ldh, j + 1, j);
        const float r = hypotf(a, b);
        const float cs = (r > 0.f) ? a / r : 1.f, sn = (r > 0.f) ? b / r : 0.f;
        mc[j] = cs;
        ms[j] = sn;
        mg[j + 1] = -sn * mg[j];
        mg[j] = cs * mg[j];
        c.ints()[4] = __float_as_int(fabsf(mg[j + 1]));
    }
    __syncthreads();
    const float est = __int_as_float(c.ints()[4]);
    __syncthreads();
    return est;
}

// One GCRO-DR cycle (kc > 0) or GMRES cycle (kc == 0) on the inner system
// A M^-1 d = r, following Algorithm 2.  rnw = ||rw|| on entry; returns the
// new ||rw||.
template <typename T>
__device__ double run_cycle(Ctx<T> &c, double rnw, double target) {
    const int kc = c.kc;
    const int Lmax = (kc == 0) ? c.m : c.m - kc;
    const int L = min(Lmax, c.maxit - c.steps);
    const int ldh = c.P.ldh;
    double *H = c.D(c.P.o_H), *Bm = c.D(c.P.o_B);
    const int cQ0 = COL_C_END - kc;   // [C, V_1, ...] start
    if (L <= 0) return rnw;
    const T tiny = (sizeof(T) == 4) ? T(1e-6) : T(1e-13);

    // Arnoldi with delayed re-orthogonalisation.  Step j holds the
    // candidate u for V_j after one classical Gram-Schmidt pass against
    // Z = [C, V_0..V_{j-1}] (u = rw for j = 0).  One operator pass gives
    // w = A M^-1 u; one reduction gives Z^T u, Z^T w, u.u, u.w, w.w.  From
    // them: the second-pass coefficients s = Z^T u finish column j-1 of
    // [B; H] and V_j = (u - Z s) / rho; A M^-1 V_j follows from w and the
    // Arnoldi relation of the finished columns, which gives column j's
    // first-pass coefficients without another pass over Z; one update pass
    // writes V_j and the next candidate.  The term A M^-1 C s_C (s_C: the
    // rounding-level second-pass coefficients against C) is not available
    // and is dropped.
    T *sv = c.tco(c.P.t_s), *al = c.tco(c.P.t_al);
    double *gq = c.D(c.P.o_dscr);   // e = B s_V (kc entries), then g = H s_V (j + 1 entries)
    double *sst = gq + c.m + 2;       // rho_j, s.t, 1/rho_j, ||A M^-1 V_{j-1}|| (one thread, shared)
    const double rinv0 = 1.0 / rnw;
    int ucol = COL_RW, wcol = COL_Y0;
    double rho = rnw, anorm = 0.0;
    int Ld = 0;
    bool early = false;
    cl_sync();   // the operator reads the neighbours' rows of rw
    for (int j = 0;; j++) {
        const bool last = (j == L);
        T *u = c.col(ucol), *w = c.col(wcol);
        if (!last) {
            operator_pass(c, u, T(1), (T *)nullptr, w);
            c.matvecs += 1;
        }
        c.tick(PH_SPMV);
        const int q = kc + j;
        T *red = c.template red<T>();
        if (j == 0)
            staged_dual_dots<T, false, true>(c, cQ0, q, ucol, wcol, red);
        else if (last)
            staged_dual_dots<T, true, false>(c, cQ0, q, ucol, wcol, red);
        else
            staged_dual_dots<T, true, true>(c, cQ0, q, ucol, wcol, red);
        allreduce<T, T>(c, 2 * q + 3);
        c.tick(PH_DOT);
        const T *vv = c.template vals<T>();
        bool stop = last, brk = false;
        double st = 0.0;
        if (j > 0) {
            // finish column j-1: add the second-pass coefficients, H(j, j-1) = rho.
            // s.s and s.t by warp 0 (lanes, then a fixed butterfly), shared
            // through shared memory: FP64 is scarce, no thread repeats it
            if (threadIdx.x < 32) {
                double a0 = 0.0, a1 = 0.0;
                for (int i = threadIdx.x; i < q; i += 32) {
                    const double si = (double)vv[i];
                    a0 += si * si;
                    if (!last) a1 += si * (double)vv[q + i];
                }
                a0 = warp_sum(a0);
                a1 = warp_sum(a1);
                if (threadIdx.x == 0) {
                    const double r2 = (double)vv[2 * q] - a0;
                    const double rh = (r2 > 0.0) ? sqrt(r2) : 0.0;
                    sst[0] = rh;
                    sst[1] = a1;
                    sst[2] = (rh > 0.0) ? 1.0 / rh : 0.0;
                }
            }
            __syncthreads();
            rho = sst[0];
            st = sst[1];
            anorm = sst[3];
            for (int i = threadIdx.x; i < q; i += blockDim.x) {
                if (i < kc)
                    M_(Bm, kc, i, j - 1) += (double)vv[i];
                else
                    M_(H, ldh, i - kc, j - 1) += (double)vv[i];
            }
            if (threadIdx.x == 0) M_(H, ldh, j, j - 1) = rho;
            for (int i = j + 1 + threadIdx.x; i <= c.m; i += blockDim.x) M_(H, ldh, i, j - 1) = 0.0;
            __syncthreads();
            c.steps += 1;
            const float est = monitor_step(c, j - 1, (float)rnw);
            brk = !(rho > (double)tiny * anorm);
            if (brk) c.breakdown = true;
            if (est <= (float)target || brk) {
                stop = true;
                early = true;
            }
        }
        const double rinv = brk ? 0.0 : ((j > 0) ? sst[2] : rinv0);
        for (int i = threadIdx.x; i < q; i += blockDim.x) sv[i] = (j > 0) ? vv[i] : T(0);
        if (stop) {
            __syncthreads();
            c.tick(PH_OTHER);
            dual_update<T, false>(c, cQ0, q, sv, al, T(0), (T)rinv, ucol, wcol, COL_V0 + j);
            c.tick(PH_UPD);
            Ld = j;
            break;
        }
        // e = B(:, 0:j) s_V, g = H(0:j+1, 0:j) s_V over the finished columns
        for (int i = threadIdx.x; i <= q; i += blockDim.x) {
            double acc = 0.0;
            for (int l = 0; l < j; l++) {
                const double sl = (double)vv[kc + l];
                acc += ((i < kc) ? M_(Bm, kc, i, l) : M_(H, ldh, i - kc, l)) * sl;
            }
            gq[i] = acc;
        }
        __syncthreads();
        // column j (first pass): Z^T A M^-1 V_j and V_j^T A M^-1 V_j.  The
        // next candidate is A M^-1 V_j - Z h1 - h1_j V_j
        //   = (w - bet u) / rho - Z (e/rho + h1 - bet s/rho),  bet = g_j/rho + h1_j,
        // written for the update pass as ((w - bet u) - Z al) / rho.
        const double h1q = (((double)vv[2 * q + 1] - st) * rinv - gq[q]) * rinv;
        const double bet = gq[q] * rinv + h1q;
        for (int i = threadIdx.x; i <= q; i += blockDim.x) {
            const double h1 = (i < q) ? ((double)vv[q + i] - gq[i]) * rinv : h1q;
            if (i < kc)
                M_(Bm, kc, i, j) = h1;
            else
                M_(H, ldh, i - kc, j) = h1;
            if (i < q) {
                const double si = (j > 0) ? (double)vv[i] : 0.0;
                al[i] = (T)(gq[i] + rho * h1 - bet * si);
            }
        }
        if (threadIdx.x == 0) sst[3] = sqrt(fmax((double)vv[2 * q + 2], 0.0)) * rinv;   // ||A M^-1 V_j||
        __syncthreads();
        c.tick(PH_OTHER);
        dual_update<T, true>(c, cQ0, q, sv, al, (T)bet, (T)rinv, ucol, wcol, COL_V0 + j);
        c.tick(PH_UPD);
        cl_sync();   // the next operator pass reads the neighbours' rows of the candidate
        ucol = wcol;
        wcol = (wcol == COL_Y0) ? COL_Y1 : COL_Y0;
    }
    const bool full = (!early) && (Ld == Lmax) && (c.k > 0);
    const int mt = kc + Ld;
    // Gram pass for the harmonic-Ritz problem: [C, V_0..V_Ld]^T U and ||u_b||^2
    T *gram = c.template red<T>();
    if (full && kc > 0) {
        staged_gram(c, cQ0, kc + Ld + 1, COL_U0, kc, gram);
        allreduce<T, T>(c, (kc + Ld + 1) * kc + kc);
    }
    c.tick(PH_GRAM);
    // ---- small dense step (FP64, every CTA)
    double *Rw = c.D(c.P.o_Rw), *gv = c.D(c.P.o_gvec), *y2 = c.D(c.P.o_y2), *gam = c.D(c.P.o_gam);
    double *av = c.D(c.P.o_avec), *gc = c.D(c.P.o_gc), *gs = c.D(c.P.o_gs), *ds = c.D(c.P.o_dscr);
    givens_lsq(H, ldh, Ld, rnw, Rw, ldh, gc, gs, gv, y2, ds);
    for (int i = threadIdx.x; i <= Ld; i += blockDim.x) {
        double sacc = 0.0;
        for (int j = 0; j < Ld; j++) sacc += M_(H, ldh, i, j) * y2[j];
        gam[i] = sacc;
    }
    for (int a = threadIdx.x; a < kc; a += blockDim.x) {
        double sacc = 0.0;
        for (int j = 0; j < Ld; j++) sacc += M_(Bm, kc, a, j) * y2[j];
        av[a] = -sacc;
    }
    __syncthreads();
    int knew = -1;
    double *Dk = c.D(c.P.o_D);
    double *Pm = c.D(c.P.o_P), *GP = c.D(c.P.o_GP), *Qc = c.D(c.P.o_Qc), *Rc = c.D(c.P.o_Rc);
    if (full) {
        double *F = c.D(c.P.o_F);
        const T *gr = c.template vals<T>();
        for (int b = threadIdx.x; b < kc; b += blockDim.x)
            Dk[b] = 1.0 / sqrt((double)gr[(kc + Ld + 1) * kc + b]);
        __syncthreads();
        // F = W^T V_hat = [[C^T U D, 0], [V^T U D, I']]  ((mt+1) x mt)
        for (int e = threadIdx.x; e < (mt + 1) * mt; e += blockDim.x) {
            const int i = e % (mt + 1), j = e / (mt + 1);
            double v;
            if (j < kc)
                v = (double)gr[i * kc + j] * Dk[j];
            else
                v = (i >= kc && i - kc == j - kc) ? 1.0 : 0.0;
            M_(F, ldh, i, j) = v;
        }
        __syncthreads();
        // Q_G^T F: the Givens rotations act on rows kc+i, kc+i+1
        for (int j = threadIdx.x; j < mt; j += blockDim.x) {
            for (int i = 0; i < Ld; i++) {
                const double a = M_(F, ldh, kc + i, j), b = M_(F, ldh, kc + i + 1, j);
                M_(F, ldh, kc + i, j) = gc[i] * a + gs[i] * b;
                M_(F, ldh, kc + i + 1, j) = -gs[i] * a + gc[i] * b;
            }
        }
        __syncthreads();
        // M = R_G^-1 (Q_G^T F)[0:mt], R_G = [[D, B], [0, R_H]], in place in F
        for (int i = mt - 1; i >= 0; i--) {
            const double rii = (i < kc) ? Dk[i] : M_(Rw, ldh, i - kc, i - kc);
            for (int j = threadIdx.x; j < mt; j += blockDim.x) M_(F, ldh, i, j) /= rii;
            __syncthreads();
            for (int e = threadIdx.x; e < i * mt; e += blockDim.x) {
                const int r = e % i, j = e / i;
                double rri;
                if (r < kc)
                    rri = (i < kc) ? 0.0 : M_(Bm, kc, r, i - kc);
                else
                    rri = M_(Rw, ldh, r - kc, i - kc);
                M_(F, ldh, r, j) -= rri * M_(F, ldh, i, j);
            }
            __syncthreads();
        }
        // the harmonic-Ritz eigenproblem in FP64 (Algorithm 2's small dense
        // step); FP32 only when the caller asks for it (skr_options.eig_fp32)
        unsigned long long *mk = reinterpret_cast<unsigned long long *>(c.D(c.P.o_sc) + 12);
        if (threadIdx.x == 0) mk[0] = mk[1] = mk[2] = 0ull;
        c.tick(PH_DENSE);
        if (sizeof(T) == 4 && c.eig32) {
            // odd leading dimension: the row updates of the Hessenberg
            // reduction and the bulge chase hit 32 distinct banks
            float *Mr = reinterpret_cast<float *>(c.D(c.P.o_Z));
            const int ldm = mt | 1;
            float *Zr = Mr + mt * ldm;
            knew = harmonic_select<float>(F, ldh, mt, c.k, Pm, mt, Mr, ldm, Zr,
                                          reinterpret_cast<float *>(c.D(c.P.o_wr)),
                                          reinterpret_cast<float *>(c.D(c.P.o_wi)),
                                          reinterpret_cast<float *>(c.D(c.P.o_xr)),
                                          reinterpret_cast<float *>(c.D(c.P.o_xi)),
                                          reinterpret_cast<float *>(c.D(c.P.o_vscr)),
                                          reinterpret_cast<float *>(c.D(c.P.o_sc)), c.ints() + 8, Rw, mk);
        } else {
            knew = harmonic_select<double>(F, ldh, mt, c.k, Pm, mt, F, ldh, c.D(c.P.o_Z), c.D(c.P.o_wr),
                                           c.D(c.P.o_wi), c.D(c.P.o_xr), c.D(c.P.o_xi), c.D(c.P.o_vscr),
                                           c.D(c.P.o_sc), c.ints() + 8, Rw, mk);
        }
        c.tick_eigen(mk);
        __syncthreads();
        if (knew > 0) {
            // G P_k, G = [[D, B], [0, Hbar]]
            for (int e = threadIdx.x; e < (mt + 1) * knew; e += blockDim.x) {
                const int i = e % (mt + 1), cc = e / (mt + 1);
                double sacc = 0.0;
                if (i < kc) {
                    sacc = Dk[i] * M_(Pm, mt, i, cc);
                    for (int j = 0; j < Ld; j++) sacc += M_(Bm, kc, i, j) * M_(Pm, mt, kc + j, cc);
                } else {
                    for (int j = 0; j < Ld; j++) sacc += M_(H, ldh, i - kc, j) * M_(Pm, mt, kc + j, cc);
                }
                M_(GP, ldh, i, cc) = sacc;
            }
            __syncthreads();
            const int bad = householder_qr(GP, ldh, mt + 1, knew, Qc, ldh, Rc, knew,
                                           c.D(c.P.o_tau), c.D(c.P.o_sc));
            __syncthreads();
            if (bad) {
                knew = -1;
            } else {
                // P R^-1 (in place in P), using R^-1 in Z
                double *Ri = c.D(c.P.o_Z);
                upper_inverse(Rc, knew, knew, Ri, knew);
                for (int i = threadIdx.x; i < mt; i += blockDim.x) {
                    double rowv[KMAX + 1];
                    for (int cc = 0; cc < knew; cc++) rowv[cc] = M_(Pm, mt, i, cc);
                    for (int cc = 0; cc < knew; cc++) {
                        double sacc = 0.0;
                        for (int q2 = 0; q2 <= cc; q2++) sacc += rowv[q2] * M_(Ri, knew, q2, cc);
                        M_(Pm, mt, i, cc) = sacc;
                    }
                }
                __syncthreads();
            }
        }
        if (knew > KMAX) knew = -1;
    }
    // ---- coefficients in working precision
    T *cC = c.tco(c.P.t_cC), *cU = c.tco(c.P.t_cU), *cr = c.tco(c.P.t_cr), *cd = c.tco(c.P.t_cd);
    const int kn = (knew > 0) ? knew : 0;
    const int KS = (kn + 3) & ~3;
    for (int i = threadIdx.x; i <= Ld; i += blockDim.x) cr[i] = (T)gam[i];
    for (int a = threadIdx.x; a < kc; a += blockDim.x) cd[a] = (T)av[a];
    for (int j = threadIdx.x; j < Ld; j += blockDim.x) cd[kc + j] = (T)y2[j];
    for (int e = threadIdx.x; e < (mt + 1) * KS; e += blockDim.x) {
        const int i = e / KS, o = e % KS;
        cC[i * KS + o] = (o < kn) ? (T)M_(Qc, ldh, i, o) : T(0);
    }
    for (int e = threadIdx.x; e < mt * KS; e += blockDim.x) {
        const int i = e / KS, o = e % KS;
        const double sc = (i < kc) ? Dk[i] : 1.0;
        cU[i * KS + o] = (o < kn) ? (T)(sc * M_(Pm, mt, i, o)) : T(0);
    }
    __syncthreads();
    c.tick(PH_DENSE);
    // ---- update pass (own rows, two rows per thread): r and C_new from
    // [C, V_0..V_Ld], then d and U_new from [U, V_0..V_{Ld-1}]
    typedef typename Vec2<T>::type T2;
    T *rw = c.col(COL_RW), *dh = c.col(COL_DH);
    const int knc = kn;   // new recycle dimension (0: keep the old C, U)
    const int nin_a = kc + Ld + 1, nin_b = kc + Ld;
    T tacc[1] = {T(0)};
    constexpr int UB = 8;
    // warp 0 asks L2 for every input column's rows two blocks ahead (a block
    // = two rows per thread): [C, V_0..V_Ld], U, r and d
    const long long brows = 2LL * blockDim.x, pend = c.lo + c.cnt;
    auto prefetch = [&](long long blk) {
        const long long r0 = c.lo + blk * brows;
        if (warp_id() != 0 || r0 >= pend) return;
        const unsigned bytes = (unsigned)(min(brows, pend - r0) * sizeof(T));
        for (int j = lane_id(); j < nin_a + kc + 2; j += 32) {
            const T *col = (j < nin_a) ? c.col(cQ0 + j) : (j < nin_a + kc) ? c.col(COL_U0 + j - nin_a)
                                                                           : (j == nin_a + kc ? rw : dh);
            prefetch_l2(col + r0, bytes);
        }
    };
    prefetch(0);
    prefetch(1);
    for (long long p = c.lo + 2 * threadIdx.x; p < c.lo + c.cnt; p += 2 * blockDim.x) {
        prefetch((p - c.lo) / brows + 2);
        T o0[KMAX], o1[KMAX];
#pragma unroll
        for (int b2 = 0; b2 < KMAX; b2++) o0[b2] = o1[b2] = T(0);
        T2 racc = *reinterpret_cast<const T2 *>(rw + p);
        for (int i0 = 0; i0 < nin_a; i0 += UB) {
            T2 xv[UB];
#pragma unroll
            for (int u = 0; u < UB; u++)
                xv[u] = (i0 + u < nin_a) ? *reinterpret_cast<const T2 *>(c.col(cQ0 + i0 + u) + p) : T2{T(0), T(0)};
#pragma unroll
            for (int u = 0; u < UB; u++) {
                const int i = i0 + u;
                if (i < nin_a) {
                    if (i >= kc) {
                        const T gmm = cr[i - kc];
                        racc.x -= gmm * xv[u].x;
                        racc.y -= gmm * xv[u].y;
                    }
                    const T *cc = cC + i * KS;
#pragma unroll
                    for (int b4 = 0; b4 < KMAX; b4 += 4) {
                        if (b4 < knc) {
                            T q0, q1, q2, q3;
                            ld4(cc + b4, q0, q1, q2, q3);
                            o0[b4] += xv[u].x * q0; o1[b4] += xv[u].y * q0;
                            o0[b4 + 1] += xv[u].x * q1; o1[b4 + 1] += xv[u].y * q1;
                            o0[b4 + 2] += xv[u].x * q2; o1[b4 + 2] += xv[u].y * q2;
                            o0[b4 + 3] += xv[u].x * q3; o1[b4 + 3] += xv[u].y * q3;
                        }
                    }
                }
            }
        }
        *reinterpret_cast<T2 *>(rw + p) = racc;
        tacc[0] += racc.x * racc.x + racc.y * racc.y;
#pragma unroll
        for (int b2 = 0; b2 < KMAX; b2++)
            if (b2 < knc) *reinterpret_cast<T2 *>(c.col(COL_C_END - knc + b2) + p) = T2{o0[b2], o1[b2]};
#pragma unroll
        for (int b2 = 0; b2 < KMAX; b2++) o0[b2] = o1[b2] = T(0);
        T2 dacc = *reinterpret_cast<const T2 *>(dh + p);
        for (int i0 = 0; i0 < nin_b; i0 += UB) {
            T2 xv[UB];
#pragma unroll
            for (int u = 0; u < UB; u++) {
                const int i = i0 + u;
                const T *src = (i < kc) ? c.col(COL_U0 + i) : c.col(COL_V0 + (i - kc));
                xv[u] = (i < nin_b) ? *reinterpret_cast<const T2 *>(src + p) : T2{T(0), T(0)};
            }
#pragma unroll
            for (int u = 0; u < UB; u++) {
                const int i = i0 + u;
                if (i < nin_b) {
                    const T dv = cd[i];
                    dacc.x += dv * xv[u].x;
                    dacc.y += dv * xv[u].y;
                    const T *cc = cU + i * KS;
#pragma unroll
                    for (int b4 = 0; b4 < KMAX; b4 += 4) {
                        if (b4 < knc) {
                            T q0, q1, q2, q3;
                            ld4(cc + b4, q0, q1, q2, q3);
                            o0[b4] += xv[u].x * q0; o1[b4] += xv[u].y * q0;
                            o0[b4 + 1] += xv[u].x * q1; o1[b4 + 1] += xv[u].y * q1;
                            o0[b4 + 2] += xv[u].x * q2; o1[b4 + 2] += xv[u].y * q2;
                            o0[b4 + 3] += xv[u].x * q3; o1[b4 + 3] += xv[u].y * q3;
                        }
                    }
                }
            }
        }
        *reinterpret_cast<T2 *>(dh + p) = dacc;
#pragma unroll
        for (int b2 = 0; b2 < KMAX; b2++)
            if (b2 < knc) *reinterpret_cast<T2 *>(c.col(COL_U0 + b2) + p) = T2{o0[b2], o1[b2]};
    }
    block_sum<1>(tacc, 1, reinterpret_cast<T *>(c.D(c.P.o_wsum)), c.template red<T>());
    allreduce<T, T>(c, 1);
    c.bytes += (unsigned long long)c.g.n * sizeof(T) *
               ((kc + Ld + 1) + (kc + Ld) + 4 + 2 * knc);
    c.tick(PH_CUPD);
    if (knc > 0) {
        c.kc = knc;
        c.updates_since_refresh += 1;
    }
    c.cycles += 1;
    return sqrt((double)c.template vals<T>()[0]);
}

// ------------------------------------------------------------------ one system

// The one-sided distance of Eq. 5, delta(Q, C) = ||(I - Pi_C) Pi_Q||_2, from
// C = the kc_in columns saved at COL_CIN when the system started to Q = the
// current C_k: with orthonormal bases and G = C^T Q, delta^2 is the largest
// eigenvalue of I - G^T G (FP64, Hessenberg + Francis QR on every CTA).
template <typename T>
__device__ __noinline__ double recycle_delta(Ctx<T> &c, int kc_in) {
    const int kq = c.kc;
    T *red = c.template red<T>();
    staged_gram(c, COL_CIN, kc_in, COL_C_END - kq, kq, red);
    allreduce<T, T>(c, kc_in * kq + kq);
    const T *gv = c.template vals<T>();   // gv[a * kq + b] = C_a . Q_b
    double *S = c.D(c.P.o_F);
    const int lds = c.P.ldh;
    for (int e = threadIdx.x; e < kq * kq; e += blockDim.x) {
        const int i = e % kq, j = e / kq;
        double acc = (i == j) ? 1.0 : 0.0;
        for (int a = 0; a < kc_in; a++) acc -= (double)gv[a * kq + i] * (double)gv[a * kq + j];
        M_(S, lds, i, j) = acc;
    }
    __syncthreads();
    double *Z = c.D(c.P.o_Z), *wr = c.D(c.P.o_wr), *wi = c.D(c.P.o_wi);
    hessenberg_reduce<double>(S, lds, Z, kq, kq, c.D(c.P.o_vscr), c.D(c.P.o_sc));
    const int fail = schur_form<double>(S, lds, Z, kq, kq, wr, wi, c.ints() + 8, c.D(c.P.o_vscr));
    double lmax = 0.0;
    for (int i = 0; i < kq; i++) lmax = fmax(lmax, wr[i]);   // symmetric: real eigenvalues
    __syncthreads();
    return fail ? -1.0 : sqrt(fmin(fmax(lmax, 0.0), 1.0));
}

// Copy the chain's final recycle space out (this CTA's rows): U_k into
// columns 0..k-1 and C_k into columns k..2k-1 of out (n doubles each),
// zeros past the carried dimension.
template <typename T>
__device__ __noinline__ void export_recycle(Ctx<T> &c, double *out) {
    __syncthreads();
    const long long n = c.g.n;
    const long long hi = min(c.lo + c.cnt, n);
    for (int j = 0; j < c.k; j++) {
        const bool have = j < c.kc;
        const T *u = c.col(COL_U0 + j);
        const T *cc = c.col(COL_C_END - c.kc + j);
        for (long long p = c.lo + threadIdx.x; p < hi; p += blockDim.x) {
            out[(long long)j * n + p] = have ? (double)u[p] : 0.0;
            out[((long long)c.k + j) * n + p] = have ? (double)cc[p] : 0.0;
        }
    }
    __syncthreads();
}

// Mixed form: recycle updates between two recomputations of C = A M^-1 U.
constexpr int RECYCLE_REFRESH = 8;

template <typename T>
__device__ void solve_system(Ctx<T> &c, const ChainArgs &a, int sysidx, bool warm) {
    const DevSystem sys = a.systems[sysidx];
    const unsigned long long t0 = global_ns();
    c.g = (sys.fmt == SKR_FMT_CSR) ? make_csr_geom(sys.nx, sys.csr_w, c.cols, c.ld)
                                   : make_geom(sys.fmt, sys.nx, sys.ny, sys.nz);
    c.pc_bs = sweep_block_rows(c.precond, c.g.n, c.pc_blocks);
    c.symc = sym_compact_form(sys.fmt, c.precond, (int)sizeof(T), c.g) ? 1 : 0;
    const long long chunk = (((c.g.n + c.cs - 1) / c.cs) + 7) / 8 * 8;
    c.lo = (long long)c.rank * chunk;
    c.cnt = chunk;
    c.steps = c.cycles = c.matvecs = c.refinements = 0;
    c.breakdown = false;
    if (c.rank == 0 && threadIdx.x == 0) c.tmark = global_ns();
    assemble_system(c, sys);
    c.tick(PH_ASM);
    // refresh the carried recycle space against the new operator (App. B.1)
    if (c.kc > 0) refresh_recycle(c);
    c.tick(PH_REFRESH);
    // diagnostics: keep the refreshed C_k to measure how far the system moves it
    int kc_in = 0;
    if (a.diagnostics && c.kc > 0) {
        kc_in = c.kc;
        for (int b = 0; b < kc_in; b++) {
            const T *src = c.col(COL_C_END - kc_in + b);
            T *dst = c.col(COL_CIN + b);
            for (long long p = c.lo + threadIdx.x; p < c.lo + c.cnt; p += blockDim.x) dst[p] = src[p];
        }
        __syncthreads();
    }
    const long long hi = c.lo + c.cnt;
    // ||b||; x_0 = 0, or the previous solution of the chain (warm start)
    double bacc[1] = {0.0};
    for (long long p = c.lo + threadIdx.x; p < hi; p += blockDim.x) {
        if (!warm) c.x[p] = 0.0;
        const double bv = c.b[p];
        c.r[p] = bv;
        bacc[0] += bv * bv;
    }
    block_sum<1>(bacc, 1, c.D(c.P.o_wsum), c.template red<double>());
    allreduce<T, double>(c, 1);
    const double bnorm = sqrt(c.template vals<double>()[0]);
    const bool fp64 = sizeof(T) == 8;
    double rnorm = warm ? true_residual(c) : bnorm;
    int flag = SKR_NOT_CONVERGED;
    for (int it = 0;; it++) {
        if (it > 0) rnorm = true_residual(c);
        c.tick(PH_RESID);
        if (isnan(rnorm) || isinf(rnorm)) {
            flag = SKR_NUMERICAL;
            break;
        }
        if (rnorm <= a.tol * bnorm) {
            flag = SKR_CONVERGED;
            break;
        }
        if (it >= a.max_refine || c.steps >= c.maxit) {
            flag = c.breakdown ? SKR_BREAKDOWN : SKR_NOT_CONVERGED;
            break;
        }
        const double target = fp64 ? a.tol * bnorm : fmax(a.inner_tol * rnorm, a.tol * bnorm);
        // mixed form: FP32 rounding makes A U = C drift with every recycle
        // update (by ~eps32 kappa each); recompute C from U (App. B.1) at
        // every refinement pass and every RECYCLE_REFRESH updates
        if (!fp64 && it > 0 && c.kc > 0 && c.updates_since_refresh > 0) {
            refresh_recycle(c);
            c.tick(PH_REFRESH);
        }
        // inner system A M^-1 d = r in working precision
        T *rw = c.col(COL_RW), *dh = c.col(COL_DH);
        for (long long p = c.lo + threadIdx.x; p < hi; p += blockDim.x) {
            rw[p] = (T)c.r[p];
            dh[p] = T(0);
        }
        __syncthreads();
        double rnw = rnorm;
        for (;;) {
            c.tick(PH_OTHER);
            if (c.kc > 0) rnw = project_recycle(c);
            c.tick(PH_PROJ);
            if (!(rnw > target) || c.steps >= c.maxit) break;
            rnw = run_cycle(c, rnw, target);
            if (isnan(rnw)) break;
            if (!fp64 && c.kc > 0 && c.updates_since_refresh >= RECYCLE_REFRESH) {
                refresh_recycle(c);
                c.tick(PH_REFRESH);
            }
        }
        // x += M^-1 d (FP64)
        if (colour_sweep_pc(c.precond)) {
            cl_sync();   // d of the neighbours
            for (long long p = c.lo + threadIdx.x; p < hi && p < c.g.n; p += blockDim.x)
                if (grid_color(c.g, p) == 1) {
                    long long blo, bhi;
                    pc_block(p, c.pc_bs, c.g.n, blo, bhi);
                    c.r[p] = ilu_sweep1_row<double, T>(c.g, c.A64, c.ld, c.dinv, dh, 1.0, p, blo, bhi);
                }
            cl_sync();
            for (long long p = c.lo + threadIdx.x; p < hi && p < c.g.n; p += blockDim.x)
                if (grid_color(c.g, p) == 0) {
                    long long blo, bhi;
                    pc_block(p, c.pc_bs, c.g.n, blo, bhi);
                    c.r[p] = ilu_sweep2_row<double, T>(c.g, c.A64, c.ld, c.dinv, dh, 1.0, c.r, p, blo, bhi);
                }
            __syncthreads();
            for (long long p = c.lo + threadIdx.x; p < hi && p < c.g.n; p += blockDim.x) c.x[p] += c.r[p];
        } else {
            for (long long p = c.lo + threadIdx.x; p < hi; p += blockDim.x)
                c.x[p] += c.dinv[p] * (double)dh[p];
        }
        __syncthreads();
        c.refinements += 1;
        c.bytes += (unsigned long long)c.g.n * (8 * 3 + sizeof(T));
    }
    const double delta = (kc_in > 0 && c.kc > 0) ? recycle_delta(c, kc_in) : -1.0;
    // write the solution
    for (long long p = c.lo + threadIdx.x; p < min(hi, c.g.n); p += blockDim.x) sys.x_out[p] = c.x[p];
    c.bytes += (unsigned long long)c.g.n * 16;
    cl_sync();
    if (c.rank == 0 && threadIdx.x == 0) {
        int stall = 0;
        for (unsigned q = 0; q < c.cs; q++) stall |= *cl_map(c.ints() + INT_STALL, q);
        if (stall) flag = SKR_DEVICE_STALL;
        DevResult res;
        res.steps = c.steps;
        res.cycles = c.cycles;
        res.matvecs = c.matvecs;
        res.refinements = c.refinements;
        res.flag = flag;
        res.k_final = c.kc;
        res.relres = (bnorm > 0.0) ? rnorm / bnorm : 0.0;
        res.t_begin = t0;
        res.t_end = global_ns();
        res.delta = delta;
        a.results[sysidx] = res;
        if (a.bytes) atomicAdd(a.bytes, c.bytes);
    }
    c.bytes = 0;
}

template <typename T>
__global__ void __launch_bounds__(CHAIN_THREADS, CHAIN_MIN_BLOCKS) chain_kernel(const __grid_constant__ ChainArgs a) {
    extern __shared__ __align__(1024) double smem_dyn[];
    Ctx<T> c;
    c.rank = cl_rank();
    c.cs = cl_size();
    const int slot = blockIdx.x / c.cs;
    c.P = make_plan(a.m, a.k, blockDim.x, (int)sizeof(T));
    c.sm = smem_dyn;
    c.parity = 0;
    c.m = a.m;
    c.k = a.k;
    c.maxit = a.maxit;
    c.precond = a.precond;
    c.pc_blocks = a.pc_blocks;
    c.eig32 = a.eig32;
    c.ld = a.ws.ld;
    c.basis = reinterpret_cast<T *>(a.ws.basis) + (long long)slot * NCOLS * c.ld;
    c.A64 = a.ws.A64 + (long long)slot * 7 * c.ld;
    c.Aw = reinterpret_cast<T *>(a.ws.Aw) + (long long)slot * AW_SLOTS * c.ld;
    c.dinv = a.ws.dinv + (long long)slot * c.ld;
    c.x = a.ws.x + (long long)slot * c.ld;
    c.r = a.ws.r + (long long)slot * c.ld;
    c.b = a.ws.b + (long long)slot * c.ld;
    c.anode = a.ws.anode + (long long)slot * a.ws.nodecap;
    c.cols = a.ws.cols ? a.ws.cols + (long long)slot * 7 * c.ld : nullptr;
    c.bytes = 0;
    c.prof = a.prof;
    c.tmark = 0;
    c.ring = reinterpret_cast<T *>(smem_dyn + c.P.o_ring);
    c.bars = reinterpret_cast<unsigned long long *>(smem_dyn + c.P.o_bar);
    c.phase = 0u;
    c.tmap = a.tmap;
    c.ybase = slot * NCOLS;
    int *ictl = c.ints();
    if (threadIdx.x == 0) {
        for (int i = 0; i < RING_MAX_NS; i++) mbar_init(c.bars + i, 1);
        mbar_init_fence();
        ictl[INT_STALL] = 0;   // sticky for the launch
    }
    __syncthreads();
    for (;;) {
        if (c.rank == 0 && threadIdx.x == 0) ictl[0] = atomicAdd(a.chain_counter, 1);
        cl_sync();
        const int chain = *cl_map(&ictl[0], 0);
        cl_sync();
        if (chain >= a.nchains) break;
        c.kc = 0;
        if (a.chain_kc) {
            const int k0 = a.chain_kc[chain];
            c.kc = (k0 > 0 && k0 <= a.k) ? k0 : 0;
        }
        c.updates_since_refresh = 0;
        bool xok = a.chain_xok ? (a.chain_xok[chain] != 0) : false;
        for (long long pos = a.chain_off[chain]; pos < a.chain_off[chain + 1]; pos++) {
            solve_system(c, a, a.order[pos], a.warm_start && xok);
            xok = true;
        }
        if (a.recycle_out) export_recycle(c, a.recycle_out[chain]);
        if (a.chain_kc && c.rank == 0 && threadIdx.x == 0) a.chain_kc[chain] = c.kc;
        if (a.chain_xok && c.rank == 0 && threadIdx.x == 0) a.chain_xok[chain] = 1;
    }
    // after a stall, give copies still in flight a bounded time to land
    if (ictl[INT_STALL]) {
        const unsigned long long t0 = global_ns();
        while (global_ns() - t0 < RING_DRAIN_NS) {
        }
    }
}

}  // namespace skr
