// Small dense FP64 linear algebra for the once-per-cycle step of GCRO-DR
// (Algorithm 2): the least-squares solve, the harmonic-Ritz eigenproblem,
// the QR of G P_k, and the Cholesky factor of the recycle refresh.
//
// All routines run on one CTA with every thread participating, operate on
// column-major matrices in shared memory, and synchronise with
// __syncthreads() on entry and exit.  The scalar control decisions of the
// iterative routines are taken from shared-memory values, so every thread
// (and every CTA of a cluster, given identical inputs) follows the same path
// and produces bit-identical results.
//
// FP64 on this GPU issues one warp instruction per 64 cycles per SM
// sub-partition regardless of how many lanes are active, so the routines
// spread independent work over lanes and warps wherever the algorithm
// allows, and keep serial sections short.
#pragma once

#include "skr_device.cuh"

namespace skr {

#define M_(A, ld, i, j) (A)[(i) + (long long)(j) * (ld)]


__device__ __forceinline__ void sync() { __syncthreads(); }

// ------------------------------------------------------------------ Givens LSQ

// Least squares min || beta e1 - Hbar y || for Hbar ((L+1) x L, upper
// Hessenberg, in H with leading dimension ldh), by Givens rotations.
// Outputs: y[0..L) and the rotations (gc, gs) for later reuse; Rw receives
// the triangular factor (L x L in its upper part); g[0..L] the rotated rhs.
// Returns |g[L]|, the residual norm (valid on every thread).
__device__ inline double givens_lsq(const double *H, int ldh, int L, double beta, double *Rw, int ldr,
                             double *gc, double *gs, double *g, double *y, double *dscr) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < (L + 1) * L; e += nt) {
        const int i = e % (L + 1), j = e / (L + 1);
        M_(Rw, ldr, i, j) = M_(H, ldh, i, j);
    }
    for (int i = tid; i <= L; i += nt) g[i] = (i == 0) ? beta : 0.0;
    sync();
    for (int i = 0; i < L; i++) {
        if (tid == 0) {
            const double a = M_(Rw, ldr, i, i), b = M_(Rw, ldr, i + 1, i);
            double c = 1.0, s = 0.0, r = a;
            if (b != 0.0) {
                const double rh = rhypot(a, b);
                c = a * rh;
                s = b * rh;
                r = a * c + b * s;
            }
            gc[i] = c;
            gs[i] = s;
            M_(Rw, ldr, i, i) = r;
            M_(Rw, ldr, i + 1, i) = 0.0;
            const double gi = g[i];
            g[i] = c * gi;
            g[i + 1] = -s * gi;
        }
        sync();
        const double c = gc[i], s = gs[i];
        for (int j = i + 1 + tid; j < L; j += nt) {
            const double a = M_(Rw, ldr, i, j), b = M_(Rw, ldr, i + 1, j);
            M_(Rw, ldr, i, j) = c * a + s * b;
            M_(Rw, ldr, i + 1, j) = -s * a + c * b;
        }
        sync();
    }
    // back substitution, column oriented; reciprocals of the diagonal first
    // (in parallel) so the serial chain holds one multiply per row
    double *rd = dscr + (L + 1);
    for (int i = tid; i < L; i += nt) {
        dscr[i] = g[i];
        rd[i] = 1.0 / M_(Rw, ldr, i, i);
    }
    sync();
    for (int i = L - 1; i >= 0; i--) {
        const double yi = dscr[i] * rd[i];
        if (tid == 0) y[i] = yi;
        for (int c = tid; c < i; c += nt) dscr[c] -= M_(Rw, ldr, c, i) * yi;
        sync();
    }
    return fabs(g[L]);
}

// ------------------------------------------------------------------ eigen-solver

// Reduce A (n x n, lda) to upper Hessenberg form by Householder reflectors,
// accumulating Z = Q (n x n, ldz) with A_in = Z H Z^T.  R is the arithmetic
// type (double, or float for the mixed form's eigen-solve).  v: n scratch
// values, sc: 4 scratch values.
template <typename R>
__device__ inline void hessenberg_reduce(R *A, int lda, R *Z, int ldz, int n, R *v, R *sc) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = lane_id(), w = warp_id(), nw = num_warps();
    for (int e = tid; e < n * n; e += nt) M_(Z, ldz, e % n, e / n) = (e % n == e / n) ? R(1) : R(0);
    sync();
    for (int c = 0; c + 2 < n; c++) {
        if (w == 0) {
            R s = R(0);
            for (int i = c + 1 + lane; i < n; i += 32) s += M_(A, lda, i, c) * M_(A, lda, i, c);
            s = warp_sum(s);
            if (lane == 0) {
                const R x0 = M_(A, lda, c + 1, c);
                const R nrm = sqrt(s);
                R tau = R(0), alpha = x0;
                if (nrm > R(0) && s - x0 * x0 > R(0)) {
                    alpha = -copysign(nrm, x0);
                    tau = (alpha - x0) / alpha;
                    sc[1] = R(1) / (x0 - alpha);
                } else {
                    sc[1] = R(0);
                }
                sc[0] = tau;
                sc[2] = alpha;
            }
        }
        sync();
        const R tau = sc[0], inv = sc[1];
        sync();                    // sc is rewritten by the next column
        if (tau == R(0)) continue;  // uniform: read from shared memory
        for (int i = c + 1 + tid; i < n; i += nt) v[i] = (i == c + 1) ? R(1) : M_(A, lda, i, c) * inv;
        sync();
        // left: A[c+1:, c:] -= tau v (v^T A[c+1:, c:]); one warp per column
        for (int j = c + w; j < n; j += nw) {
            R s = R(0);
            for (int i = c + 1 + lane; i < n; i += 32) s += v[i] * M_(A, lda, i, j);
            s = warp_sum(s) * tau;
            for (int i = c + 1 + lane; i < n; i += 32) M_(A, lda, i, j) -= s * v[i];
        }
        sync();
        // right: A[:, c+1:] -= tau (A[:, c+1:] v) v^T and Z likewise; one warp per row
        for (int r = w; r < 2 * n; r += nw) {
            R *Mx = (r < n) ? A : Z;
            const int ldm = (r < n) ? lda : ldz;
            const int i = (r < n) ? r : r - n;
            R s = R(0);
            for (int j = c + 1 + lane; j < n; j += 32) s += M_(Mx, ldm, i, j) * v[j];
            s = warp_sum(s) * tau;
            for (int j = c + 1 + lane; j < n; j += 32) M_(Mx, ldm, i, j) -= s * v[j];
        }
        sync();
        if (tid == 0) M_(A, lda, c + 1, c) = sc[2];
        for (int i = c + 2 + tid; i < n; i += nt) M_(A, lda, i, c) = R(0);
        sync();
    }
}

// hessenberg_reduce for FP64 with the dot products of each reflector
// application split over four row (or column) chunks per thread group
// instead of warp-shuffle reductions: on this GPU every FP64 instruction,
// the five additions of a warp reduction included, costs a sub-partition's
// FP64 pipe many cycles, and the chunked form issues about half as many.
// part: scratch of at least 8 n doubles.  Same reflectors as
// hessenberg_reduce (norm, tau, v), sums in a different order.
__device__ inline void hessenberg_reduce_chunked(double *A, int lda, double *Z, int ldz, int n, double *v,
                                                 double *sc, double *part) {
    typedef double R;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = lane_id(), w = warp_id();
    for (int e = tid; e < n * n; e += nt) M_(Z, ldz, e % n, e / n) = (e % n == e / n) ? R(1) : R(0);
    sync();
    for (int c = 0; c + 2 < n; c++) {
        if (w == 0) {
            R s = R(0);
            for (int i = c + 1 + lane; i < n; i += 32) s += M_(A, lda, i, c) * M_(A, lda, i, c);
            s = warp_sum(s);
            if (lane == 0) {
                const R x0 = M_(A, lda, c + 1, c);
                const R nrm = sqrt(s);
                R tau = R(0), alpha = x0;
                if (nrm > R(0) && s - x0 * x0 > R(0)) {
                    alpha = -copysign(nrm, x0);
                    tau = (alpha - x0) / alpha;
                    sc[1] = R(1) / (x0 - alpha);
                } else {
                    sc[1] = R(0);
                }
                sc[0] = tau;
                sc[2] = alpha;
            }
        }
        sync();
        const R tau = sc[0], inv = sc[1];
        sync();
        if (tau == R(0)) continue;
        for (int i = c + 1 + tid; i < n; i += nt) v[i] = (i == c + 1) ? R(1) : M_(A, lda, i, c) * inv;
        sync();
        // left: columns j in [c, n), rows in four interleaved chunks
        const int ncl = n - c;
        for (int t = tid; t < 4 * ncl; t += nt) {
            const int j = c + t % ncl, r = t / ncl;
            R s = R(0);
            for (int i = c + 1 + r; i < n; i += 4) s += v[i] * M_(A, lda, i, j);
            part[r * n + j] = s;
        }
        sync();
        for (int t = tid; t < 4 * ncl; t += nt) {
            const int j = c + t % ncl, r = t / ncl;
            const R d = tau * ((part[j] + part[n + j]) + (part[2 * n + j] + part[3 * n + j]));
            for (int i = c + 1 + r; i < n; i += 4) M_(A, lda, i, j) -= d * v[i];
        }
        sync();
        // right: rows of A and Z (2n), columns in [c+1, n) in four interleaved chunks
        for (int t = tid; t < 8 * n; t += nt) {
            const int rho = t % (2 * n), r = t / (2 * n);
            const R *Mx = (rho < n) ? A : Z;
            const int ldm = (rho < n) ? lda : ldz;
            const int i = (rho < n) ? rho : rho - n;
            R s = R(0);
            for (int j = c + 1 + r; j < n; j += 4) s += M_(Mx, ldm, i, j) * v[j];
            part[r * 2 * n + rho] = s;
        }
        sync();
        for (int t = tid; t < 8 * n; t += nt) {
            const int rho = t % (2 * n), r = t / (2 * n);
            R *Mx = (rho < n) ? A : Z;
            const int ldm = (rho < n) ? lda : ldz;
            const int i = (rho < n) ? rho : rho - n;
            const R d = tau * ((part[rho] + part[2 * n + rho]) + (part[4 * n + rho] + part[6 * n + rho]));
            for (int j = c + 1 + r; j < n; j += 4) M_(Mx, ldm, i, j) -= d * v[j];
        }
        sync();
        if (tid == 0) M_(A, lda, c + 1, c) = sc[2];
        for (int i = c + 2 + tid; i < n; i += nt) M_(A, lda, i, c) = R(0);
        sync();
    }
}

// Householder vector for u = (x, y, z): P u = alpha e1.  Writes tau, v1, v2.
// With a = -sign(x) ||u||: v = (1, y / (x - a), z / (x - a)), tau = (a - x) / a.
// Both quotients come from one reciprocal, 1 / (a (x - a)); u is rescaled
// first only when its entries are far from 1 (squares that could overflow or
// underflow), since every division and square root is a long chain of FP64
// instructions on this GPU.
template <typename R>
__device__ __forceinline__ void house3(R x, R y, R z, R &tau, R &v1, R &v2) {
    const R s = fabs(x) + fabs(y) + fabs(z);
    if (s == R(0) || (y == R(0) && z == R(0))) {
        tau = R(0);
        v1 = v2 = R(0);
        return;
    }
    constexpr R BIG = (sizeof(R) == 8) ? R(1e100) : R(1e15);
    constexpr R SMALL = (sizeof(R) == 8) ? R(1e-100) : R(1e-15);
    R xs = x, ys = y, zs = z;
    if (s > BIG || s < SMALL) {
        const R is = R(1) / s;
        xs *= is;
        ys *= is;
        zs *= is;
    }
    const R nrm = sqrt(xs * xs + ys * ys + zs * zs);
    const R a = -copysign(nrm, xs);
    const R d = xs - a;                 // = sign(x) (|x| + ||u||), never 0
    const R r = R(1) / (a * d);
    tau = -d * d * r;                   // (a - x) / a
    const R id = a * r;                 // 1 / (x - a)
    v1 = ys * id;
    v2 = zs * id;
}

// Real Schur form of an upper Hessenberg H (n x n) by the Francis
// double-shift QR algorithm (Golub & Van Loan, Alg. 7.5.1-7.5.2), with the
// Schur vectors accumulated into Z.  Run by warp 0 alone (lanes split the
// row and column updates, lane 0 takes the scalar decisions, __syncwarp
// orders them): the bulge chase is a serial chain, so a single warp with
// cheap synchronisation is the fastest executor.  Real eigenvalue pairs of
// 2x2 blocks are split by a rotation; the remaining 2x2 blocks hold complex
// pairs, with wi[p] > 0 and wi[p+1] = -wi[p].  Call from all threads.
// Returns 0, or 1 if the iteration limit was hit (valid on every thread).
template <typename R>
__device__ inline int francis_schur(R *H, int ldh, R *Z, int ldz, int n, R *wr, R *wi, int *isc) {
    constexpr R EPS = (sizeof(R) == 8) ? R(2.220446049250313e-16) : R(5.9604645e-8);
    const unsigned FULL = 0xffffffffu;
    if (warp_id() == 0) {
        const int lane = lane_id();
        int hi = n - 1, its = 0, total = 0, fail = 0;
        while (hi >= 0) {
            // every lane takes the same scalar decisions from the same shared
            // values, so no broadcast is needed.  l: the largest index <= hi
            // with a negligible subdiagonal H(l, l-1) (0 if none), 32
            // candidates per ballot
            int l = 0;
            for (int base = hi; base > 0; base -= 32) {
                const int i = base - lane;
                bool neg = false;
                if (i > 0) {
                    R s = fabs(M_(H, ldh, i - 1, i - 1)) + fabs(M_(H, ldh, i, i));
                    if (s == R(0)) s = R(1);
                    neg = fabs(M_(H, ldh, i, i - 1)) <= EPS * s;
                }
                const unsigned m = __ballot_sync(FULL, neg);
                if (m != 0u) {
                    l = base - (__ffs(m) - 1);
                    break;
                }
            }
            __syncwarp();
            if (l > 0 && lane == 0) M_(H, ldh, l, l - 1) = R(0);
            if (l == hi) {
                if (lane == 0) {
                    wr[hi] = M_(H, ldh, hi, hi);
                    wi[hi] = R(0);
                }
                hi -= 1;
                its = 0;
                __syncwarp();
                continue;
            }
            if (l == hi - 1) {
                const int p = hi - 1;
                R cs = R(1), sn = R(0);
                int rot = 0;
                const R a = M_(H, ldh, p, p), b = M_(H, ldh, p, p + 1);
                const R c = M_(H, ldh, p + 1, p), d = M_(H, ldh, p + 1, p + 1);
                const R hp = R(0.5) * (a - d);
                const R disc = hp * hp + b * c;
                R w0, w1, i0, i1;
                if (disc >= R(0)) {
                    const R q = sqrt(disc);
                    const R zz = hp + copysign(q, hp);
                    R l1, l2;
                    if (zz == R(0)) {
                        l1 = l2 = d;
                    } else {
                        l1 = d + zz;
                        l2 = d - b * c / zz;
                    }
                    R e0 = l1 - d, e1 = c;
                    if (fabs(e0) + fabs(e1) == R(0)) {
                        e0 = b;
                        e1 = l1 - a;
                    }
                    const R nrm = hypot(e0, e1);
                    if (nrm > R(0)) {
                        cs = e0 / nrm;
                        sn = e1 / nrm;
                    }
                    rot = 1;
                    w0 = l1;
                    w1 = l2;
                    i0 = i1 = R(0);
                } else {
                    const R q = sqrt(-disc);
                    w0 = w1 = hp + d;
                    i0 = q;
                    i1 = -q;
                }
                __syncwarp();
                if (lane == 0) {
                    wr[p] = w0;
                    wr[p + 1] = w1;
                    wi[p] = i0;
                    wi[p + 1] = i1;
                }
                if (rot) {
                    for (int j = p + lane; j < n; j += 32) {
                        const R a0 = M_(H, ldh, p, j), a1 = M_(H, ldh, p + 1, j);
                        M_(H, ldh, p, j) = cs * a0 + sn * a1;
                        M_(H, ldh, p + 1, j) = -sn * a0 + cs * a1;
                    }
                    __syncwarp();
                    for (int i = lane; i < p + 2; i += 32) {
                        const R a0 = M_(H, ldh, i, p), a1 = M_(H, ldh, i, p + 1);
                        M_(H, ldh, i, p) = cs * a0 + sn * a1;
                        M_(H, ldh, i, p + 1) = -sn * a0 + cs * a1;
                    }
                    for (int i = lane; i < n; i += 32) {
                        const R a0 = M_(Z, ldz, i, p), a1 = M_(Z, ldz, i, p + 1);
                        M_(Z, ldz, i, p) = cs * a0 + sn * a1;
                        M_(Z, ldz, i, p + 1) = -sn * a0 + cs * a1;
                    }
                    __syncwarp();
                    if (lane == 0) M_(H, ldh, p + 1, p) = R(0);
                }
                hi -= 2;
                its = 0;
                __syncwarp();
                continue;
            }
            its++;
            total++;
            if (total > 40 * n) {
                fail = 1;
                break;
            }
            R x, y, z;
            {
                R s, t;
                if (its == 10 || its == 20) {
                    const R w = fabs(M_(H, ldh, hi, hi - 1)) + fabs(M_(H, ldh, hi - 1, hi - 2));
                    const R xx = R(0.75) * w + M_(H, ldh, hi, hi);
                    s = R(2) * xx;
                    t = xx * xx + R(0.4375) * w * w;
                } else {
                    const R a = M_(H, ldh, hi - 1, hi - 1), b = M_(H, ldh, hi - 1, hi);
                    const R c = M_(H, ldh, hi, hi - 1), d = M_(H, ldh, hi, hi);
                    s = a + d;
                    t = a * d - b * c;
                }
                const R h00 = M_(H, ldh, l, l), h01 = M_(H, ldh, l, l + 1);
                const R h10 = M_(H, ldh, l + 1, l), h11 = M_(H, ldh, l + 1, l + 1);
                const R h21 = M_(H, ldh, l + 2, l + 1);
                x = h00 * h00 + h01 * h10 - s * h00 + t;
                y = h10 * (h00 + h11 - s);
                z = h10 * h21;
            }
            __syncwarp();
            for (int kk = l; kk <= hi - 1; kk++) {
                const int nr = (kk == hi - 1) ? 2 : 3;
                R tau, v1, v2;
                house3(x, y, nr == 3 ? z : R(0), tau, v1, v2);
                if (tau != R(0)) {
                    const int c0 = (kk > l) ? kk - 1 : l;
                    for (int j = c0 + lane; j < n; j += 32) {
                        R tt = M_(H, ldh, kk, j) + v1 * M_(H, ldh, kk + 1, j);
                        if (nr == 3) tt += v2 * M_(H, ldh, kk + 2, j);
                        tt *= tau;
                        M_(H, ldh, kk, j) -= tt;
                        M_(H, ldh, kk + 1, j) -= tt * v1;
                        if (nr == 3) M_(H, ldh, kk + 2, j) -= tt * v2;
                    }
                    __syncwarp();
                    const int rmax = min(kk + 3, hi);
                    for (int e = lane; e < (rmax + 1) + n; e += 32) {
                        R *Mx = (e <= rmax) ? H : Z;
                        const int ldm = (e <= rmax) ? ldh : ldz;
                        const int i = (e <= rmax) ? e : e - (rmax + 1);
                        R tt = M_(Mx, ldm, i, kk) + v1 * M_(Mx, ldm, i, kk + 1);
                        if (nr == 3) tt += v2 * M_(Mx, ldm, i, kk + 2);
                        tt *= tau;
                        M_(Mx, ldm, i, kk) -= tt;
                        M_(Mx, ldm, i, kk + 1) -= tt * v1;
                        if (nr == 3) M_(Mx, ldm, i, kk + 2) -= tt * v2;
                    }
                    __syncwarp();
                }
                if (kk < hi - 1) {
                    x = M_(H, ldh, kk + 1, kk);
                    y = M_(H, ldh, kk + 2, kk);
                    z = (kk < hi - 2) ? M_(H, ldh, kk + 3, kk) : R(0);
                }
                __syncwarp();
                if (lane == 0 && kk > l) {
                    M_(H, ldh, kk + 1, kk - 1) = R(0);
                    if (nr == 3) M_(H, ldh, kk + 2, kk - 1) = R(0);
                }
            }
            __syncwarp();
        }
        if (lane == 0) isc[0] = fail;
    }
    sync();
    const int fail = isc[0];
    sync();
    return fail;
}

// Named barrier among the first `nthreads` threads (whole warps) of the CTA.
__device__ __forceinline__ void named_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// francis_schur for FP64 on four warps, one per SM sub-partition: an FP64
// warp instruction occupies a sub-partition's FP64 pipe for many cycles, so
// the serial bulge chase is bound by the chain of dependent FP64
// instructions per bulge step, the reflector above all.  The chase runs with
// a one-step lookahead, in two phases per step kk separated by barriers of
// all four warps:
//   A: warp 0 computes the reflector of step kk from (x, y, z); warps 1-3
//      apply the reflector of step kk - 1 to everything outside its critical
//      block (rows kk-1..kk+1 right of column kk+2, columns kk-1..kk+1 down
//      to row kk-1, and the Schur vectors Z);
//   B: warp 0 applies the reflector of step kk to its critical block (rows
//      kk..kk+2 from column c0 to kk+3, then columns kk..kk+2 from row kk+1
//      to kk+3), which holds every entry the next reflector reads, takes the
//      next (x, y, z) from it and publishes the reflector in `pub`.
// So the reflector chain no longer waits for the long row, column and Z
// updates.  Every entry receives the same updates, in the same order and
// with the same arithmetic, as in francis_schur, hence the same results.
// The deflation scans, shifts and 2x2 blocks are computed by every warp
// alike; their few writes are warp 0's.
__device__ inline int francis_schur_4w(double *H, int ldh, double *Z, int ldz, int n, double *wr, double *wi,
                                       int *isc, double *pub) {
    typedef double R;
    constexpr R EPS = R(2.220446049250313e-16);
    const unsigned FULL = 0xffffffffu;
    constexpr int BAR_ALL = 1;
    if (warp_id() < 4) {
        const int lane = lane_id(), w = warp_id();
        int hi = n - 1, its = 0, total = 0, fail = 0;
        while (hi >= 0) {
            int l = 0;
            for (int base = hi; base > 0; base -= 32) {
                const int i = base - lane;
                bool neg = false;
                if (i > 0) {
                    R sm = fabs(M_(H, ldh, i - 1, i - 1)) + fabs(M_(H, ldh, i, i));
                    if (sm == R(0)) sm = R(1);
                    neg = fabs(M_(H, ldh, i, i - 1)) <= EPS * sm;
                }
                const unsigned m = __ballot_sync(FULL, neg);
                if (m != 0u) {
                    l = base - (__ffs(m) - 1);
                    break;
                }
            }
            named_bar(BAR_ALL, 128);   // every warp has read the subdiagonal
            if (l > 0 && w == 0 && lane == 0) M_(H, ldh, l, l - 1) = R(0);
            if (l == hi) {
                if (w == 0 && lane == 0) {
                    wr[hi] = M_(H, ldh, hi, hi);
                    wi[hi] = R(0);
                }
                hi -= 1;
                its = 0;
                named_bar(BAR_ALL, 128);
                continue;
            }
            if (l == hi - 1) {
                // a 2x2 block: warp 0 splits real pairs by a rotation (as francis_schur)
                if (w == 0) {
                    const int p = hi - 1;
                    R cs = R(1), sn = R(0);
                    int rot = 0;
                    const R a = M_(H, ldh, p, p), b = M_(H, ldh, p, p + 1);
                    const R c = M_(H, ldh, p + 1, p), d = M_(H, ldh, p + 1, p + 1);
                    const R hp = R(0.5) * (a - d);
                    const R disc = hp * hp + b * c;
                    R w0, w1, i0, i1;
                    if (disc >= R(0)) {
                        const R q = sqrt(disc);
                        const R zz = hp + copysign(q, hp);
                        R l1, l2;
                        if (zz == R(0)) {
                            l1 = l2 = d;
                        } else {
                            l1 = d + zz;
                            l2 = d - b * c / zz;
                        }
                        R e0 = l1 - d, e1 = c;
                        if (fabs(e0) + fabs(e1) == R(0)) {
                            e0 = b;
                            e1 = l1 - a;
                        }
                        const R nrm = hypot(e0, e1);
                        if (nrm > R(0)) {
                            cs = e0 / nrm;
                            sn = e1 / nrm;
                        }
                        rot = 1;
                        w0 = l1;
                        w1 = l2;
                        i0 = i1 = R(0);
                    } else {
                        const R q = sqrt(-disc);
                        w0 = w1 = hp + d;
                        i0 = q;
                        i1 = -q;
                    }
                    __syncwarp();
                    if (lane == 0) {
                        wr[p] = w0;
                        wr[p + 1] = w1;
                        wi[p] = i0;
                        wi[p + 1] = i1;
                    }
                    if (rot) {
                        for (int j = p + lane; j < n; j += 32) {
                            const R a0 = M_(H, ldh, p, j), a1 = M_(H, ldh, p + 1, j);
                            M_(H, ldh, p, j) = cs * a0 + sn * a1;
                            M_(H, ldh, p + 1, j) = -sn * a0 + cs * a1;
                        }
                        __syncwarp();
                        for (int i = lane; i < p + 2; i += 32) {
                            const R a0 = M_(H, ldh, i, p), a1 = M_(H, ldh, i, p + 1);
                            M_(H, ldh, i, p) = cs * a0 + sn * a1;
                            M_(H, ldh, i, p + 1) = -sn * a0 + cs * a1;
                        }
                        for (int i = lane; i < n; i += 32) {
                            const R a0 = M_(Z, ldz, i, p), a1 = M_(Z, ldz, i, p + 1);
                            M_(Z, ldz, i, p) = cs * a0 + sn * a1;
                            M_(Z, ldz, i, p + 1) = -sn * a0 + cs * a1;
                        }
                        __syncwarp();
                        if (lane == 0) M_(H, ldh, p + 1, p) = R(0);
                    }
                }
                hi -= 2;
                its = 0;
                named_bar(BAR_ALL, 128);
                continue;
            }
            its++;
            total++;
            if (total > 40 * n) {
                fail = 1;
                break;
            }
            R x, y, z;
            {
                R sh, t;
                if (its == 10 || its == 20) {
                    const R ww = fabs(M_(H, ldh, hi, hi - 1)) + fabs(M_(H, ldh, hi - 1, hi - 2));
                    const R xx = R(0.75) * ww + M_(H, ldh, hi, hi);
                    sh = R(2) * xx;
                    t = xx * xx + R(0.4375) * ww * ww;
                } else {
                    const R a = M_(H, ldh, hi - 1, hi - 1), b = M_(H, ldh, hi - 1, hi);
                    const R c = M_(H, ldh, hi, hi - 1), d = M_(H, ldh, hi, hi);
                    sh = a + d;
                    t = a * d - b * c;
                }
                const R h00 = M_(H, ldh, l, l), h01 = M_(H, ldh, l, l + 1);
                const R h10 = M_(H, ldh, l + 1, l), h11 = M_(H, ldh, l + 1, l + 1);
                const R h21 = M_(H, ldh, l + 2, l + 1);
                x = h00 * h00 + h01 * h10 - sh * h00 + t;
                y = h10 * (h00 + h11 - sh);
                z = h10 * h21;
            }
            named_bar(BAR_ALL, 128);   // every warp has read the shift inputs
            R tau = R(0), v1 = R(0), v2 = R(0);
            for (int kk = l; kk <= hi; kk++) {
                // phase A
                if (w == 0) {
                    if (kk <= hi - 1) house3(x, y, (kk == hi - 1) ? R(0) : z, tau, v1, v2);
                } else if (kk > l) {
                    // step pk = kk - 1 outside its critical block
                    const int pk = kk - 1;
                    const bool three = pk < hi - 1;
                    const R ptau = pub[0], pv1 = pub[1], pv2 = pub[2];
                    if (ptau != R(0)) {
                        const int cend = min(pk + 3, n - 1);
                        const int nzr = n, ncol = n - 1 - cend, nrow = pk;
                        for (int it = (w - 1) * 32 + lane; it < nzr + ncol + nrow; it += 96) {
                            if (it < nzr) {
                                // row it of the Schur vectors
                                const int i = it;
                                R tt = M_(Z, ldz, i, pk) + pv1 * M_(Z, ldz, i, pk + 1);
                                if (three) tt += pv2 * M_(Z, ldz, i, pk + 2);
                                tt *= ptau;
                                M_(Z, ldz, i, pk) -= tt;
                                M_(Z, ldz, i, pk + 1) -= tt * pv1;
                                if (three) M_(Z, ldz, i, pk + 2) -= tt * pv2;
                            } else if (it < nzr + ncol) {
                                // column j of rows pk..pk+2, right of the critical block
                                const int j = cend + 1 + (it - nzr);
                                R tt = M_(H, ldh, pk, j) + pv1 * M_(H, ldh, pk + 1, j);
                                if (three) tt += pv2 * M_(H, ldh, pk + 2, j);
                                tt *= ptau;
                                M_(H, ldh, pk, j) -= tt;
                                M_(H, ldh, pk + 1, j) -= tt * pv1;
                                if (three) M_(H, ldh, pk + 2, j) -= tt * pv2;
                            } else {
                                // row i < pk of columns pk..pk+2, above the critical block
                                const int i = it - nzr - ncol;
                                R tt = M_(H, ldh, i, pk) + pv1 * M_(H, ldh, i, pk + 1);
                                if (three) tt += pv2 * M_(H, ldh, i, pk + 2);
                                tt *= ptau;
                                M_(H, ldh, i, pk) -= tt;
                                M_(H, ldh, i, pk + 1) -= tt * pv1;
                                if (three) M_(H, ldh, i, pk + 2) -= tt * pv2;
                            }
                        }
                    }
                }
                named_bar(BAR_ALL, 128);   // reflector kk ready; step kk - 1 complete
                if (kk == hi) break;
                // phase B: the critical block of step kk (warp 0)
                if (w == 0) {
                    const bool three = kk < hi - 1;
                    if (tau != R(0)) {
                        const int c0 = (kk > l) ? kk - 1 : l;
                        const int cend = min(kk + 3, n - 1);
                        const int j = c0 + lane;
                        if (j <= cend) {
                            R tt = M_(H, ldh, kk, j) + v1 * M_(H, ldh, kk + 1, j);
                            if (three) tt += v2 * M_(H, ldh, kk + 2, j);
                            tt *= tau;
                            M_(H, ldh, kk, j) -= tt;
                            M_(H, ldh, kk + 1, j) -= tt * v1;
                            if (three) M_(H, ldh, kk + 2, j) -= tt * v2;
                        }
                        __syncwarp();
                        const int rmax = min(kk + 3, hi);
                        const int i = kk + lane;
                        if (i <= rmax) {
                            R tt = M_(H, ldh, i, kk) + v1 * M_(H, ldh, i, kk + 1);
                            if (three) tt += v2 * M_(H, ldh, i, kk + 2);
                            tt *= tau;
                            M_(H, ldh, i, kk) -= tt;
                            M_(H, ldh, i, kk + 1) -= tt * v1;
                            if (three) M_(H, ldh, i, kk + 2) -= tt * v2;
                        }
                        __syncwarp();
                    }
                    if (kk < hi - 1) {
                        x = M_(H, ldh, kk + 1, kk);
                        y = M_(H, ldh, kk + 2, kk);
                        z = (kk < hi - 2) ? M_(H, ldh, kk + 3, kk) : R(0);
                    }
                    __syncwarp();
                    if (lane == 0) {
                        if (kk > l) {
                            // the bulge entries of column kk - 1: nothing reads them again in this sweep
                            M_(H, ldh, kk + 1, kk - 1) = R(0);
                            if (three) M_(H, ldh, kk + 2, kk - 1) = R(0);
                        }
                        pub[0] = tau;
                        pub[1] = v1;
                        pub[2] = v2;
                    }
                }
                named_bar(BAR_ALL, 128);   // critical block of step kk and its reflector published
            }
        }
        if (w == 0 && lane == 0) isc[0] = fail;
    }
    sync();
    const int fail = isc[0];
    sync();
    return fail;
}

// FP64 Schur forms run on four warps, FP32 ones on one (its instructions are
// cheap enough that barriers between warps would cost more than they save).
template <typename R>
__device__ inline int schur_form(R *H, int ldh, R *Z, int ldz, int n, R *wr, R *wi, int *isc, R *pub) {
    if constexpr (sizeof(R) == 8)
        return francis_schur_4w(H, ldh, Z, ldz, n, wr, wi, isc, pub);
    else
        return francis_schur(H, ldh, Z, ldz, n, wr, wi, isc);
}
// Complex helpers (re, im pairs).
template <typename R>
__device__ __forceinline__ void cdiv(R ar, R ai, R br, R bi, R &cr, R &ci) {
    if (fabs(br) >= fabs(bi)) {
        const R r = bi / br, d = br + r * bi;
        cr = (ar + r * ai) / d;
        ci = (ai - r * ar) / d;
    } else {
        const R r = br / bi, d = bi + r * br;
        cr = (r * ar + ai) / d;
        ci = (r * ai - ar) / d;
    }
}

// Eigenvector of the quasi-triangular T for eigenvalue at position p (real,
// or the first of a complex pair when wi[p] > 0), by back substitution.
// Writes xr, xi (n entries each; xi = 0 for a real eigenvalue).
template <typename R>
__device__ inline void schur_eigvec(const R *T, int ldt, int n, const R *wr, const R *wi, int p, R *xr,
                                    R *xi, R tnorm) {
    constexpr R EPS = (sizeof(R) == 8) ? R(2.220446049250313e-16) : R(5.9604645e-8);
    const R small = EPS * fmax(tnorm, R(1e-30));
    for (int i = 0; i < n; i++) {
        xr[i] = R(0);
        xi[i] = R(0);
    }
    const R lr = wr[p], li = wi[p];
    if (li == R(0)) {
        xr[p] = R(1);
    } else {
        const R d = M_(T, ldt, p + 1, p + 1), c = M_(T, ldt, p + 1, p);
        xr[p] = lr - d;
        xi[p] = li;
        xr[p + 1] = c;
        xi[p + 1] = R(0);
    }
    const int last = (li == R(0)) ? p : p + 1;
    int i = p - 1;
    while (i >= 0) {
        const bool two = (i > 0) && (M_(T, ldt, i, i - 1) != R(0));
        if (!two) {
            R sr = R(0), si = R(0);
            for (int c = i + 1; c <= last; c++) {
                sr += M_(T, ldt, i, c) * xr[c];
                si += M_(T, ldt, i, c) * xi[c];
            }
            R dr = M_(T, ldt, i, i) - lr, di = -li;
            if (fabs(dr) + fabs(di) < small) dr = small;
            R qr, qi;
            cdiv(-sr, -si, dr, di, qr, qi);
            xr[i] = qr;
            xi[i] = qi;
            i -= 1;
        } else {
            const int a = i - 1;
            R s0r = R(0), s0i = R(0), s1r = R(0), s1i = R(0);
            for (int c = i + 1; c <= last; c++) {
                s0r += M_(T, ldt, a, c) * xr[c];
                s0i += M_(T, ldt, a, c) * xi[c];
                s1r += M_(T, ldt, i, c) * xr[c];
                s1i += M_(T, ldt, i, c) * xi[c];
            }
            const R b00r = M_(T, ldt, a, a) - lr, b00i = -li;
            const R b01 = M_(T, ldt, a, i), b10 = M_(T, ldt, i, a);
            const R b11r = M_(T, ldt, i, i) - lr, b11i = -li;
            R detr = b00r * b11r - b00i * b11i - b01 * b10;
            R deti = b00r * b11i + b00i * b11r;
            if (fabs(detr) + fabs(deti) < small * small) detr = small * small;
            const R n0r = -(s0r * b11r - s0i * b11i) + b01 * s1r;
            const R n0i = -(s0r * b11i + s0i * b11r) + b01 * s1i;
            const R n1r = -(s1r * b00r - s1i * b00i) + b10 * s0r;
            const R n1i = -(s1r * b00i + s1i * b00r) + b10 * s0i;
            cdiv(n0r, n0i, detr, deti, xr[a], xi[a]);
            cdiv(n1r, n1i, detr, deti, xr[i], xi[i]);
            i -= 2;
        }
        R mx = R(0);
        for (int c = (i + 1 > 0 ? i + 1 : 0); c <= last; c++) mx = fmax(mx, fabs(xr[c]) + fabs(xi[c]));
        const R big = (sizeof(R) == 8) ? R(1e100) : R(1e20);
        if (mx > big) {
            const R f = R(1) / mx;
            for (int c = 0; c <= last; c++) {
                xr[c] *= f;
                xi[c] *= f;
            }
        }
    }
}

// Eigenvectors of the quasi-triangular T for the npick eigenvalues at
// positions pick[0..npick) (real, or the first of a complex pair when
// wi[p] > 0), by back substitution, all at once on warp 0: lane q solves for
// pick[q] (npick <= 32), every lane stepping through the same rows in the
// same order (the 2x2 blocks of T are common to all), inactive above its own
// eigenvalue.  x is stored lane-interleaved, xr[c * npick + q] (conflict-free
// shared-memory access); xi = 0 for a real eigenvalue.  A growing vector is
// rescaled when an entry exceeds `big`, as one vector at a time would be.
template <typename R>
__device__ inline void schur_eigvecs_lanes(const R *T, int ldt, int n, const R *wr, const R *wi, const int *pick,
                                           int npick, R *xr, R *xi, R tnorm) {
    constexpr R EPS = (sizeof(R) == 8) ? R(2.220446049250313e-16) : R(5.9604645e-8);
    const R big = (sizeof(R) == 8) ? R(1e100) : R(1e20);
    if (warp_id() == 0) {
        const int q = lane_id();
        const bool on = q < npick;
        const int p = on ? pick[q] : n;
        const R lr = on ? wr[p] : R(0), li = on ? wi[p] : R(0);
        const R small = EPS * fmax(tnorm, R(1e-30));
        if (on) {
            for (int c = 0; c < n; c++) {
                xr[c * npick + q] = R(0);
                xi[c * npick + q] = R(0);
            }
            if (li == R(0)) {
                xr[p * npick + q] = R(1);
            } else {
                xr[p * npick + q] = lr - M_(T, ldt, p + 1, p + 1);
                xi[p * npick + q] = li;
                xr[(p + 1) * npick + q] = M_(T, ldt, p + 1, p);
            }
        }
        __syncwarp();
        int i = n - 1;
        while (i >= 0) {
            const bool two = (i > 0) && (M_(T, ldt, i, i - 1) != R(0));
            const bool act = on && i < p;
            R mx = R(0);
            if (!two) {
                R sr = R(0), si = R(0);
                for (int c = i + 1; c < n; c++) {
                    const R t = M_(T, ldt, i, c);
                    sr += t * xr[c * npick + q * (int)on];
                    si += t * xi[c * npick + q * (int)on];
                }
                if (act) {
                    R dr = M_(T, ldt, i, i) - lr, di = -li;
                    if (fabs(dr) + fabs(di) < small) dr = small;
                    R qr, qi;
                    cdiv(-sr, -si, dr, di, qr, qi);
                    xr[i * npick + q] = qr;
                    xi[i * npick + q] = qi;
                    mx = fabs(qr) + fabs(qi);
                }
                i -= 1;
            } else {
                const int a = i - 1;
                R s0r = R(0), s0i = R(0), s1r = R(0), s1i = R(0);
                for (int c = i + 1; c < n; c++) {
                    const R t0 = M_(T, ldt, a, c), t1 = M_(T, ldt, i, c);
                    const R vr = xr[c * npick + q * (int)on], vi = xi[c * npick + q * (int)on];
                    s0r += t0 * vr;
                    s0i += t0 * vi;
                    s1r += t1 * vr;
                    s1i += t1 * vi;
                }
                if (act) {
                    const R b00r = M_(T, ldt, a, a) - lr, b00i = -li;
                    const R b01 = M_(T, ldt, a, i), b10 = M_(T, ldt, i, a);
                    const R b11r = M_(T, ldt, i, i) - lr, b11i = -li;
                    R detr = b00r * b11r - b00i * b11i - b01 * b10;
                    R deti = b00r * b11i + b00i * b11r;
                    if (fabs(detr) + fabs(deti) < small * small) detr = small * small;
                    const R n0r = -(s0r * b11r - s0i * b11i) + b01 * s1r;
                    const R n0i = -(s0r * b11i + s0i * b11r) + b01 * s1i;
                    const R n1r = -(s1r * b00r - s1i * b00i) + b10 * s0r;
                    const R n1i = -(s1r * b00i + s1i * b00r) + b10 * s0i;
                    R ar, ai, cr, ci;
                    cdiv(n0r, n0i, detr, deti, ar, ai);
                    cdiv(n1r, n1i, detr, deti, cr, ci);
                    xr[a * npick + q] = ar;
                    xi[a * npick + q] = ai;
                    xr[i * npick + q] = cr;
                    xi[i * npick + q] = ci;
                    mx = fmax(fabs(ar) + fabs(ai), fabs(cr) + fabs(ci));
                }
                i -= 2;
            }
            if (act && mx > big) {
                const R f = R(1) / mx;
                for (int c = 0; c < n; c++) {
                    xr[c * npick + q] *= f;
                    xi[c * npick + q] *= f;
                }
            }
            __syncwarp();
        }
    }
}

// Harmonic-Ritz selection (Algorithm 2): eigen-decompose M (n x n), keep the
// eigenvectors whose eigenvalues mu have the largest |mu|, i.e. the smallest
// |theta| for theta = 1/mu (ties: smaller Re theta, then smaller Im theta,
// then lower index; keys: 3n doubles of scratch), at most kwant of them; a complex pair contributes the
// real and imaginary parts of one eigenvector and is dropped if the kwant-th
// pick would split it.  M64 (FP64, ld64) is the input; the eigen-solve runs
// in precision R on Mr (n x n, ldm; may alias M64 when R = double) with
// Schur vectors Zr (ldz = n).  Writes P (FP64, n x knew, ldp) and returns
// knew (-1 if the QR iteration failed).
// marks (optional, thread 0 writes): the device clock after the Hessenberg
// reduction, after the Schur form and after the eigenvectors.
template <typename R>
__device__ __noinline__ int harmonic_select(const double *M64, int ld64, int n, int kwant, double *P, int ldp,
                                      R *Mr, int ldm, R *Zr, R *wr, R *wi, R *xr, R *xi, R *vscr,
                                      R *scr, int *isc, double *keys, unsigned long long *marks = nullptr) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if ((const void *)Mr != (const void *)M64) {
        for (int e = tid; e < n * n; e += nt) M_(Mr, ldm, e % n, e / n) = (R)M_(M64, ld64, e % n, e / n);
        sync();
    }
    if constexpr (sizeof(R) == 8) {
        // xr, xi (contiguous, 2 (k + 1) m doubles) are free until the eigenvectors
        if (2 * (kwant + 1) * n >= 8 * n)
            hessenberg_reduce_chunked(Mr, ldm, Zr, n, n, vscr, scr, xr);
        else
            hessenberg_reduce(Mr, ldm, Zr, n, n, vscr, scr);
    } else {
        hessenberg_reduce(Mr, ldm, Zr, n, n, vscr, scr);
    }
    if (marks && threadIdx.x == 0) marks[2] = global_ns();
    const int fail = schur_form(Mr, ldm, Zr, n, n, wr, wi, isc, vscr);   // vscr: free during the Schur form
    if (marks && threadIdx.x == 0) marks[0] = global_ns();
    if (fail) return -1;
    int *rank = isc + 8;
    int *pick = isc + 8 + MMAX;
    // sort keys (|theta|, Re theta, Im theta) for theta = 1/mu, one per thread
    for (int i = tid; i < n; i += nt) {
        const double a = (double)wr[i], b = (double)wi[i];
        const double m2 = a * a + b * b;
        const double inv = (m2 == 0.0) ? 0.0 : 1.0 / m2;
        keys[i] = (m2 == 0.0) ? INFINITY : sqrt(inv);
        keys[n + i] = (m2 == 0.0) ? INFINITY : a * inv;
        keys[2 * n + i] = (m2 == 0.0) ? INFINITY : -b * inv;
    }
    sync();
    for (int i = tid; i < n; i += nt) {
        const double a0 = keys[i], a1 = keys[n + i], a2 = keys[2 * n + i];
        int r = 0;
        for (int q = 0; q < n; q++) {
            if (q == i) continue;
            const double b0 = keys[q], b1 = keys[n + q], b2 = keys[2 * n + q];
            const bool before =
                (b0 < a0) || (b0 == a0 && (b1 < a1 || (b1 == a1 && (b2 < a2 || (b2 == a2 && q < i)))));
            r += before ? 1 : 0;
        }
        rank[i] = r;
    }
    sync();
    // position of each rank, and the max-norm of the Schur form (warp 0)
    int *pos = isc + 8 + 3 * MMAX;
    for (int i = tid; i < n; i += nt) pos[rank[i]] = i;
    if (warp_id() == 0) {
        R tn = R(0);
        for (int e = lane_id(); e < n * n; e += 32) tn = fmax(tn, fabs(M_(Mr, ldm, e % n, e / n)));
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, off));
        if (lane_id() == 0) scr[3] = tn;
    }
    sync();
    if (tid == 0) {
        int cols = 0, npick = 0;
        for (int r = 0; r < kwant && r < n; r++) {
            const int q = pos[r];
            if (wi[q] == R(0)) {
                pick[npick++] = q;
                cols += 1;
            } else {
                const int p0 = (wi[q] > R(0)) ? q : q - 1;
                const int partner = (q == p0) ? p0 + 1 : p0;
                if (rank[partner] < kwant && rank[partner] > r) {
                    pick[npick++] = p0;
                    cols += 2;
                }
            }
        }
        isc[1] = npick;
        isc[2] = cols;
    }
    sync();
    const int npick = isc[1], knew = isc[2];
    const R tnorm = scr[3];
    // all picked eigenvectors at once, one per lane of warp 0
    schur_eigvecs_lanes(Mr, ldm, n, wr, wi, pick, npick, xr, xi, tnorm);
    sync();
    if (marks && threadIdx.x == 0) marks[1] = global_ns();
    int *colof = isc + 8 + 2 * MMAX;
    if (tid == 0) {
        int c = 0;
        for (int q = 0; q < npick; q++) {
            colof[q] = c;
            c += (wi[pick[q]] == R(0)) ? 1 : 2;
        }
    }
    sync();
    for (int e = tid; e < n * npick * 2; e += nt) {
        const int i = e % n, q = (e / n) % npick, part = e / (n * npick);
        const bool pair = wi[pick[q]] != R(0);
        if (part == 1 && !pair) continue;
        const R *x = (part == 0) ? xr : xi;
        R s = R(0);
        for (int c = 0; c < n; c++) s += M_(Zr, n, i, c) * x[c * npick + q];
        M_(P, ldp, i, colof[q] + part) = (double)s;
    }
    sync();
    for (int c = warp_id(); c < knew; c += num_warps()) {
        double mx = 0.0;
        for (int i = lane_id(); i < n; i += 32) mx = fmax(mx, fabs(M_(P, ldp, i, c)));
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        const double f = (mx > 0.0) ? 1.0 / mx : 1.0;
        for (int i = lane_id(); i < n; i += 32) M_(P, ldp, i, c) *= f;
    }
    sync();
    return knew;
}

// ------------------------------------------------------------------ QR / Cholesky

// Householder QR of A (rows x kc, lda), rows >= kc.  On return Q (rows x kc,
// ldq) holds the explicit orthonormal factor and R (kc x kc, ldr) the upper
// triangle, normalised so that diag(R) > 0.  A is overwritten.
// vnorm: scratch of KMAX doubles.  Returns 0, or 1 if a column is (numerically) dependent.
static __device__ __noinline__ int householder_qr(double *A, int lda, int rows, int kc, double *Q, int ldq, double *R,
                              int ldr, double *tau, double *sc) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = lane_id(), w = warp_id(), nw = num_warps();
    int bad = 0;
    for (int c = 0; c < kc; c++) {
        if (w == 0) {
            double s = 0.0;
            for (int i = c + lane; i < rows; i += 32) s += M_(A, lda, i, c) * M_(A, lda, i, c);
            s = warp_sum(s);
            if (lane == 0) {
                const double x0 = M_(A, lda, c, c);
                const double nrm = sqrt(s);
                if (nrm == 0.0) {
                    tau[c] = 0.0;
                    sc[0] = 0.0;
                    sc[1] = 0.0;
                } else {
                    const double alpha = -copysign(nrm, x0);
                    tau[c] = (alpha - x0) / alpha;
                    sc[1] = 1.0 / (x0 - alpha);
                    sc[0] = alpha;
                }
            }
        }
        sync();
        const double alpha = sc[0], inv = sc[1], tc = tau[c];
        if (alpha == 0.0) bad = 1;
        // store v below the diagonal (v0 = 1 implicit)
        for (int i = c + 1 + tid; i < rows; i += nt) M_(A, lda, i, c) *= inv;
        sync();
        if (tc != 0.0) {
            for (int j = c + 1 + w; j < kc; j += nw) {
                double s = (lane == 0) ? M_(A, lda, c, j) : 0.0;
                for (int i = c + 1 + lane; i < rows; i += 32) s += M_(A, lda, i, c) * M_(A, lda, i, j);
                s = warp_sum(s) * tc;
                if (lane == 0) M_(A, lda, c, j) -= s;
                for (int i = c + 1 + lane; i < rows; i += 32) M_(A, lda, i, j) -= s * M_(A, lda, i, c);
            }
        }
        sync();
        if (tid == 0) M_(A, lda, c, c) = (tc != 0.0) ? alpha : M_(A, lda, c, c);
        sync();
    }
    // R and explicit Q = H_0 ... H_{kc-1} [I; 0]
    for (int e = tid; e < kc * kc; e += nt) {
        const int i = e % kc, j = e / kc;
        M_(R, ldr, i, j) = (i <= j) ? M_(A, lda, i, j) : 0.0;
    }
    for (int e = tid; e < rows * kc; e += nt) {
        const int i = e % rows, j = e / rows;
        M_(Q, ldq, i, j) = (i == j) ? 1.0 : 0.0;
    }
    sync();
    for (int c = kc - 1; c >= 0; c--) {
        const double tc = tau[c];
        if (tc != 0.0) {
            for (int j = c + w; j < kc; j += nw) {
                double s = (lane == 0) ? M_(Q, ldq, c, j) : 0.0;
                for (int i = c + 1 + lane; i < rows; i += 32) s += M_(A, lda, i, c) * M_(Q, ldq, i, j);
                s = warp_sum(s) * tc;
                if (lane == 0) M_(Q, ldq, c, j) -= s;
                for (int i = c + 1 + lane; i < rows; i += 32) M_(Q, ldq, i, j) -= s * M_(A, lda, i, c);
            }
        }
        sync();
    }
    // positive diagonal: record the signs first, then flip rows of R and columns of Q
    for (int i = tid; i < kc; i += nt) tau[i] = (M_(R, ldr, i, i) < 0.0) ? -1.0 : 1.0;
    sync();
    for (int e = tid; e < kc * kc + rows * kc; e += nt) {
        if (e < kc * kc) {
            const int i = e % kc, j = e / kc;
            M_(R, ldr, i, j) *= tau[i];
        } else {
            const int f = e - kc * kc, i = f % rows, j = f / rows;
            M_(Q, ldq, i, j) *= tau[j];
        }
    }
    sync();
    return bad;
}

// Cholesky G = R^T R of a kc x kc SPD matrix (ldg), R upper (ldr).
// Returns 0, or 1 if a pivot is not positive relative to the diagonal.
static __device__ __noinline__ int cholesky_upper(const double *G, int ldg, int kc, double *R, int ldr, int *isc) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < kc * kc; e += nt) {
        const int i = e % kc, j = e / kc;
        M_(R, ldr, i, j) = (i <= j) ? M_(G, ldg, i, j) : 0.0;
    }
    if (tid == 0) isc[0] = 0;
    sync();
    double dmax = 0.0;
    for (int i = 0; i < kc; i++) dmax = fmax(dmax, M_(G, ldg, i, i));
    for (int c = 0; c < kc; c++) {
        if (tid == 0) {
            const double piv = M_(R, ldr, c, c);
            if (!(piv > 1e-13 * dmax)) {
                isc[0] = 1;
                M_(R, ldr, c, c) = 1.0;
            } else {
                M_(R, ldr, c, c) = sqrt(piv);
            }
        }
        sync();
        const double rcc = M_(R, ldr, c, c);
        for (int j = c + 1 + tid; j < kc; j += nt) M_(R, ldr, c, j) /= rcc;
        sync();
        for (int e = tid; e < kc * kc; e += nt) {
            const int i = e % kc, j = e / kc;
            if (i > c && j >= i) M_(R, ldr, i, j) -= M_(R, ldr, c, i) * M_(R, ldr, c, j);
        }
        sync();
    }
    return isc[0];
}

// Inverse of an upper-triangular kc x kc matrix R (ldr) into Ri (ldi); one
// thread per column.
static __device__ __noinline__ void upper_inverse(const double *R, int ldr, int kc, double *Ri, int ldi) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < kc * kc; e += nt) M_(Ri, ldi, e % kc, e / kc) = 0.0;
    sync();
    for (int j = tid; j < kc; j += nt) {
        // solve R x = e_j; x has support 0..j
        for (int i = j; i >= 0; i--) {
            double s = (i == j) ? 1.0 : 0.0;
            for (int c = i + 1; c <= j; c++) s -= M_(R, ldr, i, c) * M_(Ri, ldi, c, j);
            M_(Ri, ldi, i, j) = s / M_(R, ldr, i, i);
        }
    }
    sync();
}

}  // namespace skr
