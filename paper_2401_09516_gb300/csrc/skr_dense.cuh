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

constexpr double DEPS = 2.220446049250313e-16;

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
                r = hypot(a, b);
                c = a / r;
                s = b / r;
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
    // back substitution: column-oriented, the rhs lives in dscr
    for (int i = tid; i < L; i += nt) dscr[i] = g[i];
    sync();
    for (int i = L - 1; i >= 0; i--) {
        const double yi = dscr[i] / M_(Rw, ldr, i, i);
        sync();
        if (tid == 0) y[i] = yi;
        for (int c = tid; c < i; c += nt) dscr[c] -= M_(Rw, ldr, c, i) * yi;
        sync();
    }
    return fabs(g[L]);
}

// ------------------------------------------------------------------ eigen-solver

// Reduce A (n x n, lda) to upper Hessenberg form by Householder reflectors,
// accumulating Z = Q (n x n, ldz) with A_in = Z H Z^T.  v: scratch of n doubles.
__device__ inline void hessenberg_reduce(double *A, int lda, double *Z, int ldz, int n, double *v,
                                  double *sc) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = lane_id(), w = warp_id(), nw = num_warps();
    for (int e = tid; e < n * n; e += nt) M_(Z, ldz, e % n, e / n) = (e % n == e / n) ? 1.0 : 0.0;
    sync();
    for (int c = 0; c + 2 < n; c++) {
        // reflector for x = A[c+1 .. n-1, c]
        if (w == 0) {
            double s = 0.0;
            for (int i = c + 1 + lane; i < n; i += 32) s += M_(A, lda, i, c) * M_(A, lda, i, c);
            s = warp_sum(s);
            if (lane == 0) {
                const double x0 = M_(A, lda, c + 1, c);
                const double nrm = sqrt(s);
                double tau = 0.0, alpha = x0;
                if (nrm > 0.0 && s - x0 * x0 > 0.0) {
                    alpha = -copysign(nrm, x0);
                    tau = (alpha - x0) / alpha;
                    sc[1] = 1.0 / (x0 - alpha);
                } else {
                    sc[1] = 0.0;
                }
                sc[0] = tau;
                sc[2] = alpha;
            }
        }
        sync();
        const double tau = sc[0], inv = sc[1];
        sync();                    // sc is rewritten by the next column
        if (tau == 0.0) continue;  // uniform: read from shared memory
        for (int i = c + 1 + tid; i < n; i += nt) v[i] = (i == c + 1) ? 1.0 : M_(A, lda, i, c) * inv;
        sync();
        // left: A[c+1:, c:] -= tau v (v^T A[c+1:, c:]); one warp per column
        for (int j = c + w; j < n; j += nw) {
            double s = 0.0;
            for (int i = c + 1 + lane; i < n; i += 32) s += v[i] * M_(A, lda, i, j);
            s = warp_sum(s) * tau;
            for (int i = c + 1 + lane; i < n; i += 32) M_(A, lda, i, j) -= s * v[i];
        }
        sync();
        // right: A[:, c+1:] -= tau (A[:, c+1:] v) v^T ; Z likewise; one thread per row
        for (int r = tid; r < 2 * n; r += nt) {
            double *Mx = (r < n) ? A : Z;
            const int ldm = (r < n) ? lda : ldz;
            const int i = (r < n) ? r : r - n;
            double s = 0.0;
            for (int j = c + 1; j < n; j++) s += M_(Mx, ldm, i, j) * v[j];
            s *= tau;
            for (int j = c + 1; j < n; j++) M_(Mx, ldm, i, j) -= s * v[j];
        }
        sync();
        if (tid == 0) {
            M_(A, lda, c + 1, c) = sc[2];
        }
        for (int i = c + 2 + tid; i < n; i += nt) M_(A, lda, i, c) = 0.0;
        sync();
    }
}

// Apply a reflector P = I - tau v v^T (v = (1, v1, v2) or (1, v1)) to rows
// r..r+nr-1 of H (columns c0..n-1), to columns r..r+nr-1 of H (rows
// 0..rmax) and of Z (all rows).  One element of work per thread.
__device__ __forceinline__ void apply_reflector3(double *H, int ldh, double *Z, int ldz, int n, int r,
                                                 int nr, double tau, double v1, double v2, int c0,
                                                 int rmax) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = c0 + tid; j < n; j += nt) {
        double t = M_(H, ldh, r, j) + v1 * M_(H, ldh, r + 1, j);
        if (nr == 3) t += v2 * M_(H, ldh, r + 2, j);
        t *= tau;
        M_(H, ldh, r, j) -= t;
        M_(H, ldh, r + 1, j) -= t * v1;
        if (nr == 3) M_(H, ldh, r + 2, j) -= t * v2;
    }
    sync();
    for (int e = tid; e < (rmax + 1) + n; e += nt) {
        double *Mx = (e <= rmax) ? H : Z;
        const int ldm = (e <= rmax) ? ldh : ldz;
        const int i = (e <= rmax) ? e : e - (rmax + 1);
        double t = M_(Mx, ldm, i, r) + v1 * M_(Mx, ldm, i, r + 1);
        if (nr == 3) t += v2 * M_(Mx, ldm, i, r + 2);
        t *= tau;
        M_(Mx, ldm, i, r) -= t;
        M_(Mx, ldm, i, r + 1) -= t * v1;
        if (nr == 3) M_(Mx, ldm, i, r + 2) -= t * v2;
    }
    sync();
}

// Householder vector for u = (x, y, z): P u = alpha e1.  Writes tau, v1, v2.
__device__ __forceinline__ void house3(double x, double y, double z, double &tau, double &v1,
                                       double &v2, double &alpha) {
    const double s = fabs(x) + fabs(y) + fabs(z);
    if (s == 0.0 || (y == 0.0 && z == 0.0)) {
        tau = 0.0;
        v1 = v2 = 0.0;
        alpha = x;
        return;
    }
    const double xs = x / s, ys = y / s, zs = z / s;
    const double nrm = sqrt(xs * xs + ys * ys + zs * zs);
    const double a = -copysign(nrm, xs);
    tau = (a - xs) / a;
    v1 = ys / (xs - a);
    v2 = zs / (xs - a);
    alpha = a * s;
}

// Real Schur form of an upper Hessenberg H (n x n) by the Francis
// double-shift QR algorithm (Golub & Van Loan, Alg. 7.5.1-7.5.2), with the
// Schur vectors accumulated into Z.  Real eigenvalue pairs of 2x2 blocks
// are split by a rotation, so the remaining 2x2 blocks hold complex pairs;
// for such a block at (p, p+1): wi[p] > 0, wi[p+1] = -wi[p].
// Returns 0 on success, 1 if the iteration limit was hit.
__device__ inline int francis_schur(double *H, int ldh, double *Z, int ldz, int n, double *wr, double *wi,
                             double *sc, int *isc) {
    const int tid = threadIdx.x;
    int hi = n - 1, its = 0, total = 0;
    while (hi >= 0) {
        if (tid == 0) {
            int l = hi;
            while (l > 0) {
                double s = fabs(M_(H, ldh, l - 1, l - 1)) + fabs(M_(H, ldh, l, l));
                if (s == 0.0) s = 1.0;
                if (fabs(M_(H, ldh, l, l - 1)) <= DEPS * s) break;
                l--;
            }
            if (l > 0) M_(H, ldh, l, l - 1) = 0.0;
            isc[0] = l;
        }
        sync();
        const int l = isc[0];
        sync();
        if (l == hi) {
            if (tid == 0) {
                wr[hi] = M_(H, ldh, hi, hi);
                wi[hi] = 0.0;
            }
            sync();
            hi -= 1;
            its = 0;
            continue;
        }
        if (l == hi - 1) {
            const int p = hi - 1;
            if (tid == 0) {
                const double a = M_(H, ldh, p, p), b = M_(H, ldh, p, p + 1);
                const double c = M_(H, ldh, p + 1, p), d = M_(H, ldh, p + 1, p + 1);
                const double hp = 0.5 * (a - d);
                const double disc = hp * hp + b * c;
                if (disc >= 0.0) {
                    const double q = sqrt(disc);
                    const double zz = hp + copysign(q, hp);
                    double l1, l2;
                    if (zz == 0.0) {
                        l1 = l2 = d;
                    } else {
                        l1 = d + zz;
                        l2 = d - b * c / zz;
                    }
                    // rotation whose first column is an eigenvector for l1
                    double e0 = l1 - d, e1 = c;
                    if (fabs(e0) + fabs(e1) == 0.0) {
                        e0 = b;
                        e1 = l1 - a;
                    }
                    double nrm = hypot(e0, e1);
                    double cs = 1.0, sn = 0.0;
                    if (nrm > 0.0) {
                        cs = e0 / nrm;
                        sn = e1 / nrm;
                    }
                    sc[0] = cs;
                    sc[1] = sn;
                    sc[2] = 1.0;
                    wr[p] = l1;
                    wr[p + 1] = l2;
                    wi[p] = wi[p + 1] = 0.0;
                } else {
                    const double q = sqrt(-disc);
                    wr[p] = wr[p + 1] = hp + d;
                    wi[p] = q;
                    wi[p + 1] = -q;
                    sc[2] = 0.0;
                }
            }
            sync();
            if (sc[2] != 0.0) {
                const double cs = sc[0], sn = sc[1];
                const int nt = blockDim.x;
                // rows p, p+1 (columns p..n-1): [r0; r1] <- Q^T [r0; r1], Q = [[cs, -sn], [sn, cs]]
                for (int j = p + threadIdx.x; j < n; j += nt) {
                    const double a0 = M_(H, ldh, p, j), a1 = M_(H, ldh, p + 1, j);
                    M_(H, ldh, p, j) = cs * a0 + sn * a1;
                    M_(H, ldh, p + 1, j) = -sn * a0 + cs * a1;
                }
                sync();
                for (int e = threadIdx.x; e < (p + 2) + n; e += nt) {
                    double *Mx = (e < p + 2) ? H : Z;
                    const int ldm = (e < p + 2) ? ldh : ldz;
                    const int i = (e < p + 2) ? e : e - (p + 2);
                    const double a0 = M_(Mx, ldm, i, p), a1 = M_(Mx, ldm, i, p + 1);
                    M_(Mx, ldm, i, p) = cs * a0 + sn * a1;
                    M_(Mx, ldm, i, p + 1) = -sn * a0 + cs * a1;
                }
                sync();
                if (tid == 0) M_(H, ldh, p + 1, p) = 0.0;
                sync();
            }
            hi -= 2;
            its = 0;
            continue;
        }
        // Francis double-shift step on the active window [l, hi]
        its++;
        total++;
        if (total > 40 * n) return 1;
        if (tid == 0) {
            double s, t;
            if (its == 10 || its == 20) {
                const double w = fabs(M_(H, ldh, hi, hi - 1)) + fabs(M_(H, ldh, hi - 1, hi - 2));
                const double x = 0.75 * w + M_(H, ldh, hi, hi);
                s = 2.0 * x;
                t = x * x + 0.4375 * w * w;
            } else {
                const double a = M_(H, ldh, hi - 1, hi - 1), b = M_(H, ldh, hi - 1, hi);
                const double c = M_(H, ldh, hi, hi - 1), d = M_(H, ldh, hi, hi);
                s = a + d;
                t = a * d - b * c;
            }
            const double h00 = M_(H, ldh, l, l), h01 = M_(H, ldh, l, l + 1);
            const double h10 = M_(H, ldh, l + 1, l), h11 = M_(H, ldh, l + 1, l + 1);
            const double h21 = M_(H, ldh, l + 2, l + 1);
            sc[3] = h00 * h00 + h01 * h10 - s * h00 + t;
            sc[4] = h10 * (h00 + h11 - s);
            sc[5] = h10 * h21;
        }
        sync();
        for (int kk = l; kk <= hi - 1; kk++) {
            const int nr = (kk == hi - 1) ? 2 : 3;
            if (tid == 0) {
                double tau, v1, v2, alpha;
                house3(sc[3], sc[4], nr == 3 ? sc[5] : 0.0, tau, v1, v2, alpha);
                sc[6] = tau;
                sc[7] = v1;
                sc[8] = v2;
            }
            sync();
            const double tau = sc[6], v1 = sc[7], v2 = sc[8];
            if (tau != 0.0) {
                const int c0 = (kk > l) ? kk - 1 : l;
                const int rmax = min(kk + 3, hi);
                apply_reflector3(H, ldh, Z, ldz, n, kk, nr, tau, v1, v2, c0, rmax);
            }
            if (tid == 0) {
                if (kk > l) {
                    M_(H, ldh, kk + 1, kk - 1) = 0.0;
                    if (nr == 3) M_(H, ldh, kk + 2, kk - 1) = 0.0;
                }
                if (kk < hi - 1) {
                    sc[3] = M_(H, ldh, kk + 1, kk);
                    sc[4] = M_(H, ldh, kk + 2, kk);
                    sc[5] = (kk < hi - 2) ? M_(H, ldh, kk + 3, kk) : 0.0;
                }
            }
            sync();
        }
    }
    return 0;
}

// Complex helpers (re, im pairs).
__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi, double &cr,
                                     double &ci) {
    if (fabs(br) >= fabs(bi)) {
        const double r = bi / br, d = br + r * bi;
        cr = (ar + r * ai) / d;
        ci = (ai - r * ar) / d;
    } else {
        const double r = br / bi, d = bi + r * br;
        cr = (r * ar + ai) / d;
        ci = (r * ai - ar) / d;
    }
}

// Eigenvector of the quasi-triangular T for eigenvalue at position p (real,
// or the first of a complex pair when wi[p] > 0), by back substitution.
// Writes xr, xi (n entries each; xi = 0 for a real eigenvalue).
__device__ inline void schur_eigvec(const double *T, int ldt, int n, const double *wr, const double *wi,
                             int p, double *xr, double *xi, double tnorm) {
    const double small = DEPS * fmax(tnorm, 1e-300);
    for (int i = 0; i < n; i++) {
        xr[i] = 0.0;
        xi[i] = 0.0;
    }
    const double lr = wr[p], li = wi[p];
    int top;
    if (li == 0.0) {
        xr[p] = 1.0;
        top = p - 1;
    } else {
        // complex pair in rows/cols (p, p+1): u = (lambda - d, c)
        const double d = M_(T, ldt, p + 1, p + 1), c = M_(T, ldt, p + 1, p);
        xr[p] = lr - d;
        xi[p] = li;
        xr[p + 1] = c;
        xi[p + 1] = 0.0;
        top = p - 1;
    }
    const int last = (li == 0.0) ? p : p + 1;
    int i = top;
    while (i >= 0) {
        const bool two = (i > 0) && (M_(T, ldt, i, i - 1) != 0.0);
        if (!two) {
            double sr = 0.0, si = 0.0;
            for (int c = i + 1; c <= last; c++) {
                sr += M_(T, ldt, i, c) * xr[c];
                si += M_(T, ldt, i, c) * xi[c];
            }
            double dr = M_(T, ldt, i, i) - lr, di = -li;
            if (fabs(dr) + fabs(di) < small) dr = small;
            double qr, qi;
            cdiv(-sr, -si, dr, di, qr, qi);
            xr[i] = qr;
            xi[i] = qi;
            i -= 1;
        } else {
            // rows i-1, i form a 2x2 block: solve (B - lambda I) [x_{i-1}; x_i] = -s
            const int a = i - 1;
            double s0r = 0.0, s0i = 0.0, s1r = 0.0, s1i = 0.0;
            for (int c = i + 1; c <= last; c++) {
                s0r += M_(T, ldt, a, c) * xr[c];
                s0i += M_(T, ldt, a, c) * xi[c];
                s1r += M_(T, ldt, i, c) * xr[c];
                s1i += M_(T, ldt, i, c) * xi[c];
            }
            const double b00r = M_(T, ldt, a, a) - lr, b00i = -li;
            const double b01 = M_(T, ldt, a, i), b10 = M_(T, ldt, i, a);
            const double b11r = M_(T, ldt, i, i) - lr, b11i = -li;
            // det = b00 b11 - b01 b10
            double detr = b00r * b11r - b00i * b11i - b01 * b10;
            double deti = b00r * b11i + b00i * b11r;
            if (fabs(detr) + fabs(deti) < small * small) detr = small * small;
            // x0 = (-s0 b11 + b01 s1)/det ; x1 = (-s1 b00 + b10 s0)/det
            const double n0r = -(s0r * b11r - s0i * b11i) + b01 * s1r;
            const double n0i = -(s0r * b11i + s0i * b11r) + b01 * s1i;
            const double n1r = -(s1r * b00r - s1i * b00i) + b10 * s0r;
            const double n1i = -(s1r * b00i + s1i * b00r) + b10 * s0i;
            cdiv(n0r, n0i, detr, deti, xr[a], xi[a]);
            cdiv(n1r, n1i, detr, deti, xr[i], xi[i]);
            i -= 2;
        }
        // rescale to avoid overflow
        double mx = 0.0;
        for (int c = (i + 1 > 0 ? i + 1 : 0); c <= last; c++) mx = fmax(mx, fabs(xr[c]) + fabs(xi[c]));
        if (mx > 1e100) {
            const double f = 1.0 / mx;
            for (int c = 0; c <= last; c++) {
                xr[c] *= f;
                xi[c] *= f;
            }
        }
    }
}

// Harmonic-Ritz selection on M (n x n, overwritten): eigen-decompose M,
// keep the eigenvectors whose eigenvalues mu have the largest |mu|, i.e.
// the smallest |theta| for theta = 1/mu (ties: smaller Re theta, then
// smaller Im theta, then lower index), at most kwant of them; a complex
// pair contributes the real and imaginary parts of one eigenvector and is
// dropped if the kwant-th pick would split it.  Writes P (n x knew, ldp) and
// returns knew (-1 if the QR iteration failed).
// Work arrays: Z (n x n, ldz), wr/wi (n), xr/xi ((KMAX+1) x n), sc, isc.
__device__ inline int harmonic_select(double *M, int ldm, int n, int kwant, double *P, int ldp, double *Z,
                               int ldz, double *wr, double *wi, double *xr, double *xi, double *vscr,
                               double *sc, int *isc) {
    const int tid = threadIdx.x, nt = blockDim.x;
    hessenberg_reduce(M, ldm, Z, ldz, n, vscr, sc);
    const int fail = francis_schur(M, ldm, Z, ldz, n, wr, wi, sc, isc);
    if (fail) return -1;
    // ranks by (|theta|, Re theta, Im theta, index)
    int *rank = isc + 8;       // n ints
    int *pick = isc + 8 + MMAX;  // ordered list of chosen eigenvalue positions
    for (int i = tid; i < n; i += nt) {
        auto key = [&](int q, double &k0, double &k1, double &k2) {
            const double m2 = wr[q] * wr[q] + wi[q] * wi[q];
            if (m2 == 0.0) {
                k0 = k1 = k2 = INFINITY;
            } else {
                k0 = 1.0 / sqrt(m2);
                k1 = wr[q] / m2;
                k2 = -wi[q] / m2;
            }
        };
        double a0, a1, a2;
        key(i, a0, a1, a2);
        int r = 0;
        for (int q = 0; q < n; q++) {
            if (q == i) continue;
            double b0, b1, b2;
            key(q, b0, b1, b2);
            const bool before = (b0 < a0) || (b0 == a0 && (b1 < a1 || (b1 == a1 && (b2 < a2 || (b2 == a2 && q < i)))));
            r += before ? 1 : 0;
        }
        rank[i] = r;
    }
    sync();
    if (tid == 0) {
        // walk eigenvalues in rank order, build the column list
        int cols = 0, npick = 0;
        for (int r = 0; r < kwant && r < n; r++) {
            int q = 0;
            while (q < n && rank[q] != r) q++;
            if (q >= n) break;
            if (wi[q] == 0.0) {
                pick[npick++] = q;
                cols += 1;
            } else {
                // first member of the pair in the Schur form
                const int p0 = (wi[q] > 0.0) ? q : q - 1;
                const int partner = (q == p0) ? p0 + 1 : p0;
                // partner chosen iff its rank < kwant; count the pair once
                if (rank[partner] < kwant) {
                    if (rank[partner] > r) {
                        pick[npick++] = p0;
                        cols += 2;
                    }
                }
            }
        }
        isc[1] = npick;
        isc[2] = cols;
    }
    sync();
    const int npick = isc[1], knew = isc[2];
    // |T| bound for the tiny-pivot guard
    if (tid == 0) {
        double tn = 0.0;
        for (int e = 0; e < n * n; e++) tn = fmax(tn, fabs(M_(M, ldm, e % n, e / n)));
        sc[9] = tn;
    }
    sync();
    const double tnorm = sc[9];
    // eigenvectors of T, one thread per pick
    for (int q = tid; q < npick; q += nt)
        schur_eigvec(M, ldm, n, wr, wi, pick[q], xr + q * n, xi + q * n, tnorm);
    sync();
    // P columns: Z x (real), or Z Re x, Z Im x (pair); column order follows picks
    int *colof = isc + 8 + 2 * MMAX;
    if (tid == 0) {
        int c = 0;
        for (int q = 0; q < npick; q++) {
            colof[q] = c;
            c += (wi[pick[q]] == 0.0) ? 1 : 2;
        }
    }
    sync();
    for (int e = tid; e < n * npick * 2; e += nt) {
        const int i = e % n, q = (e / n) % npick, part = e / (n * npick);
        const bool pair = wi[pick[q]] != 0.0;
        if (part == 1 && !pair) continue;
        const double *x = (part == 0) ? (xr + q * n) : (xi + q * n);
        double s = 0.0;
        for (int c = 0; c < n; c++) s += M_(Z, ldz, i, c) * x[c];
        M_(P, ldp, i, colof[q] + part) = s;
    }
    sync();
    // normalise columns (max-norm) for conditioning
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
__device__ inline int householder_qr(double *A, int lda, int rows, int kc, double *Q, int ldq, double *R,
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
__device__ inline int cholesky_upper(const double *G, int ldg, int kc, double *R, int ldr, int *isc) {
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
__device__ inline void upper_inverse(const double *R, int ldr, int kc, double *Ri, int ldi) {
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
