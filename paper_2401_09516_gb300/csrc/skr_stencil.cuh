// Finite-difference assembly and the stencil operator (Sec. 3.1, App. A.2).
//
// A matrix row p holds NST = 5 (2D) or 7 (3D) coefficients, stored as NST
// arrays of length ld ("structure of arrays"): slot 0 is the diagonal, then
// the minus/plus neighbours along x, y (and z).  Unknowns are row-major with
// the last grid index fastest (p = i*ny + j in 2D, as in the paper's 2x2
// example), so the x neighbours are +-ny apart and the y neighbours +-1.
// Couplings to boundary nodes (Dirichlet u = 0) are stored as zeros, which
// lets the operator read a clamped, always-valid index without branches.
#pragma once

#include "skr_common.h"
#include "skr_device.cuh"

namespace skr {

struct Geom {
    int nx, ny, nz;      // interior grid (nz = 1 in 2D)
    int nst;             // 5 or 7 (CSR input: entries of its longest row)
    long long n;         // unknowns
    long long off[7];    // neighbour offsets by slot (off[0] = 0)
    const int *cols;     // CSR input: column of row p's entry s at cols[s * cld + p]; else nullptr
    long long cld;
};

__host__ __device__ inline Geom make_geom(int fmt, int nx, int ny, int nz) {
    Geom g;
    g.nx = nx;
    g.ny = ny;
    g.nz = (fmt == SKR_FMT_DARCY3D || fmt == SKR_FMT_STENCIL7) ? nz : 1;
    g.nst = (fmt == SKR_FMT_DARCY3D || fmt == SKR_FMT_STENCIL7) ? 7 : 5;
    g.n = (long long)nx * ny * g.nz;
    const long long sx = (long long)ny * g.nz, sy = g.nz;
    g.off[0] = 0;
    g.off[1] = -sx;
    g.off[2] = sx;
    g.off[3] = -sy;
    g.off[4] = sy;
    g.off[5] = -1;
    g.off[6] = 1;
    g.cols = nullptr;
    g.cld = 0;
    return g;
}

// Geometry of CSR input: n rows, w entries in the longest row, columns in
// cols (w arrays of stride cld, written by the assembly; row p's entries
// beyond its own count point at p with a zero coefficient).
__host__ __device__ inline Geom make_csr_geom(long long n, int w, const int *cols, long long cld) {
    Geom g = make_geom(SKR_FMT_CSR, (int)n, 1, 1);
    g.nst = w;
    g.cols = cols;
    g.cld = cld;
    return g;
}

// Neighbour index for slot s, clamped to p when outside [0, n).  The
// coefficient of an outside (boundary) neighbour is zero.
__device__ __forceinline__ long long nb_index(const Geom &g, long long p, int s) {
    if (g.cols) return g.cols[(long long)s * g.cld + p];
    long long q = p + g.off[s];
    return (q < 0 || q >= g.n) ? p : q;
}

// Row p of CSR input into the stencil slots: the diagonal in slot 0, the
// other entries in slots 1.. in their stored order, slots up to w - 1
// padded with (column p, value 0).  Input validated on the host side
// (skr_csr_check_kernel): one diagonal, at most w entries.
__device__ __forceinline__ void csr_row(const DevSystem &sys, long long p, int w, double *c, int *cidx) {
    const long long r0 = sys.rowptr[p], r1 = sys.rowptr[p + 1];
    for (int s = 0; s < w; s++) {
        c[s] = 0.0;
        cidx[s] = (int)p;
    }
    int s = 1;
    for (long long q = r0; q < r1; q++) {
        const int col = sys.colind[q];
        if (col == p) {
            c[0] = sys.coef[q];
        } else if (s < w) {
            c[s] = sys.coef[q];
            cidx[s] = col;
            s++;
        }
    }
}

// ---------------------------------------------------------------- assembly

// Darcy -div(a grad u) = f, flux form, face value = mean of the two nodes
// (2D or 3D).  anode: exp(log a) at all (nx+2)(ny+2)[(nz+2)] nodes, read
// through L2 because other CTAs of the cluster wrote it.
__device__ __forceinline__ void darcy_row(const Geom &g, const double *anode, long long p,
                                          double *c /* [7] */) {
    if (g.nst == 5) {
        const long long i = p / g.ny, j = p - i * g.ny;
        const long long W = g.ny + 2;
        const long long q = (i + 1) * W + (j + 1);
        const double ac = __ldcg(anode + q);
        const double hx = 1.0 / (double)(g.nx + 1), hy = 1.0 / (double)(g.ny + 1);
        const double hx2 = hx * hx, hy2 = hy * hy;
        const double fxm = 0.5 * (ac + __ldcg(anode + q - W)) / hx2;
        const double fxp = 0.5 * (ac + __ldcg(anode + q + W)) / hx2;
        const double fym = 0.5 * (ac + __ldcg(anode + q - 1)) / hy2;
        const double fyp = 0.5 * (ac + __ldcg(anode + q + 1)) / hy2;
        c[0] = fxm + fxp + fym + fyp;
        c[1] = (i > 0) ? -fxm : 0.0;
        c[2] = (i < g.nx - 1) ? -fxp : 0.0;
        c[3] = (j > 0) ? -fym : 0.0;
        c[4] = (j < g.ny - 1) ? -fyp : 0.0;
    } else {
        const long long nyz = (long long)g.ny * g.nz;
        const long long i = p / nyz, rem = p - i * nyz, j = rem / g.nz, l = rem - j * g.nz;
        const long long Wz = g.nz + 2, Wy = (long long)(g.ny + 2) * Wz;
        const long long q = (i + 1) * Wy + (j + 1) * Wz + (l + 1);
        const double ac = __ldcg(anode + q);
        const double hx = 1.0 / (double)(g.nx + 1), hy = 1.0 / (double)(g.ny + 1),
                     hz = 1.0 / (double)(g.nz + 1);
        const double hx2 = hx * hx, hy2 = hy * hy, hz2 = hz * hz;
        const double fxm = 0.5 * (ac + __ldcg(anode + q - Wy)) / hx2;
        const double fxp = 0.5 * (ac + __ldcg(anode + q + Wy)) / hx2;
        const double fym = 0.5 * (ac + __ldcg(anode + q - Wz)) / hy2;
        const double fyp = 0.5 * (ac + __ldcg(anode + q + Wz)) / hy2;
        const double fzm = 0.5 * (ac + __ldcg(anode + q - 1)) / hz2;
        const double fzp = 0.5 * (ac + __ldcg(anode + q + 1)) / hz2;
        c[0] = fxm + fxp + fym + fyp + fzm + fzp;
        c[1] = (i > 0) ? -fxm : 0.0;
        c[2] = (i < g.nx - 1) ? -fxp : 0.0;
        c[3] = (j > 0) ? -fym : 0.0;
        c[4] = (j < g.ny - 1) ? -fyp : 0.0;
        c[5] = (l > 0) ? -fzm : 0.0;
        c[6] = (l < g.nz - 1) ? -fzp : 0.0;
    }
}

// -nu lap u + beta . grad u = f with first-order upwinding (2D).
__device__ __forceinline__ void convdiff_row(const Geom &g, const double *prm, long long p,
                                             double *c) {
    const long long i = p / g.ny, j = p - i * g.ny;
    const double hh = 1.0 / (double)(g.nx + 1);
    const double nu = prm[0], bx = prm[1], by = prm[2];
    const double d = nu / (hh * hh);
    const double cxm = -d - fmax(bx, 0.0) / hh;
    const double cxp = -d + fmin(bx, 0.0) / hh;
    const double cym = -d - fmax(by, 0.0) / hh;
    const double cyp = -d + fmin(by, 0.0) / hh;
    c[0] = 4.0 * d + fabs(bx) / hh + fabs(by) / hh;
    c[1] = (i > 0) ? cxm : 0.0;
    c[2] = (i < g.nx - 1) ? cxp : 0.0;
    c[3] = (j > 0) ? cym : 0.0;
    c[4] = (j < g.ny - 1) ? cyp : 0.0;
}

// Helmholtz -lap u - k^2 u = f (2D, 5-point Laplacian); kfield = k at the
// interior nodes, row-major like the unknowns.
__device__ __forceinline__ void helmholtz_row(const Geom &g, const double *kfield, long long p, double *c) {
    const long long i = p / g.ny, j = p - i * g.ny;
    const double hx = 1.0 / (double)(g.nx + 1), hy = 1.0 / (double)(g.ny + 1);
    const double ix2 = 1.0 / (hx * hx), iy2 = 1.0 / (hy * hy);
    const double k = kfield[p];
    c[0] = 2.0 * ix2 + 2.0 * iy2 - k * k;
    c[1] = (i > 0) ? -ix2 : 0.0;
    c[2] = (i < g.nx - 1) ? -ix2 : 0.0;
    c[3] = (j > 0) ? -iy2 : 0.0;
    c[4] = (j < g.ny - 1) ? -iy2 : 0.0;
}

// Poisson lap u = f with the Sec. 3.1 sign (2D, 5-point).
__device__ __forceinline__ void poisson_row(const Geom &g, long long p, double *c) {
    const long long i = p / g.ny, j = p - i * g.ny;
    const double hx = 1.0 / (double)(g.nx + 1), hy = 1.0 / (double)(g.ny + 1);
    const double ix2 = 1.0 / (hx * hx), iy2 = 1.0 / (hy * hy);
    c[0] = -2.0 * ix2 - 2.0 * iy2;
    c[1] = (i > 0) ? ix2 : 0.0;
    c[2] = (i < g.nx - 1) ? ix2 : 0.0;
    c[3] = (j > 0) ? iy2 : 0.0;
    c[4] = (j < g.ny - 1) ? iy2 : 0.0;
}

// Right-hand side of row p: f, minus the Dirichlet values of the boundary
// neighbours times their coupling for the Poisson format (App. A.2); the
// rhs array (or 1) for the others.
__device__ __forceinline__ double system_rhs(const DevSystem &sys, const Geom &g, long long p) {
    if (sys.fmt != SKR_FMT_POISSON2D) return sys.rhs ? sys.rhs[p] : 1.0;
    const long long i = p / g.ny, j = p - i * g.ny;
    const double hx = 1.0 / (double)(g.nx + 1), hy = 1.0 / (double)(g.ny + 1);
    const double *f = sys.coef, *gxm = f + g.n, *gxp = gxm + g.ny, *gym = gxp + g.ny, *gyp = gym + g.nx;
    double b = f[p];
    if (i == 0) b -= gxm[j] / (hx * hx);
    if (i == g.nx - 1) b -= gxp[j] / (hx * hx);
    if (j == 0) b -= gym[i] / (hy * hy);
    if (j == g.ny - 1) b -= gyp[i] / (hy * hy);
    return b;
}

// Assembled-input formats: copy the row, zeroing couplings that leave the grid.
__device__ __forceinline__ void stencil_input_row(const Geom &g, const double *coef, long long p,
                                                  double *c) {
    for (int s = 0; s < g.nst; s++) c[s] = coef[(long long)s * g.n + p];
    if (g.nst == 5) {
        const long long i = p / g.ny, j = p - i * g.ny;
        if (i == 0) c[1] = 0.0;
        if (i == g.nx - 1) c[2] = 0.0;
        if (j == 0) c[3] = 0.0;
        if (j == g.ny - 1) c[4] = 0.0;
    } else {
        const long long nyz = (long long)g.ny * g.nz;
        const long long i = p / nyz, rem = p - i * nyz, j = rem / g.nz, l = rem - j * g.nz;
        if (i == 0) c[1] = 0.0;
        if (i == g.nx - 1) c[2] = 0.0;
        if (j == 0) c[3] = 0.0;
        if (j == g.ny - 1) c[4] = 0.0;
        if (l == 0) c[5] = 0.0;
        if (l == g.nz - 1) c[6] = 0.0;
    }
}

__device__ __forceinline__ void system_row(const DevSystem &sys, const Geom &g,
                                           const double *anode, long long p, double *c) {
    if (sys.fmt == SKR_FMT_DARCY2D || sys.fmt == SKR_FMT_DARCY3D)
        darcy_row(g, anode, p, c);
    else if (sys.fmt == SKR_FMT_CONVDIFF2D)
        convdiff_row(g, sys.params, p, c);
    else if (sys.fmt == SKR_FMT_HELMHOLTZ2D)
        helmholtz_row(g, sys.coef, p, c);
    else if (sys.fmt == SKR_FMT_POISSON2D)
        poisson_row(g, p, c);
    else
        stencil_input_row(g, sys.coef, p, c);
}

__device__ __forceinline__ long long node_count(const DevSystem &sys, const Geom &g) {
    if (sys.fmt == SKR_FMT_DARCY2D) return (long long)(g.nx + 2) * (g.ny + 2);
    if (sys.fmt == SKR_FMT_DARCY3D) return (long long)(g.nx + 2) * (g.ny + 2) * (g.nz + 2);
    return 0;
}

// ---------------------------------------------------------------- operator

// y_p = sum_s Aw[s][p] * scale * src[nb_s(p)]  (working precision T).
// src may have been written by other CTAs: read through L2.
template <typename T>
__device__ __forceinline__ T stencil_apply_row(const Geom &g, const T *Aw, long long ld,
                                               const T *src, T scale, long long p) {
    T acc = T(0);
    for (int s = 0; s < g.nst; s++) {
        const long long q = nb_index(g, p, s);
        acc += Aw[(long long)s * ld + p] * (scale * __ldcg(src + q));
    }
    return acc;
}

// ---------------------------------------------------------------- compact symmetric operator
//
// The symmetric grid formats (Darcy 2D/3D, Helmholtz, Poisson: a_pq = a_qp,
// couplings that leave the grid zero) under right Jacobi in FP32 keep the
// folded operator A D^-1 in 1 + (nst - 1) / 2 arrays instead of nst: slot 0
// holds D^-1, slot t (t = 1 .. (nst - 1) / 2) the coupling a_{p, p + off[2t]}
// of row p to its neighbour on the plus side of axis pair t.  Row p's
// coupling to its minus-side neighbour q = p - off[2t] is slot t of row q,
// and the diagonal of A D^-1 is one (the FP32 rounding of d * (1 / d) is
// exactly 1).  An operator pass then moves 5 n values in 2D (D^-1, two
// coupling arrays, the source and the result) and 6 n in 3D.  Used when the
// fastest grid extent is a multiple of 4 (one float4 of rows per thread).
__host__ __device__ inline bool sym_compact_form(int fmt, int precond, int wbytes, const Geom &g) {
    const int last = (g.nst == 5) ? g.ny : g.nz;
    return wbytes == 4 && precond == SKR_PC_JACOBI && g.cols == nullptr &&
           (fmt == SKR_FMT_DARCY2D || fmt == SKR_FMT_DARCY3D || fmt == SKR_FMT_HELMHOLTZ2D ||
            fmt == SKR_FMT_POISSON2D) &&
           last % 4 == 0;
}

// Arrays an operator pass reads in the compact form (D^-1 and the couplings).
__host__ __device__ inline int sym_compact_slots(const Geom &g) { return 1 + (g.nst - 1) / 2; }

// Compact form of row p from the FP64 rows A (slots of stride ld) and D^-1.
template <typename T>
__device__ __forceinline__ void sym_compact_fold_row(const Geom &g, const double *A, long long ld,
                                                     const double *dinv, T *Aw, long long p) {
    Aw[p] = (T)dinv[p];
    for (int t = 1; t <= (g.nst - 1) / 2; t++) Aw[(long long)t * ld + p] = (T)A[(long long)(2 * t) * ld + p];
}

// Entry of A D^-1 in row p, stencil slot s, from the compact form (zero for
// a neighbour outside [0, n)).  Neighbour rows may belong to other CTAs:
// read through L2.
template <typename T>
__device__ __forceinline__ T sym_folded(const Geom &g, const T *Aw, long long ld, long long p, int s) {
    if (s == 0) return T(1);
    const long long q = p + g.off[s];
    if (q < 0 || q >= g.n) return T(0);
    const int t = (s + 1) >> 1;
    const T a = __ldcg(Aw + (long long)t * ld + ((s & 1) ? q : p));   // odd slots: minus side
    return a * __ldcg(Aw + q);
}

// y_p = scale * (A D^-1 src)_p from the compact form.
template <typename T>
__device__ __forceinline__ T sym_apply_row(const Geom &g, const T *Aw, long long ld, const T *src, T scale,
                                           long long p) {
    T acc = scale * __ldcg(src + p);
    for (int s = 1; s < g.nst; s++) {
        const long long q = p + g.off[s];
        if (q >= 0 && q < g.n) acc += sym_folded(g, Aw, ld, p, s) * (scale * __ldcg(src + q));
    }
    return acc;
}

// r_p = b_p - sum_s A[s][p] * x[nb_s(p)]  (FP64 true residual).
__device__ __forceinline__ double residual_row(const Geom &g, const double *A, long long ld,
                                               const double *b, const double *x, long long p) {
    double acc = 0.0;
    for (int s = 0; s < g.nst; s++) {
        const long long q = nb_index(g, p, s);
        acc += A[(long long)s * ld + p] * __ldcg(x + q);
    }
    return b[p] - acc;
}

// ---------------------------------------------------------------- ILU(0), red-black
//
// ILU(0) of the matrix reordered red (even coordinate sum) before black.
// Every neighbour of a black unknown is red and vice versa, so L and U keep
// A's pattern with no elimination in the red rows: M = L U has
//   red rows:   M_rr = a_rr, M_rb = a_rb,
//   black rows: L_br = a_br / a_rr, U_bb = d_b = a_bb - sum_r a_br a_rb / a_rr,
// and M^-1 v is two sweeps: z_b = (v_b - sum_r (a_br / a_rr) v_r) / d_b, then
// z_r = (v_r - sum_b a_rb z_b) / a_rr.  The red rows of A M^-1 are unit rows,
// and A M^-1 v = v on red rows, a_bb z_b + sum_r a_br z_r on black rows.

__device__ __forceinline__ int grid_color(const Geom &g, long long p) {
    if (g.nst == 5) {
        const long long i = p / g.ny, j = p - i * g.ny;
        return (int)((i + j) & 1);
    }
    const long long nyz = (long long)g.ny * g.nz;
    const long long i = p / nyz, rem = p - i * nyz, j = rem / g.nz, l = rem - j * g.nz;
    return (int)((i + j + l) & 1);
}

// Value at index q of a vector that CTAs of the cluster write between
// passes: rows in [olo, ohi) belong to the calling CTA, whose own stores keep
// its L1 coherent, so they may come through L1; other rows come from L2
// (another SM's L1 could hold a stale copy).  olo = ohi reads everything
// from L2.
template <typename V>
__device__ __forceinline__ V ld_owned(const V *v, long long q, long long olo, long long ohi) {
    return (q >= olo && q < ohi) ? v[q] : __ldcg(v + q);
}

// slot of the coefficient that couples the neighbour back to p
__device__ __forceinline__ int opposite_slot(int s) { return (s & 1) ? s + 1 : s - 1; }

// Block-Jacobi: the rows are cut into contiguous blocks of bs rows (the
// last one ragged), like one block per process of a row-distributed matrix,
// and the factorisation keeps only the couplings inside a row's block, i.e.
// it is the red-black ILU(0) of the block-diagonal part of A.  [lo, hi) is
// the block of row p; bs >= n (ILU(0), SSOR) gives the whole matrix.
__device__ __forceinline__ void pc_block(long long p, long long bs, long long n, long long &lo, long long &hi) {
    lo = (bs >= n) ? 0 : (long long)((unsigned)p / (unsigned)bs) * bs;
    hi = min(lo + bs, n);
}

// 1 / pivot of row p: 1/a_pp (red) or 1/d_p (black), the sum over the red
// neighbours in [lo, hi).  A: FP64 rows, halo through L2.
__device__ __forceinline__ double ilu_inv_pivot(const Geom &g, const double *A, long long ld, long long p,
                                                long long lo, long long hi) {
    const double app = A[p];
    if (grid_color(g, p) == 0) return 1.0 / app;
    double d = app;
    for (int s = 1; s < g.nst; s++) {
        const double apq = A[(long long)s * ld + p];
        if (apq == 0.0) continue;
        const long long q = p + g.off[s];
        if (q < lo || q >= hi) continue;
        const double aqp = __ldcg(A + (long long)opposite_slot(s) * ld + q);
        d -= apq * aqp / __ldcg(A + q);
    }
    return 1.0 / d;
}

// Symmetric SOR with omega = 1 in red-black order, M = (D + L) D^-1 (D + U):
// its red rows are those of A and its black-black block is
// D_b + A_br D_r^-1 A_rb, so it is the factorisation above with the black
// pivots d_b = a_bb (the diagonal correction dropped): the same two sweeps.
__host__ __device__ __forceinline__ bool colour_sweep_pc(int pc) {
    return pc == SKR_PC_ILU0 || pc == SKR_PC_SSOR || pc == SKR_PC_BJACOBI;
}

// Rows per block of the sweeps: ceil(n / blocks) for block-Jacobi, n otherwise.
__host__ __device__ __forceinline__ long long sweep_block_rows(int pc, long long n, int blocks) {
    return (pc == SKR_PC_BJACOBI && blocks > 1) ? (n + blocks - 1) / blocks : n;
}

__device__ __forceinline__ double sweep_inv_pivot(const Geom &g, const double *A, long long ld, long long p, int pc,
                                                  long long bs) {
    if (pc == SKR_PC_SSOR) return 1.0 / A[p];
    long long lo, hi;
    pc_block(p, bs, g.n, lo, hi);
    return ilu_inv_pivot(g, A, ld, p, lo, hi);
}

// sweep 1 (black rows): z_b = inv_b (v_b - sum_r a_br inv_r v_r), v = scale * src
// (neighbours outside [lo, hi) are skipped: block-Jacobi)
template <typename R, typename Tv>
__device__ __forceinline__ R ilu_sweep1_row(const Geom &g, const R *Aw, long long ld, const R *inv, const Tv *src,
                                            R scale, long long p, long long lo, long long hi, long long olo = 0,
                                            long long ohi = 0) {
    R acc = scale * (R)ld_owned(src, p, olo, ohi);
    for (int s = 1; s < g.nst; s++) {
        const long long q = nb_index(g, p, s);
        if (q < lo || q >= hi) continue;
        acc -= Aw[(long long)s * ld + p] * ld_owned(inv, q, olo, ohi) * (scale * (R)ld_owned(src, q, olo, ohi));
    }
    return inv[p] * acc;
}

// sweep 2 (red rows): z_r = inv_r (v_r - sum_b a_rb z_b), b in [lo, hi)
template <typename R, typename Tv>
__device__ __forceinline__ R ilu_sweep2_row(const Geom &g, const R *Aw, long long ld, const R *inv, const Tv *src,
                                            R scale, const R *z, long long p, long long lo, long long hi,
                                            long long olo = 0, long long ohi = 0) {
    R acc = scale * (R)ld_owned(src, p, olo, ohi);
    for (int s = 1; s < g.nst; s++) {
        const long long q = nb_index(g, p, s);
        if (q < lo || q >= hi) continue;
        acc -= Aw[(long long)s * ld + p] * ld_owned(z, q, olo, ohi);
    }
    return inv[p] * acc;
}

// A z on a red row minus v_r: the couplings M leaves out, sum over the
// black neighbours outside [lo, hi) of a_rb z_b (0 without blocks, where
// the red rows of A M^-1 are unit rows)
template <typename R>
__device__ __forceinline__ R ilu_red_cross_row(const Geom &g, const R *Aw, long long ld, const R *z, long long p,
                                               long long lo, long long hi, long long olo = 0, long long ohi = 0) {
    R acc = R(0);
    for (int s = 1; s < g.nst; s++) {
        const long long q = nb_index(g, p, s);
        if (q >= lo && q < hi) continue;
        acc += Aw[(long long)s * ld + p] * ld_owned(z, q, olo, ohi);
    }
    return acc;
}

// A z on a black row: a_bb z_b + sum_r a_br z_r
template <typename R>
__device__ __forceinline__ R ilu_black_apply_row(const Geom &g, const R *Aw, long long ld, const R *z, long long p,
                                                 long long olo = 0, long long ohi = 0) {
    R acc = Aw[p] * ld_owned(z, p, olo, ohi);
    for (int s = 1; s < g.nst; s++) {
        const long long q = nb_index(g, p, s);
        acc += Aw[(long long)s * ld + p] * ld_owned(z, q, olo, ohi);
    }
    return acc;
}

}  // namespace skr
