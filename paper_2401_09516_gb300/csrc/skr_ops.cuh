// Stand-alone kernels for the operator entry points (skr_assemble,
// skr_apply).  They call the same row functions as the chain kernel, on a
// plain grid without clusters.
#pragma once

#include "skr_common.h"
#include "skr_stencil.cuh"

namespace skr {

// Checks of CSR input, one thread per row: err bits 1 (row empty or longer
// than SKR_CSR_MAX_ROW, or rowptr not ascending from 0), 2 (diagonal missing
// or repeated), 4 (column outside [0, n)), 8 (a column twice in a row);
// wmax = entries of the longest row.
__global__ void skr_csr_check_kernel(const long long *rowptr, const int *colind, long long n, int *out) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        int e = 0;
        const long long r0 = rowptr[p], r1 = rowptr[p + 1];
        const long long len = r1 - r0;
        if ((p == 0 && r0 != 0) || len < 1 || len > SKR_CSR_MAX_ROW) e |= 1;
        if (!(e & 1)) {
            int ndiag = 0;
            for (long long q = r0; q < r1; q++) {
                const int col = colind[q];
                if (col < 0 || col >= n) e |= 4;
                if (col == p) ndiag++;
                for (long long q2 = r0; q2 < q; q2++)
                    if (colind[q2] == col) e |= 8;
            }
            if (ndiag != 1) e |= 2;
            atomicMax(out + 1, (int)len);
        }
        if (e) atomicOr(out, e);
    }
}


__global__ void node_exp_kernel(const double *__restrict__ loga, long long nn, double *__restrict__ anode) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nn;
         q += (long long)gridDim.x * blockDim.x)
        anode[q] = exp(loga[q]);
}

// A (nst arrays, stride ld), b, dinv (Jacobi or 1).
// CSR input also writes its column indices into cols (g.nst arrays of stride ld).
__global__ void rows_kernel(DevSystem sys, Geom g, const double *anode, double *A, long long ld,
                            double *b, double *dinv, int precond, int *cols) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.n;
         p += (long long)gridDim.x * blockDim.x) {
        double row[7];
        if (sys.fmt == SKR_FMT_CSR) {
            int ci[7];
            csr_row(sys, p, g.nst, row, ci);
            for (int s = 0; s < g.nst; s++) cols[(long long)s * ld + p] = ci[s];
        } else {
            system_row(sys, g, anode, p, row);
        }
        for (int s = 0; s < g.nst; s++) A[(long long)s * ld + p] = row[s];
        if (b) b[p] = system_rhs(sys, g, p);
        if (dinv) dinv[p] = (precond == SKR_PC_JACOBI) ? 1.0 / row[0] : 1.0;
    }
}

template <typename T>
__global__ void fold_kernel(Geom g, const double *A, long long ld, const double *dinv, T *Aw) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.n;
         p += (long long)gridDim.x * blockDim.x) {
        for (int s = 0; s < g.nst; s++) {
            const long long q = nb_index(g, p, s);
            Aw[(long long)s * ld + p] = (T)(A[(long long)s * ld + p] * dinv[q]);
        }
    }
}

template <typename T>
__global__ void to_working_kernel(const double *v, long long n, T *out) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        out[p] = (T)v[p];
}

template <typename T>
__global__ void apply_kernel(Geom g, const T *Aw, long long ld, const T *v, double *y) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.n;
         p += (long long)gridDim.x * blockDim.x)
        y[p] = (double)stencil_apply_row(g, Aw, ld, v, T(1), p);
}

// the compact symmetric form (sym_compact_form) for the stand-alone operator entry point
__global__ void sym_fold_kernel(Geom g, const double *A, long long ld, const double *dinv, float *Aw) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.n;
         p += (long long)gridDim.x * blockDim.x)
        sym_compact_fold_row(g, A, ld, dinv, Aw, p);
}

__global__ void sym_apply_kernel(Geom g, const float *Aw, long long ld, const float *v, double *y) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.n;
         p += (long long)gridDim.x * blockDim.x)
        y[p] = (double)sym_apply_row(g, Aw, ld, v, 1.0f, p);
}

// red-black ILU(0) / SSOR for the stand-alone operator entry point
__global__ void ilu_pivot_kernel(Geom g, const double *A, long long ld, double *inv, int pc, long long bs) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.n;
         p += (long long)gridDim.x * blockDim.x)
        inv[p] = sweep_inv_pivot(g, A, ld, p, pc, bs);
}

template <typename T>
__global__ void ilu_fold_kernel(Geom g, const double *A, long long ld, const double *inv, T *Aw, T *invw) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.n;
         p += (long long)gridDim.x * blockDim.x) {
        for (int s = 0; s < g.nst; s++) Aw[(long long)s * ld + p] = (T)A[(long long)s * ld + p];
        invw[p] = (T)inv[p];
    }
}

// bs: rows per block of the sweeps (n, or ceil(n / blocks) for block-Jacobi)
template <typename T>
__global__ void ilu_sweep_kernel(Geom g, const T *Aw, long long ld, const T *inv, const T *v, T *z, double *y,
                                 int stage, long long bs) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < g.n;
         p += (long long)gridDim.x * blockDim.x) {
        const int col = grid_color(g, p);
        long long lo, hi;
        pc_block(p, bs, g.n, lo, hi);
        if (stage == 1 && col == 1) z[p] = ilu_sweep1_row<T, T>(g, Aw, ld, inv, v, T(1), p, lo, hi);
        if (stage == 2 && col == 0) z[p] = ilu_sweep2_row<T, T>(g, Aw, ld, inv, v, T(1), z, p, lo, hi);
        if (stage == 3) {
            if (col == 1)
                y[p] = (double)ilu_black_apply_row(g, Aw, ld, z, p);
            else
                y[p] = (double)(v[p] + ilu_red_cross_row(g, Aw, ld, z, p, lo, hi));
        }
    }
}

}  // namespace skr
