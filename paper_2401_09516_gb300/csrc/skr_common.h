// Internal descriptors shared by the host side of the library and its
// kernels.  Nothing here is part of the public ABI (include/skr.h).
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "../../include/skr.h"

namespace skr {

constexpr int MMAX = SKR_MAX_M;   // restart length capacity
constexpr int KMAX = SKR_MAX_K;   // recycle dimension capacity
constexpr int LDH = MMAX + 1;     // leading dimension of the small FP64 matrices

// Column layout of a slot's basis slab (working precision, column stride ld):
//   [0, KMAX)                 C_k, right-aligned: columns KMAX-kc .. KMAX-1
//   [KMAX, KMAX+MMAX+1)       V_1 .. V_{MMAX+1}
//   [UB, UB+KMAX)             U_k
//   Y0, Y1                    ping-pong scratch for the Arnoldi vector w
//   RW                        inner residual (working precision)
//   DH                        inner correction d (working precision)
//   Z                         ILU(0) sweep scratch
//   CIN, CIN+KMAX             copy of C_k at the start of a system (delta diagnostic)
// C directly precedes V, so [C_k, V_1..V_j] is one contiguous column range.
constexpr int COL_C_END = KMAX;
constexpr int COL_V0 = KMAX;
constexpr int COL_U0 = KMAX + MMAX + 1;
constexpr int COL_Y0 = COL_U0 + KMAX;
constexpr int COL_Y1 = COL_Y0 + 1;
constexpr int COL_RW = COL_Y0 + 2;
constexpr int COL_DH = COL_Y0 + 3;
constexpr int COL_Z = COL_Y0 + 4;
constexpr int COL_CIN = COL_Y0 + 5;
constexpr int NCOLS = COL_CIN + KMAX;
// Operator slots per slot: NST coefficient arrays, plus (ILU) the inverse pivots in slot 7.
constexpr int AW_SLOTS = 8;

// Streaming passes stage the basis through shared memory in blocks of rows:
// one segment is one column over RING_SEG_BYTES / sizeof(T) rows.  The TMA
// boxes are {segment rows x (16 >> i) columns}, i < NBOX, so that any run of
// columns is covered by a few boxes (16s, then a binary remainder).
constexpr int RING_SEG_BYTES = 1024;
constexpr int NBOX = 5;

// One system as the kernels see it (device pointers).
struct DevSystem {
    int fmt, nx, ny, nz;
    const double *coef;
    const double *rhs;
    double params[4];
    double *x_out;
    const long long *rowptr = nullptr;   // CSR input
    const int *colind = nullptr;
    int csr_w = 0;                        // CSR: entries of the longest row (<= SKR_CSR_MAX_ROW)
};

// Per-system outcome written by the kernel (mirrors skr_result).
struct DevResult {
    int steps, cycles, matvecs, refinements, flag, k_final;
    double relres;
    unsigned long long t_begin, t_end;
    double delta;   // one-sided distance of the recycle space, or -1
};

// Device workspace: one region per slot (cluster in flight).
struct Workspace {
    void *basis;              // NCOLS * ld elements of T per slot
    double *A64;              // 7 * ld doubles per slot (unfolded matrix)
    void *Aw;                 // AW_SLOTS * ld elements of T per slot (right-preconditioned operator)
    double *dinv;             // ld per slot (Jacobi: 1/diag, else 1)
    double *x, *r, *b;        // ld per slot each (FP64 solution, residual, rhs)
    double *anode;            // node scratch per slot (exp(log a)), nodecap doubles
    int *cols = nullptr;      // CSR input: 7 * ld column indices per slot (row p's entry s at s * ld + p)
    long long ld;             // column stride (elements), multiple of 64
    long long nodecap;        // node scratch capacity per slot
    int nslots;
};

struct ChainArgs {
    const DevSystem *systems;
    const int *order;
    const long long *chain_off;   // nchains + 1
    int nchains;
    int *chain_counter;           // dynamic chain assignment (zeroed by the host)
    Workspace ws;
    DevResult *results;
    int m, k, maxit, max_refine, precond;
    double tol, inner_tol;
    unsigned long long *bytes;    // algorithmic bytes counter (optional)
    unsigned long long *prof;     // SKR_NPHASE per-phase ns accumulators (optional)
    int warm_start;               // x_0 = previous solution of the chain
    int diagnostics;              // nonzero: compute delta per system
    int pc_blocks;                // SKR_PC_BJACOBI: row blocks of the preconditioner
    int eig32 = 0;                // mixed form: harmonic-Ritz eigen-solve in FP32 instead of FP64
    int *chain_xok;               // per chain, optional: nonzero when the slot's x holds the
                                  // previous solution (read at chain start, set at chain end)
    double *const *recycle_out = nullptr;   // per chain, optional: its final U_k then C_k,
                                  // k columns of n doubles each (zero past the carried dimension)
    int *chain_kc;                // per-chain recycle dimension carried between launches
                                  // (optional: read at chain start, written at chain end;
                                  // the chain's U_k, C_k stay in its workspace slot)
    // TMA descriptors of the basis slab of all slots, seen as one 2D array:
    // ld rows (contiguous) x nslots * NCOLS columns (stride ld elements);
    // tmap[i] has boxes of 16 >> i columns
    CUtensorMap tmap[NBOX];
};

enum Phase { PH_ASM, PH_REFRESH, PH_PROJ, PH_SPMV, PH_DOT, PH_UPD, PH_GRAM, PH_DENSE, PH_CUPD, PH_RESID, PH_OTHER,
             PH_SCHUR, PH_EIGVEC, PH_HESS };

}  // namespace skr
