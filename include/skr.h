/*
 * skr.h -- C ABI of the GB300 sorted-recycling (SKR) solver library.
 *
 * The library solves a sequence of sparse linear systems A(i) x(i) = b(i)
 * that come from one PDE family (Sec. 3.1, Eq. 1 of arXiv 2401.09516).  It
 * first orders them with the greedy nearest-neighbour sort of Algorithm 1
 * (Sec. 4.1), then solves them in that order with GCRO-DR (Sec. 4.2,
 * Algorithm 2), carrying the recycle space U_k, C_k = A U_k from one system
 * to the next and refreshing it against each new matrix (App. B.1).  k = 0
 * gives plain restarted GMRES(m), the comparator of Sec. 6.
 *
 * Everything runs in hand-written CUDA kernels for sm_103a; there is no CPU
 * fallback.  All arithmetic is real: the paper allows complex systems, this
 * library does not.
 *
 * Conventions for every entry point:
 *   - the return value is SKR_OK (0) or a negative SKR_ERR_*; on error,
 *     skr_last_error() returns a message for the calling thread;
 *   - "mem" says where the caller's data pointers live: SKR_MEM_DEVICE
 *     (device memory of the current CUDA device) or SKR_MEM_HOST (host
 *     memory; the library copies in and out, pinned memory is faster);
 *   - the caller owns every buffer it passes; the library only borrows them
 *     for the duration of the call, and the call returns after all of its
 *     device work has finished;
 *   - "stream" is a cudaStream_t (NULL = the legacy default stream);
 *   - arrays are dense, row-major for matrices, 64-bit sizes.
 */
#ifndef SKR_H
#define SKR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t skr_status;

/* call-level status */
#define SKR_OK                0
#define SKR_NOT_READY         1   /* skr_poll: the request is still in flight */
#define SKR_ERR_INVALID_ARG  (-1)
#define SKR_ERR_OOM          (-2)
#define SKR_ERR_CUDA         (-3)
#define SKR_ERR_TIMEOUT      (-4)
#define SKR_ERR_BUSY         (-5)

/* per-system outcome (skr_result.flag); a system that does not converge
 * does not fail the call */
#define SKR_CONVERGED         0   /* true relative residual <= tol */
#define SKR_NOT_CONVERGED     1   /* Arnoldi step cap (maxit) or refinement cap hit */
#define SKR_BREAKDOWN         2   /* Arnoldi or QR breakdown without convergence */
#define SKR_NUMERICAL         3   /* NaN or Inf in a residual */
#define SKR_DEVICE_STALL      4   /* a bounded device-side wait for a staged copy ran out (2 s);
                                     the system's result is not valid */

/* problem formats (skr_system.fmt).  Unknowns are numbered row-major with
 * the last grid index fastest: p = i*ny + j (2D), p = (i*ny + j)*nz + l (3D),
 * as in the 2x2 example of Sec. 3.1.  Grids are the unit square / cube with
 * nx (ny, nz) interior nodes per side and h = 1/(nx+1) per axis. */
#define SKR_FMT_DARCY2D       1   /* -div(a grad u) = f; coef = log a at the (nx+2)*(ny+2) nodes */
#define SKR_FMT_DARCY3D       2   /* 3D analogue; coef = log a at (nx+2)*(ny+2)*(nz+2) nodes */
#define SKR_FMT_CONVDIFF2D    3   /* -nu lap u + beta.grad u = f, upwind; params = {nu, beta_x, beta_y} */
#define SKR_FMT_STENCIL5      4   /* assembled 2D 5-point matrix; coef = 5 arrays of n doubles:
                                     diagonal, x-minus (p-ny), x-plus (p+ny), y-minus (p-1), y-plus (p+1) */
#define SKR_FMT_STENCIL7      5   /* assembled 3D 7-point matrix; coef = 7 arrays: diagonal,
                                     x-minus, x-plus, y-minus, y-plus, z-minus, z-plus */
#define SKR_FMT_POISSON2D     7   /* Poisson lap u = f (App. E, the third dataset) with Dirichlet data,
                                     the Sec. 3.1 sign (diagonal -2/hx^2 - 2/hy^2); coef = f at the nx*ny
                                     interior nodes, then u on the boundary lines x = 0 (ny values,
                                     j order), x = 1 (ny), y = 0 (nx, i order), y = 1 (nx); b = f minus
                                     the boundary neighbours' values over h^2 (App. A.2); rhs must be NULL */
#define SKR_FMT_HELMHOLTZ2D   6   /* Helmholtz (App. E, the fourth dataset), read as -lap u - k^2 u = f
                                     with u = 0 on the boundary, 5-point Laplacian; coef = k at the
                                     nx*ny interior nodes.  Indefinite once k^2 exceeds the smallest
                                     eigenvalues of the discrete -lap (2 pi^2 for the unit square) */

#define SKR_FMT_CSR           8   /* an assembled sparse matrix in compressed sparse row form (Sec. 3.1's
                                     A: any numbering of the unknowns): nx = n rows (ny = nz = 1);
                                     rowptr = n + 1 int64 offsets (rowptr[0] = 0), colind = int32 column
                                     indices, coef = the values (rowptr[n] doubles); every row holds its
                                     diagonal once and at most SKR_CSR_MAX_ROW entries in all, no column
                                     twice, columns in [0, n).  Preconditioners: SKR_PC_NONE and
                                     SKR_PC_JACOBI (the colour sweeps need a grid) */
#define SKR_CSR_MAX_ROW       7   /* entries per CSR row (the 5- and 7-point stencils fit) */

/* right preconditioner M (App. D.3): the Krylov method solves A M^-1 y = b, x = M^-1 y */
#define SKR_PC_NONE           0
#define SKR_PC_JACOBI         1   /* M = diag(A) */
#define SKR_PC_SSOR           3   /* symmetric SOR, omega = 1 (App. D.3's SOR; PETSc's default local
                                     symmetric sweep): M = (D + L) D^-1 (D + U) of A in red-black order,
                                     applied as the same two parallel colour sweeps as SKR_PC_ILU0 */
#define SKR_PC_ILU0           2   /* M = L U, ILU(0) of A in red-black order (no fill; both
                                     triangular solves are two parallel colour sweeps) */
#define SKR_PC_BJACOBI        4   /* block Jacobi (App. D.3): the rows are cut into pc_blocks
                                     contiguous blocks of ceil(n / pc_blocks) rows (the last one
                                     ragged), one per process of a row-distributed matrix, and each
                                     diagonal block is factored by ILU(0) in red-black order, as
                                     SKR_PC_ILU0 (PETSc's default sub-preconditioner); couplings
                                     between blocks are left out of M.  pc_blocks = 1 is SKR_PC_ILU0 */

/* precision form */
#define SKR_PREC_FP64         0   /* all vectors and reductions in FP64 */
#define SKR_PREC_MIXED        1   /* FP32 SpMV/Arnoldi/recycle vectors with FP32 accumulation,
                                     FP64 true residual, solution, refinement and small dense step
                                     (least squares, harmonic-Ritz eigenproblem, QR, Cholesky) */

#define SKR_MEM_DEVICE        0
#define SKR_MEM_HOST          1

/* compile-time capacity of the small dense step */
#define SKR_MAX_M            48   /* maximum restart length m */
#define SKR_MAX_K            24   /* maximum recycle dimension k */

/* One linear system of the sequence (Eq. 1).  Pointers are borrowed for the
 * call and live where skr_options.mem says. */
typedef struct skr_system {
    int32_t fmt;            /* SKR_FMT_* */
    int32_t nx, ny, nz;     /* interior grid (nz = 1 for 2D) */
    const double *coef;     /* format data, see SKR_FMT_* (NULL for CONVDIFF2D) */
    const double *rhs;      /* f at the n unknowns, or NULL for f = 1 */
    double params[4];       /* CONVDIFF2D: nu, beta_x, beta_y; otherwise unused */
    const int64_t *rowptr;  /* CSR: n + 1 row offsets; otherwise unused */
    const int32_t *colind;  /* CSR: column index of every value; otherwise unused */
} skr_system;

typedef struct skr_options {
    int32_t m;              /* maximum subspace size (Algorithm 2), 2 <= m <= SKR_MAX_M */
    int32_t k;              /* recycle dimension, 0 <= k <= min(SKR_MAX_K, m-2); 0 = GMRES(m) */
    int32_t maxit;          /* cap on Arnoldi steps per system (default 10000) */
    int32_t max_refine;     /* cap on residual-refinement passes per system (default 10) */
    double  tol;            /* target true relative residual ||b - A x|| / ||b|| (default 1e-8) */
    double  inner_tol;      /* SKR_PREC_MIXED: relative reduction per inner solve (default 1e-5) */
    int32_t precond;        /* SKR_PC_* (default SKR_PC_NONE) */
    int32_t precision;      /* SKR_PREC_* (default SKR_PREC_FP64) */
    int32_t cluster_size;   /* CTAs cooperating on one system, 1..16 (0 = planned per chain from
                               the measured launch table, see skr_last_plan) */
    int32_t max_slots;      /* clusters (chains in flight) at once over all launches (0 = as many
                               as fit on the GPU) */
    int32_t mem;            /* SKR_MEM_DEVICE or SKR_MEM_HOST */
    int32_t profile;        /* nonzero: accumulate device time per phase (skr_last_profile) */
    void   *stream;         /* cudaStream_t */
    int32_t warm_start;     /* nonzero: x_0 of a system is the solution of the previous system of
                               its chain (Algorithm 2 leaves x_0 free); the first system of a chain,
                               and every system when zero (default), starts from x_0 = 0 */
    int32_t diagnostics;    /* nonzero: report skr_result.delta (one extra Gram pass per system) */
    int32_t pc_blocks;      /* SKR_PC_BJACOBI: number of row blocks, >= 1 (default 1) */
    int32_t eig_fp32;       /* SKR_PREC_MIXED: 1 runs the harmonic-Ritz eigenproblem of each cycle end
                               (Algorithm 2) in FP32 instead of FP64 (default 0: FP64, like the rest
                               of the small dense step); ignored in the FP64 form */
    double *const *recycle_out;  /* NULL (default), or a host array of nchains pointers to DEVICE
                               memory (skr_solve_sequence with mem = SKR_MEM_DEVICE only): chain c's
                               final recycle space, U_k (Algorithm 2) in columns 0..k-1 and C_k in
                               columns k..2k-1, column-major with n rows; columns past the carried
                               dimension (k_final of the chain's last system) are zero.  For
                               checking A M^-1 U_k = C_k, C_k^T C_k = I (Sec. 4.2, App. B.1) */
} skr_options;

typedef struct skr_result {
    int32_t steps;          /* Arnoldi steps (one A M^-1 product each) */
    int32_t cycles;         /* GCRO-DR / GMRES cycles */
    int32_t matvecs;        /* all A M^-1 products, including the k of the recycle refresh */
    int32_t refinements;    /* inner solves (residual-refinement passes) */
    int32_t flag;           /* SKR_CONVERGED, ... */
    int32_t k_final;        /* recycle dimension carried out of this system */
    double  relres;         /* true ||b - A x||_2 / ||b||_2, computed in FP64 on the device */
    double  seconds;        /* device time spent on this system (globaltimer) */
    double  delta;          /* with diagnostics: the one-sided distance (Sec. 5.1, Eq. 5)
                               delta(Q, C) = ||(I - Pi_C) Pi_Q||_2 from C = range(C_k) entering the
                               system (after the App. B.1 refresh) to Q = range(C_k) leaving it,
                               i.e. the sine of the largest principal angle; -1 when either space
                               is empty or diagnostics are off */
} skr_result;

/* Fill *opt with the defaults named above. */
skr_status skr_options_default(skr_options *opt);

/*
 * skr_sort -- Algorithm 1 (Sec. 4.1): greedy nearest-neighbour order.
 *
 * params    N x p doubles, row i = the flattened parameter matrix P(i)
 * start     index of the first system (0 = the paper's system 1)
 * perm_out  N int32: the solve order, perm_out[0] = start
 * Distances are squared Frobenius norms summed in one fixed order (element
 * t into lane t mod 256, lanes added left to right without fused
 * multiply-add, then combined pairwise); ties go to the lowest index.
 * Scratch: an N x N FP64 distance matrix in device memory, allocated and
 * freed by the call.  Errors: N < 0, p < 1 (when N > 0), start outside
 * [0, N), or a non-finite parameter -> SKR_ERR_INVALID_ARG.
 */
skr_status skr_sort(const double *params, int64_t N, int64_t p, int64_t start,
                    int32_t mem, void *stream, int32_t *perm_out);

/*
 * skr_sort_noalloc -- the order of skr_sort, for callers that cannot
 * allocate device memory.  The paper has no counterpart: this entry point
 * exists for deployment, not for the method.
 *
 * Some callers cannot let a library call cudaMalloc: applications that hand
 * all device memory to their own pool allocator and forbid hidden
 * allocations, and loops with a latency budget in which a cudaMalloc /
 * cudaFree pair (each may synchronise the device) is not acceptable.  This
 * call computes the same permutation as skr_sort, bit for bit, and allocates
 * nothing: its scratch (the N x N distance matrix, the per-system "placed"
 * flags and an error word, about 2 MiB in all) lives in one fixed array of
 * device memory that every GPU loading this library holds until the process
 * exits.
 *
 * params    N x p doubles in DEVICE memory of the current device, row i = P(i) flattened
 * perm_out  N int32 in DEVICE memory of the current device
 * The call works on the current device; pointers to another device's
 * memory are rejected with SKR_ERR_INVALID_ARG.
 * N         at most SKR_SORT_NOALLOC_MAX_N; a larger N is rejected with
 *           SKR_ERR_INVALID_ARG before any device work
 * The first call on a device looks up the device address of the array
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  Every call on a device uses the same array and leaves its
 * contents behind: each call resets what must start at zero (the error word;
 * the kernel resets the flags), but two calls whose work overlaps on the GPU
 * (different streams or host threads) race on the array, so serialise them.
 * Host-memory pointers are rejected; other errors as skr_sort.
 */
#define SKR_SORT_NOALLOC_MAX_N 512
skr_status skr_sort_noalloc(const double *params, int64_t N, int64_t p, int64_t start,
                            void *stream, int32_t *perm_out);

/*
 * skr_sort_grouped -- the large-N order of Sec. 4.1 (the paragraph after
 * Algorithm 1): divide the systems into groups of at most group_max by
 * their coordinates, order each group by Algorithm 1, concatenate.
 *
 * params         N x p doubles, row i = P(i) flattened (memory per mem)
 * group_max      G >= 1, the largest group
 * perm_out       N int32 (memory per mem): the solve order
 * group_offsets  NULL, or a HOST array of at least ngroups + 1 int64 (N + 1
 *                always suffice): group g is perm_out[off[g] .. off[g+1])
 * ngroups        NULL, or HOST int64: the number of groups
 * Groups: recursive coordinate bisection.  A set of s > G systems is split
 * along the coordinate (entry of P(i)) whose spread max - min over the set
 * is largest, the lowest coordinate on ties: ordered by (value of that
 * coordinate, index), its first floor(s/2) systems form the first half,
 * the rest the second; sets of at most G systems are groups, concatenated
 * first half first.  Every set's size, hence every group offset, depends
 * on N and G only.  Inside a group, Algorithm 1 scans its systems in
 * ascending index order from its lowest index, with the distances of
 * skr_sort (bit for bit).  With G >= N the result equals skr_sort's with
 * start = 0.
 * Scratch (allocated and freed by the call): the working index array, the
 * sort keys (16 bytes per system, padded to a power of two >= 1024), per
 * split set 16 bytes per coordinate, and the groups' distance matrices
 * (sum of size^2 doubles, at most N x G).
 * Errors: N < 0, p < 1 (when N > 0), group_max < 1, a non-finite parameter
 * or distance -> SKR_ERR_INVALID_ARG; allocation failure -> SKR_ERR_OOM.
 */
skr_status skr_sort_grouped(const double *params, int64_t N, int64_t p, int64_t group_max,
                            int32_t mem, void *stream, int32_t *perm_out,
                            int64_t *group_offsets, int64_t *ngroups);

/*
 * skr_solve_sequence -- Algorithm 2 over a sorted sequence (Sec. 4.2,
 * App. B), with the sorted list cut into independent chains (App. E.2.2).
 *
 * systems        N system descriptors (host array; their data pointers per opt->mem)
 * order          N indices: the solve order (e.g. from skr_sort), or NULL = 0..N-1
 * chain_offsets  nchains+1 offsets into order (chain c = order[off[c] .. off[c+1]) ),
 *                or NULL = nchains contiguous near-equal pieces
 * nchains        >= 1; every system of one chain must share fmt and grid
 * opt            options (NULL = defaults)
 * x_out          N pointers (host array); x_out[i] receives n doubles, the
 *                solution of systems[i] (memory per opt->mem)
 * results        N entries (host array), indexed like systems
 * Each chain carries its own U_k, C_k; a chain's first system starts
 * without a recycle space.  Per system: residual refinement in FP64
 * around GCRO-DR inner solves (x = 0; repeat r = b - A x, stop when
 * ||r|| <= tol ||b||, solve A M^-1 d = r, x += M^-1 d).
 * Device memory for the Krylov basis and recycle vectors is allocated by
 * the call (or reused from the previous call) and kept by the library until
 * skr_release_workspace().
 */
skr_status skr_solve_sequence(const skr_system *systems, int64_t N, const int32_t *order,
                              const int64_t *chain_offsets, int32_t nchains,
                              const skr_options *opt, double *const *x_out,
                              skr_result *results);

/*
 * skr_assemble -- the discretisation of one system (Sec. 3.1, App. A.2) as
 * the solver builds it.
 *
 * coef_out    5 (2D) or 7 (3D) arrays of n doubles, the matrix A in the
 *             layout of SKR_FMT_STENCIL5/7 (may be NULL)
 * rhs_out     n doubles, b (may be NULL)
 * Uses the same device code as the solver.  Memory per mem.
 */
skr_status skr_assemble(const skr_system *sys, int32_t mem, void *stream,
                        double *coef_out, double *rhs_out);

/*
 * skr_apply -- y = A M^-1 v for one system, in the working precision of
 * `precision` (SKR_PREC_MIXED: FP32 arithmetic, v rounded to FP32 on
 * input and y widened to FP64 on output), using the solver's own operator
 * code.  v, y: n doubles each, memory per mem.  pc_blocks: the block count
 * of SKR_PC_BJACOBI (>= 1; ignored by the other preconditioners).
 */
skr_status skr_apply(const skr_system *sys, int32_t precond, int32_t pc_blocks, int32_t precision,
                     const double *v, double *y, int32_t mem, void *stream);

/* ------------------------------------------------------------------ serving
 *
 * A request loop over the same solver: systems arrive one at a time (as in
 * data generation for a neural operator, Sec. 1 and Fig. 1, where a stream
 * of PDE instances is solved), are admitted as device memory and slots free
 * up, are routed to the resident recycle chain nearest to them in parameter
 * space (the sort's distance, Algorithm 1, applied online), and run
 * concurrently with the requests of other chains (continuous batching: a new
 * request starts as soon as it is admitted, while others are on the GPU).
 * Each chain keeps its U_k, C_k in device memory between requests and
 * refreshes them against every new matrix (App. B.1).
 */
typedef struct skr_server skr_server;

typedef struct skr_server_info {
    int64_t submitted, completed, queued, running;
    int32_t chains;           /* recycle chains resident now */
    int32_t evicted;          /* chains evicted so far to make room for a request of a new shape */
    double  p50_ms, p99_ms, mean_ms;   /* submit-to-completion latency of completed requests */
    double  hbm_bytes;        /* device memory held by the server's chains */
} skr_server_info;

/*
 * skr_server_create -- start a server on the current CUDA device.
 *
 * opt          solver options (m, k, tol, precond, precision, cluster_size, ...);
 *              opt->mem and opt->stream are ignored (requests are host memory,
 *              every chain has its own stream)
 * hbm_budget   bytes of device memory the server may hold for chains (each
 *              chain holds one workspace slot sized for its grid plus its
 *              request buffers); 0 = no limit
 * max_chains   upper bound on resident chains (0 = as many as chain-kernel CTAs fit on the GPU)
 * A host thread owned by the server admits, routes, launches and collects
 * requests.  Every chain has its own stream; streams share the device's
 * hardware work queues (CUDA_DEVICE_MAX_CONNECTIONS, 8 by default), and a
 * request whose stream shares a queue with a running solve can start only
 * after it, so processes that serve many chains should set that variable to
 * 32 before CUDA starts.  Errors: bad options -> SKR_ERR_INVALID_ARG.
 */
skr_status skr_server_create(const skr_options *opt, size_t hbm_budget, int32_t max_chains,
                             skr_server **srv);

/*
 * skr_submit -- enqueue one system; returns at once with a ticket.
 *
 * sys    the system, its data in HOST memory; the server copies it before
 *        returning, so the caller may reuse or free the buffers
 * key    p doubles, the routing parameter vector (e.g. log a flattened, or
 *        (nu, beta)); only chains of the same format, grid and p are
 *        candidates.  key may be NULL (p = 0): the system's own coefficient
 *        data is then the key
 * Requests are admitted in arrival order, a waiting one not holding back
 * later ones.  A request waits until its cluster's CTAs fit on the GPU
 * beside the running requests (one request always runs).  It then goes to
 * the nearest idle chain of its shape (format, grid and p); else to a new
 * chain if max_chains and the budget leave room; else to a new chain that
 * replaces the least recently used idle chains (evicted: their recycle
 * spaces are dropped).  So every request that fits the budget on its own is
 * eventually served, and no SM waits while a request could use it.
 * A request larger than the whole budget is rejected (SKR_ERR_OOM).
 */
skr_status skr_submit(skr_server *srv, const skr_system *sys, const double *key, int64_t p,
                      uint64_t *ticket);

/*
 * skr_poll -- SKR_NOT_READY while the request is queued or running; once it
 * is done, copies the n-vector solution to x_out (host memory) and the
 * outcome to *res, forgets the ticket and returns SKR_OK.  An unknown ticket
 * -> SKR_ERR_INVALID_ARG.
 */
skr_status skr_poll(skr_server *srv, uint64_t ticket, double *x_out, skr_result *res);

/* Counters and latency percentiles of the server so far. */
skr_status skr_server_stats(skr_server *srv, skr_server_info *info);

/* Wait for the running requests, stop the loop and free every resource;
 * queued requests are dropped. */
skr_status skr_server_destroy(skr_server *srv);

/*
 * skr_last_stats -- figures of the last skr_solve_sequence call on the
 * calling thread: the algorithmic bytes its kernel streamed (the compulsory
 * traffic of each pass, counted by the kernel from the pass sizes, not
 * measured), the kernels' duration from CUDA events recorded around the
 * launches on the call's stream, the cluster size (0 when the call made
 * launches of several sizes, see skr_last_plan), the number of clusters in
 * flight over all launches, and the number of kernel launches.  Any
 * pointer may be NULL.
 */
skr_status skr_last_stats(uint64_t *bytes, double *kernel_ms, int32_t *cluster_size,
                          int32_t *slots, int32_t *launches);

/*
 * skr_last_plan -- the launches of the last skr_solve_sequence call on the
 * calling thread.  With opt->cluster_size = 0 the library cuts the chains
 * into launches by cluster size (App. E.2.2's independent chains, each a
 * thread-block cluster): each chain gets the cluster size that a table
 * measured on this GPU (the project's autotuner, paper_2401_09516_gb300/
 * tune.py) makes cheapest in CTA time per Arnoldi step, chains longer than
 * the batch's ideal makespan get larger clusters, the launches share the
 * GPU's CTAs in proportion to their estimated work and run concurrently,
 * and each launch hands out its chains longest first.  With
 * opt->cluster_size > 0 there is one launch of that cluster size.
 * For launch i < min(cap, *nlaunch): cluster_size[i] CTAs per cluster,
 * clusters[i] clusters, chains[i] chains.  Any array may be NULL.
 */
skr_status skr_last_plan(int32_t *cluster_size, int32_t *clusters, int32_t *chains, int32_t cap,
                         int32_t *nlaunch);

/*
 * skr_last_profile -- device time per phase of the last skr_solve_sequence
 * call made with opt->profile != 0, summed over all clusters (rank-0 CTA
 * clocks, globaltimer): ns_out[i] for phase i < min(nphase, SKR_NPHASE),
 * in the order assembly, refresh, projection, operator, multi-dot, update,
 * gram, dense, cycle-update, true-residual, other, schur, eigenvectors,
 * hessenberg (the last three are the parts of the dense step spent on the
 * Francis iteration to the Schur form of the harmonic-Ritz matrix, on its
 * selected eigenvectors, and on its Hessenberg reduction; "dense" holds the
 * rest of the cycle-end small step).
 */
#define SKR_NPHASE 14
skr_status skr_last_profile(double *ns_out, int32_t nphase);

/* Free the device workspace cached by skr_solve_sequence (all devices). */
skr_status skr_release_workspace(void);

/* Message describing the last error on the calling thread ("" if none). */
const char *skr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SKR_H */
