// C ABI of the SKR library (include/skr.h): validation, device workspace,
// staging of host data, kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "skr_common.h"
#include "skr_launch.h"
#include "skr_plan.h"
#include "skr_tma.h"
#include "skr_workspace.h"
#include "skr_ops.cuh"
#include "skr_sort.cuh"

using namespace skr;

namespace {

thread_local std::string g_err;

skr_status fail(skr_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? SKR_ERR_OOM : SKR_ERR_CUDA,          \
                        "%s failed: %s", #expr, cudaGetErrorString(e_));                      \
        }                                                                                     \
    } while (0)

// RAII device buffer (per call).
struct DBuf {
    void *p = nullptr;
    ~DBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 16); }
    template <typename X> X *as() const { return reinterpret_cast<X *>(p); }
};

// Workspace cached across calls (per device), grown on demand.
struct CachedWs {
    int device = -1;
    size_t bytes = 0;
    void *base = nullptr;
};
std::mutex g_ws_mu;
std::vector<CachedWs> g_ws;

cudaError_t ws_get(size_t bytes, void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_ws_mu);
    for (auto &w : g_ws) {
        if (w.device == dev) {
            if (w.bytes >= bytes) {
                *out = w.base;
                return cudaSuccess;
            }
            cudaFree(w.base);
            w.base = nullptr;
            w.bytes = 0;
            e = cudaMalloc(&w.base, bytes);
            if (e != cudaSuccess) return e;
            w.bytes = bytes;
            *out = w.base;
            return cudaSuccess;
        }
    }
    CachedWs w;
    w.device = dev;
    e = cudaMalloc(&w.base, bytes);
    if (e != cudaSuccess) return e;
    w.bytes = bytes;
    g_ws.push_back(w);
    *out = w.base;
    return cudaSuccess;
}

// Streams of the concurrent launches of one call (per device, created on
// first use, kept until exit).
std::vector<std::pair<int, cudaStream_t>> g_streams;

cudaError_t launch_streams(int count, cudaStream_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_ws_mu);
    int have = 0;
    for (auto &ps : g_streams)
        if (ps.first == dev && have < count) out[have++] = ps.second;
    while (have < count) {
        cudaStream_t s2 = nullptr;
        e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        g_streams.push_back({dev, s2});
        out[have++] = s2;
    }
    return cudaSuccess;
}

bool is_3d(int fmt) { return fmt == SKR_FMT_DARCY3D || fmt == SKR_FMT_STENCIL7; }

long long sys_n(const skr_system &s) {
    if (s.fmt == SKR_FMT_CSR) return (long long)s.nx;
    return (long long)s.nx * s.ny * (is_3d(s.fmt) ? s.nz : 1);
}

long long sys_coef_len(const skr_system &s) {
    const long long n = sys_n(s);
    switch (s.fmt) {
        case SKR_FMT_DARCY2D: return (long long)(s.nx + 2) * (s.ny + 2);
        case SKR_FMT_DARCY3D: return (long long)(s.nx + 2) * (s.ny + 2) * (s.nz + 2);
        case SKR_FMT_STENCIL5: return 5 * n;
        case SKR_FMT_STENCIL7: return 7 * n;
        case SKR_FMT_HELMHOLTZ2D: return n;
        case SKR_FMT_POISSON2D: return n + 2LL * (s.nx + s.ny);
        default: return 0;   // CSR: the value count lives in rowptr[n]
    }
}

skr_status check_system(const skr_system &s, long long idx) {
    if (s.fmt < SKR_FMT_DARCY2D || s.fmt > SKR_FMT_CSR)
        return fail(SKR_ERR_INVALID_ARG, "system %lld: unknown format %d", idx, s.fmt);
    if (s.fmt == SKR_FMT_CSR) {
        if (s.nx < 1) return fail(SKR_ERR_INVALID_ARG, "system %lld: CSR with no rows", idx);
        if (!s.rowptr || !s.colind || !s.coef)
            return fail(SKR_ERR_INVALID_ARG, "system %lld: CSR needs rowptr, colind and coef (the values)", idx);
        return SKR_OK;
    }
    if (s.nx < 1 || s.ny < 1 || (is_3d(s.fmt) && s.nz < 1))
        return fail(SKR_ERR_INVALID_ARG, "system %lld: empty grid", idx);
    if (s.fmt == SKR_FMT_CONVDIFF2D && s.nx != s.ny)
        return fail(SKR_ERR_INVALID_ARG, "system %lld: convection-diffusion needs nx == ny", idx);
    if (s.fmt == SKR_FMT_CONVDIFF2D && !(s.params[0] > 0.0))
        return fail(SKR_ERR_INVALID_ARG, "system %lld: nu must be positive", idx);
    if (s.fmt != SKR_FMT_CONVDIFF2D && s.coef == nullptr)
        return fail(SKR_ERR_INVALID_ARG, "system %lld: coef is NULL", idx);
    if (s.fmt == SKR_FMT_POISSON2D && s.rhs != nullptr)
        return fail(SKR_ERR_INVALID_ARG, "system %lld: the Poisson format takes f in coef; rhs must be NULL", idx);
    if (sys_n(s) > (1LL << 31) - 1024)
        return fail(SKR_ERR_INVALID_ARG, "system %lld: too many unknowns", idx);
    return SKR_OK;
}

bool same_shape(const skr_system &a, const skr_system &b) {
    if (a.fmt == SKR_FMT_CSR || b.fmt == SKR_FMT_CSR) return a.fmt == b.fmt && a.nx == b.nx;
    return a.fmt == b.fmt && a.nx == b.nx && a.ny == b.ny && (!is_3d(a.fmt) || a.nz == b.nz);
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (int)std::max(1LL, std::min(b, 152LL * 16));
}

// Stage one system's data on the device when mem == HOST.
struct Staged {
    DBuf coef, rhs, rowptr, colind;
    DevSystem dev;
};

skr_status stage_system(const skr_system &s, int mem, cudaStream_t st, Staged &out) {
    out.dev.fmt = s.fmt;
    out.dev.nx = s.nx;
    out.dev.ny = s.ny;
    out.dev.nz = is_3d(s.fmt) ? s.nz : 1;
    for (int i = 0; i < 4; i++) out.dev.params[i] = s.params[i];
    out.dev.x_out = nullptr;
    const long long n = sys_n(s);
    long long clen = sys_coef_len(s);
    out.dev.rowptr = nullptr;
    out.dev.colind = nullptr;
    out.dev.csr_w = 0;
    if (s.fmt == SKR_FMT_CSR) {
        out.dev.ny = out.dev.nz = 1;
        if (mem == SKR_MEM_HOST) {
            const long long nnz = s.rowptr[n];
            if (nnz < n || nnz > (long long)SKR_CSR_MAX_ROW * n)
                return fail(SKR_ERR_INVALID_ARG, "CSR: rowptr[n] = %lld is not a value count of n = %lld rows "
                            "with 1..%d entries each", nnz, n, SKR_CSR_MAX_ROW);
            clen = nnz;
            CUDA_TRY(out.rowptr.alloc((n + 1) * 8));
            CUDA_TRY(cudaMemcpyAsync(out.rowptr.p, s.rowptr, (n + 1) * 8, cudaMemcpyHostToDevice, st));
            CUDA_TRY(out.colind.alloc(nnz * 4));
            CUDA_TRY(cudaMemcpyAsync(out.colind.p, s.colind, nnz * 4, cudaMemcpyHostToDevice, st));
            out.dev.rowptr = out.rowptr.as<long long>();
            out.dev.colind = out.colind.as<int>();
        } else {
            out.dev.rowptr = reinterpret_cast<const long long *>(s.rowptr);
            out.dev.colind = s.colind;
        }
    }
    if (mem == SKR_MEM_HOST) {
        if (clen > 0) {
            CUDA_TRY(out.coef.alloc(clen * 8));
            CUDA_TRY(cudaMemcpyAsync(out.coef.p, s.coef, clen * 8, cudaMemcpyHostToDevice, st));
        }
        if (s.rhs) {
            CUDA_TRY(out.rhs.alloc(n * 8));
            CUDA_TRY(cudaMemcpyAsync(out.rhs.p, s.rhs, n * 8, cudaMemcpyHostToDevice, st));
        }
        out.dev.coef = out.coef.as<double>();
        out.dev.rhs = s.rhs ? out.rhs.as<double>() : nullptr;
    } else {
        out.dev.coef = s.coef;
        out.dev.rhs = s.rhs;
    }
    return SKR_OK;
}

// Check the CSR systems among hs (device descriptors; ns[i] rows) with one
// kernel each and a single read-back, and set their row width.
skr_status check_csr(std::vector<DevSystem> &hs, const std::vector<long long> &ns, cudaStream_t st) {
    std::vector<int> idx;
    for (size_t i = 0; i < hs.size(); i++)
        if (hs[i].fmt == SKR_FMT_CSR) idx.push_back((int)i);
    if (idx.empty()) return SKR_OK;
    DBuf dout;
    CUDA_TRY(dout.alloc(sizeof(int) * 2 * idx.size()));
    CUDA_TRY(cudaMemsetAsync(dout.p, 0, sizeof(int) * 2 * idx.size(), st));
    for (size_t q = 0; q < idx.size(); q++) {
        const long long n = ns[idx[q]];
        skr_csr_check_kernel<<<grid_for(n, 256), 256, 0, st>>>(hs[idx[q]].rowptr, hs[idx[q]].colind, n,
                                                               dout.as<int>() + 2 * q);
    }
    CUDA_TRY(cudaGetLastError());
    std::vector<int> h(2 * idx.size());
    CUDA_TRY(cudaMemcpyAsync(h.data(), dout.p, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (size_t q = 0; q < idx.size(); q++) {
        const int e = h[2 * q];
        if (e & 1)
            return fail(SKR_ERR_INVALID_ARG, "system %d: CSR rowptr not ascending from 0, or a row with no entry "
                        "or more than %d", idx[q], SKR_CSR_MAX_ROW);
        if (e & 2) return fail(SKR_ERR_INVALID_ARG, "system %d: CSR row without exactly one diagonal entry", idx[q]);
        if (e & 4) return fail(SKR_ERR_INVALID_ARG, "system %d: CSR column index outside [0, n)", idx[q]);
        if (e & 8) return fail(SKR_ERR_INVALID_ARG, "system %d: CSR column repeated within a row", idx[q]);
        hs[idx[q]].csr_w = h[2 * q + 1];
    }
    return SKR_OK;
}

}  // namespace

namespace skr {
// Record an error message for the calling thread (used by the server unit).
skr_status set_last_error(skr_status code, const char *msg) {
    g_err = msg;
    return code;
}
}  // namespace skr

namespace {

struct LastStats {
    unsigned long long prof[SKR_NPHASE] = {0};
    unsigned long long bytes = 0;
    float kernel_ms = 0.f;
    int cluster_size = 0, slots = 0, launches = 0;
    struct Shape {
        int cs, slots, chains;
    };
    std::vector<Shape> plan;   // per launch of the last call
};
thread_local LastStats g_last;

}  // namespace

namespace {

// Pairwise distance matrix of Algorithm 1 (full sort): short parameter
// vectors take one thread per pair, long ones a CTA per 4 x 4 tile of pairs;
// both follow the same summation order.
cudaError_t launch_sort_dist(const double *P, long long N, long long p, double *dist, int *err, cudaStream_t st) {
    if (p <= SORT_SMALL_P) {
        launch_pair_dist_small(P, p, nullptr, nullptr, nullptr, 0, N, dist, err, st);
    } else {
        const long long nt = (N + SORT_TILE - 1) / SORT_TILE;
        const long long blocks = nt * (nt + 1) / 2;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
        sort_dist_kernel<<<(unsigned)blocks, SORT_LANES, 0, st>>>(P, N, p, dist, err);
    }
    return cudaGetLastError();
}

// Sort the working positions by (set, split value, index): a bitonic
// network over M = 2^e >= BITONIC_LOCAL keys, the steps with partner
// distance below BITONIC_LOCAL in shared memory.
cudaError_t bitonic_sort(GroupKey *keys, long long M, cudaStream_t st) {
    const unsigned nb = (unsigned)(M / BITONIC_LOCAL);
    bitonic_local_kernel<<<nb, BITONIC_LOCAL / 2, 0, st>>>(keys, 0);
    for (long long k = 2 * BITONIC_LOCAL; k <= M; k <<= 1) {
        for (long long j = k >> 1; j >= BITONIC_LOCAL; j >>= 1)
            bitonic_global_kernel<<<grid_for(M / 2, 256), 256, 0, st>>>(keys, M, k, j);
        bitonic_local_kernel<<<nb, BITONIC_LOCAL / 2, 0, st>>>(keys, k);
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" {

skr_status skr_options_default(skr_options *opt) {
    if (!opt) return fail(SKR_ERR_INVALID_ARG, "opt is NULL");
    memset(opt, 0, sizeof(*opt));
    opt->m = 30;
    opt->k = 10;
    opt->maxit = 10000;
    opt->max_refine = 10;
    opt->tol = 1e-8;
    opt->inner_tol = 1e-5;
    opt->precond = SKR_PC_NONE;
    opt->precision = SKR_PREC_FP64;
    opt->cluster_size = 0;
    opt->max_slots = 0;
    opt->mem = SKR_MEM_DEVICE;
    opt->stream = nullptr;
    opt->pc_blocks = 1;
    return SKR_OK;
}

const char *skr_last_error(void) { return g_err.c_str(); }

skr_status skr_sort(const double *params, int64_t N, int64_t p, int64_t start, int32_t mem, void *stream,
                    int32_t *perm_out) {
    g_err.clear();
    if (N < 0) return fail(SKR_ERR_INVALID_ARG, "N < 0");
    if (N == 0) return SKR_OK;
    if (!params || !perm_out) return fail(SKR_ERR_INVALID_ARG, "NULL pointer");
    if (p < 1) return fail(SKR_ERR_INVALID_ARG, "p < 1");
    if (start < 0 || start >= N) return fail(SKR_ERR_INVALID_ARG, "start out of range");
    if (mem != SKR_MEM_DEVICE && mem != SKR_MEM_HOST) return fail(SKR_ERR_INVALID_ARG, "bad mem");
    if (N > (1LL << 20)) return fail(SKR_ERR_INVALID_ARG, "N too large for the N x N distance matrix");
    cudaStream_t st = (cudaStream_t)stream;
    DBuf dparams, ddist, dperm, dtaken, derr;
    const double *P = params;
    if (mem == SKR_MEM_HOST) {
        CUDA_TRY(dparams.alloc((size_t)N * p * 8));
        CUDA_TRY(cudaMemcpyAsync(dparams.p, params, (size_t)N * p * 8, cudaMemcpyHostToDevice, st));
        P = dparams.as<double>();
    }
    CUDA_TRY(ddist.alloc((size_t)N * N * 8));
    CUDA_TRY(dtaken.alloc((size_t)N));
    CUDA_TRY(derr.alloc(sizeof(int)));
    CUDA_TRY(cudaMemsetAsync(derr.p, 0, sizeof(int), st));
    int *perm = perm_out;
    if (mem == SKR_MEM_HOST) {
        CUDA_TRY(dperm.alloc((size_t)N * 4));
        perm = dperm.as<int>();
    }
    {
        const cudaError_t e = launch_sort_dist(P, N, p, ddist.as<double>(), derr.as<int>(), st);
        if (e == cudaErrorInvalidValue) return fail(SKR_ERR_INVALID_ARG, "N too large");
        CUDA_TRY(e);
    }
    int herr = 0;
    CUDA_TRY(cudaMemcpyAsync(&herr, derr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (herr) return fail(SKR_ERR_INVALID_ARG, "non-finite parameter distance");
    sort_chain_kernel<<<1, 1024, 0, st>>>(ddist.as<double>(), N, start, perm, dtaken.as<unsigned char>());
    CUDA_TRY(cudaGetLastError());
    if (mem == SKR_MEM_HOST)
        CUDA_TRY(cudaMemcpyAsync(perm_out, perm, (size_t)N * 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return SKR_OK;
}

skr_status skr_sort_grouped(const double *params, int64_t N, int64_t p, int64_t group_max, int32_t mem,
                            void *stream, int32_t *perm_out, int64_t *group_offsets, int64_t *ngroups) {
    g_err.clear();
    if (N < 0) return fail(SKR_ERR_INVALID_ARG, "N < 0");
    if (group_max < 1) return fail(SKR_ERR_INVALID_ARG, "group_max < 1");
    if (mem != SKR_MEM_DEVICE && mem != SKR_MEM_HOST) return fail(SKR_ERR_INVALID_ARG, "bad mem");
    if (N == 0) {
        if (group_offsets) group_offsets[0] = 0;
        if (ngroups) *ngroups = 0;
        return SKR_OK;
    }
    if (!params || !perm_out) return fail(SKR_ERR_INVALID_ARG, "NULL pointer");
    if (p < 1) return fail(SKR_ERR_INVALID_ARG, "p < 1");
    if (N > (1LL << 30)) return fail(SKR_ERR_INVALID_ARG, "N too large");
    if (p > 65535LL * SPREAD_THREADS) return fail(SKR_ERR_INVALID_ARG, "p too large");
    cudaStream_t st = (cudaStream_t)stream;
    DBuf dparams, dperm, derr, didx, dkeys;
    const double *P = params;
    if (mem == SKR_MEM_HOST) {
        CUDA_TRY(dparams.alloc((size_t)N * p * 8));
        CUDA_TRY(cudaMemcpyAsync(dparams.p, params, (size_t)N * p * 8, cudaMemcpyHostToDevice, st));
        P = dparams.as<double>();
    }
    int *perm = perm_out;
    if (mem == SKR_MEM_HOST) {
        CUDA_TRY(dperm.alloc((size_t)N * 4));
        perm = dperm.as<int>();
    }
    CUDA_TRY(derr.alloc(sizeof(int)));
    CUDA_TRY(cudaMemsetAsync(derr.p, 0, sizeof(int), st));
    finite_kernel<<<1024, 256, 0, st>>>(P, N * p, derr.as<int>());
    CUDA_TRY(cudaGetLastError());
    int herr = 0;
    CUDA_TRY(cudaMemcpyAsync(&herr, derr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (herr) return fail(SKR_ERR_INVALID_ARG, "non-finite parameter");

    long long M = BITONIC_LOCAL;
    while (M < N) M <<= 1;
    CUDA_TRY(didx.alloc((size_t)N * 4));
    CUDA_TRY(dkeys.alloc((size_t)M * sizeof(GroupKey)));
    iota_kernel<<<grid_for(N, 256), 256, 0, st>>>(didx.as<int>(), N);
    CUDA_TRY(cudaGetLastError());
    // bisection levels: the set offsets are known here, the members are not
    std::vector<long long> off = {0, (long long)N};
    const long long spread_cap = 1LL << 25;   // coordinates x sets per spread batch (2 x 256 MB of keys)
    const long long batch_sets = std::max(1LL, spread_cap / p);
    for (int final_pass = 0; final_pass < 2;) {
        const int nn = (int)off.size() - 1;
        std::vector<long long> soff, ssize, sslot;
        if (!final_pass)
            for (int q = 0; q < nn; q++)
                if (off[q + 1] - off[q] > group_max) {
                    soff.push_back(off[q]);
                    ssize.push_back(off[q + 1] - off[q]);
                    sslot.push_back(q);
                }
        if (!final_pass && soff.empty()) {
            final_pass = 1;   // leaves only: one more sort puts each group in index order
            continue;
        }
        DBuf dcoord, doff;
        CUDA_TRY(dcoord.alloc((size_t)nn * 4));
        CUDA_TRY(cudaMemsetAsync(dcoord.p, 0xff, (size_t)nn * 4, st));   // -1: not split
        CUDA_TRY(doff.alloc((size_t)(nn + 1) * 8));
        CUDA_TRY(cudaMemcpyAsync(doff.p, off.data(), (size_t)(nn + 1) * 8, cudaMemcpyHostToDevice, st));
        for (size_t b0 = 0; b0 < soff.size(); b0 += (size_t)batch_sets) {
            const long long nb = std::min((long long)(soff.size() - b0), batch_sets);
            long long smax = 0;
            for (long long q = 0; q < nb; q++) smax = std::max(smax, ssize[b0 + q]);
            const long long cps = (smax + SPREAD_CHUNK - 1) / SPREAD_CHUNK;
            if (nb * cps > 0x7fffffffLL) return fail(SKR_ERR_INVALID_ARG, "N too large");
            DBuf dmn, dmx, dso, dss, dsl;
            CUDA_TRY(dmn.alloc((size_t)nb * p * 8));
            CUDA_TRY(dmx.alloc((size_t)nb * p * 8));
            CUDA_TRY(dso.alloc((size_t)nb * 8));
            CUDA_TRY(dss.alloc((size_t)nb * 8));
            CUDA_TRY(dsl.alloc((size_t)nb * 8));
            CUDA_TRY(cudaMemcpyAsync(dso.p, soff.data() + b0, (size_t)nb * 8, cudaMemcpyHostToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(dss.p, ssize.data() + b0, (size_t)nb * 8, cudaMemcpyHostToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(dsl.p, sslot.data() + b0, (size_t)nb * 8, cudaMemcpyHostToDevice, st));
            spread_init_kernel<<<grid_for(nb * p, 256), 256, 0, st>>>(dmn.as<unsigned long long>(),
                                                                     dmx.as<unsigned long long>(), nb * p);
            const dim3 grid((unsigned)(nb * cps), (unsigned)((p + SPREAD_THREADS - 1) / SPREAD_THREADS));
            spread_kernel<<<grid, SPREAD_THREADS, 0, st>>>(P, p, didx.as<int>(), dso.as<long long>(),
                                                           dss.as<long long>(), cps, dmn.as<unsigned long long>(),
                                                           dmx.as<unsigned long long>());
            spread_argmax_kernel<<<(unsigned)nb, SPREAD_THREADS, 0, st>>>(
                dmn.as<unsigned long long>(), dmx.as<unsigned long long>(), p, dsl.as<long long>(),
                dcoord.as<int>());
            CUDA_TRY(cudaGetLastError());
            CUDA_TRY(cudaStreamSynchronize(st));   // the batch's buffers are freed on return
        }
        group_keys_kernel<<<grid_for(M, 256), 256, 0, st>>>(P, p, didx.as<int>(), N, M, doff.as<long long>(), nn,
                                                          dcoord.as<int>(), dkeys.as<GroupKey>());
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(bitonic_sort(dkeys.as<GroupKey>(), M, st));
        keys_to_idx_kernel<<<grid_for(N, 256), 256, 0, st>>>(dkeys.as<GroupKey>(), N, didx.as<int>());
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaStreamSynchronize(st));   // doff, dcoord are freed on return
        if (final_pass) break;
        std::vector<long long> next;
        for (int q = 0; q < nn; q++) {
            next.push_back(off[q]);
            const long long sz = off[q + 1] - off[q];
            if (sz > group_max) next.push_back(off[q] + sz / 2);
        }
        next.push_back(N);
        off.swap(next);
    }
    // Algorithm 1 inside each group
    const int ng = (int)off.size() - 1;
    // long parameter vectors: a CTA per 4 x 4 tile of pairs; short ones: a
    // CTA per row, a thread per pair
    const bool small = p <= SORT_SMALL_P;
    std::vector<long long> boff(ng + 1), doffs(ng + 1);
    boff[0] = doffs[0] = 0;
    for (int g = 0; g < ng; g++) {
        const long long s = off[g + 1] - off[g], nt = (s + SORT_TILE - 1) / SORT_TILE;
        boff[g + 1] = boff[g] + nt * (nt + 1) / 2;
        doffs[g + 1] = doffs[g] + s * s;
    }
    const long long nblk = small ? (long long)N : boff[ng];
    if (nblk > 0x7fffffffLL) return fail(SKR_ERR_INVALID_ARG, "groups too large for one launch");
    DBuf dgoff, dboff, ddoff, ddist, dtaken;
    CUDA_TRY(dgoff.alloc((size_t)(ng + 1) * 8));
    CUDA_TRY(dboff.alloc((size_t)(ng + 1) * 8));
    CUDA_TRY(ddoff.alloc((size_t)(ng + 1) * 8));
    CUDA_TRY(ddist.alloc((size_t)doffs[ng] * 8));
    CUDA_TRY(dtaken.alloc((size_t)N));
    CUDA_TRY(cudaMemcpyAsync(dgoff.p, off.data(), (size_t)(ng + 1) * 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(dboff.p, boff.data(), (size_t)(ng + 1) * 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(ddoff.p, doffs.data(), (size_t)(ng + 1) * 8, cudaMemcpyHostToDevice, st));
    if (small)
        launch_pair_dist_small(P, p, didx.as<int>(), dgoff.as<long long>(), ddoff.as<long long>(), ng, N,
                               ddist.as<double>(), derr.as<int>(), st);
    else
        group_dist_kernel<<<(unsigned)nblk, SORT_LANES, 0, st>>>(P, p, didx.as<int>(), dgoff.as<long long>(),
                                                                 dboff.as<long long>(), ddoff.as<long long>(), ng,
                                                                 ddist.as<double>(), derr.as<int>());
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(&herr, derr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (herr) return fail(SKR_ERR_INVALID_ARG, "non-finite parameter distance");
    group_chain_kernel<<<(unsigned)ng, 256, 0, st>>>(ddist.as<double>(), ddoff.as<long long>(),
                                                     dgoff.as<long long>(), didx.as<int>(), perm,
                                                     dtaken.as<unsigned char>());
    CUDA_TRY(cudaGetLastError());
    if (mem == SKR_MEM_HOST)
        CUDA_TRY(cudaMemcpyAsync(perm_out, perm, (size_t)N * 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (group_offsets)
        for (int g = 0; g <= ng; g++) group_offsets[g] = off[g];
    if (ngroups) *ngroups = ng;
    return SKR_OK;
}

skr_status skr_assemble(const skr_system *sys, int32_t mem, void *stream, double *coef_out, double *rhs_out) {
    g_err.clear();
    if (!sys) return fail(SKR_ERR_INVALID_ARG, "sys is NULL");
    skr_status s0 = check_system(*sys, 0);
    if (s0 != SKR_OK) return s0;
    if (sys->fmt == SKR_FMT_CSR) return fail(SKR_ERR_INVALID_ARG, "a CSR system is already assembled");
    cudaStream_t st = (cudaStream_t)stream;
    Staged sg;
    s0 = stage_system(*sys, mem, st, sg);
    if (s0 != SKR_OK) return s0;
    const Geom g = make_geom(sys->fmt, sys->nx, sys->ny, sys->nz);
    DBuf anode, A, b;
    long long nn = (sys->fmt == SKR_FMT_DARCY2D || sys->fmt == SKR_FMT_DARCY3D) ? sys_coef_len(*sys) : 0;
    if (nn > 0) {
        CUDA_TRY(anode.alloc(nn * 8));
        node_exp_kernel<<<grid_for(nn, 256), 256, 0, st>>>(sg.dev.coef, nn, anode.as<double>());
        CUDA_TRY(cudaGetLastError());
    }
    CUDA_TRY(A.alloc((size_t)g.nst * g.n * 8));
    CUDA_TRY(b.alloc((size_t)g.n * 8));
    rows_kernel<<<grid_for(g.n, 256), 256, 0, st>>>(sg.dev, g, anode.as<double>(), A.as<double>(), g.n,
                                                     b.as<double>(), nullptr, SKR_PC_NONE, nullptr);
    CUDA_TRY(cudaGetLastError());
    const cudaMemcpyKind kind = (mem == SKR_MEM_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (coef_out) CUDA_TRY(cudaMemcpyAsync(coef_out, A.p, (size_t)g.nst * g.n * 8, kind, st));
    if (rhs_out) CUDA_TRY(cudaMemcpyAsync(rhs_out, b.p, (size_t)g.n * 8, kind, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return SKR_OK;
}

skr_status skr_apply(const skr_system *sys, int32_t precond, int32_t pc_blocks, int32_t precision,
                     const double *v, double *y, int32_t mem, void *stream) {
    g_err.clear();
    if (!sys || !v || !y) return fail(SKR_ERR_INVALID_ARG, "NULL pointer");
    skr_status s0 = check_system(*sys, 0);
    if (s0 != SKR_OK) return s0;
    if (precond != SKR_PC_NONE && precond != SKR_PC_JACOBI && precond != SKR_PC_ILU0 && precond != SKR_PC_SSOR &&
        precond != SKR_PC_BJACOBI)
        return fail(SKR_ERR_INVALID_ARG, "unknown preconditioner %d", precond);
    if (precond == SKR_PC_BJACOBI && pc_blocks < 1) return fail(SKR_ERR_INVALID_ARG, "pc_blocks < 1");
    if (precision != SKR_PREC_FP64 && precision != SKR_PREC_MIXED)
        return fail(SKR_ERR_INVALID_ARG, "bad precision");
    if (sys->fmt == SKR_FMT_CSR && colour_sweep_pc(precond))
        return fail(SKR_ERR_INVALID_ARG, "CSR input takes SKR_PC_NONE or SKR_PC_JACOBI only");
    cudaStream_t st = (cudaStream_t)stream;
    Staged sg;
    s0 = stage_system(*sys, mem, st, sg);
    if (s0 != SKR_OK) return s0;
    DBuf cols;
    Geom g = make_geom(sys->fmt, sys->nx, sys->ny, sys->nz);
    if (sys->fmt == SKR_FMT_CSR) {
        std::vector<DevSystem> one(1, sg.dev);
        s0 = check_csr(one, std::vector<long long>(1, sys_n(*sys)), st);
        if (s0 != SKR_OK) return s0;
        sg.dev.csr_w = one[0].csr_w;
        CUDA_TRY(cols.alloc((size_t)one[0].csr_w * sys_n(*sys) * 4));
        g = make_csr_geom(sys_n(*sys), one[0].csr_w, cols.as<int>(), sys_n(*sys));
    }
    DBuf anode, A, dinv, Aw, vw, dv, dy;
    long long nn = (sys->fmt == SKR_FMT_DARCY2D || sys->fmt == SKR_FMT_DARCY3D) ? sys_coef_len(*sys) : 0;
    if (nn > 0) {
        CUDA_TRY(anode.alloc(nn * 8));
        node_exp_kernel<<<grid_for(nn, 256), 256, 0, st>>>(sg.dev.coef, nn, anode.as<double>());
        CUDA_TRY(cudaGetLastError());
    }
    CUDA_TRY(A.alloc((size_t)g.nst * g.n * 8));
    CUDA_TRY(dinv.alloc((size_t)g.n * 8));
    rows_kernel<<<grid_for(g.n, 256), 256, 0, st>>>(sg.dev, g, anode.as<double>(), A.as<double>(), g.n, nullptr,
                                                     dinv.as<double>(), colour_sweep_pc(precond) ? SKR_PC_NONE : precond,
                                                     cols.as<int>());
    CUDA_TRY(cudaGetLastError());
    const double *vin = v;
    double *yout = y;
    if (mem == SKR_MEM_HOST) {
        CUDA_TRY(dv.alloc((size_t)g.n * 8));
        CUDA_TRY(dy.alloc((size_t)g.n * 8));
        CUDA_TRY(cudaMemcpyAsync(dv.p, v, (size_t)g.n * 8, cudaMemcpyHostToDevice, st));
        vin = dv.as<double>();
        yout = dy.as<double>();
    }
    const int gb = grid_for(g.n, 256);
    if (colour_sweep_pc(precond)) {
        DBuf inv, invw, zb;
        const long long bs = sweep_block_rows(precond, g.n, pc_blocks);
        CUDA_TRY(inv.alloc((size_t)g.n * 8));
        ilu_pivot_kernel<<<gb, 256, 0, st>>>(g, A.as<double>(), g.n, inv.as<double>(), precond, bs);
        const size_t es = (precision == SKR_PREC_MIXED) ? 4 : 8;
        CUDA_TRY(Aw.alloc((size_t)g.nst * g.n * es));
        CUDA_TRY(invw.alloc((size_t)g.n * es));
        CUDA_TRY(vw.alloc((size_t)g.n * es));
        CUDA_TRY(zb.alloc((size_t)g.n * es));
        if (precision == SKR_PREC_MIXED) {
            ilu_fold_kernel<float><<<gb, 256, 0, st>>>(g, A.as<double>(), g.n, inv.as<double>(), Aw.as<float>(), invw.as<float>());
            to_working_kernel<float><<<gb, 256, 0, st>>>(vin, g.n, vw.as<float>());
            for (int stage = 1; stage <= 3; stage++)
                ilu_sweep_kernel<float><<<gb, 256, 0, st>>>(g, Aw.as<float>(), g.n, invw.as<float>(), vw.as<float>(),
                                                            zb.as<float>(), yout, stage, bs);
        } else {
            ilu_fold_kernel<double><<<gb, 256, 0, st>>>(g, A.as<double>(), g.n, inv.as<double>(), Aw.as<double>(), invw.as<double>());
            to_working_kernel<double><<<gb, 256, 0, st>>>(vin, g.n, vw.as<double>());
            for (int stage = 1; stage <= 3; stage++)
                ilu_sweep_kernel<double><<<gb, 256, 0, st>>>(g, Aw.as<double>(), g.n, invw.as<double>(), vw.as<double>(),
                                                             zb.as<double>(), yout, stage, bs);
        }
        CUDA_TRY(cudaGetLastError());
    } else if (precision == SKR_PREC_MIXED && sym_compact_form(sys->fmt, precond, 4, g)) {
        // the chain kernel's compact symmetric operator
        CUDA_TRY(Aw.alloc((size_t)sym_compact_slots(g) * g.n * 4));
        CUDA_TRY(vw.alloc((size_t)g.n * 4));
        sym_fold_kernel<<<gb, 256, 0, st>>>(g, A.as<double>(), g.n, dinv.as<double>(), Aw.as<float>());
        to_working_kernel<float><<<gb, 256, 0, st>>>(vin, g.n, vw.as<float>());
        sym_apply_kernel<<<gb, 256, 0, st>>>(g, Aw.as<float>(), g.n, vw.as<float>(), yout);
    } else if (precision == SKR_PREC_MIXED) {
        CUDA_TRY(Aw.alloc((size_t)g.nst * g.n * 4));
        CUDA_TRY(vw.alloc((size_t)g.n * 4));
        fold_kernel<float><<<gb, 256, 0, st>>>(g, A.as<double>(), g.n, dinv.as<double>(), Aw.as<float>());
        to_working_kernel<float><<<gb, 256, 0, st>>>(vin, g.n, vw.as<float>());
        apply_kernel<float><<<gb, 256, 0, st>>>(g, Aw.as<float>(), g.n, vw.as<float>(), yout);
    } else {
        CUDA_TRY(Aw.alloc((size_t)g.nst * g.n * 8));
        fold_kernel<double><<<gb, 256, 0, st>>>(g, A.as<double>(), g.n, dinv.as<double>(), Aw.as<double>());
        apply_kernel<double><<<gb, 256, 0, st>>>(g, Aw.as<double>(), g.n, vin, yout);
    }
    CUDA_TRY(cudaGetLastError());
    if (mem == SKR_MEM_HOST) CUDA_TRY(cudaMemcpyAsync(y, yout, (size_t)g.n * 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return SKR_OK;
}

skr_status skr_solve_sequence(const skr_system *systems, int64_t N, const int32_t *order,
                              const int64_t *chain_offsets, int32_t nchains, const skr_options *opt_in,
                              double *const *x_out, skr_result *results) {
    g_err.clear();
    g_last = LastStats();
    skr_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        skr_options_default(&opt);
    if (N < 0) return fail(SKR_ERR_INVALID_ARG, "N < 0");
    if (N == 0) return SKR_OK;
    if (!systems || !x_out || !results) return fail(SKR_ERR_INVALID_ARG, "NULL pointer");
    if (nchains < 1 || nchains > N) return fail(SKR_ERR_INVALID_ARG, "nchains must be in [1, N]");
    if (opt.m < 2 || opt.m > SKR_MAX_M) return fail(SKR_ERR_INVALID_ARG, "m must be in [2, %d]", SKR_MAX_M);
    if (opt.k < 0 || opt.k > SKR_MAX_K || (opt.k > 0 && opt.k > opt.m - 2))
        return fail(SKR_ERR_INVALID_ARG, "k must be in [0, min(%d, m-2)]", SKR_MAX_K);
    if (opt.maxit < 1) return fail(SKR_ERR_INVALID_ARG, "maxit < 1");
    if (opt.max_refine < 1) return fail(SKR_ERR_INVALID_ARG, "max_refine < 1");
    if (!(opt.tol > 0.0) || !(opt.tol < 1.0)) return fail(SKR_ERR_INVALID_ARG, "tol must be in (0, 1)");
    if (opt.precision == SKR_PREC_MIXED && !(opt.inner_tol > 0.0 && opt.inner_tol < 1.0))
        return fail(SKR_ERR_INVALID_ARG, "inner_tol must be in (0, 1)");
    if (opt.precond != SKR_PC_NONE && opt.precond != SKR_PC_JACOBI && opt.precond != SKR_PC_ILU0 &&
        opt.precond != SKR_PC_SSOR && opt.precond != SKR_PC_BJACOBI)
        return fail(SKR_ERR_INVALID_ARG, "unknown preconditioner %d", opt.precond);
    if (opt.precond == SKR_PC_BJACOBI && opt.pc_blocks < 1) return fail(SKR_ERR_INVALID_ARG, "pc_blocks < 1");
    if (opt.precision != SKR_PREC_FP64 && opt.precision != SKR_PREC_MIXED)
        return fail(SKR_ERR_INVALID_ARG, "bad precision");
    if (opt.mem != SKR_MEM_DEVICE && opt.mem != SKR_MEM_HOST) return fail(SKR_ERR_INVALID_ARG, "bad mem");
    if (opt.cluster_size < 0 || opt.cluster_size > 16) return fail(SKR_ERR_INVALID_ARG, "cluster_size in [0, 16]");
    if (opt.warm_start != 0 && opt.warm_start != 1) return fail(SKR_ERR_INVALID_ARG, "warm_start must be 0 or 1");
    if (opt.diagnostics != 0 && opt.diagnostics != 1) return fail(SKR_ERR_INVALID_ARG, "diagnostics must be 0 or 1");
    if (opt.eig_fp32 != 0 && opt.eig_fp32 != 1) return fail(SKR_ERR_INVALID_ARG, "eig_fp32 must be 0 or 1");
    if (opt.recycle_out) {
        if (opt.mem != SKR_MEM_DEVICE) return fail(SKR_ERR_INVALID_ARG, "recycle_out needs mem = SKR_MEM_DEVICE");
        for (int c = 0; c < nchains; c++)
            if (!opt.recycle_out[c]) return fail(SKR_ERR_INVALID_ARG, "recycle_out[%d] is NULL", c);
    }
    cudaStream_t st = (cudaStream_t)opt.stream;

    // order and chains
    std::vector<int> ord(N);
    if (order) {
        std::vector<char> seen(N, 0);
        for (long long i = 0; i < N; i++) {
            if (order[i] < 0 || order[i] >= N || seen[order[i]])
                return fail(SKR_ERR_INVALID_ARG, "order is not a permutation of 0..N-1");
            seen[order[i]] = 1;
            ord[i] = order[i];
        }
    } else {
        for (long long i = 0; i < N; i++) ord[i] = (int)i;
    }
    std::vector<long long> off(nchains + 1);
    if (chain_offsets) {
        for (int c = 0; c <= nchains; c++) off[c] = chain_offsets[c];
        if (off[0] != 0 || off[nchains] != N) return fail(SKR_ERR_INVALID_ARG, "chain_offsets must span 0..N");
        for (int c = 0; c < nchains; c++)
            if (off[c + 1] <= off[c]) return fail(SKR_ERR_INVALID_ARG, "empty or decreasing chain");
    } else {
        for (int c = 0; c <= nchains; c++) off[c] = (long long)c * N / nchains;
    }
    long long nmax = 0, nodemax = 0;
    for (long long i = 0; i < N; i++) {
        skr_status s0 = check_system(systems[i], i);
        if (s0 != SKR_OK) return s0;
        if (!x_out[i]) return fail(SKR_ERR_INVALID_ARG, "x_out[%lld] is NULL", i);
        nmax = std::max(nmax, sys_n(systems[i]));
        if (systems[i].fmt == SKR_FMT_DARCY2D || systems[i].fmt == SKR_FMT_DARCY3D)
            nodemax = std::max(nodemax, sys_coef_len(systems[i]));
    }
    for (int c = 0; c < nchains; c++)
        for (long long q = off[c] + 1; q < off[c + 1]; q++)
            if (!same_shape(systems[ord[q]], systems[ord[off[c]]]))
                return fail(SKR_ERR_INVALID_ARG, "chain %d mixes grids or formats", c);
    if (colour_sweep_pc(opt.precond))
        for (long long i = 0; i < N; i++)
            if (systems[i].fmt == SKR_FMT_CSR)
                return fail(SKR_ERR_INVALID_ARG, "CSR input takes SKR_PC_NONE or SKR_PC_JACOBI only");

    // launch geometry: one launch per cluster size (skr_plan.h)
    const bool fp64 = opt.precision == SKR_PREC_FP64;
    const int threads = chain_threads();
    const size_t smem = chain_smem_bytes(opt.m, opt.k, threads, fp64 ? 8 : 4);
    if (smem > 227 * 1024) return fail(SKR_ERR_INVALID_ARG, "m, k too large for shared memory (%zu bytes)", smem);
    auto maxc = [&](int cs) {
        return fp64 ? max_active_clusters_f64(cs, threads, smem) : max_active_clusters_f32(cs, threads, smem);
    };
    std::vector<LaunchClass> plan;
    if (opt.cluster_size > 0) {
        LaunchClass k;
        k.cs = opt.cluster_size;
        for (int c = 0; c < nchains; c++) k.chains.push_back(c);
        const int mc = maxc(k.cs);
        if (mc < 1)
            return fail(SKR_ERR_CUDA, "cluster of %d CTAs with %zu bytes of shared memory cannot be scheduled", k.cs,
                        smem);
        k.slots = std::min(nchains, mc);
        if (opt.max_slots > 0) k.slots = std::min(k.slots, opt.max_slots);
        plan.push_back(k);
    } else {
        std::vector<long long> cn(nchains), cl(nchains);
        std::vector<char> c3(nchains);
        for (int c = 0; c < nchains; c++) {
            cn[c] = sys_n(systems[ord[off[c]]]);
            cl[c] = off[c + 1] - off[c];
            c3[c] = is_3d(systems[ord[off[c]]].fmt) ? 1 : 0;
        }
        plan = plan_launches(cn, cl, maxc(1), maxc, opt.max_slots, &c3);
        if (plan.empty()) return fail(SKR_ERR_CUDA, "no launch shape of the chain kernel can be scheduled");
    }
    const int nlaunch = (int)plan.size();
    const size_t esz = fp64 ? 8 : 4;
    // per launch: its chains' order positions, offsets and workspace
    struct LaunchGeo {
        long long ld = 0, nodecap = 1, ord0 = 0, off0 = 0;
        SlabLayout L;
        size_t ws0 = 0;
    };
    std::vector<LaunchGeo> geo(nlaunch);
    std::vector<int> ordk;
    std::vector<long long> offk;
    size_t wtotal = 0;
    for (int li = 0; li < nlaunch; li++) {
        LaunchGeo &g = geo[li];
        long long nm = 1, nodem = 0;
        bool csr = false;
        g.ord0 = (long long)ordk.size();
        g.off0 = (long long)offk.size();
        offk.push_back(0);
        for (int c : plan[li].chains) {
            for (long long q = off[c]; q < off[c + 1]; q++) {
                const skr_system &sy = systems[ord[q]];
                nm = std::max(nm, sys_n(sy));
                if (sy.fmt == SKR_FMT_DARCY2D || sy.fmt == SKR_FMT_DARCY3D) nodem = std::max(nodem, sys_coef_len(sy));
                csr = csr || sy.fmt == SKR_FMT_CSR;
                ordk.push_back(ord[q]);
            }
            offk.push_back((long long)ordk.size() - g.ord0);
        }
        g.ld = chain_ld(nm, plan[li].cs);
        g.nodecap = std::max<long long>(nodem, 1);
        g.L = slab_layout(plan[li].slots, g.ld, g.nodecap, esz, csr);
        g.ws0 = wtotal;
        wtotal += (g.L.total + 255) / 256 * 256;
    }
    void *wbase = nullptr;
    CUDA_TRY(ws_get(wtotal, &wbase));
    char *wb = reinterpret_cast<char *>(wbase);
    // the basis must start zeroed: padded rows are never written by the passes that read them
    for (int li = 0; li < nlaunch; li++)
        CUDA_TRY(cudaMemsetAsync(wb + geo[li].ws0 + geo[li].L.o_basis, 0,
                                 (size_t)plan[li].slots * NCOLS * geo[li].ld * esz, st));

    // per-call device arrays
    std::vector<Staged> staged(N);
    std::vector<DevSystem> hsys(N);
    for (long long i = 0; i < N; i++) {
        skr_status s0 = stage_system(systems[i], opt.mem, st, staged[i]);
        if (s0 != SKR_OK) return s0;
        hsys[i] = staged[i].dev;
    }
    std::vector<DBuf> xstage;
    if (opt.mem == SKR_MEM_HOST) {
        xstage.resize(N);
        for (long long i = 0; i < N; i++) {
            CUDA_TRY(xstage[i].alloc((size_t)sys_n(systems[i]) * 8));
            hsys[i].x_out = xstage[i].as<double>();
        }
    } else {
        for (long long i = 0; i < N; i++) hsys[i].x_out = x_out[i];
    }
    {
        std::vector<long long> ns(N);
        for (long long i = 0; i < N; i++) ns[i] = sys_n(systems[i]);
        skr_status s0 = check_csr(hsys, ns, st);
        if (s0 != SKR_OK) return s0;
    }
    // counters: one chain counter per launch (64 bytes apart), then the
    // algorithmic-bytes accumulator, then the per-phase accumulators
    const size_t ctr_bytes = 64 * (size_t)nlaunch + 64 + 8 * SKR_NPHASE;
    DBuf dsys, dord, doff, dres, dctr;
    CUDA_TRY(dsys.alloc(sizeof(DevSystem) * N));
    CUDA_TRY(dord.alloc(sizeof(int) * N));
    CUDA_TRY(doff.alloc(sizeof(long long) * offk.size()));
    CUDA_TRY(dres.alloc(sizeof(DevResult) * N));
    CUDA_TRY(dctr.alloc(ctr_bytes));
    CUDA_TRY(cudaMemcpyAsync(dsys.p, hsys.data(), sizeof(DevSystem) * N, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(dord.p, ordk.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(doff.p, offk.data(), sizeof(long long) * offk.size(), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(dctr.p, 0, ctr_bytes, st));
    CUDA_TRY(cudaMemsetAsync(dres.p, 0, sizeof(DevResult) * N, st));

    ChainArgs a;
    a.systems = dsys.as<DevSystem>();
    a.results = dres.as<DevResult>();
    a.m = opt.m;
    a.k = opt.k;
    a.maxit = opt.maxit;
    a.max_refine = opt.max_refine;
    a.precond = opt.precond;
    a.pc_blocks = opt.pc_blocks;
    a.eig32 = opt.eig_fp32;
    a.tol = opt.tol;
    a.inner_tol = opt.inner_tol;
    a.bytes = reinterpret_cast<unsigned long long *>(dctr.as<char>() + 64 * nlaunch);
    a.prof = opt.profile ? reinterpret_cast<unsigned long long *>(dctr.as<char>() + 64 * nlaunch + 64) : nullptr;
    a.chain_kc = nullptr;
    a.warm_start = opt.warm_start;
    a.diagnostics = opt.diagnostics;
    a.chain_xok = nullptr;   // every chain of the call starts from x_0 = 0
    // recycle export: per launch, the caller's pointers in the launch's chain order
    DBuf drec;
    if (opt.recycle_out) {
        std::vector<double *> rec;
        for (int li = 0; li < nlaunch; li++)
            for (int c : plan[li].chains) rec.push_back(opt.recycle_out[c]);
        CUDA_TRY(drec.alloc(sizeof(double *) * rec.size()));
        CUDA_TRY(cudaMemcpyAsync(drec.p, rec.data(), sizeof(double *) * rec.size(), cudaMemcpyHostToDevice, st));
    }
    std::vector<ChainArgs> args(nlaunch, a);
    int rec0 = 0;
    for (int li = 0; li < nlaunch; li++) {
        ChainArgs &ak = args[li];
        ak.order = dord.as<int>() + geo[li].ord0;
        ak.chain_off = doff.as<long long>() + geo[li].off0;
        ak.nchains = (int)plan[li].chains.size();
        ak.chain_counter = reinterpret_cast<int *>(dctr.as<char>() + 64 * li);
        ak.recycle_out = opt.recycle_out ? drec.as<double *>() + rec0 : nullptr;
        rec0 += (int)plan[li].chains.size();
        ak.ws = slab_bind(wb + geo[li].ws0, geo[li].L, plan[li].slots, geo[li].ld, geo[li].nodecap);
        if (encode_basis_maps(ak.ws.basis, geo[li].ld, plan[li].slots, (int)esz, ak.tmap) != cudaSuccess)
            return fail(SKR_ERR_CUDA, "TMA descriptors of the basis could not be encoded");
    }
    std::vector<cudaStream_t> lst(nlaunch, st);
    if (nlaunch > 1) CUDA_TRY(launch_streams(nlaunch, lst.data()));

    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    std::vector<cudaEvent_t> joins(nlaunch, nullptr);
    auto drop_events = [&]() {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (cudaEvent_t ev : joins)
            if (ev) cudaEventDestroy(ev);
    };
    CUDA_TRY(cudaEventRecord(e0, st));
    cudaError_t le = cudaSuccess;
    for (int li = 0; li < nlaunch && le == cudaSuccess; li++) {
        if (lst[li] != st) {
            le = cudaStreamWaitEvent(lst[li], e0, 0);
            if (le != cudaSuccess) break;
        }
        le = fp64 ? launch_chain_f64(args[li], plan[li].slots, plan[li].cs, threads, smem, lst[li])
                  : launch_chain_f32(args[li], plan[li].slots, plan[li].cs, threads, smem, lst[li]);
        if (le == cudaSuccess && lst[li] != st) {
            le = cudaEventCreateWithFlags(&joins[li], cudaEventDisableTiming);
            if (le == cudaSuccess) le = cudaEventRecord(joins[li], lst[li]);
            if (le == cudaSuccess) le = cudaStreamWaitEvent(st, joins[li], 0);
        }
    }
    if (le != cudaSuccess) {
        cudaStreamSynchronize(st);
        for (cudaStream_t s2 : lst) cudaStreamSynchronize(s2);
        drop_events();
        return fail(SKR_ERR_CUDA, "chain kernel launch failed: %s", cudaGetErrorString(le));
    }
    CUDA_TRY(cudaEventRecord(e1, st));
    std::vector<DevResult> hres(N);
    unsigned long long hbytes = 0;
    CUDA_TRY(cudaMemcpyAsync(hres.data(), dres.p, sizeof(DevResult) * N, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&hbytes, a.bytes, sizeof(hbytes), cudaMemcpyDeviceToHost, st));
    unsigned long long hprof[SKR_NPHASE] = {0};
    if (a.prof) CUDA_TRY(cudaMemcpyAsync(hprof, a.prof, sizeof(hprof), cudaMemcpyDeviceToHost, st));
    if (opt.mem == SKR_MEM_HOST) {
        for (long long i = 0; i < N; i++)
            CUDA_TRY(cudaMemcpyAsync(x_out[i], xstage[i].p, (size_t)sys_n(systems[i]) * 8,
                                     cudaMemcpyDeviceToHost, st));
    }
    cudaError_t se = cudaStreamSynchronize(st);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    drop_events();
    if (se != cudaSuccess) return fail(SKR_ERR_CUDA, "solve failed: %s", cudaGetErrorString(se));
    for (long long i = 0; i < N; i++) {
        skr_result &r = results[i];
        const DevResult &d = hres[i];
        r.steps = d.steps;
        r.cycles = d.cycles;
        r.matvecs = d.matvecs;
        r.refinements = d.refinements;
        r.flag = d.flag;
        r.k_final = d.k_final;
        r.relres = d.relres;
        r.seconds = (d.t_end >= d.t_begin) ? (double)(d.t_end - d.t_begin) * 1e-9 : 0.0;
        r.delta = d.delta;
    }
    g_last.bytes = hbytes;
    for (int i = 0; i < SKR_NPHASE; i++) g_last.prof[i] = hprof[i];
    g_last.kernel_ms = ms;
    g_last.cluster_size = nlaunch == 1 ? plan[0].cs : 0;
    g_last.slots = 0;
    g_last.launches = nlaunch;
    g_last.plan.clear();
    for (const LaunchClass &k : plan) {
        g_last.slots += k.slots;
        g_last.plan.push_back({k.cs, k.slots, (int)k.chains.size()});
    }
    return SKR_OK;
}

skr_status skr_last_stats(uint64_t *bytes, double *kernel_ms, int32_t *cluster_size, int32_t *slots,
                          int32_t *launches) {
    if (bytes) *bytes = g_last.bytes;
    if (kernel_ms) *kernel_ms = g_last.kernel_ms;
    if (cluster_size) *cluster_size = g_last.cluster_size;
    if (slots) *slots = g_last.slots;
    if (launches) *launches = g_last.launches;
    return SKR_OK;
}

skr_status skr_last_plan(int32_t *cluster_size, int32_t *clusters, int32_t *chains, int32_t cap,
                         int32_t *nlaunch) {
    if (cap < 0) return fail(SKR_ERR_INVALID_ARG, "cap < 0");
    const int n = (int)g_last.plan.size();
    for (int i = 0; i < n && i < cap; i++) {
        if (cluster_size) cluster_size[i] = g_last.plan[i].cs;
        if (clusters) clusters[i] = g_last.plan[i].slots;
        if (chains) chains[i] = g_last.plan[i].chains;
    }
    if (nlaunch) *nlaunch = n;
    return SKR_OK;
}

skr_status skr_last_profile(double *ns_out, int32_t nphase) {
    if (!ns_out || nphase < 0) return fail(SKR_ERR_INVALID_ARG, "bad arguments");
    for (int i = 0; i < nphase && i < SKR_NPHASE; i++) ns_out[i] = (double)g_last.prof[i];
    return SKR_OK;
}

skr_status skr_release_workspace(void) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &w : g_ws) {
        if (w.base) {
            cudaSetDevice(w.device);
            cudaFree(w.base);
        }
    }
    g_ws.clear();
    cudaSetDevice(cur);
    return SKR_OK;
}

}  // extern "C"
// ---------------------------------------------------------------- sort without allocation
//
// skr_sort_noalloc keeps its scratch (the N x N distance matrix, the
// per-system "placed" flags and an error word) in one fixed array in
// device memory that every GPU loading this library holds until the process
// exits, so the call itself never allocates.  Host code must not pass the
// array's name to a kernel: in host code that name denotes a host-side
// stand-in, not the device address.  The device address is looked up once
// per device with cudaGetSymbolAddress and cached.
namespace {
constexpr long long NOALLOC_MAX_N = SKR_SORT_NOALLOC_MAX_N;
constexpr size_t NOALLOC_DIST_BYTES = (size_t)NOALLOC_MAX_N * NOALLOC_MAX_N * sizeof(double);
constexpr size_t NOALLOC_FLAGS_OFF = NOALLOC_DIST_BYTES;                  // N bytes
constexpr size_t NOALLOC_ERR_OFF = NOALLOC_DIST_BYTES + NOALLOC_MAX_N;    // one int
constexpr size_t NOALLOC_BYTES = NOALLOC_ERR_OFF + 256;
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_sort_scratch[NOALLOC_BYTES];

namespace {
// Device address of g_sort_scratch on the current device (set-up on first use).
skr_status noalloc_scratch(unsigned char **out) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(SKR_ERR_INVALID_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess || p == nullptr)
            return fail(SKR_ERR_CUDA, "cudaGetSymbolAddress of the sort scratch failed: %s", cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = reinterpret_cast<unsigned char *>(g_noalloc_addr[dev]);
    return SKR_OK;
}

// Device memory of device `dev`, or managed memory (which any device reaches).
bool is_device_pointer(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged;
}
}  // namespace

extern "C" skr_status skr_sort_noalloc(const double *params, int64_t N, int64_t p, int64_t start,
                                       void *stream, int32_t *perm_out) {
    g_err.clear();
    if (N < 0) return fail(SKR_ERR_INVALID_ARG, "N < 0");
    if (N == 0) return SKR_OK;
    if (N > NOALLOC_MAX_N)
        return fail(SKR_ERR_INVALID_ARG, "N = %lld exceeds SKR_SORT_NOALLOC_MAX_N = %lld", (long long)N,
                    NOALLOC_MAX_N);
    if (!params || !perm_out) return fail(SKR_ERR_INVALID_ARG, "NULL pointer");
    if (p < 1) return fail(SKR_ERR_INVALID_ARG, "p < 1");
    if (start < 0 || start >= N) return fail(SKR_ERR_INVALID_ARG, "start out of range");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (!is_device_pointer(params, dev) || !is_device_pointer(perm_out, dev))
        return fail(SKR_ERR_INVALID_ARG, "params and perm_out must be device memory of the current device (%d)", dev);
    unsigned char *base = nullptr;
    skr_status s0 = noalloc_scratch(&base);
    if (s0 != SKR_OK) return s0;
    double *dist = reinterpret_cast<double *>(base);
    unsigned char *taken = base + NOALLOC_FLAGS_OFF;
    int *err = reinterpret_cast<int *>(base + NOALLOC_ERR_OFF);
    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's contents: reset the error word
    // (the chain kernel clears the placed flags itself)
    CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    CUDA_TRY(launch_sort_dist(params, N, p, dist, err, st));
    int herr = 0;
    CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (herr) return fail(SKR_ERR_INVALID_ARG, "non-finite parameter distance");
    sort_chain_kernel<<<1, 1024, 0, st>>>(dist, N, start, perm_out, taken);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(st));
    return SKR_OK;
}
