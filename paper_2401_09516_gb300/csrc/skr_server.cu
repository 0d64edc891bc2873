// Serving loop over the chain kernel (include/skr.h, skr_server_*).
//
// One host thread per server owns every CUDA call: it collects finished
// requests (event queries), admits queued ones (nearest idle chain of the
// same shape, or a new chain if the device-memory budget and the chain limit
// allow, else a new chain in place of the least recently used idle chains
// when the request's shape has no chain at all), and launches each admitted
// request as a one-cluster chain-kernel launch on the chain's own stream,
// as long as the running requests leave enough CTAs free on the GPU.
// Requests of different chains therefore run concurrently on the GPU; a
// request that arrives while others run starts as soon as a chain of its
// shape (or room for one) is free.  skr_submit and skr_poll only touch host
// data under the server's mutex.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "skr_common.h"
#include "skr_launch.h"
#include "skr_plan.h"
#include "skr_tma.h"
#include "skr_workspace.h"

namespace skr {
skr_status set_last_error(skr_status code, const char *msg);
}

using namespace skr;

namespace {

using Clock = std::chrono::steady_clock;

skr_status err(skr_status code, const std::string &msg) { return set_last_error(code, msg.c_str()); }

bool fmt3d(int fmt) { return fmt == SKR_FMT_DARCY3D || fmt == SKR_FMT_STENCIL7; }

long long n_of(int fmt, int nx, int ny, int nz) { return (long long)nx * ny * (fmt3d(fmt) ? nz : 1); }

long long coef_len(int fmt, int nx, int ny, int nz) {
    const long long n = n_of(fmt, nx, ny, nz);
    switch (fmt) {
        case SKR_FMT_DARCY2D: return (long long)(nx + 2) * (ny + 2);
        case SKR_FMT_DARCY3D: return (long long)(nx + 2) * (ny + 2) * (nz + 2);
        case SKR_FMT_STENCIL5: return 5 * n;
        case SKR_FMT_STENCIL7: return 7 * n;
        case SKR_FMT_HELMHOLTZ2D: return n;
        case SKR_FMT_POISSON2D: return n + 2LL * (nx + ny);
        default: return 0;
    }
}

struct Request {
    uint64_t ticket = 0;
    int fmt = 0, nx = 0, ny = 0, nz = 1;
    long long n = 0;
    double params[4] = {0, 0, 0, 0};
    std::vector<double> coef, rhs, key;
    int state = 0;   // 0 queued, 1 running, 2 done
    std::vector<double> x;
    skr_result res{};
    Clock::time_point t_submit, t_done;
};

struct Chain {
    int fmt = 0, nx = 0, ny = 0, nz = 1;
    long long n = 0, clen = 0;
    size_t p = 0;
    std::vector<double> key;
    int cs = 1;
    long long ld = 0, nodecap = 1;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    char *slab = nullptr;
    size_t bytes = 0;
    Workspace ws{};
    double *dcoef = nullptr, *drhs = nullptr, *dx = nullptr;
    DevSystem *dsys = nullptr;
    DevResult *dres = nullptr;
    int *dorder = nullptr, *dctr = nullptr, *dkc = nullptr;
    long long *doff = nullptr;
    unsigned long long *dbytes = nullptr;
    bool busy = false;
    uint64_t ticket = 0;
    uint64_t last_used = 0;   // launch counter at this chain's last launch (LRU eviction)
};

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

struct skr_server {
    skr_options opt{};
    size_t budget = 0, used = 0, smem = 0;
    int max_chains = 64, device = 0, threads = 0;
    int cap_ctas = 0;          // CTAs of the chain kernel that fit on the GPU at once
    int maxc[SKR_TUNE_COLS] = {};   // clusters of each table size that fit at once
    uint64_t launches = 0;     // launch counter (chain recency)
    int64_t evicted = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request *> reqs;
    std::vector<Chain *> chains;
    std::vector<double> lat_ms;
    uint64_t next = 1;
    int64_t submitted = 0, completed = 0;
    bool stop = false;
    std::thread th;
};

namespace {

// Cluster size of one request of n unknowns: the caller's if set; else,
// from the measured launch table (skr_plan.h), the fastest size whose CTA
// time per Arnoldi step is within 1.6x of the cheapest size's and that is
// at most `share` CTAs.  The share is the request's part of the GPU's CTAs
// in proportion to its estimated work (n times the grid side, the planner's
// weight)
// among the running and waiting requests, and never more than the CTAs
// free now: one fast cluster per request under light load, and under load
// clusters sized so that the largest requests do not straggle on one SM.
int request_cs(const skr_server *S, long long n, int share);


struct ChainPlan {
    SlabLayout L;
    long long ld = 0, nodecap = 1, clen = 1;
    int cs = 1;
    size_t o_coef = 0, o_rhs = 0, o_x = 0, o_sys = 0, o_res = 0, o_ord = 0, o_off = 0, o_ctr = 0, o_kc = 0;
    size_t bytes = 0, pin = 0;
};

// Device layout of a chain shaped like request r.
ChainPlan chain_plan(const skr_server *S, const Request &r) {
    ChainPlan P;
    const size_t esz = S->opt.precision == SKR_PREC_FP64 ? 8 : 4;
    // a chain may run each request on another cluster size: its column
    // stride holds the row split of every size
    P.cs = 1;
    P.ld = 0;
    for (int j = 0; j < SKR_TUNE_COLS; j++) P.ld = std::max(P.ld, chain_ld(r.n, SKR_TUNE_CS[j]));
    if (S->opt.cluster_size > 0) P.ld = std::max(P.ld, chain_ld(r.n, S->opt.cluster_size));
    P.nodecap = std::max<long long>(1, (r.fmt == SKR_FMT_DARCY2D || r.fmt == SKR_FMT_DARCY3D)
                                           ? coef_len(r.fmt, r.nx, r.ny, r.nz)
                                           : 1);
    P.clen = std::max<long long>(1, coef_len(r.fmt, r.nx, r.ny, r.nz));
    P.L = slab_layout(1, P.ld, P.nodecap, esz);
    size_t o = P.L.total;
    P.o_coef = o;  o += al256(P.clen * 8);
    P.o_rhs = o;   o += al256(r.n * 8);
    P.o_x = o;     o += al256(r.n * 8);
    P.o_sys = o;   o += 256;
    P.o_res = o;   o += 256;
    P.o_ord = o;   o += 256;
    P.o_off = o;   o += 256;
    P.o_ctr = o;   o += 256;
    P.o_kc = o;    o += 256;
    P.bytes = o;
    return P;
}

size_t chain_bytes(const skr_server *S, const Request &r) { return chain_plan(S, r).bytes; }

void destroy_chain(Chain *c) {
    if (c->st) cudaStreamSynchronize(c->st);
    if (c->slab) cudaFree(c->slab);
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->st) cudaStreamDestroy(c->st);
    delete c;
}

// Shape an idle chain (its device slab already large enough) like request r: bind the layout, forget any recycle space and
// previous solution, and set the constant descriptors of a one-system chain.
// Returns false on a CUDA error.
bool shape_chain(skr_server *S, Chain *c, const Request &r, const ChainPlan &P) {
    const size_t esz = S->opt.precision == SKR_PREC_FP64 ? 8 : 4;
    c->fmt = r.fmt;
    c->nx = r.nx;
    c->ny = r.ny;
    c->nz = r.nz;
    c->n = r.n;
    c->p = r.key.size();
    c->key.clear();
    c->clen = P.clen;
    c->cs = P.cs;
    c->ld = P.ld;
    c->nodecap = P.nodecap;
    c->ws = slab_bind(c->slab, P.L, 1, c->ld, c->nodecap);
    c->dcoef = reinterpret_cast<double *>(c->slab + P.o_coef);
    c->drhs = reinterpret_cast<double *>(c->slab + P.o_rhs);
    c->dx = reinterpret_cast<double *>(c->slab + P.o_x);
    c->dsys = reinterpret_cast<DevSystem *>(c->slab + P.o_sys);
    c->dres = reinterpret_cast<DevResult *>(c->slab + P.o_res);
    c->dorder = reinterpret_cast<int *>(c->slab + P.o_ord);
    c->doff = reinterpret_cast<long long *>(c->slab + P.o_off);
    c->dctr = reinterpret_cast<int *>(c->slab + P.o_ctr);
    c->dbytes = reinterpret_cast<unsigned long long *>(c->slab + P.o_ctr + 64);
    c->dkc = reinterpret_cast<int *>(c->slab + P.o_kc);
    // one chain of one system, starting with no recycle space
    cudaMemsetAsync(c->ws.basis, 0, (size_t)NCOLS * c->ld * esz, c->st);
    cudaMemsetAsync(c->slab + P.o_ord, 0, P.bytes - P.o_ord, c->st);
    const long long off[2] = {0, 1};
    cudaMemcpyAsync(c->doff, off, sizeof(off), cudaMemcpyHostToDevice, c->st);
    cudaStreamSynchronize(c->st);
    return cudaGetLastError() == cudaSuccess;
}

// New chain shaped like request r (called with the server lock held).
Chain *create_chain(skr_server *S, const Request &r) {
    const ChainPlan P = chain_plan(S, r);
    Chain *c = new Chain();
    c->bytes = P.bytes;
    if (cudaMalloc(&c->slab, c->bytes) != cudaSuccess) {
        cudaGetLastError();
        c->slab = nullptr;
        destroy_chain(c);
        return nullptr;
    }
    if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        destroy_chain(c);
        return nullptr;
    }
    if (!shape_chain(S, c, r, P)) {
        destroy_chain(c);
        return nullptr;
    }
    return c;
}

// Launch request r on chain c (without the server lock: this touches only
// the chain's own device memory and stream).  Returns false on a CUDA error.
bool launch(skr_server *S, Chain *c, Request *r, int cs) {
    cudaStream_t st = c->st;
    // copies from the request's own (pageable) host memory: the call returns
    // once the data is staged, and the request outlives it
    if (!r->coef.empty()) cudaMemcpyAsync(c->dcoef, r->coef.data(), r->coef.size() * 8, cudaMemcpyHostToDevice, st);
    if (!r->rhs.empty()) {
        cudaMemcpyAsync(c->drhs, r->rhs.data(), r->n * 8, cudaMemcpyHostToDevice, st);
    }
    DevSystem ds;
    ds.fmt = r->fmt;
    ds.nx = r->nx;
    ds.ny = r->ny;
    ds.nz = r->nz;
    ds.coef = r->coef.empty() ? nullptr : c->dcoef;
    ds.rhs = r->rhs.empty() ? nullptr : c->drhs;
    for (int i = 0; i < 4; i++) ds.params[i] = r->params[i];
    ds.x_out = c->dx;
    cudaMemcpyAsync(c->dsys, &ds, sizeof(DevSystem), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(c->dctr, 0, 128, st);
    ChainArgs a;
    a.systems = c->dsys;
    a.order = c->dorder;
    a.chain_off = c->doff;
    a.nchains = 1;
    a.chain_counter = c->dctr;
    a.ws = c->ws;
    a.results = c->dres;
    a.m = S->opt.m;
    a.k = S->opt.k;
    a.maxit = S->opt.maxit;
    a.max_refine = S->opt.max_refine;
    a.precond = S->opt.precond;
    a.pc_blocks = S->opt.pc_blocks;
    a.eig32 = S->opt.eig_fp32;
    a.tol = S->opt.tol;
    a.inner_tol = S->opt.inner_tol;
    a.bytes = c->dbytes;
    a.prof = nullptr;
    a.chain_kc = c->dkc;
    a.warm_start = S->opt.warm_start;
    a.diagnostics = S->opt.diagnostics;
    a.chain_xok = c->dkc + 16;   // the chain's x holds its previous request's solution
    c->cs = cs;
    if (encode_basis_maps(a.ws.basis, a.ws.ld, a.ws.nslots, S->opt.precision == SKR_PREC_FP64 ? 8 : 4, a.tmap) !=
        cudaSuccess)
        return false;
    const cudaError_t e = (S->opt.precision == SKR_PREC_FP64)
                              ? launch_chain_f64(a, 1, c->cs, S->threads, S->smem, st)
                              : launch_chain_f32(a, 1, c->cs, S->threads, S->smem, st);
    if (e != cudaSuccess) return false;
    cudaEventRecord(c->ev, st);
    return cudaGetLastError() == cudaSuccess;
}

void finish(skr_server *S, Request *r, const DevResult *d, bool ok) {
    r->t_done = Clock::now();
    if (ok) {
        r->res.steps = d->steps;
        r->res.cycles = d->cycles;
        r->res.matvecs = d->matvecs;
        r->res.refinements = d->refinements;
        r->res.flag = d->flag;
        r->res.k_final = d->k_final;
        r->res.relres = d->relres;
        r->res.seconds = (d->t_end >= d->t_begin) ? (double)(d->t_end - d->t_begin) * 1e-9 : 0.0;
        r->res.delta = d->delta;
    } else {
        r->res = skr_result{};
        r->res.flag = SKR_NUMERICAL;
        r->res.relres = NAN;
        r->res.delta = -1.0;
    }
    r->state = 2;
    S->completed += 1;
    S->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
}

double sqdist(const std::vector<double> &a, const std::vector<double> &b) {
    double s = 0.0;
    for (size_t i = 0; i < a.size(); i++) {
        const double d = a[i] - b[i];
        s += d * d;
    }
    return s;
}

// The server thread.  Each round: under the lock, collect the chains whose
// launch finished and take a snapshot of the queue; without the lock, copy
// their results to the requests and plan the admissions;
// under the lock again, publish the results, evict, create chains and
// launch.  The chain list and every chain's state are written by this
// thread only, and only under the lock, so the unlocked reads race with
// nothing; a request that is queued or running is never touched by
// skr_poll, and its key is immutable.  skr_submit and skr_poll therefore
// wait for the lock only while results are published and requests launched,
// not while keys are compared.
//
// Admission, in arrival order (a request that must wait does not hold back
// later ones):
//   1. the CTAs of the request's cluster must fit beside the running and
//      already admitted requests (at least one request always runs);
//   2. the nearest idle chain of the request's shape (format, grid, key
//      length) takes it;
//   3. else a new chain, if the chain limit and the device-memory budget
//      leave room;
//   4. else the least recently used idle chains are evicted until the new
//      chain fits (an evicted chain's memory is reused in place when it is
//      large enough).
// A request reaches 2-4 only when its cluster fits on the free SMs, so
// chains are evicted only for work that starts at once: while the GPU is
// full, requests wait instead of evicting back and forth.  No request is
// starved by idle chains of other shapes.
void dequeue(skr_server *S, uint64_t ticket) {
    auto it = std::find(S->queue.begin(), S->queue.end(), ticket);
    if (it != S->queue.end()) S->queue.erase(it);
}

struct Admit {
    Request *r;
    Chain *chain;                  // an idle chain of r's shape, or nullptr: a new chain
    std::vector<Chain *> victims;  // idle chains to evict first (new chain only)
    int cs;                        // cluster size of this request's launch
};

int request_cs(const skr_server *S, long long n, int share) {
    if (S->opt.cluster_size > 0) return S->opt.cluster_size;
    double cheapest = 1e300;
    for (int j = 0; j < SKR_TUNE_COLS; j++)
        if (S->maxc[j] > 0) cheapest = std::min(cheapest, tuned_step_us(n, SKR_TUNE_CS[j]) * SKR_TUNE_CS[j]);
    int best = 1;
    double bt = 1e300;
    for (int j = 0; j < SKR_TUNE_COLS; j++) {
        const int cs = SKR_TUNE_CS[j];
        if (S->maxc[j] <= 0 || cs > std::max(1, share)) continue;
        const double t = tuned_step_us(n, cs);
        if (t * cs > 1.6 * cheapest) continue;
        if (t < bt) {
            bt = t;
            best = cs;
        }
    }
    return best;
}

bool same_shape(const Chain *c, const Request *r) {
    return c->fmt == r->fmt && c->nx == r->nx && c->ny == r->ny && c->nz == r->nz && c->p == r->key.size();
}

void loop(skr_server *S) {
    cudaSetDevice(S->device);
    struct Done {
        Chain *c;
        Request *r;
        bool ok;
        DevResult res;
    };
    std::vector<Done> done;
    std::vector<Request *> queued;
    std::vector<Admit> plan;
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        done.clear();
        queued.clear();
        plan.clear();
        bool any_busy = false;
        for (Chain *c : S->chains) {
            if (!c->busy) continue;
            const cudaError_t q = cudaEventQuery(c->ev);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            if (q != cudaSuccess) cudaGetLastError();
            auto it = S->reqs.find(c->ticket);
            done.push_back({c, it != S->reqs.end() ? it->second : nullptr, q == cudaSuccess, DevResult{}});
        }
        if (S->stop && !any_busy && done.empty()) break;
        if (!S->stop)
            for (uint64_t t : S->queue) queued.push_back(S->reqs[t]);
        const size_t nchains = S->chains.size();
        const size_t used = S->used;
        lk.unlock();
        // results of finished launches: the chain's stream is idle, so these
        // copies wait for nothing but themselves
        for (Done &d : done) {
            if (!d.r || !d.ok) continue;
            d.r->x.resize(d.r->n);
            if (cudaMemcpyAsync(d.r->x.data(), d.c->dx, d.r->n * 8, cudaMemcpyDeviceToHost, d.c->st) != cudaSuccess ||
                cudaMemcpyAsync(&d.res, d.c->dres, sizeof(DevResult), cudaMemcpyDeviceToHost, d.c->st) != cudaSuccess ||
                cudaStreamSynchronize(d.c->st) != cudaSuccess) {
                cudaGetLastError();
                d.ok = false;
            }
        }
        {
            // 0 idle, 1 busy, 2 taken this round (admitted onto or evicted)
            std::vector<char> state(nchains, 0);
            int free_ctas = S->cap_ctas;
            int running = 0;
            for (size_t ci = 0; ci < nchains; ci++) {
                const Chain *c = S->chains[ci];
                bool fin = false;
                for (const Done &d : done) fin = fin || d.c == c;
                if (c->busy && !fin) {
                    state[ci] = 1;
                    free_ctas -= c->cs;
                    running++;
                }
            }
            // estimated work of the running and waiting requests (the share of each)
            double work_total = 0.0;
            for (size_t ci = 0; ci < nchains; ci++)
                if (state[ci] == 1)
                    work_total += (double)S->chains[ci]->n * plan_step_weight(S->chains[ci]->n, fmt3d(S->chains[ci]->fmt));
            for (Request *r : queued) work_total += (double)r->n * plan_step_weight(r->n, fmt3d(r->fmt));
            long long free_slots = (long long)S->max_chains - (long long)nchains;
            long long free_bytes = S->budget == 0 ? (1LL << 62) : (long long)S->budget - (long long)used;
            for (size_t qi = 0; qi < queued.size(); qi++) {
                Request *r = queued[qi];
                const double wr = (double)r->n * plan_step_weight(r->n, fmt3d(r->fmt));
                const int want = (int)std::floor(S->cap_ctas * wr / std::max(wr, work_total));
                const int cs = request_cs(S, r->n, std::min(std::max(1, want), std::max(1, free_ctas)));
                if (cs > free_ctas && running > 0) continue;      // wait for SMs
                int best = -1;
                double bd = INFINITY;
                for (size_t ci = 0; ci < nchains; ci++) {
                    const Chain *c = S->chains[ci];
                    if (!same_shape(c, r)) continue;
                    if (state[ci] != 0) continue;
                    const double dist = c->key.empty() ? 0.0 : sqdist(c->key, r->key);
                    if (dist < bd) {
                        bd = dist;
                        best = (int)ci;
                    }
                }
                if (best >= 0) {
                    state[best] = 2;
                    plan.push_back({r, S->chains[best], {}, cs});
                } else {
                    const long long need = (long long)chain_bytes(S, *r);
                    std::vector<Chain *> victims;
                    if (free_slots < 1 || need > free_bytes) {
                        // the request's cluster fits on free SMs (checked above):
                        // run it now on a new chain in place of idle ones
                        std::vector<size_t> idle;
                        for (size_t ci = 0; ci < nchains; ci++)
                            if (state[ci] == 0) idle.push_back(ci);
                        std::sort(idle.begin(), idle.end(), [&](size_t a, size_t b) {
                            return S->chains[a]->last_used < S->chains[b]->last_used;
                        });
                        long long slots = free_slots, bytes = free_bytes;
                        size_t v = 0;
                        for (; v < idle.size() && (slots < 1 || need > bytes); v++) {
                            slots += 1;
                            bytes += (long long)S->chains[idle[v]]->bytes;
                        }
                        if (slots < 1 || need > bytes) continue;  // not enough idle chains: wait
                        for (size_t q = 0; q < v; q++) {
                            state[idle[q]] = 2;
                            victims.push_back(S->chains[idle[q]]);
                        }
                        free_slots = slots;
                        free_bytes = bytes;
                    }
                    free_slots -= 1;
                    free_bytes -= need;
                    plan.push_back({r, nullptr, victims, cs});
                }
                free_ctas -= cs;
                running++;
            }
        }
        lk.lock();
        for (const Done &d : done) {
            if (d.r) finish(S, d.r, d.ok ? &d.res : nullptr, d.ok);
            d.c->busy = false;
        }
        // victims leave the chain list under the lock (stats reads it); the
        // one whose memory will be reshaped in place stays
        std::vector<Chain *> dead;
        std::vector<Chain *> reuse(plan.size(), nullptr);
        for (size_t a = 0; a < plan.size(); a++) {
            Admit &ad = plan[a];
            if (ad.chain || ad.victims.empty()) continue;
            const ChainPlan P = chain_plan(S, *ad.r);
            if (ad.victims.back()->bytes >= P.bytes) {
                reuse[a] = ad.victims.back();
                ad.victims.pop_back();
            }
            for (Chain *v : ad.victims) {
                S->chains.erase(std::find(S->chains.begin(), S->chains.end(), v));
                S->used -= v->bytes;
                S->evicted += 1;
                dead.push_back(v);
            }
        }
        const bool stopping = S->stop;
        lk.unlock();
        // every CUDA call of the admissions runs without the lock, so that
        // skr_submit and skr_poll never wait for one (a copy from pageable
        // memory can wait behind a running solve)
        for (Chain *v : dead) destroy_chain(v);
        std::vector<Chain *> fresh(plan.size(), nullptr), ran(plan.size(), nullptr);
        std::vector<char> failed(plan.size(), 0);
        size_t used_after = S->used;
        for (size_t a = 0; a < plan.size() && !stopping; a++) {
            Admit &ad = plan[a];
            Request *r = ad.r;
            Chain *c = ad.chain;
            if (!c) {
                const ChainPlan P = chain_plan(S, *r);
                if (reuse[a]) {
                    if (shape_chain(S, reuse[a], *r, P)) c = reuse[a];
                } else if (S->budget == 0 || used_after + P.bytes <= S->budget) {
                    c = create_chain(S, *r);
                    if (c) {
                        fresh[a] = c;
                        used_after += c->bytes;
                    }
                } else {
                    continue;   // stays queued
                }
                if (!c) {
                    failed[a] = 1;   // device memory could not be obtained
                    continue;
                }
            }
            if (launch(S, c, r, ad.cs))
                ran[a] = c;
            else
                failed[a] = 1;
        }
        lk.lock();
        for (size_t a = 0; a < plan.size(); a++) {
            Request *r = plan[a].r;
            if (fresh[a]) {
                S->chains.push_back(fresh[a]);
                S->used += fresh[a]->bytes;
            }
            if (reuse[a] && !ran[a] && failed[a]) {
                // the reshape failed: drop the chain (rare; its stream is idle)
                S->chains.erase(std::find(S->chains.begin(), S->chains.end(), reuse[a]));
                S->used -= reuse[a]->bytes;
                S->evicted += 1;
                destroy_chain(reuse[a]);
            } else if (reuse[a]) {
                S->evicted += 1;
            }
            if (ran[a]) {
                Chain *c = ran[a];
                c->busy = true;
                c->ticket = r->ticket;
                c->key = r->key;
                c->last_used = ++S->launches;
                r->state = 1;
                dequeue(S, r->ticket);
            } else if (failed[a]) {
                cudaGetLastError();
                finish(S, r, nullptr, false);
                dequeue(S, r->ticket);
            }
        }
        S->cv.wait_for(lk, std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" {

skr_status skr_server_create(const skr_options *opt_in, size_t hbm_budget, int32_t max_chains, skr_server **out) {
    if (!out) return err(SKR_ERR_INVALID_ARG, "srv is NULL");
    *out = nullptr;
    skr_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        skr_options_default(&opt);
    if (opt.m < 2 || opt.m > SKR_MAX_M) return err(SKR_ERR_INVALID_ARG, "m out of range");
    if (opt.k < 0 || opt.k > SKR_MAX_K || (opt.k > 0 && opt.k > opt.m - 2)) return err(SKR_ERR_INVALID_ARG, "k out of range");
    if (opt.maxit < 1 || opt.max_refine < 1 || !(opt.tol > 0.0 && opt.tol < 1.0))
        return err(SKR_ERR_INVALID_ARG, "bad maxit, max_refine or tol");
    if (opt.precision == SKR_PREC_MIXED && !(opt.inner_tol > 0.0 && opt.inner_tol < 1.0))
        return err(SKR_ERR_INVALID_ARG, "inner_tol must be in (0, 1)");
    if (opt.precond != SKR_PC_NONE && opt.precond != SKR_PC_JACOBI && opt.precond != SKR_PC_ILU0 &&
        opt.precond != SKR_PC_SSOR && opt.precond != SKR_PC_BJACOBI)
        return err(SKR_ERR_INVALID_ARG, "unknown preconditioner");
    if (opt.precond == SKR_PC_BJACOBI && opt.pc_blocks < 1) return err(SKR_ERR_INVALID_ARG, "pc_blocks < 1");
    if ((opt.warm_start != 0 && opt.warm_start != 1) || (opt.diagnostics != 0 && opt.diagnostics != 1))
        return err(SKR_ERR_INVALID_ARG, "warm_start and diagnostics must be 0 or 1");
    if (opt.precision != SKR_PREC_FP64 && opt.precision != SKR_PREC_MIXED) return err(SKR_ERR_INVALID_ARG, "bad precision");
    if (opt.cluster_size < 0 || opt.cluster_size > 16) return err(SKR_ERR_INVALID_ARG, "cluster_size in [0, 16]");
    if (max_chains < 0) return err(SKR_ERR_INVALID_ARG, "max_chains < 0");
    skr_server *S = new skr_server();
    S->opt = opt;
    S->budget = hbm_budget;
    S->max_chains = max_chains;   // 0: set below, one chain per resident CTA
    S->threads = chain_threads();
    S->smem = chain_smem_bytes(opt.m, opt.k, S->threads, opt.precision == SKR_PREC_FP64 ? 8 : 4);
    if (S->smem > 227 * 1024) {
        delete S;
        return err(SKR_ERR_INVALID_ARG, "m, k too large for shared memory");
    }
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return err(SKR_ERR_CUDA, "no CUDA device");
    }
    // CTAs of the chain kernel resident at once (clusters of one CTA)
    S->cap_ctas = opt.precision == SKR_PREC_FP64 ? max_active_clusters_f64(1, S->threads, S->smem)
                                                 : max_active_clusters_f32(1, S->threads, S->smem);
    for (int j = 0; j < SKR_TUNE_COLS; j++)
        S->maxc[j] = opt.precision == SKR_PREC_FP64 ? max_active_clusters_f64(SKR_TUNE_CS[j], S->threads, S->smem)
                                                    : max_active_clusters_f32(SKR_TUNE_CS[j], S->threads, S->smem);
    if (S->max_chains == 0) S->max_chains = std::max(1, S->cap_ctas);
    if (S->cap_ctas < 1) {
        delete S;
        return err(SKR_ERR_CUDA, "the chain kernel cannot be scheduled with this shared memory");
    }
    S->th = std::thread(loop, S);
    *out = S;
    return SKR_OK;
}

skr_status skr_submit(skr_server *S, const skr_system *sys, const double *key, int64_t p, uint64_t *ticket) {
    if (!S || !sys || !ticket) return err(SKR_ERR_INVALID_ARG, "NULL pointer");
    if (sys->fmt == SKR_FMT_CSR)
        return err(SKR_ERR_INVALID_ARG, "the serving loop takes the grid formats; CSR input goes to skr_solve_sequence");
    if (sys->fmt < SKR_FMT_DARCY2D || sys->fmt > SKR_FMT_POISSON2D) return err(SKR_ERR_INVALID_ARG, "unknown format");
    if (sys->fmt == SKR_FMT_POISSON2D && sys->rhs) return err(SKR_ERR_INVALID_ARG, "Poisson format: rhs must be NULL");
    if (sys->nx < 1 || sys->ny < 1 || (fmt3d(sys->fmt) && sys->nz < 1)) return err(SKR_ERR_INVALID_ARG, "empty grid");
    if (sys->fmt == SKR_FMT_CONVDIFF2D && (sys->nx != sys->ny || !(sys->params[0] > 0.0)))
        return err(SKR_ERR_INVALID_ARG, "convection-diffusion needs nx == ny and nu > 0");
    if (sys->fmt != SKR_FMT_CONVDIFF2D && !sys->coef) return err(SKR_ERR_INVALID_ARG, "coef is NULL");
    if (p < 0 || (p > 0 && !key)) return err(SKR_ERR_INVALID_ARG, "bad key");
    Request *r = new Request();
    r->fmt = sys->fmt;
    r->nx = sys->nx;
    r->ny = sys->ny;
    r->nz = fmt3d(sys->fmt) ? sys->nz : 1;
    r->n = n_of(r->fmt, r->nx, r->ny, r->nz);
    for (int i = 0; i < 4; i++) r->params[i] = sys->params[i];
    const long long clen = coef_len(r->fmt, r->nx, r->ny, r->nz);
    if (clen > 0) r->coef.assign(sys->coef, sys->coef + clen);
    if (sys->rhs) r->rhs.assign(sys->rhs, sys->rhs + r->n);
    if (p > 0)
        r->key.assign(key, key + p);
    else if (clen > 0)
        r->key = r->coef;
    else
        r->key.assign(r->params, r->params + 3);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->budget > 0 && chain_bytes(S, *r) > S->budget) {
            delete r;
            return err(SKR_ERR_OOM, "request does not fit in the server's device-memory budget");
        }
        r->ticket = S->next++;
        S->reqs[r->ticket] = r;
        S->queue.push_back(r->ticket);
        S->submitted += 1;
        *ticket = r->ticket;
    }
    S->cv.notify_one();
    return SKR_OK;
}

skr_status skr_poll(skr_server *S, uint64_t ticket, double *x_out, skr_result *res) {
    if (!S) return err(SKR_ERR_INVALID_ARG, "srv is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return err(SKR_ERR_INVALID_ARG, "unknown ticket");
    Request *r = it->second;
    if (r->state != 2) return SKR_NOT_READY;
    if (x_out && !r->x.empty()) std::memcpy(x_out, r->x.data(), r->x.size() * 8);
    if (res) *res = r->res;
    S->reqs.erase(it);
    delete r;
    return SKR_OK;
}

skr_status skr_server_stats(skr_server *S, skr_server_info *info) {
    if (!S || !info) return err(SKR_ERR_INVALID_ARG, "NULL pointer");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(info, 0, sizeof(*info));
    info->submitted = S->submitted;
    info->completed = S->completed;
    info->queued = (int64_t)S->queue.size();
    int64_t running = 0;
    for (Chain *c : S->chains) running += c->busy ? 1 : 0;
    info->running = running;
    info->chains = (int32_t)S->chains.size();
    info->evicted = (int32_t)S->evicted;
    info->hbm_bytes = (double)S->used;
    if (!S->lat_ms.empty()) {
        std::vector<double> v = S->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            const size_t i = std::min(v.size() - 1, (size_t)std::floor(q * (double)(v.size() - 1) + 0.5));
            return v[i];
        };
        info->p50_ms = pct(0.50);
        info->p99_ms = pct(0.99);
        double s = 0.0;
        for (double x : v) s += x;
        info->mean_ms = s / (double)v.size();
    }
    return SKR_OK;
}

skr_status skr_server_destroy(skr_server *S) {
    if (!S) return SKR_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->queue.clear();
    }
    S->cv.notify_one();
    if (S->th.joinable()) S->th.join();
    for (Chain *c : S->chains) destroy_chain(c);
    for (auto &kv : S->reqs) delete kv.second;
    delete S;
    return SKR_OK;
}

}  // extern "C"
