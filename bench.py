"""Benchmark: sorted Krylov recycling (SKR) vs plain restarted GMRES on one GB300.

One step = the whole hot path over one batch: the greedy sort of the 200
Darcy systems (Algorithm 1) and their recycled GCRO-DR solves to a true
relative residual of 1e-8 (Algorithm 2 with residual refinement), inputs
already resident in device memory.  Workload: 2D Darcy -div(a grad u) = 1
on a 256 x 256 interior grid (n = 65,536), a = exp(GRF, ell = 0.1,
sigma = 1), Jacobi preconditioner, m = 40, k = 20, mixed precision (FP32
Krylov vectors, FP64 refinement, solution and small dense step).  The
synthetic fields stand in for the paper's Darcy dataset.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU
oracle instead, on a bounded sample of the same workload.  `--workload
helmholtz100` measures the paper's Helmholtz set the same way (100^2
unknowns, -lap u - k^2 u = 1 with k from a GRF: indefinite systems).
"""
import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "systems/s to rel-res 1e-8, SKR vs plain GMRES on 1 GB300; HBM GB/s frac; p99"
WORKLOADS = {
    # Darcy 32^2, 20 systems, no preconditioner, FP64 throughout: the small
    # case the oracle finishes in seconds.  Latency-bound: the sorted order is
    # cut into 4 chains and the planner gives each a 16-CTA cluster (measured
    # 45 against 12 systems/s for one chain on one CTA)
    "darcy32_fp64": dict(kind="darcy2d", nside=32, nsys=20, ell=0.2, sigma=1.0, seed=1, m=30, k=10,
                         precond="none", precision="fp64", tol=1e-8, inner_tol=1e-5, chains=4, cluster_size=0,
                         desc="darcy2d 32x32 (n=1024), %d systems, a=exp(GRF ell=0.2 sigma=1), f=1, "
                              "no preconditioner, GCRO-DR m=30 k=10, FP64, tol 1e-8"),
    # Darcy on 256^2 (n = 65,536), 200 systems
    "darcy256": dict(kind="darcy2d", nside=256, nsys=200, ell=0.1, sigma=1.0, seed=2, m=40, k=20,
                     precond="jacobi", precision="mixed", tol=1e-8, inner_tol=1e-5, chains=76, cluster_size=2,
                     desc="darcy2d 256x256 (n=65536), %d systems, a=exp(GRF ell=0.1 sigma=1), f=1, "
                          "Jacobi, GCRO-DR m=40 k=20, mixed precision, tol 1e-8"),
    # convection-diffusion on 512^2 (n = 262,144), 500 systems, red-black ILU(0);
    # sort keys (nu, beta_x, beta_y) z-scored by their drawing distributions
    "convdiff512_ilu": dict(kind="convdiff2d", nside=512, nsys=500, seed=3, m=40, k=20,
                            precond="ilu0", precision="mixed", tol=1e-8, inner_tol=1e-5, chains=38, cluster_size=0,
                            desc="convdiff2d 512x512 (n=262144), %d systems, -nu lap u + beta.grad u = f "
                                 "(first-order upwind), nu~U[0.01,0.1], beta=U[0,50](cos phi, sin phi), "
                                 "f=GRF(ell=0.1 sigma=1), red-black ILU(0), GCRO-DR m=40 k=20, mixed precision, "
                                 "tol 1e-8; sort keys (nu, beta) z-scored"),
    # 64 independent chains of 50 Darcy systems, grid side per chain from
    # {64, 128, 192, 256, 384}, ell per chain ~ U[0.05, 0.3]; each chain sorted on its own
    "batched64x50": dict(kind="batched", nchains=64, chain_len=50, nsys=3200, seed=4, m=40, k=20,
                         sides=(64, 128, 192, 256, 384), ell_range=(0.05, 0.3), sigma=1.0,
                         precond="jacobi", precision="mixed", tol=1e-8, inner_tol=1e-5, cluster_size=0,
                         desc="batched Darcy: %d systems in 64 independent sorted chains of 50, side per chain "
                              "from {64,128,192,256,384}, a=exp(GRF ell~U[0.05,0.3] sigma=1), f=1, Jacobi, "
                              "GCRO-DR m=40 k=20, mixed precision, tol 1e-8"),
    # Darcy at the ablation's matrix size (10^4 unknowns, 100^2)
    "darcy100": dict(kind="darcy2d", nside=100, nsys=200, ell=0.1, sigma=1.0, seed=8, m=40, k=20,
                     precond="jacobi", precision="mixed", tol=1e-8, inner_tol=1e-5,
                     desc="darcy2d 100x100 (n=10000), %d systems, a=exp(GRF ell=0.1 sigma=1), f=1, "
                          "Jacobi, GCRO-DR m=40 k=20, mixed precision, tol 1e-8"),
    # Darcy 100^2 on a closed curve of GRF samples: close neighbours exist, so
    # the sort's effect on the recycle spaces (Table 2's mechanism) can show
    "darcy100_circle": dict(kind="darcy2d", family="circle", nside=100, nsys=200, ell=0.1, sigma=1.0, seed=9,
                            m=40, k=20, precond="jacobi", precision="mixed", tol=1e-8, inner_tol=1e-5,
                            desc="darcy2d 100x100 (n=10000), %d systems, a=exp(cos t G1 + sin t G2), G1, G2 "
                                 "GRF ell=0.1 sigma=1, t ~ U[0, 2pi), f=1, Jacobi, GCRO-DR m=40 k=20, "
                                 "mixed precision, tol 1e-8"),
    "darcy256_circle": dict(kind="darcy2d", family="circle", nside=256, nsys=200, ell=0.1, sigma=1.0, seed=10,
                            m=40, k=20, precond="jacobi", precision="mixed", tol=1e-8, inner_tol=1e-5,
                            desc="darcy2d 256x256 (n=65536), %d systems, a=exp(cos t G1 + sin t G2), G1, G2 "
                                 "GRF ell=0.1 sigma=1, t ~ U[0, 2pi), f=1, Jacobi, GCRO-DR m=40 k=20, "
                                 "mixed precision, tol 1e-8"),
    # Poisson with Dirichlet data and forcing from truncated Chebyshev series (App. E);
    # one fixed matrix, the right-hand sides differ; sort keys = the 96 coefficients
    "poisson_cheb256": dict(kind="poisson2d", nside=256, nsys=200, ncoef=8, decay=0.6, seed=7, m=40, k=20,
                            precond="jacobi", precision="mixed", tol=1e-8, inner_tol=1e-5,
                            desc="poisson2d 256x256 (n=65536), %d systems, lap u = f, f and boundary data "
                                 "from truncated Chebyshev series (8 coefficients each, decay 0.6), "
                                 "Jacobi, GCRO-DR m=40 k=20, mixed precision, tol 1e-8"),
    # the paper's Helmholtz set (App. E): 100^2 unknowns, k from a GRF; indefinite
    "helmholtz100": dict(kind="helmholtz2d", nside=100, nsys=200, kbar=10.0, ell=0.1, sigma=1.0, spread=0.2,
                         seed=6, m=40, k=20, precond="jacobi", precision="mixed", tol=1e-8, inner_tol=1e-5,
                         # n = 10^4 needs no cluster: one CTA per chain, fewer and longer chains
                         chains=100, cluster_size=1,
                         desc="helmholtz2d 100x100 (n=10000), %d systems, -lap u - k^2 u = 1, "
                              "k=10 exp(0.2 GRF(ell=0.1 sigma=1)), Jacobi, GCRO-DR m=40 k=20, mixed precision, tol 1e-8"),
}
DEFAULT_WORKLOAD = "darcy256"


PRECOND_NAMES = {"none": "no preconditioner", "jacobi": "Jacobi", "ssor": "SSOR", "ilu0": "red-black ILU(0)",
                 "bjacobi": "block Jacobi"}


def _workload(args):
    """The named workload, with the preconditioner overridden if asked."""
    W = dict(WORKLOADS[args.workload])
    W["pc_blocks"] = 1
    for key in ("m", "k"):
        val = getattr(args, key, None)
        if val is not None and val != W[key]:
            W["desc"] = W["desc"].replace("m=%d k=%d" % (W["m"], W["k"]),
                                          "m=%d k=%d" % (val if key == "m" else W["m"], val if key == "k" else W["k"]))
            W[key] = val
    if args.precond and args.precond != W["precond"]:
        name = PRECOND_NAMES[args.precond]
        if args.precond == "bjacobi":
            W["pc_blocks"] = args.pc_blocks
            name = "block Jacobi (%d row blocks, red-black ILU(0) each)" % args.pc_blocks
        W["desc"] = W["desc"].replace(PRECOND_NAMES[W["precond"]], name)
        W["precond"] = args.precond
    return W


def _inputs(W, nsys, seed):
    """Seeded inputs of nsys systems of a one-group workload: (sort keys [nsys, p], per-system payload)."""
    if W["kind"] == "darcy2d":
        from workloads import darcy2d_sequence, darcy2d_circle_sequence
        if W.get("family") == "circle":
            L, _ = darcy2d_circle_sequence(W["nside"], nsys, W["ell"], W["sigma"], seed=seed)
        else:
            L = darcy2d_sequence(W["nside"], nsys, W["ell"], W["sigma"], seed=seed)
        return L.reshape(nsys, -1), [L[i] for i in range(nsys)]
    if W["kind"] == "helmholtz2d":
        from workloads import helmholtz2d_sequence
        L = helmholtz2d_sequence(W["nside"], nsys, W["kbar"], W["ell"], W["sigma"], spread=W["spread"], seed=seed)
        return L.reshape(nsys, -1), [L[i] for i in range(nsys)]
    if W["kind"] == "convdiff2d":
        from workloads import convdiff2d_sequence, convdiff_keys
        nu, beta, f = convdiff2d_sequence(W["nside"], nsys, seed=seed)
        return convdiff_keys(nu, beta), [(float(nu[i]), (float(beta[i, 0]), float(beta[i, 1])), f[i])
                                         for i in range(nsys)]
    from workloads import chebyshev_poisson_sequence
    K, F, G = chebyshev_poisson_sequence(W["nside"], nsys, W["ncoef"], W["decay"], seed=seed)
    return K, [(F[i], G[i]) for i in range(nsys)]


class Batch:
    """The inputs of one bench step.

    groups   list of (first system, keys [count, p]): the systems of a group
             are sorted together (Algorithm 1) and are consecutive here
    chains   chains per group: a group's sorted order is cut into that many
             contiguous chains (App. E.2.2)
    payload  per-system arrays the system is built from
    n        unknowns per system
    """

    def __init__(self, groups, chains, payload, n):
        self.groups, self.chains, self.payload, self.n = groups, chains, payload, n

    @property
    def nsys(self):
        return len(self.payload)

    def chain_offsets(self):
        offs = [0]
        for (first, keys), q in zip(self.groups, self.chains):
            c = keys.shape[0]
            offs += [first + (i * c) // q for i in range(1, q + 1)]
        return offs

    def order(self, perms):
        """The solve order from one permutation per group (group-local indices)."""
        import numpy as np
        return np.concatenate([first + np.asarray(pm, dtype=np.int64)
                               for (first, _), pm in zip(self.groups, perms)]).astype(np.int32)


def _batch(W, nsys, seed, nchains=None):
    """Seeded inputs of one bench step of workload W (nsys systems)."""
    if W["kind"] == "batched":
        from workloads import batched_chains
        clen = W["chain_len"]
        nch = max(1, nsys // clen)
        chains = batched_chains(nch, clen, sides=W["sides"], ell_range=W["ell_range"], sigma=W["sigma"],
                                seed=seed)
        groups, payload, n = [], [], []
        for side, _, sub in chains:
            groups.append((len(payload), sub.reshape(clen, -1)))
            for i in range(clen):
                payload.append(sub[i])
                n.append(side * side)
        return Batch(groups, [1] * len(groups), payload, n)
    K, payload = _inputs(W, nsys, seed)
    q = nchains if nchains is not None else W.get("chains", 76)
    n = [W["nside"] ** 2] * nsys
    return Batch([(0, K)], [max(1, min(q, nsys))], payload, n)


def _to(payload, conv):
    return tuple(conv(a) for a in payload) if isinstance(payload, tuple) else conv(payload)


def _to_payload(W, payload, conv):
    """Move a system's arrays with conv (scalars stay)."""
    if W["kind"] == "convdiff2d":
        nu, beta, f = payload
        return (nu, beta, conv(f))
    return _to(payload, conv)


def _system(skr, W, payload):
    if W["kind"] in ("darcy2d", "batched"):
        return skr.darcy2d(payload)
    if W["kind"] == "helmholtz2d":
        return skr.helmholtz2d(payload)
    if W["kind"] == "convdiff2d":
        nu, beta, f = payload
        return skr.convdiff2d(nu, beta, W["nside"], rhs=f)
    f, g = payload
    return skr.poisson2d(f, tuple(g[e] for e in range(4)))


def _oracle_system(W, payload):
    if W["kind"] in ("darcy2d", "batched"):
        return dict(kind="darcy2d", loga=payload)
    if W["kind"] == "helmholtz2d":
        return dict(kind="helmholtz2d", k=payload)
    if W["kind"] == "convdiff2d":
        nu, beta, f = payload
        return dict(kind="convdiff2d", nu=nu, beta=beta, nside=W["nside"], rhs=f)
    f, g = payload
    return dict(kind="poisson2d", f=f, g=tuple(g))


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one chain-
# kernel launch on the default workload, from a one-pass ncu capture; valid
# only for the sources it was taken with (sha256 over the files that build
# or launch the chain kernel and the public header, as computed by
# _kernel_sources_sha256).
TRAFFIC = {"workload": "darcy256", "sources_sha256": "98dd06aa31b4e802d4e1fa77088f198d03fe160a3cb4e88f5cb239e4680338b6",
           "bytes_per_launch": 5684345175552 + 413036297984}


# the chain kernel's translation units, their headers and the host code
# that launches it from skr_solve_sequence (the server and the sort kernels
# do not change a chain-kernel launch)
CHAIN_KERNEL_SOURCES = ("skr_api.cu", "skr_chain.cuh", "skr_chain_f32.cu", "skr_chain_f64.cu",
                        "skr_chain_launch.cuh", "skr_common.h", "skr_dense.cuh", "skr_device.cuh",
                        "skr_launch.h", "skr_plan.h", "skr_stencil.cuh", "skr_tma.h", "skr_tuned.inc",
                        "skr_workspace.h")


def _kernel_sources_sha256():
    files = [os.path.join(ROOT, "paper_2401_09516_gb300", "csrc", f) for f in CHAIN_KERNEL_SOURCES]
    files = files + [os.path.join(ROOT, "include", "skr.h")]
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.relpath(f, ROOT).encode())
        h.update(b"\0")
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _rank_seed(W, rank):
    """Seed of a rank's batch: ranks solve independent batches (weak scaling)."""
    return W["seed"] + 1000 * rank


def _agg_ms(ms_list, ws, device):
    """Mean step time of this rank; with several ranks the maximum over the
    ranks, since the job is as slow as its slowest rank."""
    mean = sum(ms_list) / len(ms_list)
    if ws > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([mean], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        return float(tt.item())
    return mean


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    def barrier():
        if ws > 1:
            dist.barrier()

    import paper_2401_09516_gb300 as skr
    W = _workload(args)
    # weak scaling: every rank solves its own batch (independent chains)
    N = args.nsys if args.nsys is not None else W["nsys"]
    B = _batch(W, N, _rank_seed(W, rank), args.chains)
    N = B.nsys
    P_dev = [torch.tensor(keys, device=dev) for _, keys in B.groups]
    if W["kind"] in ("darcy2d", "helmholtz2d", "batched"):
        # the keys are the fields themselves: the systems read them in place
        pay_dev = []
        for (first, keys), Pg in zip(B.groups, P_dev):
            pay_dev += [Pg[i].view(*B.payload[first + i].shape) for i in range(keys.shape[0])]
    else:
        pay_dev = [_to_payload(W, pl, lambda a: torch.tensor(a, device=dev)) for pl in B.payload]
    systems = [_system(skr, W, pl) for pl in pay_dev]
    x_dev = [torch.empty(B.n[i], dtype=torch.float64, device=dev) for i in range(N)]
    stream = torch.cuda.current_stream(dev)
    offs = B.chain_offsets()
    cluster_size = args.cluster_size if args.cluster_size is not None else W.get("cluster_size", 0)

    def opts(k, precision=None, profile=0):
        return skr.skr_options_default(m=W["m"], k=k, tol=W["tol"], inner_tol=W["inner_tol"],
                                       maxit=args.maxit, precond=W["precond"], pc_blocks=W["pc_blocks"],
                                       precision=precision or W["precision"], cluster_size=cluster_size,
                                       stream=stream, warm_start=int(args.warm_start),
                                       diagnostics=int(args.diagnostics), profile=profile,
                                       eig_fp32=int(args.eig_fp32))

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    sort_ev = []   # (start, end) events around the sorts of each step
    ident = [np.arange(keys.shape[0]) for _, keys in B.groups]

    def step(k, precision=None, profile=0):
        if args.no_sort:
            order = B.order(ident)
        else:
            es0 = torch.cuda.Event(enable_timing=True)
            es1 = torch.cuda.Event(enable_timing=True)
            es0.record(stream)
            perms = [skr.skr_sort(Pg, stream=stream) for Pg in P_dev]
            es1.record(stream)
            sort_ev.append((es0, es1))
            order = B.order([pm.cpu().numpy() for pm in perms])
        _, res = skr.skr_solve_sequence(systems, order=order, chain_offsets=offs, nchains=len(offs) - 1,
                                        options=opts(k, precision, profile), x_out=x_dev)
        st = skr.skr_last_stats()
        st["plan"] = skr.skr_last_plan()
        return res, st

    def timed(k, steps, warmup, precision=None):
        for _ in range(warmup):
            step(k, precision)
        torch.cuda.synchronize()
        times, stats, allres = [], [], []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res, st = step(k, precision)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            times.append(e0.elapsed_time(e1))
            stats.append(st)
            allres.append(res)
        return times, stats, allres

    sampler = ClockSampler(local)
    sampler.start()
    t_skr, st_skr, res_skr = timed(W["k"], args.steps, args.warmup)
    clocks = sampler.stop()
    timed_sorts = sort_ev[-args.steps:] if (sort_ev and not args.no_sort) else []
    sort_ms = (sum(a.elapsed_time(b) for a, b in timed_sorts) / len(timed_sorts)) if timed_sorts else None

    def agg(ms_list):
        return _agg_ms(ms_list, ws, dev)

    def arm_summary(times, allres):
        ms = agg(times)
        last = allres[-1]
        flags = [r["flag"] for r in last]
        return {"value": round(N * ws / (ms / 1e3), 3), "ms_per_step": round(ms, 3), "steps_timed": len(times),
                "avg_arnoldi_steps": round(sum(r["steps"] for r in last) / N, 1),
                "converged": sum(1 for f in flags if f == 0), "not_converged": sum(1 for f in flags if f != 0),
                "flags": sorted(set(flags)), "max_relres": max(r["relres"] for r in last)}

    ms_step = agg(t_skr)
    value = N * ws / (ms_step / 1e3)
    gmres = None
    if args.gmres_steps > 0:
        t_gm, _, res_gm = timed(0, args.gmres_steps, 1)
        gmres = arm_summary(t_gm, res_gm)
        gmres["maxit"] = args.maxit
    fp64 = None
    if args.fp64_steps > 0 and W["precision"] == "mixed":
        t_64, _, res_64 = timed(W["k"], args.fp64_steps, 1, precision="fp64")
        fp64 = arm_summary(t_64, res_64)
    # per-phase device time of one more (untimed) SKR step with the phase timers on
    phases = None
    if args.phases:
        step(W["k"], profile=1)
        torch.cuda.synchronize()
        prof = skr.skr_last_profile()
        tot = sum(prof.values())
        phases = {"ms_per_system": {k: round(v / N, 3) for k, v in prof.items()},
                  "share": {k: round(v / tot, 4) for k, v in prof.items()} if tot > 0 else None,
                  "measured": "device timers (globaltimer) of each cluster's rank-0 CTA, summed over clusters, "
                              "divided by the systems of the step; one extra untimed step"}
    # roofline of the dominant kernel (the chain kernel), measured per launch
    peak, peak_kind = _peaks()
    kbytes = sum(s["bytes"] for s in st_skr) / len(st_skr)
    kms = sum(s["kernel_ms"] for s in st_skr) / len(st_skr)
    achieved = kbytes / (kms / 1e3) / 1e9
    traffic = None
    if (args.workload == TRAFFIC.get("workload") and N == W["nsys"] and args.chains is None
            and args.cluster_size is None and TRAFFIC["sources_sha256"] == _kernel_sources_sha256()):
        traffic = TRAFFIC["bytes_per_launch"]
    # correctness of the timed results
    relmax = max(r["relres"] for r in res_skr[-1])
    flags = sorted({r["flag"] for r in res_skr[-1]})
    lat = sorted(r["seconds"] * 1e3 for r in res_skr[-1])
    steps_skr = sum(r["steps"] for r in res_skr[-1]) / N
    launches_per_step = (0 if args.no_sort else 2 * len(B.groups)) + st_skr[-1]["launches"]

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if args.e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()   # noqa: E731
        Lh = [_to_payload(W, pl, pin) for pl in B.payload]
        Ph = [pin(keys) for _, keys in B.groups]
        xh = [torch.empty(B.n[i], dtype=torch.float64).pin_memory() for i in range(N)]
        sys_h = [_system(skr, W, _to_payload(W, Lh[i], lambda t: t.numpy())) for i in range(N)]
        xh_np = [x.numpy() for x in xh]

        def e2e_step():
            if args.no_sort:
                order = B.order(ident)
            else:
                order = B.order([skr.skr_sort(Pg.numpy(), stream=stream) for Pg in Ph])
            skr.skr_solve_sequence(sys_h, order=order, chain_offsets=offs, nchains=len(offs) - 1,
                                   options=opts(W["k"]), x_out=xh_np)

        e2e_step()
        torch.cuda.synchronize()
        e2e_ms = []
        for _ in range(max(1, args.e2e_steps)):
            flush.zero_()
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            barrier()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e_val = N * ws / (agg(e2e_ms) / 1e3)

        def nbytes(pl):
            if W["kind"] == "convdiff2d":
                return pl[2].numel() * 8
            return sum(t.numel() for t in pl) * 8 if isinstance(pl, tuple) else pl.numel() * 8
        h2d = (0 if args.no_sort else sum(P.numel() * 8 for P in Ph))
        h2d += sum(nbytes(pl) for pl in Lh)
        d2h = sum(B.n) * 8 + (0 if args.no_sort else N * 4)
        e2e = {"value": round(e2e_val, 3), "unit": "systems/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps_timed": len(e2e_ms)}

    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "systems/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if W["precision"] == "mixed" else "f64",
        "data": "synthetic",
        "config": {
            "workload": W["desc"] % N,
            "chains": len(offs) - 1, "cluster_size": st_skr[-1]["cluster_size"],
            "warm_start": bool(args.warm_start), "sorted": not args.no_sort,
            "eigen_solve": "fp32" if (args.eig_fp32 and W["precision"] == "mixed") else "fp64",
            "slots": st_skr[-1]["slots"], "launches": st_skr[-1]["plan"],
            "maxit": args.maxit, "l2": "flushed between steps (256 MB write)",
            "parallelism": "replicas" if ws > 1 else "single GPU",
        },
        "sort_ms": None if sort_ms is None else round(sort_ms, 3),
        "avg_steps_skr": round(steps_skr, 1),
        "max_relres": relmax,
        "flags": flags,
        "gmres": gmres,
        "speedup_vs_gmres": None if gmres is None else round(value / gmres["value"], 3),
        "fp64": fp64,
        "latency_ms": {"p50": round(lat[len(lat) // 2], 3), "p99": round(lat[min(len(lat) - 1, int(0.99 * len(lat)))], 3),
                       "measured": "device time of each system inside the batch (first to last kernel work on it)"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": "chain_kernel<%s>" % ("float" if W["precision"] == "mixed" else "double"),
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": int(kbytes), "kernel_ms": round(kms, 3)},
        "phases": phases,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if args.diagnostics:
        ds = [r["delta"] for r in res_skr[-1] if r["delta"] >= 0.0]
        line["delta_mean"] = round(sum(ds) / len(ds), 4) if ds else None
        line["delta_systems"] = len(ds)
    if args.cpu_baseline and rank == 0:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, W, args.warm_start, B)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def _oracle_worker(conn, W, segments, warm):
    """One host core walking its chain segments with the FP64 oracle, as it stands.

    segments: lists of system payloads; the recycle state (and the warm
    start) resets at the first system of each segment, and the worker wraps
    around to its first segment after the last.  On "go" it solves systems
    back to back; between systems it checks for "stop", then replies with
    the (start, end) monotonic clock times of every system it finished.
    """
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    from oracle import skr as oskr
    from oracle.krylov import RecycleState

    conn.send("ready")
    if conn.recv() != "go":
        return
    spans = []
    seg, pos, state, prev = 0, 0, RecycleState(), None
    while not conn.poll():
        if pos == len(segments[seg]):
            seg, pos, state, prev = (seg + 1) % len(segments), 0, RecycleState(), None
        t0 = time.monotonic()
        sysd = _oracle_system(W, segments[seg][pos])
        A, b = oskr.assemble(sysd)
        x, _ = oskr.solve_system(A, b, W["precond"], W["m"], W["k"], W["tol"], state,
                                 precision=W["precision"], inner_tol=W["inner_tol"],
                                 x0=prev if warm else None, grid=oskr.grid_of(sysd),
                                 pc_blocks=W["pc_blocks"])
        spans.append((t0, time.monotonic()))
        prev = x
        pos += 1
    conn.recv()
    conn.send(spans)


def _progress(spans, a, b):
    """Systems finished inside [a, b], a system that straddles an edge
    counted by the fraction of its solve time inside."""
    tot = 0.0
    for t0, t1 in spans:
        if t1 > t0:
            tot += max(0.0, min(t1, b) - max(t0, a)) / (t1 - t0)
    return tot


class OracleChains:
    """The FP64 oracle in the paper's decomposition: each sort group ordered
    by the oracle's Algorithm 1 (once, on one core), the sorted order cut
    into chain segments, the segments dealt to the host cores, every core
    solving its segments.

    Workers are spawned processes (no fork after the GPU is in use).  `run`
    lets them solve for a number of back-to-back windows and returns, per
    window, the systems finished inside it (fractions for systems that
    straddle a window edge; the run waits for the systems in flight at the
    end to finish so that their fractions are known).
    """

    def __init__(self, W, batch, warm=False, cores=None):
        import multiprocessing as mp
        from oracle import sort as osort
        from oracle import skr as oskr

        self.W = W
        self.nsys = batch.nsys
        t0 = time.perf_counter()
        perms = [osort.greedy_sort(keys) for _, keys in batch.groups]
        self.t_sort = time.perf_counter() - t0
        order = batch.order(perms)
        offs = batch.chain_offsets()
        chains = [order[offs[c]:offs[c + 1]] for c in range(len(offs) - 1)]
        self.cores = max(1, min(cores or os.cpu_count() or 1, batch.nsys))
        if len(chains) < self.cores:
            # one group cut into fewer chains than cores: one segment per core instead
            chains = [c for (first, keys), pm in zip(batch.groups, perms)
                      for c in oskr.split_chains([first + int(i) for i in pm],
                                                 max(1, round(self.cores * keys.shape[0] / batch.nsys)))]
        self.cores = min(self.cores, len(chains))
        segs = [[] for _ in range(self.cores)]
        for c, ch in enumerate(chains):
            segs[c % self.cores].append([batch.payload[int(i)] for i in ch])
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for sg in segs:
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, W, sg, warm), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for cn in self.conns:
            assert cn.recv() == "ready"

    def run(self, windows, window_s):
        """Solve for `windows` back-to-back windows of window_s seconds;
        returns (systems finished per window, measured window lengths in s)."""
        for cn in self.conns:
            cn.send("go")
        t0 = time.monotonic()
        edges = [t0 + i * window_s for i in range(windows + 1)]
        while time.monotonic() < edges[-1]:
            time.sleep(min(0.05, max(0.0, edges[-1] - time.monotonic())))
        for cn in self.conns:
            cn.send("stop")
        spans = [sp for cn in self.conns for sp in cn.recv()]
        prog = [_progress(spans, edges[i], edges[i + 1]) for i in range(windows)]
        return prog, [edges[i + 1] - edges[i] for i in range(windows)]

    def rate(self, systems, seconds):
        """Whole-host systems/s with the one-core sort amortised over all systems."""
        if systems <= 0:
            return 0.0
        return 1.0 / (seconds / systems + self.t_sort / self.nsys)

    def close(self):
        for p in self.procs:
            p.join(timeout=5)
            if p.is_alive():
                p.terminate()
                p.join(timeout=5)


def _cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def cpu_baseline(budget_s, W, warm=False, batch=None):
    """One bounded oracle sample beside the GPU line, on every host core."""
    if batch is None:
        batch = _batch(W, W["nsys"], W["seed"])
    ch = OracleChains(W, batch, warm)
    try:
        prog, secs = ch.run(1, budget_s)
    finally:
        ch.close()
    v = ch.rate(prog[0], secs[0])
    return {"value": round(v, 4), "unit": "systems/s", "cores": ch.cores, "kind": "oracle",
            "cpu": _cpu_model(),
            "sample": "%.1f systems finished in a %.0f s window on %d cores (a system straddling the window "
                      "edge counts by its fraction inside), chain segments of the sorted order dealt to the "
                      "cores (the paper's decomposition); the oracle's sort of all %d systems amortised; "
                      "numpy/scipy FP64, BLAS threads = 1 per core"
                      % (prog[0], secs[0], ch.cores, batch.nsys)}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    W = _workload(args)
    batch = _batch(W, W["nsys"], W["seed"], getattr(args, "chains", None))
    ch = OracleChains(W, batch, args.warm_start)
    window = max(1.0, min(args.ref_seconds, 120.0 / max(1, args.steps + args.warmup)))
    try:
        prog, secs = ch.run(args.warmup + args.steps, window)
    finally:
        ch.close()
    prog, secs = prog[args.warmup:], secs[args.warmup:]
    done, wall = sum(prog), sum(secs)
    value = ch.rate(done, wall)
    cb = {"value": round(value, 4), "unit": "systems/s", "cores": ch.cores, "kind": "oracle", "cpu": _cpu_model(),
          "sample": "%d timed windows of %.1f s after %d untimed ones, the oracle solving back to back on %d "
                    "cores, chain segments of the sorted order dealt to the cores (the paper's decomposition); "
                    "%.1f systems finished in the timed windows (a system straddling a window edge counts by "
                    "its fraction inside); the oracle's sort of all %d systems amortised; numpy/scipy FP64, "
                    "BLAS threads = 1 per core"
                    % (args.steps, window, args.warmup, ch.cores, done, batch.nsys)}
    line = {
        "metric": METRIC, "value": cb["value"], "unit": "systems/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(wall / max(1, len(secs)) * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": W["desc"].replace("mixed precision", "mixed-form refinement in FP64")
                   % batch.nsys},
        "cpu_baseline": cb,
        "e2e": {"value": cb["value"], "unit": "systems/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


SERVING_SIZES = {
    # the request mix of the serving workload: 2D Darcy 128^2 - 1024^2 and
    # 3D 7-point Darcy 64^3 - 128^3 (n up to 2.1M), half of each
    "full": ((128, 256, 512, 1024), (64, 96, 128)),
    # a mix that runs in seconds, for quick checks
    "small": ((128, 256), (48, 64)),
}


def _serve(skr, opts, reqs, systems, budget, max_chains):
    """Replay the arrival stream in real time against one server; returns
    (client latencies in ms, server stats, results, wall seconds, submit span)."""
    done, t_done = {}, {}
    with skr.Server(opts, hbm_budget=budget, max_chains=max_chains) as srv:
        tickets, pending = [], []
        t0 = time.perf_counter()

        def collect():
            for t in list(pending):
                out = srv.poll(t)
                if out is not None:
                    done[t] = out
                    t_done[t] = time.perf_counter() - t0
                    pending.remove(t)

        for r, sysr in zip(reqs, systems):
            while time.perf_counter() - t0 < r["t"]:   # arrival time of the request
                collect()
                time.sleep(0.0002)
            t = srv.submit(sysr)
            tickets.append(t)
            pending.append(t)
        submit_span = time.perf_counter() - t0
        while pending:
            if time.perf_counter() - t0 > 1800.0:
                raise TimeoutError("serving stream not drained after 1800 s")
            collect()
            time.sleep(0.0002)
        elapsed = time.perf_counter() - t0
        st = srv.stats()
    # client view: from the scheduled arrival to the poll that returned the result
    lat = sorted((t_done[t] - r["t"]) * 1e3 for r, t in zip(reqs, tickets))
    return lat, st, [done[t][1] for t in tickets], elapsed, submit_span


def _serving_summary(reqs, lat, st, res, elapsed, submit_span):
    pct = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]   # noqa: E731
    return {"value": round(len(reqs) / elapsed, 3), "wall_s": round(elapsed, 2),
            "latency_ms": {"p50": round(pct(0.50), 1), "p99": round(pct(0.99), 1),
                           "mean": round(sum(lat) / len(lat), 1),
                           "measured": "scheduled arrival to the poll that returned the result"},
            "server_latency_ms": {"p50": round(st["p50_ms"], 1), "p99": round(st["p99_ms"], 1),
                                  "measured": "skr_submit return to completion, by the server"},
            "avg_steps": round(sum(r["steps"] for r in res) / len(res), 1),
            "flags": sorted({r["flag"] for r in res}), "max_relres": max(r["relres"] for r in res),
            "chains": st["chains"], "evicted": st["evicted"], "submit_span_s": round(submit_span, 3)}


def run_serving(args):
    """Serving: a seeded Poisson arrival stream of 2D and 3D Darcy requests
    replayed in real time against the server (skr_server_*), with recycling
    (SKR) and, with --serving-plain, again as plain GMRES (k = 0)."""
    # every resident chain has its own stream: give them the most hardware
    # work queues, so that a new request does not queue behind another
    # chain's running solve (must be set before CUDA starts)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch

    _, _, local = _dist()
    torch.cuda.set_device(local)
    import paper_2401_09516_gb300 as skr
    from workloads import serving_stream
    sides2d, sides3d = SERVING_SIZES[args.serving_sizes]
    reqs = serving_stream(args.serving_requests, args.serving_rate, seed=5, sides2d=sides2d, sides3d=sides3d)
    systems = [skr.darcy3d(r["loga"]) if r["ndim"] == 3 else skr.darcy2d(r["loga"]) for r in reqs]

    def opts(k):
        return skr.skr_options_default(m=40, k=k, tol=1e-8, inner_tol=1e-5, precond="jacobi", precision="mixed",
                                       maxit=args.maxit)

    # warm-up on a server of its own (context, module load, first chains)
    with skr.Server(opts(20)) as srv:
        for t in [srv.submit(systems[i]) for i in range(min(4, len(systems)))]:
            srv.wait(t, timeout=600.0)
    budget = int(args.serving_budget_gb * 2**30)
    sampler = ClockSampler(local)
    sampler.start()
    skr_arm = _serving_summary(reqs, *_serve(skr, opts(20), reqs, systems, budget, args.serving_chains))
    plain = None
    if args.serving_plain:
        plain = _serving_summary(reqs, *_serve(skr, opts(0), reqs, systems, budget, args.serving_chains))
    clocks = sampler.stop()
    n3 = sum(1 for r in reqs if r["ndim"] == 3)
    line = {
        "metric": "serving: completed systems/s and arrival-to-result p50/p99 under Poisson arrivals, SKR vs plain GMRES",
        "value": skr_arm["value"], "unit": "systems/s", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": round(skr_arm["wall_s"] * 1e3, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "the first %d requests of the seeded Darcy stream (seed 5), Poisson arrivals at %.0f/s: "
                               "%d 2D (sides %s), %d 3D 7-point (sides %s), a=exp(GRF ell=0.1 sigma=1), Jacobi, "
                               "GCRO-DR m=40 k=20, mixed, tol 1e-8"
                               % (len(reqs), args.serving_rate, len(reqs) - n3, list(sides2d), n3, list(sides3d)),
                   "hbm_budget_gb": args.serving_budget_gb or None, "max_chains": args.serving_chains or 64,
                   "arrival_span_s": round(reqs[-1]["t"], 3)},
        "skr": skr_arm, "plain_gmres": plain,
        "speedup_vs_gmres": None if plain is None else round(skr_arm["value"] / plain["value"], 3),
        "latency_ms": skr_arm["latency_ms"],
        "gpu_launches": len(reqs) * (2 if plain else 1), "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def _grouped_sort_launches(N, p, G):
    """Kernel launches of one skr_sort_grouped call (its host loop, counted)."""
    M = 1024
    while M < N:
        M <<= 1
    bitonic, k = 1, 2048
    while k <= M:
        bitonic += (k.bit_length() - 1) - 10 + 1   # global steps j = k/2 .. 1024, then one local pass
        k <<= 1
    batch = max(1, (1 << 25) // p)
    launches, sets = 2, [N]
    while any(s > G for s in sets):
        nsplit = sum(1 for s in sets if s > G)
        launches += 3 * (-(-nsplit // batch)) + 1 + bitonic + 1
        sets = [h for s in sets for h in ((s // 2, s - s // 2) if s > G else (s,))]
    return launches + (1 + bitonic + 1) + 2


def run_sort_only(args):
    """Time the large-N grouped sort (Sec. 4.1) on N seeded coefficient keys."""
    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2401_09516_gb300 as skr
    N, p, G = (args.nsys or 100000), args.keys_p, args.group_max
    rng = np.random.default_rng(4000 + rank)
    # coefficient keys with a decaying spectrum, like the Chebyshev data of the Poisson workload
    Kh = rng.standard_normal((N, p)) / (1.0 + np.arange(p))[None, :]
    P = torch.tensor(Kh, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        perm, offs = skr.skr_sort_grouped(P, G, stream=stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        perm, offs = skr.skr_sort_grouped(P, G, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    ms = sum(times) / len(times)
    sizes = np.diff(offs)
    line = {
        "metric": "systems/s through the grouped greedy sort (Sec. 4.1, large N)",
        "value": round(N / (ms / 1e3), 1), "unit": "systems/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "grouped sort, N=%d keys of p=%d decaying Gaussian coefficients, groups of at most %d"
                               % (N, p, G),
                   "groups": int(len(sizes)), "group_sizes": [int(sizes.min()), int(sizes.max())],
                   "l2": "flushed between steps (256 MB write)"},
        "gpu_launches": _grouped_sort_launches(N, p, G) * args.steps,
        "clocks": clocks,
    }
    if args.cpu_baseline:
        from oracle import sort as osort
        ns = min(N, 20000)
        t0 = time.perf_counter()
        osort.grouped_sort(Kh[:ns], G)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": round(ns / dt, 1), "unit": "systems/s", "cores": 1, "kind": "oracle",
                                "cpu": _cpu_model(),
                                "sample": "the first %d keys, grouped sort with the same G, numpy FP64, one core" % ns}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="skr", choices=["skr", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS),
                    help="named workload (default %s)" % DEFAULT_WORKLOAD)
    ap.add_argument("--warm-start", action="store_true", help="x_0 = previous solution of the chain")
    ap.add_argument("--eig-fp32", action="store_true",
                    help="mixed form: harmonic-Ritz eigen-solve in FP32 instead of FP64")
    ap.add_argument("--no-sort", action="store_true", help="solve in input order (ablation)")
    ap.add_argument("--precond", default=None, choices=sorted(PRECOND_NAMES),
                    help="override the workload's preconditioner")
    ap.add_argument("--pc-blocks", type=int, default=72,
                    help="row blocks of --precond bjacobi (72: the paper's Darcy runs, one per process)")
    ap.add_argument("--diagnostics", action="store_true", help="report the mean one-sided distance delta")
    ap.add_argument("--chains", type=int, default=None,
                    help="chains the sorted order of a one-group workload is cut into (default: the workload's)")
    ap.add_argument("--cluster-size", type=int, default=None,
                    help="CTAs per chain, a thread-block cluster (default: the workload's; 0 = the library's choice)")
    ap.add_argument("--nsys", type=int, default=None, help="systems per batch (default: the full workload)")
    ap.add_argument("--m", type=int, default=None, help="override the workload's restart length m")
    ap.add_argument("--k", type=int, default=None, help="override the workload's recycle dimension k")
    ap.add_argument("--maxit", type=int, default=100000,
                    help="cap on Arnoldi steps per system, both arms (high enough that plain GMRES converges)")
    ap.add_argument("--gmres-steps", type=int, default=3, help="timed steps of the plain GMRES(m) arm (k = 0)")
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="timed steps of the same SKR solve in the FP64 form (mixed workloads only)")
    ap.add_argument("--no-phases", dest="phases", action="store_false",
                    help="skip the untimed profiled step that reports device time per phase")
    ap.add_argument("--e2e-steps", type=int, default=3, help="timed steps of the end-to-end (host buffers) arm")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--sort-only", action="store_true",
                    help="time the large-N grouped sort instead of the solves (use with --nsys)")
    ap.add_argument("--keys-p", type=int, default=16, help="coordinates per key for --sort-only")
    ap.add_argument("--group-max", type=int, default=1000, help="largest group for --sort-only")
    ap.add_argument("--serving", action="store_true",
                    help="replay a Poisson arrival stream against the serving loop instead of the batch")
    ap.add_argument("--serving-requests", type=int, default=200,
                    help="prefix of the seeded request stream to replay")
    ap.add_argument("--serving-rate", type=float, default=200.0, help="arrivals per second")
    ap.add_argument("--serving-sizes", default="full", choices=sorted(SERVING_SIZES),
                    help="full: 2D 128^2-1024^2 and 3D 64^3-128^3; small: a mix that runs in seconds")
    ap.add_argument("--serving-budget-gb", type=float, default=0.0,
                    help="device-memory budget of the server in GiB (0 = none)")
    ap.add_argument("--serving-chains", type=int, default=0, help="resident chain limit (0 = 64)")
    ap.add_argument("--serving-plain", action="store_true",
                    help="replay the same stream again with plain GMRES (k = 0); on the full mix plain GMRES "
                         "needs tens of thousands of steps on the 1024^2 and 128^3 requests")
    ap.add_argument("--ref-seconds", type=float, default=20.0,
                    help="upper bound on one reference sample")
    args = ap.parse_args()
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    if args.sort_only:
        run_sort_only(args)
    elif args.serving:
        run_serving(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
