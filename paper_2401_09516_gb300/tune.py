"""Launch-shape autotuner: measures the chain kernel on this GPU and writes
the table the library plans its launches with (csrc/skr_tuned.inc).

For every grid size n in a ladder of 2D Darcy problems and every cluster
size cs in {1, 2, 4, 8, 16}, it fills the GPU with as many clusters of cs
CTAs as fit at once, each solving a short chain of two systems (so the
recycled path, the App. B.1 refresh included, is part of the sample) with
the Arnoldi step count capped, and records the time per Arnoldi step of one
cluster: kernel time x clusters / total Arnoldi steps.  With every SM busy,
that is the time a chain of such systems takes per step when batched with
others.  The library then sizes each chain's cluster from the table and
shares the SMs between chains of different sizes (skr_solve_sequence with
cluster_size = 0; the serving loop).

Run on the GPU the library will run on:
    python -m paper_2401_09516_gb300.tune [--out path] [--quick]
"""
import argparse
import datetime
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
TABLE = os.path.join(HERE, "csrc", "skr_tuned.inc")
CLUSTER_SIZES = (1, 2, 4, 8, 16)
SIDES = (32, 64, 96, 128, 192, 256, 384, 512, 768)


def measure(skr, torch, side, cs, steps_cap=240, systems_per_chain=2, seed=0):
    """Microseconds per Arnoldi step of one cluster of cs CTAs on side^2
    Darcy systems (Jacobi, mixed precision, m = 40, k = 20) with the GPU full."""
    from workloads import darcy2d_sequence

    dev = torch.device("cuda", torch.cuda.current_device())
    opt = skr.skr_options_default(m=40, k=20, tol=1e-12, inner_tol=1e-5, precond="jacobi", precision="mixed",
                                  cluster_size=cs, maxit=steps_cap, max_refine=2)
    # as many clusters as can be resident (one chain each): a probe launch of
    # more tiny chains than clusters fit reports the resident count as its slots
    tiny = torch.tensor(darcy2d_sequence(8, 1, 0.1, seed=seed)[0], device=dev)
    nprobe = 2 * (160 // cs) + 8
    skr.skr_solve_sequence([skr.darcy2d(tiny)] * nprobe, nchains=nprobe, options=opt)
    slots = max(1, skr.skr_last_stats()["slots"])
    nsys = systems_per_chain * slots
    # fields are reused across chains: the timing does not depend on them
    L = darcy2d_sequence(side, systems_per_chain, 0.1, seed=seed)
    fields = [torch.tensor(L[i], device=dev) for i in range(systems_per_chain)]
    systems = [skr.darcy2d(fields[i % systems_per_chain]) for i in range(nsys)]
    x = [torch.empty(side * side, dtype=torch.float64, device=dev) for _ in range(nsys)]
    opt.max_slots = slots
    for rep in range(2):            # the first launch warms up
        _, res = skr.skr_solve_sequence(systems, nchains=slots, options=opt, x_out=x)
        st = skr.skr_last_stats()
    steps = sum(r["steps"] for r in res)
    return st["kernel_ms"] * 1e3 * st["slots"] / max(1, steps), st["slots"]


def write_table(rows, path, gpu, note):
    ns = [r["n"] for r in rows]
    lines = [
        "// Measured launch-shape table of the chain kernel (written by",
        "// paper_2401_09516_gb300/tune.py; do not edit by hand).",
        "// %s" % note,
        "// GPU: %s" % gpu,
        "// Row i: 2D Darcy systems of SKR_TUNE_N[i] unknowns (Jacobi, mixed precision,",
        "// m = 40, k = 20); column j: clusters of SKR_TUNE_CS[j] CTAs, as many as fit at",
        "// once; value: microseconds per Arnoldi step of one cluster (cycle ends and",
        "// the recycle refresh included, amortised).",
        "#define SKR_TUNE_ROWS %d" % len(rows),
        "#define SKR_TUNE_COLS %d" % len(CLUSTER_SIZES),
        "static const int SKR_TUNE_CS[SKR_TUNE_COLS] = {%s};" % ", ".join(str(c) for c in CLUSTER_SIZES),
        "static const long long SKR_TUNE_N[SKR_TUNE_ROWS] = {%s};" % ", ".join(str(n) for n in ns),
        "static const double SKR_TUNE_US[SKR_TUNE_ROWS][SKR_TUNE_COLS] = {",
    ]
    for r in rows:
        lines.append("    {%s}," % ", ".join("%.3f" % r["us"][str(c)] for c in CLUSTER_SIZES))
    lines.append("};")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--json", default=None, help="also write the raw measurements here")
    ap.add_argument("--quick", action="store_true", help="fewer grid sizes (a smoke run)")
    args = ap.parse_args()
    sys.path.insert(0, ROOT)
    import torch
    import paper_2401_09516_gb300 as skr

    sides = (32, 128, 384) if args.quick else SIDES
    rows = []
    t0 = time.time()
    for side in sides:
        us = {}
        for cs in CLUSTER_SIZES:
            try:
                v, slots = measure(skr, torch, side, cs)
            except skr.SkrError as e:      # a shape that cannot be scheduled is never planned
                print("side %d cs %d: %s" % (side, cs, e), flush=True)
                v, slots = 1e30, 0
            us[str(cs)] = v
            print("side %4d n %7d cs %2d clusters %3d: %9.2f us/step" % (side, side * side, cs, slots, v), flush=True)
        rows.append({"side": side, "n": side * side, "us": us})
    gpu = torch.cuda.get_device_name()
    note = "measured %s in %.0f s" % (datetime.datetime.utcnow().strftime("%Y-%m-%d"), time.time() - t0)
    write_table(rows, args.out, gpu, note)
    if args.json:
        with open(args.json, "w") as fh:
            json.dump({"gpu": gpu, "rows": rows}, fh, indent=1)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
