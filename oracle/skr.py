"""A sorted sequence of systems solved with recycling (oracle, float64).

Fig. 2 steps c-e: sort the systems (Algorithm 1), then solve them in that
order, carrying U_k from each solve to the next (Algorithm 2, last line)
and refreshing it against the new matrix (App. B.1).  App. E.2.2 cuts the
sorted list into independent chains; `solve_sequence` does the same when
nchains > 1 (contiguous, near-equal pieces).

Each system is solved by residual refinement around GCRO-DR:
  x = 0; repeat: r = b - A x (float64); stop if ||r|| <= tol ||b||;
  solve A M^-1 d = r by GCRO-DR to the inner target; x += M^-1 d.
For the "fp64" form the inner target is tol ||b|| (one pass normally
suffices; the loop only confirms it on the true residual).  For the
"mixed" form the inner target is max(inner_tol ||r||, tol ||b||), the
structure the GPU path runs with single-precision inner solves; the oracle
runs that same structure in float64.  The "fp32-emulated" form runs the
mixed structure with every vector of the inner solves (and the carried
U_k, C_k) rounded to float32 after each vector operation, the small dense
step, x, the true residual and the refinement staying float64: it states
the error the mixed form should show, without the GPU's summation orders.
"""
import numpy as np

from . import assembly
from .precond import RightPreconditioner
from .krylov import RecycleState, refresh, gcrodr_solve, one_sided_distance, round32


def grid_of(system):
    """Interior grid shape of a system description (None for a bare matrix)."""
    kind = system["kind"]
    if kind in ("darcy2d", "darcy3d"):
        return tuple(s - 2 for s in np.shape(system["loga"]))
    if kind == "convdiff2d":
        return (system["nside"], system["nside"])
    if kind == "helmholtz2d":
        return tuple(np.shape(system["k"]))
    if kind == "poisson2d":
        return tuple(np.shape(system["f"]))
    return system.get("grid")


def assemble(system):
    """Build (A, b) for one system description (a dict from the workload module)."""
    kind = system["kind"]
    if kind == "darcy2d":
        return assembly.darcy2d(system["loga"], rhs=system.get("rhs"))
    if kind == "darcy3d":
        return assembly.darcy3d(system["loga"], rhs=system.get("rhs"))
    if kind == "convdiff2d":
        return assembly.convdiff2d(system["nu"], system["beta"], system["nside"],
                                   rhs=system.get("rhs"))
    if kind == "helmholtz2d":
        return assembly.helmholtz2d(system["k"], rhs=system.get("rhs"))
    if kind == "poisson2d":
        return assembly.poisson2d_dirichlet(system["f"], *system["g"])
    if kind == "matrix":
        return system["A"], system["b"]
    raise ValueError(kind)


def solve_system(A, b, precond, m, k, tol, state, precision="fp64", inner_tol=1e-5,
                 max_refine=10, max_steps=10**4, grid=None, x0=None, pc_blocks=1):
    """Solve one system, updating the carried recycle state in place.

    x0 is Algorithm 2's initial guess (default 0); pc_blocks is block
    Jacobi's block count.

    Returns (x, info) with info = dict(steps, cycles, matvecs, refinements,
    relres, converged).  `steps` counts Arnoldi steps (one operator
    application each); `matvecs` also counts the k products of the refresh.
    """
    if precision not in ("fp64", "mixed", "fp32-emulated"):
        raise ValueError(precision)
    rnd = round32 if precision == "fp32-emulated" else None
    M = RightPreconditioner(A, precond, grid, blocks=pc_blocks)

    def op(v):
        return A @ M.apply(v)

    stats = dict(steps=0, cycles=0, matvecs=0, refinements=0, delta=-1.0)
    stats["matvecs"] += refresh(op, state, rnd)
    C_in = None if state.C is None else state.C.copy()
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    if bnorm == 0.0:
        stats.update(relres=0.0, converged=True)
        return x, stats
    for _ in range(max_refine):
        r = b - A @ x
        rn = np.linalg.norm(r)
        if rn <= tol * bnorm or stats["steps"] >= max_steps:
            break
        if precision == "fp64":
            tol_abs = tol * bnorm
        else:
            tol_abs = max(inner_tol * rn, tol * bnorm)
        d, _ = gcrodr_solve(op, r, m, k, tol_abs, state, max_steps, stats, rnd=rnd)
        x = x + M.apply(d)
        stats["refinements"] += 1
    relres = np.linalg.norm(b - A @ x) / bnorm
    stats.update(relres=relres, converged=bool(relres <= tol))
    if C_in is not None and state.C is not None and state.C.shape[1] > 0:
        # how far this system moved the recycle space it was handed (Eq. 5)
        stats["delta"] = one_sided_distance(state.C, C_in)
    return x, stats


def split_chains(order, nchains):
    """Cut an order into nchains contiguous, near-equal chains (App. E.2.2)."""
    order = list(order)
    N = len(order)
    nchains = max(1, min(nchains, N)) if N else 1
    bounds = [(c * N) // nchains for c in range(nchains + 1)]
    return [order[bounds[c]:bounds[c + 1]] for c in range(nchains)]


def solve_sequence(systems, order, precond, m, k, tol, precision="fp64", nchains=1,
                   inner_tol=1e-5, max_refine=10, max_steps=10**4, warm_start=False, pc_blocks=1):
    """Solve systems[order[0]], systems[order[1]], ... carrying U_k along each chain.

    warm_start: x0 of a system is the previous solution of its chain (the
    first system of every chain starts from 0).  Returns (xs, infos), lists
    indexed like `systems`.
    """
    xs = [None] * len(systems)
    infos = [None] * len(systems)
    for chain in split_chains(order, nchains):
        state = RecycleState()
        prev = None
        for idx in chain:
            A, b = assemble(systems[idx])
            x, info = solve_system(A, b, precond, m, k, tol, state, precision, inner_tol,
                                   max_refine, max_steps, grid=grid_of(systems[idx]),
                                   x0=prev if warm_start else None, pc_blocks=pc_blocks)
            xs[idx] = x
            infos[idx] = info
            prev = x
    return xs, infos
