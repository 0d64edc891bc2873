"""Arnoldi, restarted GMRES and GCRO-DR with recycling (oracle, float64).

Sec. 3.2 (Eq. 2-3): the Arnoldi relation A V_m = V_{m+1} Hbar_m.
Sec. 4.2 (Eq. 4) and Algorithm 2 (App. B.2): GCRO-DR, whose Arnoldi steps
use the projected operator (I - C C^T) A.  App. B.1: the recycle refresh
C = Q, U = U_old R^-1 from the reduced QR of A_new U_old.
GMRES is GCRO-DR with k = 0 (Sec. 4.2), and `gcrodr_solve` with k = 0 is
exactly restarted GMRES(m).

Everything is real (the paper allows complex systems; this build does not).

Readings taken where Algorithm 2 is silent:
  * a cycle stops early at the first Arnoldi step whose least-squares
    residual is <= tol; such a cycle still updates x and r but does not
    recompute the recycle space (the stopping test of the while loop then
    ends the solve);
  * when the first cycle stops early, no recycle space exists yet and the
    next solve starts in the "no recycle space" branch again;
  * the LSQ right-hand side W^T r is formed explicitly;
  * every cycle that has a recycle space starts with the projection of the
    first step of Algorithm 2 (x += U C^T r, r -= C C^T r), which is a no-op
    in exact arithmetic and keeps v_1 orthogonal to C in floating point;
  * D_k = diag(1/||u_j||);
  * QR factorisations are normalised to a positive diagonal of R;
  * harmonic Ritz selection: the k eigenvalues of smallest modulus, ties
    broken by real then imaginary part; a complex conjugate pair contributes
    the real and imaginary parts of one eigenvector; a pair that the k-th
    pick would split is dropped, leaving k-1 vectors;
  * orthogonalisation: two Gram-Schmidt passes (classical against C_k,
    modified against V_j), accumulating the coefficients.

Pins (tests/test_oracle_krylov.py): dense-LU solutions on small grids;
orthonormality of V and C; A U = C; the projected Arnoldi relation (Eq. 4);
k = 0 reproduces GMRES; identical consecutive systems converge in far fewer
steps (delta = gamma = 0, Sec. 5.1); harmonic Ritz values on a complete
Krylov space equal the closed-form Laplacian eigenvalues; the harmonic
Petrov-Galerkin condition for both branches of Algorithm 2; the selection
rule on a hand-made spectrum (order, ties, conjugate pairs, the split
rule); and, on a complete space, the subspace selected by either branch
spans the closed-form eigenvectors of the k smallest eigenvalues.
"""
import numpy as np
import scipy.linalg as sla


def qr_pos(X):
    """Reduced QR with diag(R) > 0 (the unique normalisation)."""
    Q, R = np.linalg.qr(X)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :], R * s[:, None]


def select_smallest(theta, Z, k):
    """Real basis of the eigenvectors of the k smallest-|theta| eigenvalues.

    theta complex[m], Z complex[m, m] (columns are eigenvectors).
    Returns P real[m, k_eff] with k_eff in {k-1, k} (see module readings).
    """
    theta = np.asarray(theta, dtype=np.complex128)
    mag = np.abs(theta)
    mag = np.where(np.isfinite(mag), mag, np.inf)
    order = sorted(range(len(theta)),
                   key=lambda i: (mag[i], np.nan_to_num(theta[i].real, nan=np.inf),
                                  np.nan_to_num(theta[i].imag, nan=np.inf)))
    chosen = order[:k]
    chosen_set = set(chosen)
    cols = []
    done = set()
    for i in chosen:
        if i in done:
            continue
        if theta[i].imag == 0.0:
            cols.append(np.real(Z[:, i]))
            done.add(i)
            continue
        # complex: find its conjugate partner
        partner = None
        for j in range(len(theta)):
            if j != i and j not in done and theta[j] == np.conj(theta[i]):
                partner = j
                break
        if partner is None or partner not in chosen_set:
            done.add(i)          # split pair: drop it
            continue
        cols.append(np.real(Z[:, i]))
        cols.append(np.imag(Z[:, i]))
        done.add(i)
        done.add(partner)
    if not cols:
        return np.zeros((Z.shape[0], 0))
    return np.stack(cols, axis=1)


def round32(a):
    """Round to the nearest float32 and back: the FP32-emulating variant's
    rounding after every vector-level operation."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def _same(a):
    return a


def lsq_residual(Hbar, beta):
    """min_y || beta e1 - Hbar y || and its minimiser."""
    rhs = np.zeros(Hbar.shape[0])
    rhs[0] = beta
    y = np.linalg.lstsq(Hbar, rhs, rcond=None)[0]
    return np.linalg.norm(rhs - Hbar @ y), y


def arnoldi(op, r, steps, C, tol_abs, rnd=None):
    """Arnoldi with the operator (I - C C^T) op, v1 = r/||r|| (Eq. 2-4).

    Returns dict(V n x (j+1), Hbar (j+1) x j, B kc x j, j, early, matvecs).
    Stops early when the GMRES least-squares residual on Hbar is <= tol_abs
    (for GCRO-DR this equals the residual of the full LSQ problem, because
    the D_k block of G can always cancel the C rows).  rnd (default: none)
    rounds the result of every vector operation and reduction.
    """
    rnd = rnd or _same
    n = r.size
    beta = float(rnd(np.linalg.norm(r)))
    kc = 0 if C is None else C.shape[1]
    V = np.zeros((n, steps + 1))
    H = np.zeros((steps + 1, steps))
    B = np.zeros((kc, steps))
    V[:, 0] = rnd(r / beta)
    j_done = steps
    early = False
    for j in range(steps):
        w = rnd(op(V[:, j]))
        nrm_in = np.linalg.norm(w)
        for _ in range(2):
            if kc:
                c = rnd(C.T @ w)
                B[:, j] += c
                w = rnd(w - C @ c)
            for i in range(j + 1):
                hij = float(rnd(V[:, i] @ w))
                H[i, j] += hij
                w = rnd(w - hij * V[:, i])
        hn = float(rnd(np.linalg.norm(w)))
        H[j + 1, j] = hn
        breakdown = hn <= 1e-14 * max(nrm_in, 1e-300)
        if not breakdown:
            V[:, j + 1] = rnd(w / hn)
        res, _ = lsq_residual(H[: j + 2, : j + 1], beta)
        if res <= tol_abs or breakdown:
            j_done = j + 1
            early = j_done < steps or breakdown
            break
    return dict(V=V[:, : j_done + 1], Hbar=H[: j_done + 1, : j_done], B=B[:, :j_done],
                j=j_done, early=early, beta=beta)


def harmonic_ritz_first(Hbar, k):
    """Algorithm 2, no-recycle branch: eigenvectors of
    H_m + h_{m+1,m}^2 H_m^-T e_m e_m^T for the k smallest |theta|."""
    m = Hbar.shape[1]
    Hm = Hbar[:m, :m]
    em = np.zeros(m)
    em[-1] = 1.0
    f = np.linalg.solve(Hm.T, em)
    T = Hm + Hbar[m, m - 1] ** 2 * np.outer(f, em)
    theta, Z = np.linalg.eig(T)
    return select_smallest(theta, Z, k), theta


def harmonic_ritz_general(G, What, Vhat, k):
    """Algorithm 2, recycle branch: G^T G z = theta G^T W^T V z, k smallest |theta|."""
    A1 = G.T @ G
    A2 = G.T @ (What.T @ Vhat)
    theta, Z = sla.eig(A1, A2)
    return select_smallest(theta, Z, k), theta


def one_sided_distance(Q, C):
    """Eq. 5 (Sec. 5.1): delta(Q, C) = ||(I - Pi_C) Pi_Q||_2 for orthonormal bases Q, C.

    With G = C^T Q, (I - Pi_C) Pi_Q restricted to range(Q) has Gram matrix
    I - G^T G, so delta is the square root of its largest eigenvalue.
    """
    G = C.T @ Q
    lam = np.linalg.eigvalsh(np.eye(Q.shape[1]) - G.T @ G)
    return float(np.sqrt(min(max(lam[-1], 0.0), 1.0)))


class RecycleState:
    """What one system hands to the next: U_k (as Y_tilde) and C_k."""

    def __init__(self):
        self.U = None
        self.C = None

    @property
    def k(self):
        return 0 if self.U is None else self.U.shape[1]


def refresh(op, state, rnd=None):
    """App. B.1: [Q, R] = qr(A_new U_old); C = Q; U = U_old R^-1.  Returns matvecs used."""
    rnd = rnd or _same
    if state.U is None or state.k == 0:
        return 0
    AY = np.stack([rnd(op(state.U[:, i])) for i in range(state.k)], axis=1)
    Q, R = qr_pos(AY)
    state.C = rnd(Q)
    state.U = rnd(np.linalg.solve(R.T, state.U.T).T)   # U_old R^-1
    return state.k


def gcrodr_solve(op, r0, m, k, tol_abs, state, max_steps=10**4, stats=None, rnd=None):
    """Solve op(d) = r0 from d = 0 by GCRO-DR(m, k) (Algorithm 2).

    op        callable v -> A_hat v (the right-preconditioned operator)
    state     RecycleState, updated in place (U, C valid for op on return)
    tol_abs   stop when ||r|| <= tol_abs
    rnd       rounding after every vector operation (default: none); the
              small dense step (least squares, eigenproblem, QR) stays FP64
    Returns (d, r); `stats` (dict) accumulates steps, cycles, matvecs.
    """
    rnd = rnd or _same
    if stats is None:
        stats = {}
    for key in ("steps", "cycles", "matvecs"):
        stats.setdefault(key, 0)
    history = stats.setdefault("history", [])
    n = r0.size
    d = np.zeros(n)
    r = rnd(np.array(r0, dtype=np.float64, copy=True))
    if state.U is not None and state.k > 0:
        z = rnd(state.C.T @ r)                  # x1 = x0 + U C^T r0
        d = rnd(d + state.U @ z)
        r = rnd(r - state.C @ z)                # r1 = r0 - C C^T r0
    while np.linalg.norm(r) > tol_abs and stats["steps"] < max_steps:
        kc = state.k
        budget = max_steps - stats["steps"]
        if kc == 0:
            # GMRES cycle of m steps (the "else" branch of Algorithm 2)
            ar = arnoldi(op, r, min(m, budget), None, tol_abs, rnd)
            j = ar["j"]
            stats["steps"] += j
            stats["matvecs"] += j
            stats["cycles"] += 1
            Hbar, V = ar["Hbar"], ar["V"]
            _, y = lsq_residual(Hbar, ar["beta"])
            d = rnd(d + V[:, :j] @ y)
            r = rnd(r - V @ (Hbar @ y))
            if k > 0 and not ar["early"] and j == m:
                P, _ = harmonic_ritz_first(Hbar, k)
                if P.shape[1] > 0:
                    Yt = V[:, :m] @ P
                    Q, R = qr_pos(Hbar @ P)
                    state.C = rnd(V @ Q)
                    state.U = rnd(np.linalg.solve(R.T, Yt.T).T)
        else:
            # re-apply the projection of Algorithm 2's first step (x += U C^T r,
            # r -= C C^T r): a no-op in exact arithmetic (r is orthogonal to C
            # after every cycle), it keeps v_1 = r/||r|| orthogonal to C in
            # floating point once ||r|| has dropped far below its earlier values
            z = rnd(state.C.T @ r)
            d = rnd(d + state.U @ z)
            r = rnd(r - state.C @ z)
            steps = min(m - kc, budget)
            ar = arnoldi(op, r, steps, state.C, tol_abs, rnd)
            j = ar["j"]
            stats["steps"] += j
            stats["matvecs"] += j
            stats["cycles"] += 1
            U, C = state.U, state.C
            Dk = 1.0 / np.linalg.norm(U, axis=0)
            Ut = U * Dk[None, :]
            Vhat = np.concatenate([Ut, ar["V"][:, :j]], axis=1)
            What = np.concatenate([C, ar["V"]], axis=1)
            G = np.zeros((kc + j + 1, kc + j))
            G[:kc, :kc] = np.diag(Dk)
            G[:kc, kc:] = ar["B"]
            G[kc:, kc:] = ar["Hbar"]
            y = np.linalg.lstsq(G, rnd(What.T @ r), rcond=None)[0]
            d = rnd(d + Vhat @ y)
            r = rnd(r - What @ (G @ y))
            if not ar["early"] and j == m - kc:
                P, _ = harmonic_ritz_general(G, What, Vhat, k)
                if P.shape[1] > 0:
                    Yt = Vhat @ P
                    Q, R = qr_pos(G @ P)
                    state.C = rnd(What @ Q)
                    state.U = rnd(np.linalg.solve(R.T, Yt.T).T)
        history.append(np.linalg.norm(r))
    return d, r
