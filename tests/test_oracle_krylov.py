"""Pins for the oracle's preconditioners, Arnoldi, GMRES and GCRO-DR."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import assembly, krylov, precond, skr
from oracle import precond as oprecond
from workloads import darcy2d_sequence


def _darcy(N, seed=0, ell=0.2):
    loga = darcy2d_sequence(N, 1, ell, seed=seed)[0]
    return assembly.darcy2d(loga)


# ---------------------------------------------------------------- preconditioners

def test_ilu0_of_tridiagonal_is_exact_lu():
    n = 12
    rng = np.random.default_rng(0)
    main = 4.0 + rng.uniform(size=n)
    A = sp.diags([rng.uniform(-1, 0, n - 1), main, rng.uniform(-1, 0, n - 1)], [-1, 0, 1], format="csr")
    L, U = precond.ilu0(A)
    np.testing.assert_allclose((L @ U).toarray(), A.toarray(), rtol=1e-14, atol=1e-14)


def test_ilu0_matches_a_on_its_pattern_and_has_no_fill():
    A, _ = assembly.convdiff2d(0.05, (20.0, 7.0), 6)
    L, U = precond.ilu0(A)
    LU = (L @ U).toarray()
    Ad = A.toarray()
    mask = Ad != 0
    np.testing.assert_allclose(LU[mask], Ad[mask], rtol=1e-13, atol=1e-12)
    assert set(zip(*L.nonzero())) <= set(zip(*np.nonzero(np.tril(Ad, -1) + np.eye(36))))
    assert set(zip(*U.nonzero())) <= set(zip(*np.nonzero(np.triu(Ad))))
    # and ILU(0) is not the exact LU for the 5-point pattern (fill is dropped)
    assert np.abs(LU - Ad).max() > 1e-6


@pytest.mark.parametrize("grid", [(6, 5), (6, 6), (4, 3, 5)])
def test_redblack_ilu0_closed_form(grid):
    # in red-black order the red rows of L and U carry no elimination, the
    # black pivots are a_bb - sum_r a_br a_rb / a_rr, and the red rows of
    # A M^-1 are unit rows
    rng = np.random.default_rng(len(grid))
    if len(grid) == 2:
        A, _ = assembly.convdiff2d(0.05, (17.0, -9.0), grid[0]) if grid[0] == grid[1] else \
            assembly.darcy2d(rng.standard_normal((grid[0] + 2, grid[1] + 2)))
    else:
        A, _ = assembly.darcy3d(rng.standard_normal(tuple(g + 2 for g in grid)))
    perm, L, U = oprecond.ilu0_redblack(A, grid)
    Ap = A.toarray()[perm][:, perm]
    nred = int((np.indices(grid).reshape(len(grid), -1).sum(0) % 2 == 0).sum())
    Ud = U.diagonal()
    np.testing.assert_allclose(Ud[:nred], np.diag(Ap)[:nred], rtol=1e-15)
    for bi in range(nred, Ap.shape[0]):
        reds = np.nonzero(Ap[bi, :nred])[0]
        want = Ap[bi, bi] - sum(Ap[bi, r] * Ap[r, bi] / Ap[r, r] for r in reds)
        assert np.isclose(Ud[bi], want, rtol=1e-13)
    M = oprecond.RightPreconditioner(A, "ilu0", grid)
    AM = np.stack([A @ M.apply(e) for e in np.eye(A.shape[0])], axis=1)
    reds_nat = perm[:nred]
    np.testing.assert_allclose(AM[reds_nat], np.eye(A.shape[0])[reds_nat], atol=1e-12)


def test_jacobi_right_preconditioner():
    A, _ = _darcy(5)
    M = precond.RightPreconditioner(A, "jacobi")
    v = np.arange(25.0)
    np.testing.assert_allclose(M.apply(v), v / A.diagonal(), rtol=1e-15)


# ---------------------------------------------------------------- Arnoldi (Eq. 2-4)

def test_arnoldi_relation_and_orthonormality():
    A, b = _darcy(8)
    op = lambda v: A @ v
    ar = krylov.arnoldi(op, b, 20, None, 0.0)
    V, H = ar["V"], ar["Hbar"]
    j = ar["j"]
    assert j == 20
    AV = np.stack([op(V[:, i]) for i in range(j)], axis=1)
    np.testing.assert_allclose(AV, V @ H, atol=1e-10 * np.abs(AV).max())
    np.testing.assert_allclose(V.T @ V, np.eye(j + 1), atol=1e-12)


def test_projected_arnoldi_relation_eq4():
    A, b = _darcy(8)
    op = lambda v: A @ v
    rng = np.random.default_rng(1)
    C, _ = krylov.qr_pos(rng.standard_normal((64, 5)))
    r = b - C @ (C.T @ b)
    ar = krylov.arnoldi(op, r, 15, C, 0.0)
    V, H, B = ar["V"], ar["Hbar"], ar["B"]
    AV = np.stack([op(V[:, i]) for i in range(15)], axis=1)
    lhs = AV - C @ (C.T @ AV)
    np.testing.assert_allclose(lhs, V @ H, atol=1e-10 * np.abs(AV).max())
    np.testing.assert_allclose(B, C.T @ AV, atol=1e-10 * np.abs(AV).max())
    assert np.abs(C.T @ V).max() < 1e-12


# ---------------------------------------------------------------- GMRES / GCRO-DR solves

@pytest.mark.parametrize("k", [0, 4])
@pytest.mark.parametrize("pc", ["none", "jacobi", "ilu0"])
def test_solution_matches_dense_lu(k, pc):
    A, b = _darcy(10, seed=2)
    state = krylov.RecycleState()
    x, info = skr.solve_system(A, b, pc, 12, k, 1e-10, state, grid=(10, 10))
    xd = np.linalg.solve(A.toarray(), b)
    assert info["converged"] and info["relres"] <= 1e-10
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)


def test_k0_is_restarted_gmres_library():
    # GCRO-DR with k = 0 is GMRES(m) (Sec. 4.2); compare with SciPy's GMRES(m)
    A, b = _darcy(12, seed=4)
    m, tol = 10, 1e-9
    state = krylov.RecycleState()
    stats = {}
    d, r = krylov.gcrodr_solve(lambda v: A @ v, b, m, 0, tol * np.linalg.norm(b), state, 5000, stats)
    count = []
    xs, _ = spla.gmres(A, b, rtol=tol, atol=0.0, restart=m, maxiter=1000,
                       callback=lambda pr: count.append(pr), callback_type="pr_norm")
    assert abs(stats["steps"] - len(count)) <= 2, (stats["steps"], len(count))
    np.testing.assert_allclose(d, xs, rtol=0, atol=1e-6 * np.linalg.norm(xs))


def test_gmres_cycle_residuals_monotone():
    A, b = _darcy(12, seed=5)
    for k in (0, 5):
        stats = {}
        krylov.gcrodr_solve(lambda v: A @ v, b, 10, k, 1e-9 * np.linalg.norm(b),
                            krylov.RecycleState(), 5000, stats)
        h = np.array(stats["history"])
        assert np.all(np.diff(h) <= 1e-12 * h[:-1]), h


def test_recycle_invariants_after_solve():
    A, b = _darcy(12, seed=6)
    op = lambda v: A @ v
    state = krylov.RecycleState()
    krylov.gcrodr_solve(op, b, 20, 6, 1e-10 * np.linalg.norm(b), state, 5000, {})
    U, C = state.U, state.C
    assert U.shape[1] in (5, 6)
    np.testing.assert_allclose(C.T @ C, np.eye(C.shape[1]), atol=1e-12)
    AU = np.stack([op(U[:, i]) for i in range(U.shape[1])], axis=1)
    assert np.linalg.norm(AU - C) <= 1e-10 * np.linalg.norm(C)


def test_refresh_gives_orthonormal_c_and_au_equals_c():
    A1, b1 = _darcy(12, seed=7)
    A2, _ = _darcy(12, seed=8)
    state = krylov.RecycleState()
    krylov.gcrodr_solve(lambda v: A1 @ v, b1, 20, 6, 1e-9 * np.linalg.norm(b1), state, 5000, {})
    U_old = state.U.copy()
    krylov.refresh(lambda v: A2 @ v, state)
    AU = A2 @ state.U
    np.testing.assert_allclose(AU, state.C, atol=1e-10 * np.abs(AU).max())
    np.testing.assert_allclose(state.C.T @ state.C, np.eye(state.k), atol=1e-12)
    # span(U) unchanged by the refresh
    Qo, _ = np.linalg.qr(U_old)
    Qn, _ = np.linalg.qr(state.U)
    s = np.linalg.svd(Qo.T @ Qn, compute_uv=False)
    assert np.all(s > 1 - 1e-10)


def test_identical_consecutive_systems_converge_much_faster():
    # C spans an approximate invariant subspace of the same matrix: the
    # delta = gamma = 0 case of the convergence bound (Sec. 5.1)
    loga = darcy2d_sequence(16, 1, 0.2, seed=11)[0]
    systems = [dict(kind="darcy2d", loga=loga)] * 3
    xs, infos = skr.solve_sequence(systems, [0, 1, 2], "none", 20, 8, 1e-8)
    _, plain = skr.solve_sequence(systems, [0, 1, 2], "none", 20, 0, 1e-8)
    steps = [i["steps"] for i in infos]
    assert steps[1] < 0.75 * steps[0], steps
    assert steps[1] < 0.5 * plain[1]["steps"], (steps, plain[1]["steps"])
    for i in infos:
        assert i["converged"]


def test_recycling_beats_gmres_on_a_sorted_sequence():
    L = darcy2d_sequence(16, 6, 0.2, seed=12)
    systems = [dict(kind="darcy2d", loga=l) for l in L]
    from oracle import sort
    order = sort.greedy_sort(L.reshape(6, -1))
    _, g = skr.solve_sequence(systems, order, "none", 20, 0, 1e-8)
    _, s = skr.solve_sequence(systems, order, "none", 20, 8, 1e-8)
    assert sum(i["steps"] for i in s) < 0.7 * sum(i["steps"] for i in g)


# ---------------------------------------------------------------- harmonic Ritz

def test_harmonic_ritz_full_space_gives_exact_eigenvalues():
    # with m = n the Krylov space is the whole space, h_{m+1,m} = 0 and the
    # harmonic Ritz values are the eigenvalues (closed form for a = 1; a
    # 3 x 5 grid has distinct eigenvalues, so the Krylov space is complete)
    nx, ny = 3, 5
    A, _ = assembly.darcy2d(np.zeros((nx + 2, ny + 2)))
    n = nx * ny
    rng = np.random.default_rng(2)
    ar = krylov.arnoldi(lambda v: A @ v, rng.standard_normal(n), n, None, 0.0)
    H = ar["Hbar"]
    assert H.shape[1] == n
    _, theta = krylov.harmonic_ritz_first(H, 3)
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    lx = 4.0 / hx**2 * np.sin(np.arange(1, nx + 1) * np.pi * hx / 2) ** 2
    ly = 4.0 / hy**2 * np.sin(np.arange(1, ny + 1) * np.pi * hy / 2) ** 2
    closed = np.sort((lx[:, None] + ly[None, :]).ravel())
    np.testing.assert_allclose(np.sort(theta.real), closed, rtol=1e-8)
    assert np.abs(theta.imag).max() < 1e-8 * closed.max()


def test_first_cycle_pairs_satisfy_harmonic_petrov_galerkin():
    A, b = _darcy(10, seed=3)
    op = lambda v: A @ v
    ar = krylov.arnoldi(op, b, 15, None, 0.0)
    V, H = ar["V"], ar["Hbar"]
    m = H.shape[1]
    Hm = H[:m, :m]
    em = np.zeros(m); em[-1] = 1
    T = Hm + H[m, m - 1] ** 2 * np.outer(np.linalg.solve(Hm.T, em), em)
    theta, Z = np.linalg.eig(T)
    AV = np.stack([op(V[:, i]) for i in range(m)], axis=1)
    for i in range(m):
        y = V[:, :m] @ Z[:, i]
        res = AV @ Z[:, i] - theta[i] * y
        assert np.abs(AV.T @ res).max() <= 1e-8 * np.abs(theta[i]) * np.linalg.norm(AV) * np.linalg.norm(y)


def test_general_cycle_pairs_satisfy_harmonic_petrov_galerkin():
    A, b = _darcy(10, seed=4)
    op = lambda v: A @ v
    state = krylov.RecycleState()
    krylov.gcrodr_solve(op, b, 15, 5, 1e-3 * np.linalg.norm(b), state, 15, {})
    U, C = state.U, state.C
    kc = U.shape[1]
    r = b - C @ (C.T @ b)
    ar = krylov.arnoldi(op, r, 15 - kc, C, 0.0)
    j = ar["j"]
    Dk = 1.0 / np.linalg.norm(U, axis=0)
    Vhat = np.concatenate([U * Dk, ar["V"][:, :j]], axis=1)
    What = np.concatenate([C, ar["V"]], axis=1)
    G = np.zeros((kc + j + 1, kc + j))
    G[:kc, :kc] = np.diag(Dk); G[:kc, kc:] = ar["B"]; G[kc:, kc:] = ar["Hbar"]
    AVhat = np.stack([op(Vhat[:, i]) for i in range(Vhat.shape[1])], axis=1)
    np.testing.assert_allclose(AVhat, What @ G, atol=1e-9 * np.abs(AVhat).max())
    import scipy.linalg as sla
    theta, Z = sla.eig(G.T @ G, G.T @ (What.T @ Vhat))
    for i in range(len(theta)):
        if not np.isfinite(theta[i]):
            continue
        y = Vhat @ Z[:, i]
        res = AVhat @ Z[:, i] - theta[i] * y
        assert np.abs(AVhat.T @ res).max() <= 1e-7 * abs(theta[i]) * np.linalg.norm(AVhat) * np.linalg.norm(y)


def test_select_smallest_pairs_and_split_rule():
    theta = np.array([5.0, 1 + 1j, 1 - 1j, 0.5, 3.0])
    Z = np.eye(5, dtype=complex) + 1j * np.roll(np.eye(5), 1, axis=0)
    P = krylov.select_smallest(theta, Z, 3)        # 0.5, pair (|.|=1.41) -> 3 cols
    assert P.shape == (5, 3)
    np.testing.assert_array_equal(P[:, 0], np.real(Z[:, 3]))
    P2 = krylov.select_smallest(theta, Z, 2)       # 0.5 then half a pair: drop it
    assert P2.shape == (5, 1)
    theta2 = np.array([-1.0, 1.0, 2.0])
    P3 = krylov.select_smallest(theta2, np.eye(3, dtype=complex), 1)
    np.testing.assert_array_equal(P3[:, 0], [1.0, 0.0, 0.0])   # tie on |theta|: smaller real part


def test_qr_pos_normalisation():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((10, 4))
    Q, R = krylov.qr_pos(X)
    assert np.all(np.diag(R) > 0)
    np.testing.assert_allclose(Q @ R, X, atol=1e-13)
    np.testing.assert_allclose(Q.T @ Q, np.eye(4), atol=1e-14)


def test_recycling_solves_an_indefinite_helmholtz_sequence():
    # -lap u - k^2 u = 1 with k from a GRF (App. E): indefinite, where
    # restarted GMRES needs several times more steps than GCRO-DR
    from workloads import helmholtz2d_sequence
    from oracle import sort as osort
    K = helmholtz2d_sequence(24, 4, 7.0, 0.15, seed=7)
    A0, _ = assembly.helmholtz2d(K[0])
    ev = np.linalg.eigvalsh(A0.toarray())
    assert (ev < 0).any() and (ev > 0).any()
    order = osort.greedy_sort(K.reshape(4, -1))
    sysd = [dict(kind="helmholtz2d", k=K[i]) for i in range(4)]
    x_r, info_r = skr.solve_sequence(sysd, order, "jacobi", 20, 8, 1e-8, precision="fp64")
    x_g, info_g = skr.solve_sequence(sysd, order, "jacobi", 20, 0, 1e-8, precision="fp64")
    for i in range(4):
        A, b = assembly.helmholtz2d(K[i])
        ev = np.abs(np.linalg.eigvalsh(A.toarray()))
        kappa = ev.max() / ev.min()
        xd = spla.spsolve(A.tocsc(), b)
        assert np.linalg.norm(b - A @ x_r[i]) <= 1e-8 * np.linalg.norm(b) * 1.01
        assert np.linalg.norm(x_r[i] - xd) <= 10 * kappa * 1e-8 * np.linalg.norm(xd)
    assert sum(i["steps"] for i in info_r) * 3 < sum(i["steps"] for i in info_g)


def test_warm_start_takes_no_steps_on_a_repeated_system():
    # Algorithm 2 leaves x_0 free; with x_0 = the previous solution of an
    # identical system the initial residual already meets the tolerance
    L = darcy2d_sequence(12, 1, 0.2, seed=3)
    sysd = [dict(kind="darcy2d", loga=L[0])] * 2
    xs, info = skr.solve_sequence(sysd, [0, 1], "jacobi", 20, 6, 1e-8, warm_start=True)
    assert info[0]["steps"] > 0 and info[1]["steps"] == 0
    np.testing.assert_array_equal(xs[1], xs[0])
    xs_c, info_c = skr.solve_sequence(sysd, [0, 1], "jacobi", 20, 6, 1e-8, warm_start=False)
    assert info_c[1]["steps"] > 0


def test_warm_start_on_a_sorted_chebyshev_poisson_sequence():
    from workloads import chebyshev_poisson_sequence
    from oracle import sort as osort
    K, F, G = chebyshev_poisson_sequence(20, 8, seed=2)
    order = osort.greedy_sort(K)
    sysd = [dict(kind="poisson2d", f=F[i], g=tuple(G[i])) for i in range(8)]
    xw, iw = skr.solve_sequence(sysd, order, "jacobi", 20, 6, 1e-8, warm_start=True)
    xc, ic = skr.solve_sequence(sysd, order, "jacobi", 20, 6, 1e-8, warm_start=False)
    for i in range(8):
        A, b = assembly.poisson2d_dirichlet(F[i], *G[i])
        xd = spla.spsolve(A.tocsc(), b)
        for x in (xw[i], xc[i]):
            assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b) * 1.01
            assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
    assert iw[order[0]]["steps"] == ic[order[0]]["steps"]   # the first system starts from 0 either way


def test_one_sided_distance_is_the_sine_of_the_largest_principal_angle():
    import scipy.linalg as sla
    rng = np.random.default_rng(12)
    n = 40
    for dq, dc in ((3, 5), (4, 4), (1, 6)):
        Q = np.linalg.qr(rng.standard_normal((n, dq)))[0]
        C = np.linalg.qr(rng.standard_normal((n, dc)))[0]
        ang = sla.subspace_angles(Q, C)
        assert abs(krylov.one_sided_distance(Q, C) - np.sin(ang.max())) < 1e-12
    C = np.linalg.qr(rng.standard_normal((n, 5)))[0]
    assert krylov.one_sided_distance(C[:, :3], C) < 1e-7          # Q inside C
    P = np.eye(n)[:, :3]
    Cp = np.eye(n)[:, 3:8]
    assert abs(krylov.one_sided_distance(P, Cp) - 1.0) < 1e-12     # orthogonal
    assert abs(krylov.one_sided_distance(C, C[:, :2]) - 1.0) < 1e-12  # dim Q > dim C


def test_sequence_reports_delta_per_system():
    L = darcy2d_sequence(14, 4, 0.2, seed=5)
    sysd = [dict(kind="darcy2d", loga=l) for l in L]
    _, info = skr.solve_sequence(sysd, [0, 1, 2, 3], "none", 20, 6, 1e-8)
    assert info[0]["delta"] == -1.0                      # nothing recycled into the first system
    assert all(0.0 <= info[i]["delta"] <= 1.0 for i in (1, 2, 3))


def _gauss_seidel_ssor(A, v):
    """One forward then one backward Gauss-Seidel sweep from x = 0 (the SSOR
    iteration with omega = 1, written as scalar loops)."""
    A = A.toarray()
    n = len(v)
    x = np.zeros(n)
    for i in range(n):
        x[i] = (v[i] - A[i, :i] @ x[:i] - A[i, i + 1:] @ x[i + 1:]) / A[i, i]
    for i in reversed(range(n)):
        x[i] = (v[i] - A[i, :i] @ x[:i] - A[i, i + 1:] @ x[i + 1:]) / A[i, i]
    return x


def test_ssor_is_a_symmetric_gauss_seidel_sweep_in_redblack_order():
    L = darcy2d_sequence(5, 1, 0.3, seed=6)
    A, _ = assembly.darcy2d(L[0])
    grid = (5, 5)
    M = oprecond.RightPreconditioner(A, "ssor", grid)
    perm = oprecond.redblack_permutation(grid)
    Ap = sp.csr_matrix(A)[perm][:, perm]
    v = np.random.default_rng(1).standard_normal(25)
    z = M.apply(v)
    np.testing.assert_allclose(z[perm], _gauss_seidel_ssor(Ap, v[perm]), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("grid", [(6, 5), (4, 3, 5)])
def test_redblack_ssor_closed_form(grid):
    # red rows of M are those of A; the black-black block is D_b + A_br D_r^-1 A_rb
    if len(grid) == 2:
        A, _ = assembly.darcy2d(darcy2d_sequence(grid[0], 1, 0.3, seed=7)[0][: grid[0] + 2, : grid[1] + 2])
    else:
        from workloads import darcy3d_sequence
        A, _ = assembly.darcy3d(darcy3d_sequence(max(grid), 1, 0.3, seed=7)[0][: grid[0] + 2, : grid[1] + 2, : grid[2] + 2])
    perm, Lp, Up = oprecond.ssor_redblack(A, grid)
    M = (Lp @ Up).toarray()
    Ap = sp.csr_matrix(A)[perm][:, perm].toarray()
    nr = (np.indices(grid).reshape(len(grid), -1).sum(axis=0) % 2 == 0).sum()
    np.testing.assert_allclose(M[:nr], Ap[:nr], rtol=1e-13, atol=1e-13 * np.abs(Ap).max())
    Dr = np.diag(Ap)[:nr]
    want_bb = np.diag(np.diag(Ap)[nr:]) + Ap[nr:, :nr] @ np.diag(1.0 / Dr) @ Ap[:nr, nr:]
    np.testing.assert_allclose(M[nr:, nr:], want_bb, rtol=1e-13, atol=1e-13 * np.abs(Ap).max())


# ---------------------------------------------------------------- block Jacobi (App. D.3 item 3)

def _grid_matrix(grid, seed):
    rng = np.random.default_rng(seed)
    if len(grid) == 2:
        return assembly.darcy2d(rng.standard_normal((grid[0] + 2, grid[1] + 2)))[0]
    return assembly.darcy3d(rng.standard_normal(tuple(g + 2 for g in grid)))[0]


def test_block_ranges_are_contiguous_with_a_ragged_last_block():
    assert precond.block_ranges(30, 4) == [(0, 8), (8, 16), (16, 24), (24, 30)]
    assert precond.block_ranges(7, 1) == [(0, 7)]
    assert precond.block_ranges(5, 5) == [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)]


def test_bjacobi_one_block_is_ilu0_and_unit_blocks_are_jacobi():
    grid = (6, 5)
    A = _grid_matrix(grid, 1)
    v = np.random.default_rng(2).standard_normal(30)
    one = precond.RightPreconditioner(A, "bjacobi", grid, blocks=1).apply(v)
    np.testing.assert_array_equal(one, precond.RightPreconditioner(A, "ilu0", grid).apply(v))
    unit = precond.RightPreconditioner(A, "bjacobi", grid, blocks=30).apply(v)
    np.testing.assert_allclose(unit, v / A.diagonal(), rtol=1e-15)


@pytest.mark.parametrize("grid,blocks", [((6, 5), 4), ((7, 7), 3), ((4, 3, 5), 5)])
def test_bjacobi_closed_form(grid, blocks):
    # M is block diagonal over the row blocks; inside a block it is the
    # red-black ILU(0) of the block alone: M_rr = a_rr, M_rb = a_rb and
    # M_br = a_br for r, b in the block, and on the black rows
    # M_bb = a_bb and, for b != b', M_bb' = sum over the block's reds r of
    # a_br a_rb' / a_rr (the fill that ILU(0) drops from U)
    A = _grid_matrix(grid, 3)
    Ad = A.toarray()
    n = Ad.shape[0]
    Mop = precond.RightPreconditioner(A, "bjacobi", grid, blocks=blocks)
    M = np.linalg.inv(np.stack([Mop.apply(e) for e in np.eye(n)], axis=1))
    color = np.indices(grid).reshape(len(grid), -1).sum(axis=0) % 2
    want = np.zeros((n, n))
    for lo, hi in precond.block_ranges(n, blocks):
        for i in range(lo, hi):
            for j in range(lo, hi):
                if color[i] == 0 or color[j] == 0:
                    want[i, j] = Ad[i, j]
                else:
                    want[i, j] = Ad[i, i] if i == j else sum(
                        Ad[i, r] * Ad[r, j] / Ad[r, r] for r in range(lo, hi) if color[r] == 0)
    np.testing.assert_allclose(M, want, rtol=1e-10, atol=1e-10 * np.abs(Ad).max())
    assert blocks > 1 and np.abs(want - Ad * (want != 0)).max() > 0   # not plain A


def test_bjacobi_gcrodr_converges_on_darcy():
    A, b = _darcy(12, seed=4)
    st = krylov.RecycleState()
    x, info = skr.solve_system(A, b, "bjacobi", 20, 6, 1e-10, st, grid=(12, 12), pc_blocks=5)
    assert info["converged"] and np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    _, info1 = skr.solve_system(A, b, "ilu0", 20, 6, 1e-10, krylov.RecycleState(), grid=(12, 12))
    _, infoj = skr.solve_system(A, b, "jacobi", 20, 6, 1e-10, krylov.RecycleState(), grid=(12, 12))
    # between ILU(0) (one block) and Jacobi (one row per block) in strength
    assert info1["steps"] <= info["steps"] <= infoj["steps"]


# ---------------------------------------------------------------- harmonic-Ritz selection on a complete space

def _laplacian_3x5_and_smallest_eigvecs(k):
    # a = 1 Darcy on a 3 x 5 grid: A = -lap_h, eigenvectors
    # sin(p pi x_i) sin(q pi y_j), eigenvalues lx[p] + ly[q] (closed form)
    nx, ny = 3, 5
    A, _ = assembly.darcy2d(np.zeros((nx + 2, ny + 2)))
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    pairs = [(p, q) for p in range(1, nx + 1) for q in range(1, ny + 1)]
    lam = {pq: 4.0 / hx**2 * np.sin(pq[0] * np.pi * hx / 2) ** 2 + 4.0 / hy**2 * np.sin(pq[1] * np.pi * hy / 2) ** 2
           for pq in pairs}
    order = sorted(pairs, key=lambda pq: lam[pq])
    assert lam[order[k]] - lam[order[k - 1]] > 1.0        # a gap after the k-th: the span is unique
    i, j = np.meshgrid(np.arange(1, nx + 1), np.arange(1, ny + 1), indexing="ij")
    E = np.stack([(np.sin(p * np.pi * i * hx) * np.sin(q * np.pi * j * hy)).ravel() for p, q in order[:k]], axis=1)
    return A, E


def test_first_cycle_selection_spans_the_smallest_closed_form_eigenvectors():
    import scipy.linalg as sla
    k = 3
    A, E = _laplacian_3x5_and_smallest_eigvecs(k)
    n = A.shape[0]
    ar = krylov.arnoldi(lambda v: A @ v, np.random.default_rng(5).standard_normal(n), n, None, 0.0)
    P, _ = krylov.harmonic_ritz_first(ar["Hbar"], k)
    assert P.shape[1] == k
    Y = ar["V"][:, :n] @ P
    assert sla.subspace_angles(Y, E).max() < 1e-6


def test_recycled_cycle_selection_spans_the_smallest_closed_form_eigenvectors():
    # the augmented space [U, V] of a recycled cycle covers R^n: the
    # generalized harmonic-Ritz problem of Algorithm 2 is exact, and the k
    # smallest |theta| select the closed-form eigenvectors
    import scipy.linalg as sla
    k = 3
    A, E = _laplacian_3x5_and_smallest_eigvecs(k)
    n = A.shape[0]
    rng = np.random.default_rng(6)
    kc = 4
    state = krylov.RecycleState()
    state.U = rng.standard_normal((n, kc))
    state.C = None
    krylov.refresh(lambda v: A @ v, state)            # C = qr(A U).Q, U = U R^-1
    U, C = state.U, state.C
    r = rng.standard_normal(n)
    r = r - C @ (C.T @ r)
    ar = krylov.arnoldi(lambda v: A @ v, r, n - kc, C, 0.0)
    j = ar["j"]
    assert kc + j == n
    Dk = 1.0 / np.linalg.norm(U, axis=0)
    Vhat = np.concatenate([U * Dk, ar["V"][:, :j]], axis=1)
    What = np.concatenate([C, ar["V"]], axis=1)
    G = np.zeros((kc + j + 1, kc + j))
    G[:kc, :kc] = np.diag(Dk)
    G[:kc, kc:] = ar["B"]
    G[kc:, kc:] = ar["Hbar"]
    P, _ = krylov.harmonic_ritz_general(G, What, Vhat, k)
    assert P.shape[1] == k
    assert sla.subspace_angles(Vhat @ P, E).max() < 1e-6


# ---------------------------------------------------------------- FP32-emulating variant (mixed-form error)

def test_round32_is_float32_rounding():
    assert krylov.round32(1.0 + 2.0 ** -30) == 1.0                     # below float32's 24-bit mantissa
    assert krylov.round32(1.0 + 2.0 ** -20) == 1.0 + 2.0 ** -20
    assert krylov.round32(1.0 + 3 * 2.0 ** -24) == 1.0 + 2.0 ** -22   # nearest, ties to even
    v = np.random.default_rng(0).standard_normal(50)
    assert np.array_equal(krylov.round32(v), v.astype(np.float32).astype(np.float64))


def test_emulated_arnoldi_keeps_float32_vectors():
    A, b = _darcy(8, seed=5)
    ar = krylov.arnoldi(lambda v: A @ v, b, 10, None, 0.0, rnd=krylov.round32)
    V = ar["V"]
    assert np.array_equal(krylov.round32(V), V)
    # orthonormal to float32 accuracy, not to float64's
    err = np.abs(V.T @ V - np.eye(V.shape[1])).max()
    assert 1e-9 < err < 1e-5


def test_fp32_emulated_sequence_stays_within_the_mixed_form_bound():
    L = darcy2d_sequence(24, 4, 0.15, seed=23)
    order = list(range(4))
    sysd = [dict(kind="darcy2d", loga=l) for l in L]
    x64, _ = skr.solve_sequence(sysd, order, "jacobi", 30, 10, 1e-8, precision="fp64")
    xm, _ = skr.solve_sequence(sysd, order, "jacobi", 30, 10, 1e-8, precision="mixed")
    xe, ie = skr.solve_sequence(sysd, order, "jacobi", 30, 10, 1e-8, precision="fp32-emulated")
    for i in range(4):
        A, b = assembly.darcy2d(L[i])
        assert ie[i]["converged"] and ie[i]["refinements"] >= 2       # FP32 inner solves need refinement
        assert np.linalg.norm(b - A @ xe[i]) <= 1e-8 * np.linalg.norm(b)
        assert np.linalg.norm(xe[i] - x64[i]) <= 1e-6 * np.linalg.norm(x64[i])
        assert not np.array_equal(xe[i], xm[i])                        # the rounding is active
