"""Pins for the oracle's finite-difference assembly (Sec. 3.1, App. A.2)."""
import os

import numpy as np
import scipy.sparse.linalg as spla

from oracle import assembly

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_matrix():
    rows = []
    with open(os.path.join(GOLDEN, "paper_poisson_2x2.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return np.array(rows)


def test_paper_worked_example_poisson():
    A = assembly.poisson2d_paper(2, 2, 1.0, 1.0).toarray()
    np.testing.assert_array_equal(A, _paper_matrix())


def test_darcy_unit_coefficient_is_minus_paper_laplacian():
    # -div(1 grad u) = -lap u: with h = 1 the Darcy matrix is the negation.
    A, b = assembly.darcy2d(np.zeros((4, 4)), h=1.0)
    np.testing.assert_array_equal(A.toarray(), -_paper_matrix())
    np.testing.assert_array_equal(b, np.ones(4))


def test_darcy_rectangular_ordering():
    # nx = 3, ny = 2: neighbours in x are +-ny apart, in y +-1 (second index fastest)
    A, _ = assembly.darcy2d(np.zeros((5, 4)), h=1.0)
    A = A.toarray()
    assert A[0, 1] == -1 and A[0, 2] == -1 and A[1, 2] == 0 and A[2, 4] == -1


def _manufactured_error(N):
    # u = sin(pi x) sin(pi y) solves -lap u = 2 pi^2 u with u = 0 on the boundary
    h = 1.0 / (N + 1)
    x = np.arange(1, N + 1) * h
    X, Y = np.meshgrid(x, x, indexing="ij")
    u = np.sin(np.pi * X) * np.sin(np.pi * Y)
    f = 2.0 * np.pi**2 * u
    A, b = assembly.darcy2d(np.zeros((N + 2, N + 2)), rhs=f.ravel())
    uh = spla.spsolve(A.tocsc(), b)
    return np.max(np.abs(uh - u.ravel()))


def test_manufactured_solution_second_order():
    e1, e2 = _manufactured_error(15), _manufactured_error(31)
    ratio = e1 / e2
    assert 3.6 < ratio < 4.4, ratio


def test_constant_coefficient_eigenvalues_closed_form():
    N = 6
    h = 1.0 / (N + 1)
    A, _ = assembly.darcy2d(np.zeros((N + 2, N + 2)))
    ev = np.sort(np.linalg.eigvalsh(A.toarray()))
    p = np.arange(1, N + 1)
    lam1 = 4.0 / h**2 * np.sin(p * np.pi * h / 2) ** 2
    closed = np.sort((lam1[:, None] + lam1[None, :]).ravel())
    np.testing.assert_allclose(ev, closed, rtol=1e-12)


def test_darcy_flux_form_symmetric_and_face_means():
    rng = np.random.default_rng(3)
    loga = rng.standard_normal((6, 5))
    A, _ = assembly.darcy2d(loga, h=1.0)
    D = A.toarray()
    np.testing.assert_allclose(D, D.T, rtol=0, atol=0)
    a = np.exp(loga)
    # row of interior node (1,1) of the node array = unknown 0; its +x neighbour is unknown ny=3
    assert np.isclose(D[0, 3], -0.5 * (a[1, 1] + a[2, 1]))
    assert np.isclose(D[0, 1], -0.5 * (a[1, 1] + a[1, 2]))
    faces = 0.5 * (a[1, 1] + a[0, 1]) + 0.5 * (a[1, 1] + a[2, 1]) + 0.5 * (a[1, 1] + a[1, 0]) + 0.5 * (a[1, 1] + a[1, 2])
    assert np.isclose(D[0, 0], faces)
    # zero row sums for rows away from the boundary (flux form conserves)
    assert abs(D[4].sum()) < 1e-12 * abs(D[4, 4])


def test_darcy3d_reduces_to_closed_form():
    N = 3
    h = 1.0 / (N + 1)
    A, _ = assembly.darcy3d(np.zeros((N + 2,) * 3))
    ev = np.sort(np.linalg.eigvalsh(A.toarray()))
    p = np.arange(1, N + 1)
    lam1 = 4.0 / h**2 * np.sin(p * np.pi * h / 2) ** 2
    closed = np.sort((lam1[:, None, None] + lam1[None, :, None] + lam1[None, None, :]).ravel())
    np.testing.assert_allclose(ev, closed, rtol=1e-12)


def test_convdiff_upwind_is_m_matrix_and_pure_diffusion_limit():
    A, _ = assembly.convdiff2d(0.05, (30.0, -20.0), 8)
    D = A.toarray()
    off = D - np.diag(np.diag(D))
    assert np.all(off <= 0)
    assert np.all(np.diag(D) > 0)
    assert np.all(D.sum(axis=1) >= -1e-9)        # weak diagonal dominance
    B, _ = assembly.convdiff2d(1.0, (0.0, 0.0), 8)
    L, _ = assembly.darcy2d(np.zeros((10, 10)))
    np.testing.assert_allclose(B.toarray(), L.toarray(), rtol=1e-14)
    # nonsymmetric when beta != 0
    assert np.abs(D - D.T).max() > 0


# ------------------------------------------------------------------ Helmholtz (App. E)

def test_helmholtz_zero_wavenumber_is_unit_coefficient_darcy():
    A0, b0 = assembly.helmholtz2d(np.zeros((7, 5)))
    Ad, bd = assembly.darcy2d(np.zeros((9, 7)))
    assert abs(A0 - Ad).max() == 0.0
    np.testing.assert_array_equal(b0, bd)


def test_helmholtz_constant_wavenumber_closed_form_spectrum():
    # -lap_h - k^2 I on the unit square: lambda_ij - k^2 with the closed-form
    # Dirichlet Laplacian eigenvalues; k = 9 makes it indefinite
    nx = ny = 8
    h = 1.0 / (nx + 1)
    kk = 9.0
    A, _ = assembly.helmholtz2d(np.full((nx, ny), kk))
    ev = np.sort(np.linalg.eigvalsh(A.toarray()))
    lam = np.sort([(4.0 / h**2) * (np.sin(i * np.pi * h / 2) ** 2 + np.sin(j * np.pi * h / 2) ** 2) - kk**2
                   for i in range(1, nx + 1) for j in range(1, ny + 1)])
    np.testing.assert_allclose(ev, lam, rtol=1e-12, atol=1e-9)
    assert 0 < (ev < 0).sum() < ev.size


def test_helmholtz_variable_wavenumber_enters_the_diagonal_only():
    rng = np.random.default_rng(3)
    k = rng.uniform(2.0, 9.0, size=(6, 4))
    A, _ = assembly.helmholtz2d(k)
    A0, _ = assembly.helmholtz2d(np.zeros((6, 4)))
    D = (A0 - A).toarray()
    np.testing.assert_allclose(D, np.diag(k.ravel() ** 2), rtol=1e-14, atol=0.0)


def test_helmholtz_manufactured_solution_second_order():
    kk = 3.0
    errs = []
    for N in (15, 31):
        h = 1.0 / (N + 1)
        x = np.arange(1, N + 1) * h
        X, Y = np.meshgrid(x, x, indexing="ij")
        u = np.sin(np.pi * X) * np.sin(2 * np.pi * Y)
        f = (5 * np.pi**2 - kk**2) * u
        A, b = assembly.helmholtz2d(np.full((N, N), kk), rhs=f.ravel())
        xh = spla.spsolve(A.tocsc(), b)
        errs.append(np.abs(xh - u.ravel()).max())
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


# ------------------------------------------------------------------ Poisson with Dirichlet data

def test_poisson_dirichlet_zero_data_is_the_paper_example():
    f = np.array([[1.0, 2.0], [3.0, 4.0]])
    z = np.zeros(2)
    A, b = assembly.poisson2d_dirichlet(f, z, z, z, z, h=1.0)
    np.testing.assert_array_equal(A.toarray(), _paper_matrix())
    np.testing.assert_array_equal(b, f.ravel())


def test_poisson_dirichlet_exact_on_a_quadratic():
    # the 5-point Laplacian is exact on quadratics, so the discrete solution
    # equals u at the nodes; the x/y asymmetry of u pins which boundary line
    # is which and the sign of the folded values
    nx, ny = 9, 6
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    x = np.arange(1, nx + 1) * hx
    y = np.arange(1, ny + 1) * hy
    u = lambda X, Y: X**2 + 2.0 * Y**2 + 0.5 * X * Y + X - 3.0 * Y + 0.25   # noqa: E731
    X, Y = np.meshgrid(x, y, indexing="ij")
    f = np.full((nx, ny), 2.0 + 4.0)
    A, b = assembly.poisson2d_dirichlet(f, u(0.0, y), u(1.0, y), u(x, 0.0), u(x, 1.0))
    xs = spla.spsolve(A.tocsc(), b)
    np.testing.assert_allclose(xs, u(X, Y).ravel(), rtol=0, atol=1e-11)


# ------------------------------------------------------------------ convection-diffusion: upwind scale and direction
#
# These pins hold the convection-diffusion assembly to closed forms that a
# wrong diffusion scale, a wrong upwind scale (beta/(2h) instead of beta/h) or
# an upwind taken from the wrong side each break.

def _convdiff_interior_residual(conv, nu, beta, M, u):
    """(A u)_p at the rows whose four neighbours are all unknowns of an M x M
    grid, u evaluated at the nodes (i+1)h, (j+1)h with h = 1/(M+1); no
    Dirichlet coupling is dropped on those rows, so A u is the full stencil."""
    h = 1.0 / (M + 1)
    x = np.arange(1, M + 1) * h
    X, Y = np.meshgrid(x, x, indexing="ij")
    A, _ = conv(nu, beta, M)
    r = (A @ u(X, Y).ravel()).reshape(M, M)
    return r[1:-1, 1:-1], X[1:-1, 1:-1], Y[1:-1, 1:-1], h


def _check_convdiff_closed_forms(conv):
    """Both closed forms below, for beta in all four sign quadrants."""
    nu, M = 0.037, 11
    for beta in ((23.0, 7.5), (-23.0, 7.5), (23.0, -7.5), (-31.0, -4.0)):
        # linear u: the 5-point Laplacian and one-sided differences are exact,
        # so every full row gives beta . grad u = beta_x c1 + beta_y c2
        c0, c1, c2 = 0.3, 1.7, -2.9
        r, _, _, _ = _convdiff_interior_residual(conv, nu, beta, M, lambda X, Y: c0 + c1 * X + c2 * Y)
        np.testing.assert_allclose(r, beta[0] * c1 + beta[1] * c2, rtol=0, atol=1e-9)
        # quadratic u = a x^2 + b y^2: -nu lap_h u = -2 nu (a + b) exactly, and
        # the upwind difference of x^2 on the side beta points from is
        # 2x - sign(beta_x) h (similarly in y)
        qa, qb = 1.3, -0.8
        r, X, Y, h = _convdiff_interior_residual(conv, nu, beta, M, lambda X, Y: qa * X**2 + qb * Y**2)
        sx, sy = np.sign(beta[0]), np.sign(beta[1])
        want = (-2.0 * nu * (qa + qb) + beta[0] * qa * (2.0 * X - sx * h) + beta[1] * qb * (2.0 * Y - sy * h))
        np.testing.assert_allclose(r, want, rtol=0, atol=1e-9)


def _convdiff_manufactured_errors(conv, sizes=(15, 31)):
    """Max nodal error against u = sin(pi x) sin(pi y) (zero on the boundary)
    with f = -nu lap u + beta . grad u, on the given grids."""
    nu, beta = 0.05, (20.0, -12.0)
    errs = []
    for N in sizes:
        h = 1.0 / (N + 1)
        x = np.arange(1, N + 1) * h
        X, Y = np.meshgrid(x, x, indexing="ij")
        u = np.sin(np.pi * X) * np.sin(np.pi * Y)
        f = (2.0 * np.pi**2 * nu * u + beta[0] * np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
             + beta[1] * np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y))
        A, b = conv(nu, beta, N, rhs=f.ravel())
        errs.append(np.abs(spla.spsolve(A.tocsc(), b) - u.ravel()).max())
    return errs


def _check_convdiff_first_order(conv):
    e1, e2 = _convdiff_manufactured_errors(conv)
    # first-order upwinding: the error halves with h (measured 0.249 -> 0.132)
    assert e2 < 0.2 and 1.7 < e1 / e2 < 2.3, (e1, e2)


def test_convdiff_exact_on_linear_and_quadratic_fields():
    _check_convdiff_closed_forms(assembly.convdiff2d)


def test_convdiff_manufactured_solution_first_order():
    _check_convdiff_first_order(assembly.convdiff2d)


# ------------------------------------------------------------------ 3D Darcy: face means, axis order, O(h^2)

def _check_darcy3d_row_by_hand(d3):
    """Every entry of every row of a 3 x 4 x 5 grid (three distinct sides, so
    three distinct h and strides) against face means computed node by node."""
    rng = np.random.default_rng(11)
    nx, ny, nz = 3, 4, 5
    loga = rng.standard_normal((nx + 2, ny + 2, nz + 2))
    a = np.exp(loga)
    hs = (1.0 / (nx + 1), 1.0 / (ny + 1), 1.0 / (nz + 1))
    A, b = d3(loga)
    D = A.toarray()
    n = nx * ny * nz
    want = np.zeros((n, n))
    for i in range(nx):
        for j in range(ny):
            for l in range(nz):
                p = (i * ny + j) * nz + l
                c = a[i + 1, j + 1, l + 1]
                for (di, dj, dl), hh in (((-1, 0, 0), hs[0]), ((1, 0, 0), hs[0]), ((0, -1, 0), hs[1]),
                                         ((0, 1, 0), hs[1]), ((0, 0, -1), hs[2]), ((0, 0, 1), hs[2])):
                    face = 0.5 * (c + a[i + 1 + di, j + 1 + dj, l + 1 + dl]) / hh**2
                    want[p, p] += face
                    ii, jj, ll = i + di, j + dj, l + dl
                    if 0 <= ii < nx and 0 <= jj < ny and 0 <= ll < nz:
                        want[p, (ii * ny + jj) * nz + ll] = -face
    np.testing.assert_allclose(D, want, rtol=1e-14, atol=0.0)
    np.testing.assert_array_equal(b, np.ones(n))


def _darcy3d_manufactured_errors(d3, sizes=(7, 15)):
    """Max nodal error for u = sin(pi x) sin(2 pi y) sin(pi z) and the smooth,
    axis-anisotropic a = exp(0.6 x - 0.3 y + 0.9 z + 0.4 x y); f =
    -div(a grad u) in closed form."""
    errs = []
    for N in sizes:
        nx, ny, nz = N, N + 1, N + 2
        g = [np.arange(0, s + 2) / (s + 1.0) for s in (nx, ny, nz)]
        X, Y, Z = np.meshgrid(*g, indexing="ij")
        la = 0.6 * X - 0.3 * Y + 0.9 * Z + 0.4 * X * Y
        a = np.exp(la)
        ax, ay, az = a * (0.6 + 0.4 * Y), a * (-0.3 + 0.4 * X), a * 0.9
        sx, sy, sz = np.sin(np.pi * X), np.sin(2 * np.pi * Y), np.sin(np.pi * Z)
        cx, cy, cz = np.cos(np.pi * X), np.cos(2 * np.pi * Y), np.cos(np.pi * Z)
        u = sx * sy * sz
        ux, uy, uz = np.pi * cx * sy * sz, 2 * np.pi * sx * cy * sz, np.pi * sx * sy * cz
        lap = -(np.pi**2 + 4 * np.pi**2 + np.pi**2) * u
        f = -(a * lap + ax * ux + ay * uy + az * uz)
        inner = (slice(1, -1),) * 3
        A, b = d3(la, rhs=f[inner].ravel())
        errs.append(np.abs(spla.spsolve(A.tocsc(), b) - u[inner].ravel()).max())
    return errs


def _check_darcy3d_second_order(d3):
    e1, e2 = _darcy3d_manufactured_errors(d3)
    assert e2 < 0.05 and 3.3 < e1 / e2 < 4.7, (e1, e2)


def test_darcy3d_rows_by_hand_on_a_non_cubic_grid():
    _check_darcy3d_row_by_hand(assembly.darcy3d)


def test_darcy3d_manufactured_solution_second_order():
    _check_darcy3d_second_order(assembly.darcy3d)


# ------------------------------------------------------------------ the pins catch planted mistakes
#
# Each mutant is the oracle's own source with one plausible mistake planted
# (text substitution, then exec); the pins above must reject every one.

def _mutant(func_name, old, new):
    import inspect
    src = inspect.getsource(assembly)
    assert src.count(old) >= 1, old
    ns = {}
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    return ns[func_name]


def _fails(check, fn):
    """True when the pin rejects fn: an assertion fails, or the mutant's
    matrix cannot even be built (an index outside the grid)."""
    try:
        check(fn)
    except (AssertionError, ValueError, IndexError):
        return True
    return False


def test_convdiff_pins_reject_planted_mistakes():
    mutants = [
        _mutant("convdiff2d", "cxm = -d - max(bx, 0.0) / hh", "cxm = -d - max(bx, 0.0) / (2.0 * hh)"),
        _mutant("convdiff2d", "cpp = 4.0 * d + abs(bx) / hh", "cpp = 4.0 * d + abs(bx) / (2.0 * hh)"),
        _mutant("convdiff2d", "d = nu / hh**2", "d = 0.5 * nu / hh**2"),
        # upwind from the wrong side in x: the diagonal stays |bx|/h, the
        # coupling moves to the downstream neighbour
        _mutant("convdiff2d", "cxm = -d - max(bx, 0.0) / hh\n    cxp = -d + min(bx, 0.0) / hh",
                "cxm = -d + min(bx, 0.0) / hh\n    cxp = -d - max(bx, 0.0) / hh"),
    ]
    for mu in mutants:
        assert _fails(_check_convdiff_closed_forms, mu) or _fails(_check_convdiff_first_order, mu)


def test_darcy3d_pins_reject_planted_mistakes():
    harmonic = _mutant("darcy3d", "f = 0.5 * (c + a[tuple(nb)]) / hs[ax] ** 2",
                       "f = 2.0 * c * a[tuple(nb)] / (c + a[tuple(nb)]) / hs[ax] ** 2")
    swapped = _mutant("darcy3d", "strides = (ny * nz, nz, 1)", "strides = (nz, ny * nz, 1)")
    wrong_h = _mutant("darcy3d", "f = 0.5 * (c + a[tuple(nb)]) / hs[ax] ** 2",
                      "f = 0.5 * (c + a[tuple(nb)]) / hs[2 - ax] ** 2")
    for mu in (harmonic, swapped, wrong_h):
        assert _fails(_check_darcy3d_row_by_hand, mu)
    # the axis mistakes also break second-order convergence on the anisotropic field
    for mu in (swapped, wrong_h):
        assert _fails(_check_darcy3d_second_order, mu)
