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
