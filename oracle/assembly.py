"""Finite-difference assembly of the linear systems A x = b (oracle).

Follows the paper's FDM recipe (Sec. 3.1 and App. A.2): central differences
on a uniform grid, one matrix row per interior node, unknowns in row-major
order with the second grid index fastest (u11, u12, u21, u22 in the 2x2
example of Sec. 3.1), Dirichlet data folded into b (zero here).

Readings where the paper is silent:
  * Darcy -div(a grad u) = f is discretised in conservative (flux) form; the
    face coefficient is the arithmetic mean of the two node values of a.
  * The Poisson dataset with Chebyshev data (App. E) keeps the Sec. 3.1 sign
    (lap u = f, diagonal -2/hx^2 - 2/hy^2) and folds the Dirichlet values of
    boundary neighbours into b as f - g/h^2 (App. A.2).
  * The Helmholtz dataset (App. E, lap u + k^2 u = 0 with k from a GRF) is
    taken as -lap u - k^2 u = f with u = 0 on the boundary and f = 1 by
    default: the homogeneous equation with zero boundary data has only the
    zero solution.
  * Convection-diffusion uses first-order upwinding for beta . grad u.
  * The unit square (cube) has h = 1/(N+1) for N interior nodes per side,
    unless h is passed explicitly (the worked example uses h = 1).

Pins: the 2x2 worked example of Sec. 3.1 (Poisson, h = 1) and its Darcy
negation for a = 1; O(h^2) convergence to a manufactured solution; the
closed-form eigenvalues of the constant-coefficient Laplacian, shifted by
-k^2 for the Helmholtz operator.  Convection-diffusion: A u equals
beta . grad u exactly on linear u and the closed-form upwind value on
quadratic u (all four sign quadrants of beta), and first-order convergence
to a manufactured solution.  3D Darcy: every entry of a 3 x 4 x 5 grid's
matrix against face means computed node by node, and O(h^2) convergence
with an axis-anisotropic coefficient.  The tests also plant plausible
mistakes in copies of this file (upwind scale beta/(2h), halved diffusion,
upwind side swapped, harmonic face means, swapped strides, an axis's h
taken from another axis) and check that the pins reject each one.
"""
import numpy as np
import scipy.sparse as sp


def _coo_to_csr(rows, cols, vals, n):
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def poisson2d_paper(nx, ny, hx=1.0, hy=1.0):
    """The paper's discretisation of lap u = f (App. A.2, Sec. 3.1 example).

    Row for interior node (i, j): -2(1/hx^2 + 1/hy^2) u_ij + (u_i+1,j +
    u_i-1,j)/hx^2 + (u_i,j+1 + u_i,j-1)/hy^2.  Unknown index p = i*ny + j.
    """
    n = nx * ny
    rows, cols, vals = [], [], []
    for i in range(nx):
        for j in range(ny):
            p = i * ny + j
            rows.append(p); cols.append(p); vals.append(-2.0 * (1.0 / hx**2 + 1.0 / hy**2))
            for di, dj, w in ((-1, 0, 1.0 / hx**2), (1, 0, 1.0 / hx**2),
                              (0, -1, 1.0 / hy**2), (0, 1, 1.0 / hy**2)):
                ii, jj = i + di, j + dj
                if 0 <= ii < nx and 0 <= jj < ny:
                    rows.append(p); cols.append(ii * ny + jj); vals.append(w)
    return _coo_to_csr(np.array(rows), np.array(cols), np.array(vals), n)


def darcy2d(loga, h=None, rhs=None):
    """-div(a grad u) = f on an nx x ny interior grid, a = exp(loga).

    loga  (nx+2, ny+2) node values of log a, boundary nodes included
    h     grid spacing (default 1/(nx+1) in x and 1/(ny+1) in y)
    rhs   f at the interior nodes (n values); default f = 1
    Returns (A as scipy CSR float64, b float64[n]).

    Row p = i*ny + j (interior node (i+1, j+1) of the node array):
      A[p, p-ny] = -a(i-1/2, j)/hx^2, A[p, p+ny] = -a(i+1/2, j)/hx^2,
      A[p, p-1]  = -a(i, j-1/2)/hy^2, A[p, p+1]  = -a(i, j+1/2)/hy^2,
      A[p, p]    = sum of the four face coefficients (each over h^2),
    with face values a(i+-1/2, j) = (a(i, j) + a(i+-1, j))/2.  Couplings to
    boundary nodes are dropped (Dirichlet u = 0).
    """
    loga = np.asarray(loga, dtype=np.float64)
    nx, ny = loga.shape[0] - 2, loga.shape[1] - 2
    hx = 1.0 / (nx + 1) if h is None else float(h)
    hy = 1.0 / (ny + 1) if h is None else float(h)
    a = np.exp(loga)
    c = a[1:-1, 1:-1]
    fxm = 0.5 * (c + a[:-2, 1:-1]) / hx**2
    fxp = 0.5 * (c + a[2:, 1:-1]) / hx**2
    fym = 0.5 * (c + a[1:-1, :-2]) / hy**2
    fyp = 0.5 * (c + a[1:-1, 2:]) / hy**2
    n = nx * ny
    p = np.arange(n).reshape(nx, ny)
    rows = [p.ravel()]
    cols = [p.ravel()]
    vals = [(fxm + fxp + fym + fyp).ravel()]
    for f, sl_row, shift in ((fxm, (slice(1, None), slice(None)), -ny),
                             (fxp, (slice(None, -1), slice(None)), ny),
                             (fym, (slice(None), slice(1, None)), -1),
                             (fyp, (slice(None), slice(None, -1)), 1)):
        pr = p[sl_row].ravel()
        rows.append(pr)
        cols.append(pr + shift)
        vals.append(-f[sl_row].ravel())
    A = _coo_to_csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)
    b = np.ones(n) if rhs is None else np.asarray(rhs, dtype=np.float64).copy()
    return A, b


def darcy3d(loga, h=None, rhs=None):
    """3D analogue of darcy2d: 7-point flux stencil, p = (i*ny + j)*nz + k."""
    loga = np.asarray(loga, dtype=np.float64)
    nx, ny, nz = (s - 2 for s in loga.shape)
    hs = [1.0 / (s + 1) if h is None else float(h) for s in (nx, ny, nz)]
    a = np.exp(loga)
    c = a[1:-1, 1:-1, 1:-1]
    n = nx * ny * nz
    p = np.arange(n).reshape(nx, ny, nz)
    strides = (ny * nz, nz, 1)
    diag = np.zeros_like(c)
    rows, cols, vals = [], [], []
    for ax in range(3):
        for sgn in (-1, 1):
            nb = [slice(1, -1)] * 3
            nb[ax] = slice(0, -2) if sgn < 0 else slice(2, None)
            f = 0.5 * (c + a[tuple(nb)]) / hs[ax] ** 2
            diag = diag + f
            keep = [slice(None)] * 3
            keep[ax] = slice(1, None) if sgn < 0 else slice(None, -1)
            pr = p[tuple(keep)].ravel()
            rows.append(pr)
            cols.append(pr + sgn * strides[ax])
            vals.append(-f[tuple(keep)].ravel())
    rows.insert(0, p.ravel()); cols.insert(0, p.ravel()); vals.insert(0, diag.ravel())
    A = _coo_to_csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)
    b = np.ones(n) if rhs is None else np.asarray(rhs, dtype=np.float64).copy()
    return A, b


def convdiff2d(nu, beta, nside, rhs=None, h=None):
    """-nu lap u + beta . grad u = f, 5-point diffusion, first-order upwind convection.

    For beta_x >= 0 the x-derivative is (u_P - u_{i-1})/h, otherwise
    (u_{i+1} - u_P)/h (same in y); the matrix is then an M-matrix for any
    cell Peclet number.  Unknown index p = i*nside + j, h = 1/(nside+1).
    """
    nx = ny = int(nside)
    hh = 1.0 / (nx + 1) if h is None else float(h)
    bx, by = float(beta[0]), float(beta[1])
    d = nu / hh**2
    cxm = -d - max(bx, 0.0) / hh
    cxp = -d + min(bx, 0.0) / hh
    cym = -d - max(by, 0.0) / hh
    cyp = -d + min(by, 0.0) / hh
    cpp = 4.0 * d + abs(bx) / hh + abs(by) / hh
    n = nx * ny
    p = np.arange(n).reshape(nx, ny)
    rows, cols, vals = [p.ravel()], [p.ravel()], [np.full(n, cpp)]
    for cval, sl_row, shift in ((cxm, (slice(1, None), slice(None)), -ny),
                                (cxp, (slice(None, -1), slice(None)), ny),
                                (cym, (slice(None), slice(1, None)), -1),
                                (cyp, (slice(None), slice(None, -1)), 1)):
        pr = p[sl_row].ravel()
        rows.append(pr); cols.append(pr + shift); vals.append(np.full(pr.size, cval))
    A = _coo_to_csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)
    b = np.ones(n) if rhs is None else np.asarray(rhs, dtype=np.float64).copy()
    return A, b


def helmholtz2d(k, h=None, rhs=None):
    """-lap u - k^2 u = f on an nx x ny interior grid (App. E, Helmholtz).

    k     (nx, ny) wavenumber at the interior nodes
    h     grid spacing (default 1/(nx+1) in x and 1/(ny+1) in y)
    rhs   f at the interior nodes (n values); default f = 1
    Returns (A as scipy CSR float64, b float64[n]).

    Row p = i*ny + j: A[p, p] = 2/hx^2 + 2/hy^2 - k_p^2, A[p, p+-ny] = -1/hx^2,
    A[p, p+-1] = -1/hy^2 (couplings to boundary nodes dropped, u = 0 there).
    """
    k = np.asarray(k, dtype=np.float64)
    nx, ny = k.shape
    hx = 1.0 / (nx + 1) if h is None else float(h)
    hy = 1.0 / (ny + 1) if h is None else float(h)
    n = nx * ny
    p = np.arange(n).reshape(nx, ny)
    rows = [p.ravel()]
    cols = [p.ravel()]
    vals = [(2.0 / hx**2 + 2.0 / hy**2 - k**2).ravel()]
    for sl_row, shift, w in (((slice(1, None), slice(None)), -ny, 1.0 / hx**2),
                             ((slice(None, -1), slice(None)), ny, 1.0 / hx**2),
                             ((slice(None), slice(1, None)), -1, 1.0 / hy**2),
                             ((slice(None), slice(None, -1)), 1, 1.0 / hy**2)):
        pr = p[sl_row].ravel()
        rows.append(pr)
        cols.append(pr + shift)
        vals.append(np.full(pr.size, -w))
    A = _coo_to_csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)
    b = np.ones(n) if rhs is None else np.asarray(rhs, dtype=np.float64).copy()
    return A, b


def poisson2d_dirichlet(f, g_x0, g_x1, g_y0, g_y1, h=None):
    """lap u = f on an nx x ny interior grid with u = g on the boundary (Sec. 3.1 sign).

    f (nx, ny) at the interior nodes; g_x0, g_x1 (ny values): u on the lines
    x = 0 and x = 1 at y_j; g_y0, g_y1 (nx values): u on y = 0 and y = 1 at
    x_i.  Row p = i*ny + j of A is poisson2d_paper's; b_p = f_p minus each
    boundary neighbour's value times its coupling (1/hx^2 or 1/hy^2).
    Returns (A as scipy CSR float64, b float64[n]).
    """
    f = np.asarray(f, dtype=np.float64)
    nx, ny = f.shape
    hx = 1.0 / (nx + 1) if h is None else float(h)
    hy = 1.0 / (ny + 1) if h is None else float(h)
    A = poisson2d_paper(nx, ny, hx, hy)
    b = f.copy()
    b[0, :] -= np.asarray(g_x0, dtype=np.float64) / hx**2
    b[-1, :] -= np.asarray(g_x1, dtype=np.float64) / hx**2
    b[:, 0] -= np.asarray(g_y0, dtype=np.float64) / hy**2
    b[:, -1] -= np.asarray(g_y1, dtype=np.float64) / hy**2
    return A, b.ravel()
