"""Preconditioners applied from the right (oracle).

App. D.3 lists the preconditioners; this build uses five of them:
  * none:   M = I
  * jacobi: M = diag(A) ("the inverse of the diagonal elements")
  * ssor:   symmetric SOR with omega = 1 (App. D.3's SOR, as PETSc applies it
            by default: one local symmetric sweep), M = (D + L) D^-1 (D + U)
            with A = L + D + U
  * ilu0:   M = L U, the incomplete LU factorisation with no fill, i.e. L
            and U keep exactly the sparsity pattern of A (App. D.3 item 7).
  * bjacobi: block Jacobi (App. D.3 item 3): M = blockdiag(M_1, ..., M_B)
            over B contiguous row blocks of ceil(n / B) rows (the last one
            ragged), M_b the ILU(0) below of the diagonal block A[b, b].

Reading for block Jacobi: the paper says only that each block is
preconditioned independently from its diagonal part; its runs are PETSc's,
whose default is one block per process of the row distribution and ILU(0)
on each block, and its Darcy block-Jacobi table is for 72 processes.  So
the blocks are contiguous row ranges, B is a parameter, and each block is
factored by the red-black ILU(0) below (red and black as in the whole grid).

Reading for SSOR: omega = 1 (not stated) and the same red-black ordering
as ILU(0) below, so that both sweeps are parallel over one colour each.

Reading for ILU(0) (the paper does not fix the ordering): the unknowns of
the 5/7-point grid are taken in red-black order (red: even i + j [+ l]),
ILU(0) is computed for that reordered matrix, and M is mapped back to the
natural numbering.  With this ordering both triangular solves are two
parallel sweeps over one colour each.

Right preconditioning (a reading; the paper does not state the side): the
Krylov method solves (A M^-1) x_hat = b and x = M^-1 x_hat, so its residual
is the unpreconditioned residual b - A x.

ILU(0) follows the textbook row-by-row (IKJ) elimination restricted to the
pattern of A.  Pins: for a tridiagonal matrix ILU(0) is the exact LU (no
fill is ever produced), and for any pattern the product L U agrees with A
at every position of A's pattern.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def jacobi_inv_diag(A):
    """1 / diag(A)."""
    d = A.diagonal()
    if np.any(d == 0):
        raise ZeroDivisionError("zero diagonal entry")
    return 1.0 / d


def ilu0(A):
    """ILU(0) of a CSR matrix: returns (L unit-lower CSR, U upper CSR).

    For each row i in order, for each k < i in the pattern of row i:
    a_ik <- a_ik / a_kk, then a_ij <- a_ij - a_ik a_kj for every j > k that
    is in the pattern of row i.  Entries outside the pattern are never
    created.
    """
    A = sp.csr_matrix(A, dtype=np.float64, copy=True)
    A.sort_indices()
    n = A.shape[0]
    indptr, indices, data = A.indptr, A.indices, A.data
    diag_pos = np.full(n, -1)
    for i in range(n):
        for q in range(indptr[i], indptr[i + 1]):
            if indices[q] == i:
                diag_pos[i] = q
    if np.any(diag_pos < 0):
        raise ValueError("ILU(0) needs a structurally nonzero diagonal")
    for i in range(n):
        row = {indices[q]: q for q in range(indptr[i], indptr[i + 1])}
        for q in range(indptr[i], indptr[i + 1]):
            kcol = indices[q]
            if kcol >= i:
                break
            data[q] = data[q] / data[diag_pos[kcol]]
            aik = data[q]
            for r in range(indptr[kcol], indptr[kcol + 1]):
                j = indices[r]
                if j > kcol and j in row:
                    data[row[j]] -= aik * data[r]
    L = sp.tril(A, k=-1, format="csr") + sp.identity(n, format="csr")
    U = sp.triu(A, k=0, format="csr")
    return L.tocsr(), U.tocsr()


def redblack_permutation(grid):
    """Red unknowns (even coordinate sum) first, then black; ascending within a colour.

    grid: (nx, ny) or (nx, ny, nz), unknowns numbered with the last index fastest.
    Returns perm with perm[new] = old.
    """
    coords = np.indices(grid).reshape(len(grid), -1)
    color = coords.sum(axis=0) % 2
    return np.concatenate([np.nonzero(color == 0)[0], np.nonzero(color == 1)[0]])


def ilu0_redblack(A, grid):
    """ILU(0) of the red-black reordered matrix: (perm, L, U) with
    A[perm][:, perm] ~ L U on the pattern."""
    perm = redblack_permutation(grid)
    Ap = sp.csr_matrix(A)[perm][:, perm]
    L, U = ilu0(Ap)
    return perm, L, U


def ssor_redblack(A, grid):
    """Symmetric SOR (omega = 1) of the red-black reordered matrix:
    (perm, L', U') with M = (D + L) D^-1 (D + U) = L' U', L' = I + L D^-1 unit
    lower, U' = D + U, where Ap = A[perm][:, perm] = L + D + U."""
    perm = redblack_permutation(grid)
    Ap = sp.csr_matrix(A)[perm][:, perm]
    d = Ap.diagonal()
    if np.any(d == 0):
        raise ZeroDivisionError("zero diagonal entry")
    Lo = sp.tril(Ap, k=-1, format="csr")
    Up = sp.triu(Ap, k=0, format="csr")
    Lp = (sp.identity(Ap.shape[0], format="csr") + Lo @ sp.diags(1.0 / d)).tocsr()
    return perm, Lp, Up


def block_ranges(n, blocks):
    """The B contiguous row blocks of block Jacobi: ceil(n / B) rows each, the last ragged."""
    bs = -(-n // blocks)
    return [(lo, min(lo + bs, n)) for lo in range(0, n, bs)]


class BlockILU0:
    """Block Jacobi with red-black ILU(0) on every diagonal block."""

    def __init__(self, A, grid, blocks):
        A = sp.csr_matrix(A)
        n = A.shape[0]
        coords = np.indices(grid).reshape(len(grid), -1)
        color = coords.sum(axis=0) % 2
        self.parts = []
        for lo, hi in block_ranges(n, blocks):
            rows = np.arange(lo, hi)
            perm = np.concatenate([rows[color[rows] == 0], rows[color[rows] == 1]])
            Ab = A[perm][:, perm]
            L, U = ilu0(Ab)
            self.parts.append((perm, L, U))

    def solve(self, v):
        v = np.asarray(v, dtype=np.float64)
        out = np.empty_like(v)
        for perm, L, U in self.parts:
            y = spla.spsolve_triangular(L, v[perm], lower=True, unit_diagonal=True)
            out[perm] = spla.spsolve_triangular(U, y, lower=False)
        return out


class RightPreconditioner:
    """M^-1 as an operator, for M in {none, jacobi, ssor, ilu0, bjacobi}.

    ssor, ilu0 and bjacobi need the grid shape (red-black ordering, see the
    module readings); blocks is block Jacobi's block count.
    """

    def __init__(self, A, kind, grid=None, blocks=1):
        self.kind = kind
        if kind == "none":
            pass
        elif kind == "jacobi":
            self.dinv = jacobi_inv_diag(A)
        elif kind == "bjacobi":
            if grid is None:
                raise ValueError(kind + " needs the grid shape")
            if blocks < 1:
                raise ValueError("blocks < 1")
            self.block = BlockILU0(A, grid, blocks)
        elif kind in ("ilu0", "ssor"):
            if grid is None:
                raise ValueError(kind + " needs the grid shape")
            self.perm, self.L, self.U = (ilu0_redblack if kind == "ilu0" else ssor_redblack)(A, grid)
        else:
            raise ValueError(kind)

    def apply(self, v):
        if self.kind == "none":
            return np.array(v, dtype=np.float64, copy=True)
        if self.kind == "jacobi":
            return self.dinv * v
        if self.kind == "bjacobi":
            return self.block.solve(v)
        vp = np.asarray(v, dtype=np.float64)[self.perm]
        y = spla.spsolve_triangular(self.L, vp, lower=True, unit_diagonal=True)
        z = spla.spsolve_triangular(self.U, y, lower=False)
        out = np.empty_like(z)
        out[self.perm] = z
        return out
