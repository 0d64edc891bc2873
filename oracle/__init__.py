"""FP64 CPU oracle for the sorted-recycling (SKR) solve.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
of the build entry point and the CPU-baseline leg of the benchmark may import
anything from this package.  The CUDA library never calls it, and it calls
nothing of the CUDA library: the two share no code.

It is a plain, slow, obviously checkable restatement of what the method
computes, in float64, following the paper step by step:

  assembly.py   finite-difference discretisation (Sec. 3.1, App. A.2)
  sort.py       the greedy nearest-neighbour sort (Sec. 4.1, Algorithm 1)
                and its large-N grouped form
  precond.py    Jacobi, SSOR, ILU(0) and block-Jacobi preconditioners (App. D.3)
  krylov.py     Arnoldi (Eq. 2-3), restarted GMRES (Sec. 3.2) and GCRO-DR
                with the recycle refresh (Sec. 4.2, Eq. 4, App. B.1,
                Algorithm 2)
  skr.py        a whole sorted sequence with residual refinement

Library primitives used as single steps: numpy/scipy sparse products,
np.linalg.qr, np.linalg.lstsq, np.linalg.eig, scipy.linalg.eig (QZ),
scipy triangular solves.

The pins of each function are listed in the module docstrings.  The paper
prints no worked example of Algorithm 2, so GCRO-DR is pinned by closed
forms and invariants: dense-LU solutions, the Arnoldi relations, exact
harmonic Ritz pairs and the selected eigenvectors on a complete space.
"""
