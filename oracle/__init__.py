"""FP64 CPU oracle for the refined-IGA shift-and-invert eigensolution.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA library in
``paper_2009_08167_gb300/`` and imports nothing from it.

Every function states the passage of arXiv 2009.08167 ("Refined isogeometric
analysis for generalized Hermitian eigenproblems") it follows.  The code is
plain and slow on purpose: numpy arrays, fp64, library primitives (matmul,
sort, a small dense ``eigh``) used only as single steps.

Modules
-------
bspline   open knot vectors with inserted C0 knots, Cox-de Boor basis,
          Gauss-Legendre rule, 1D stiffness/mass matrices (Sec. 3.1, Eq. U,
          Eq. N, Eq. 1Dmatrix, Sec. 3.2)
assembly  Kronecker and per-element assembly of K and M, CSR helpers
          (Eq. 2Dmatrix, Eq. dofs)
symbolic  separator-induced nested-dissection order, fronts, elimination
          tree and column counts (Sec. 3.2, Sec. 5.1, Sec. 6)
factor    LDL^T without pivoting, Sylvester inertia, solves (Sec. 4.2,
          Remark on inertia)
eigen     Kronecker-sum spectra, dense GHEP, shift-and-invert Lanczos with
          full reorthogonalization and locking (Sec. 4.1, Sec. 4.2)
adjoint   per-element eigenvalue sensitivities (not in the paper; the
          definition d lambda = u^T (dK - lambda dM) u for M-normalised u)
"""
