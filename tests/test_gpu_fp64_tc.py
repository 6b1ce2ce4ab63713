"""FP64 fronts with the Schur updates on the tensor cores (digit slices:
riga_set_fp64_update(ctx, 1)) against the oracle at the FP64 bars.

Pins: the oracle's dense LDL^T of the permuted shifted matrix (pivots 1e-8,
L entries, componentwise backward error 1e-13 (|L||D||L^T| + |K| + |sigma||M|)),
Sylvester's law (the inertia exactly), the dense generalized eigensolver
(eigenvalues 1e-10 relative, residuals 1e-10, eigenvector subspaces), and
the FP64 residual of plain (unrefined) solves on a mesh with fronts of 1820
variables, whose trailing matrices span many 128 x 64 tiles and end in
ragged ones.  The update's error is about 2^-53 of 32 2^(e_i + f_j) per
entry and panel (2^e_i, 2^f_j the row bounds of L21 and L21 D), below an
FP64 dot product's 32 2^-53 of the same bound, so every FP64 bar holds
unchanged.  The operands are balanced by power-of-two |D|^(1/2) column
scalings: without them, near-zero pivots at shifts inside the spectrum put
the row maxima of L21 and L21 D in different columns, and a first version
missed the 1e-10 solve bar (1.5e-10 on the 24^2 p=3 mesh, about 300 times
the FMA path's error there)."""
import numpy as np
import pytest

from oracle import eigen
from paper_2009_08167_gb300.inputs import Mesh, normal
from tests.gpu_helpers import oracle_matrices, riga_ctx
from tests.test_gpu_parity import FACT_CASES, _check_eigs, factor_parity

pytestmark = pytest.mark.gpu

CASES = FACT_CASES + [Mesh(3, [8, 8, 8], 2, 4, 4), Mesh(2, 40, 4, 10, 8)]
LARGE = Mesh(3, 32, 2, 8, 8)  # N = 42,875; largest front 1820 variables


@pytest.fixture(scope="module")
def R():
    r = riga_ctx()
    r.set_fp64_update(1)
    yield r
    r.set_fp64_update(0)
    r.set_eig_options(slice=0, precision=0, extra=2, seed=1)
    r.close()


@pytest.mark.parametrize("mesh", CASES, ids=[repr(m) for m in CASES])
def test_fp64_tc_factor_parity(R, mesh):
    factor_parity(R, mesh)


@pytest.mark.parametrize("mesh", CASES[1:4], ids=[repr(m) for m in CASES[1:4]])
def test_fp64_fma_factor_parity(R, mesh):
    """The CUDA-core FP64 update (riga_set_fp64_update(ctx, 0)) at the same bars."""
    R.set_fp64_update(0)
    try:
        factor_parity(R, mesh)
    finally:
        R.set_fp64_update(1)


def test_fp64_tc_large_fronts_against_fp64_fma(R):
    """Both FP64 update paths on fronts of up to 1820 variables, at sigma = 0
    (SPD: pivots within 1e-12 of each other) and sigma = 40 (indefinite,
    inertia exactly 1: the only eigenvalue below is about 3 pi^2); plain
    FP64 solves (no refinement) reach residual 1e-10 with the tensor-core
    factor."""
    K, M = oracle_matrices(LARGE)
    R.assemble(LARGE)
    B = np.random.default_rng(7).normal(size=(K.n, 2))
    for sigma, nneg, bar in [(0.0, 0, 1e-12), (40.0, 1, 1e-9)]:
        R.set_fp64_update(0)
        assert R.factor(sigma) == nneg
        D0, _, _ = R.get_factor()
        R.set_fp64_update(1)
        assert R.factor(sigma) == nneg
        D1, _, _ = R.get_factor()
        assert np.max(np.abs(D1 - D0) / np.abs(D0)) <= bar, sigma
        X, sweeps = R.solve(np.asfortranarray(B), tol=0.0)
        X = np.asarray(X).reshape(K.n, 2, order="F")
        for j in range(2):
            r = B[:, j] - (K.matvec(X[:, j]) - sigma * M.matvec(X[:, j]))
            assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(B[:, j]), (sigma, j)


def test_fp64_tc_eigs(R):
    R.set_eig_options(slice=8, extra=2, seed=3)
    _check_eigs(R, Mesh(2, 24, 3, 8, 8), 24)
    R.set_eig_options(slice=0, extra=3, seed=5)
    _check_eigs(R, Mesh(3, [8, 8, 8], 2, 4, 4), 15)
    R.set_eig_options(slice=0, extra=2, seed=1)


def test_fp64_tc_eigs_interval(R):
    """Spectrum slicing (inertia-only factorizations skip the extra rows'
    tiles): every pair of an interval ending in a gap."""
    mesh = Mesh(2, 20, 2, 5, 6)
    K, M = oracle_matrices(mesh)
    lam, _ = eigen.ghep_dense(K.todense(), M.todense())
    i = next(t for t in range(30, lam.size - 1) if lam[t + 1] - lam[t] > 1e-3 * lam[t + 1])
    hi = 0.5 * (lam[i] + lam[i + 1])
    R.set_eig_options(slice=12, extra=2, seed=8)
    R.assemble(mesh)
    ev, U, rs, _ = R.eigs_interval(0.0, hi, kmax=200, tol=1e-10)
    assert ev.size == i + 1
    assert np.max(np.abs(ev - lam[:i + 1]) / lam[:i + 1]) <= 1e-10
    assert np.max(rs) <= 1e-10
    R.set_eig_options(slice=0, extra=2, seed=1)


def test_fp64_tc_batch(R):
    """The batch forest (factorizations replayed as CUDA graphs, per-problem
    shifts and inertia) with the tensor-core FP64 updates."""
    meshes = [Mesh(2, 12, 2, 4, 4), Mesh(2, [9, 14], 3, 5, 6), Mesh(1, 40, 2, 8, 8), Mesh(3, [4, 5, 3], 2, 2, 3)]
    cK = [np.exp(normal(100 + b, m.n_elem, 0.5)) for b, m in enumerate(meshes)]
    R.assemble_batch(meshes, cK)
    k = 6
    ev, rs, nc = R.eigs_batch(k, 0.0, 1e-12)
    assert np.all(nc == k) and np.all(rs <= 1e-10)
    for b, (m, c) in enumerate(zip(meshes, cK)):
        K, M = oracle_matrices(m, c, None)
        lam = eigen.ghep_dense(K.todense(), M.todense())[0][:k]
        assert np.max(np.abs(ev[b] - lam) / lam) <= 1e-10, b
