"""Several right-hand sides per tree traversal: parity with the oracle's
dense solve, and bit-identical columns whether solved alone or together
(each column's sums run in the same order in every kernel width)."""
import numpy as np
import pytest

from paper_2009_08167_gb300.inputs import Mesh, normal
from tests.gpu_helpers import oracle_matrices, riga_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    r = riga_ctx()
    yield r
    r.close()


def _check(R, N, solve_dense, sigma):
    rng = np.random.default_rng(7)
    B = np.asfortranarray(rng.normal(size=(N, 7)))
    X, _ = R.solve(B)
    for j in range(7):
        xr = solve_dense(B[:, j])
        assert np.linalg.norm(X[:, j] - xr) <= 1e-10 * np.linalg.norm(xr), j
        xs, _ = R.solve(np.ascontiguousarray(B[:, j]))
        assert np.array_equal(xs, X[:, j]), j  # grouping does not change a column


@pytest.mark.parametrize("mesh", [Mesh(2, 24, 3, 8, 8), Mesh(2, [20, 13], 2, 5, 4)], ids=["2d_p3", "2d_p2"])
def test_multirhs_single_problem(R, mesh):
    R.assemble(mesh)
    K, M = oracle_matrices(mesh)
    A = K.todense() - 37.0 * M.todense()
    R.factor(37.0)
    _check(R, K.n, lambda b: np.linalg.solve(A, b), 37.0)


def test_multirhs_batch_of_many_trees(R):
    meshes = [Mesh(2, 6 + b % 7, 2 + b % 2, 3 + b % 3, 3) for b in range(18)]
    cK = [np.exp(normal(500 + b, m.n_elem, 0.3)) for b, m in enumerate(meshes)]
    R.assemble_batch(meshes, cK)
    mats = [oracle_matrices(m, c, None) for m, c in zip(meshes, cK)]
    R.factor(11.0)
    offs = np.cumsum([0] + [K.n for K, _ in mats])

    def solve_dense(b):
        out = np.empty_like(b)
        for i, (K, M) in enumerate(mats):
            out[offs[i]:offs[i + 1]] = np.linalg.solve(K.todense() - 11.0 * M.todense(), b[offs[i]:offs[i + 1]])
        return out
    _check(R, int(offs[-1]), solve_dense, 11.0)


def test_multirhs_fp32_refined(R):
    from paper_2009_08167_gb300.riga import RIGA_FP32
    mesh = Mesh(2, 24, 3, 8, 8)
    R.assemble(mesh)
    K, M = oracle_matrices(mesh)
    A = K.todense() - 5.0 * M.todense()
    R.factor(5.0, RIGA_FP32)
    B = np.asfortranarray(np.random.default_rng(3).normal(size=(K.n, 5)))
    X, _ = R.solve(B, tol=1e-12)
    for j in range(5):
        xr = np.linalg.solve(A, B[:, j])
        assert np.linalg.norm(X[:, j] - xr) <= 1e-10 * np.linalg.norm(xr), j
