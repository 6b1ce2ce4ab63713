"""TF32 fronts (Schur updates on the tensor cores, head + tail products):
pivots against the FP64 factorization at about FP32 accuracy, the exact
inertia, refined solves and eigenpairs at the FP64 bars."""
import numpy as np
import pytest

from paper_2009_08167_gb300.inputs import Mesh
from tests.gpu_helpers import oracle_matrices, riga_ctx
from tests.test_gpu_parity import _check_eigs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    r = riga_ctx()
    yield r
    r.set_eig_options(slice=0, precision=0, extra=2, seed=1)
    r.close()


@pytest.mark.parametrize("mesh", [Mesh(2, 24, 3, 8, 8), Mesh(2, 48, 2, 16, 8), Mesh(3, [8, 8, 8], 2, 4, 4)],
                         ids=["2d_p3", "2d_p2_bs16", "3d"])
def test_tf32_factor_matches_fp64(R, mesh):
    from paper_2009_08167_gb300.riga import RIGA_FP64, RIGA_TF32
    R.assemble(mesh)
    n64 = R.factor(17.0, RIGA_FP64)
    D64, _, _ = R.get_factor()
    n32 = R.factor(17.0, RIGA_TF32)
    D32, _, _ = R.get_factor()
    assert n32 == n64
    assert np.max(np.abs(D32 - D64) / np.abs(D64)) <= 1e-4
    K, M = oracle_matrices(mesh)
    A = K.todense() - 17.0 * M.todense()
    b = np.random.default_rng(5).normal(size=K.n)
    x, sweeps = R.solve(b, tol=1e-12)
    xr = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)


def test_tf32_eigs(R):
    R.set_eig_options(slice=0, precision=2, extra=2, seed=7)
    _check_eigs(R, Mesh(2, 24, 3, 8, 8), 16)
    R.set_eig_options(slice=0, precision=0, extra=2, seed=1)
