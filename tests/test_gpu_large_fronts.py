"""GPU: factor and tree solve on a 3D mesh whose fronts exceed 1536 variables.

That is the large-front shape of the solve: 256-thread CTAs, up to 256 parts
per front, two panel slots per CTA (the next item's copies run while the
current item computes).  The 2D and small 3D cases of the other files never
reach it.

Pins: the oracle's K and M (Kronecker assembly) and Sylvester's law.  At
sigma = 40 the only eigenvalue below the shift is lambda_1 (about 3 pi^2 =
29.6; the next, 6 pi^2 = 59.2, is triple), so the inertia is exactly 1.  Each
solve is checked by its FP64 residual ||b - (K - sigma M) x|| <= 1e-10 ||b||:
the FP64 factor is backward stable and cond(K - sigma M) of this mesh is
about 1e4 at this shift (residuals near 1e-13 are expected); the FP32 and
TF32 factors reach the bar through FP64 iterative refinement (tol 1e-12); so does
the BF16 one (about 2^-16 relative per update term, cond about 1e4: a
contraction of roughly 0.15 per sweep).
"""
import numpy as np
import pytest

from paper_2009_08167_gb300.inputs import Mesh
from tests.gpu_helpers import oracle_matrices, riga_ctx

pytestmark = pytest.mark.gpu

LARGE = Mesh(3, 32, 2, 8, 8)  # N = 42,875; largest front 1820 variables


@pytest.fixture(scope="module")
def R():
    r = riga_ctx()
    yield r
    r.close()


@pytest.fixture(scope="module")
def KM():
    return oracle_matrices(LARGE)


def test_large_front_shape(R):
    R.assemble(LARGE)
    sym = R.get_symbolic()
    assert int(np.max(np.diff(sym["front_ptr"]))) > 1536


@pytest.mark.parametrize("precision", [0, 1, 2, 3], ids=["fp64", "fp32", "tf32", "bf16"])
def test_large_front_factor_and_solve(R, KM, precision):
    K, M = KM
    R.assemble(LARGE)
    sigma = 40.0
    assert R.factor(sigma, precision=precision) == 1
    B = np.random.default_rng(7).normal(size=(K.n, 3))
    X, sweeps = R.solve(np.asfortranarray(B), tol=0.0 if precision == 0 else 1e-12)
    X = np.asarray(X).reshape(K.n, 3, order="F")
    for j in range(3):
        r = B[:, j] - (K.matvec(X[:, j]) - sigma * M.matvec(X[:, j]))
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(B[:, j]), (precision, j)
    if precision != 0:
        assert sweeps >= 2
