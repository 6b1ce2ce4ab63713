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


@pytest.mark.parametrize("mesh", [Mesh(2, 24, 3, 8, 8), Mesh(2, 48, 2, 16, 8), Mesh(3, [8, 8, 8], 2, 4, 4)],
                         ids=["2d_p3", "2d_p2_bs16", "3d"])
def test_bf16_factor_matches_fp64(R, mesh):
    """BF16 tensor-core Schur updates (head + tail BF16 products, FP32
    accumulation, power-of-two block scaling): each update term carries a
    relative error of about 2^-16 (two 8-bit significands), so the pivots
    stay within 5e-3 of FP64 (rounding accumulated over the eliminated
    columns, amplified by the growth of an unpivoted indefinite
    factorization); the inertia at a shift in a wide gap is exact; FP64
    refinement recovers solves to 1e-10 when cond(A) 2^-16 < 1."""
    from paper_2009_08167_gb300.riga import RIGA_BF16, RIGA_FP64
    R.assemble(mesh)
    n64 = R.factor(17.0, RIGA_FP64)
    D64, _, _ = R.get_factor()
    nb = R.factor(17.0, RIGA_BF16)
    Db, _, _ = R.get_factor()
    assert nb == n64
    assert np.max(np.abs(Db - D64) / np.abs(D64)) <= 5e-3
    K, M = oracle_matrices(mesh)
    A = K.todense() - 17.0 * M.todense()
    b = np.random.default_rng(6).normal(size=K.n)
    x, sweeps = R.solve(b, tol=1e-12)
    xr = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)


def test_bf16_and_tf32_agree_on_larger_fronts(R):
    """Both tensor-core modes on a 3D mesh with fronts above 1000 variables,
    at a shift inside the spectrum (A indefinite): the inertia of FP64
    exactly; the median pivot within 1e-6 (TF32 head + tail) / 1e-4 (BF16
    head + tail) relative of FP64 and the pivots normwise within 5e-2 (a
    pivot close to zero carries the absolute error of the sum it comes
    from: its relative error is unbounded in any working precision, FP32
    FFMA's included); refined solves at the FP64 bar, the criterion the
    eigensolver relies on."""
    from paper_2009_08167_gb300.riga import RIGA_BF16, RIGA_FP64, RIGA_TF32
    mesh = Mesh(3, [16, 16, 16], 2, 8, 8)
    R.assemble(mesh)
    sigma = 40.0
    n64 = R.factor(sigma, RIGA_FP64)
    D64, _, _ = R.get_factor()
    K, M = oracle_matrices(mesh)
    b = np.random.default_rng(8).normal(size=K.n)
    for prec, med in ((RIGA_TF32, 1e-6), (RIGA_BF16, 1e-4)):
        assert R.factor(sigma, prec) == n64
        Dp, _, _ = R.get_factor()
        ep = np.abs(Dp - D64)
        assert np.median(ep / np.abs(D64)) <= med, prec
        assert np.max(ep) <= 5e-2 * np.max(np.abs(D64)), prec
        x, sweeps = R.solve(b, tol=1e-12)
        r = b - (K.matvec(x) - sigma * M.matvec(x))
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b), prec


def test_bf16_eigs(R):
    R.set_eig_options(slice=0, precision=3, extra=2, seed=7)
    _check_eigs(R, Mesh(2, 24, 3, 8, 8), 16)
    R.set_eig_options(slice=0, precision=0, extra=2, seed=1)
