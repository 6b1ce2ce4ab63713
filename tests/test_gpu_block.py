"""Block shift-and-invert Lanczos (block sizes 2 and 4) against the oracle:
eigenvalues, FP64 residuals, M-orthonormality and eigenvector subspaces, on
meshes with exact multiplicities (symmetric squares and cubes), spectrum
slicing, an interior shift, FP32 fronts, and the full-size 2D workload
against its Kronecker-sum spectrum.  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from oracle import eigen
from paper_2009_08167_gb300.inputs import Mesh
from tests.gpu_helpers import compare_eigvecs, oracle_matrices, riga_ctx
from tests.test_gpu_parity import _check_eigs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    r = riga_ctx()
    yield r
    r.set_eig_block(1)
    r.close()


@pytest.mark.parametrize("block", [2, 4])
def test_block_c1(R, block):
    R.set_eig_block(block)
    R.set_eig_options(slice=0, extra=2, seed=1)
    _check_eigs(R, Mesh(2, 16, 2, None), 10)


@pytest.mark.parametrize("block", [2, 4])
def test_block_slicing_shift_3d(R, block):
    R.set_eig_block(block)
    R.set_eig_options(slice=8, extra=2, seed=3)
    _check_eigs(R, Mesh(2, 24, 3, 8, 8), 24)
    mesh = Mesh(2, 20, 2, 5, 6)
    K, M = oracle_matrices(mesh)
    lam, V = eigen.ghep_dense(K.todense(), M.todense())
    s = 0.5 * (lam[15] + lam[16]) if lam[16] - lam[15] > 1e-3 * lam[15] else 0.5 * (lam[16] + lam[17])
    R.set_eig_options(slice=0, extra=2, seed=4)
    _check_eigs(R, mesh, 12, sigma=s)
    R.set_eig_options(slice=0, extra=3, seed=5)
    _check_eigs(R, Mesh(3, [6, 6, 6], 2, 3, 4), 15)  # multiplicities 3 and 6


def test_block_fp32_fronts(R):
    R.set_eig_block(4)
    R.set_eig_options(slice=0, precision=1, extra=2, seed=7)
    _check_eigs(R, Mesh(2, 24, 3, 8, 8), 16)
    R.set_eig_options(slice=0, precision=0, extra=2, seed=1)


def test_block_c2_full_size(R):
    mesh = Mesh(2, 256, 3, 16, 8)
    lam_r, idx, V_r = eigen.kron_sum_eigs(2, mesh.ne, 3, mesh.mults, k=104)
    R.set_eig_block(4)
    R.set_eig_options(slice=50, extra=2, seed=11)
    R.assemble(mesh)
    ev, U, rs = R.eigs(100, 0.0, 1e-10)
    assert np.max(np.abs(ev - lam_r[:100]) / lam_r[:100]) <= 1e-10
    assert np.max(rs) <= 1e-10
    K, M = oracle_matrices(mesh)
    compare_eigvecs(V_r[:, :100], U, M, lam_r[:100], rel=1e-6, lam_next=lam_r[100])


def test_block_size_errors(R):
    from paper_2009_08167_gb300.riga import RigaError, RIGA_EINVAL
    with pytest.raises(RigaError) as e:
        R.set_eig_block(3)
    assert e.value.code == RIGA_EINVAL
    R.set_eig_block(1)
