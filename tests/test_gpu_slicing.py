"""Dynamic spectrum slicing with thick-restart Lanczos (riga_eigs_interval;
Sec. 4.1, Sec. 4.2 Eq. LanczosRestart, Remark on inertia, Sec. 6) against
the Kronecker-sum oracle (Eq. 2Dmatrix): every eigenpair of an interval,
more than 500 of them, with a Lanczos basis bounded by the restart length
and the slice size, not by the number of pairs.

Bars: the count equals the oracle's count in the interval exactly (it comes
from two inertias); eigenvalues 1e-10 relative; residuals rho <= 1e-10;
eigenvector subspaces per cluster 1e-9 in cosine (compare_eigvecs)."""
import numpy as np
import pytest

from oracle import eigen
from paper_2009_08167_gb300.inputs import Mesh
from tests.gpu_helpers import compare_eigvecs_kron, kron_residuals, riga_ctx

pytestmark = pytest.mark.gpu

MESH = Mesh(2, 64, 3, 16, 8)  # N = 71^2 = 5,041


@pytest.fixture(scope="module")
def R():
    r = riga_ctx()
    yield r
    r.set_eig_options(slice=0, precision=0, extra=2, seed=1)
    r.close()


@pytest.fixture(scope="module")
def oracle():
    return eigen.kron_sum_eigs(2, MESH.ne, MESH.p, MESH.mults, k=700)


def _gap_after(lam, i, rel=1e-3):
    """Midpoint of the first relative gap > rel at or after index i."""
    for t in range(i, lam.size - 1):
        if lam[t + 1] - lam[t] > rel * lam[t + 1]:
            return 0.5 * (lam[t] + lam[t + 1]), t + 1
    raise AssertionError("no gap")


def _check(mesh, lam_r, V_r, ev, U, rs, lo_idx, count):
    ref = lam_r[lo_idx:lo_idx + count]
    assert ev.shape == (count,)
    rel = np.abs(ev - ref) / ref
    assert np.max(rel) <= 1e-10, (int(np.argmax(rel)), float(np.max(rel)))
    assert np.max(rs) <= 1e-10
    rho, _ = kron_residuals(mesh, ev, U)
    assert np.max(rho) <= 1e-10
    # the interval ends in gaps, so no cluster is cut
    compare_eigvecs_kron(mesh, V_r[:, lo_idx:lo_idx + count], U, ref, rel=1e-8, tol=1e-9)


def test_interval_over_500_pairs_bounded_basis(R, oracle):
    lam_r, _, V_r = oracle
    hi, count = _gap_after(lam_r, 520)
    assert count >= 520
    R.set_eig_options(slice=50, extra=2, seed=21)
    R.assemble(MESH)
    ev, U, rs, basis = R.eigs_interval(0.0, hi, kmax=700, tol=1e-10)
    _check(MESH, lam_r, V_r, ev, U, rs, 0, count)
    m = max(2 * (50 + 2), 50 + 2 + 40)
    assert basis == 2 * (50 + 2 + 8) + 16 + m + 2
    assert basis < count / 2  # memory bounded by the slices and m, not by the pairs


def test_interior_interval_and_explicit_basis(R, oracle):
    lam_r, _, V_r = oracle
    lo, i0 = _gap_after(lam_r, 200)
    hi, i1 = _gap_after(lam_r, i0 + 90)
    R.set_eig_options(slice=30, extra=2, seed=22)
    R.assemble(MESH)
    ev, U, rs, basis = R.eigs_interval(lo, hi, kmax=400, tol=1e-10, m_basis=48)
    _check(MESH, lam_r, V_r, ev, U, rs, i0, i1 - i0)
    assert basis == 2 * (30 + 2 + 8) + 16 + 48 + 2


def test_interval_count_above_kmax(R, oracle):
    from paper_2009_08167_gb300.riga import RIGA_EINVAL, RigaError
    lam_r, _, _ = oracle
    hi, count = _gap_after(lam_r, 100)
    R.assemble(MESH)
    with pytest.raises(RigaError) as e:
        R.eigs_interval(0.0, hi, kmax=count - 1, tol=1e-10)
    assert e.value.code == RIGA_EINVAL and e.value.count == count
