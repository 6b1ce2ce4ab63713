"""GPU accuracy module (riga_eig_errors; Sec. 2 Eq. eigerrors, Sec. 8)
against the oracle's error module (oracle/accuracy.py, pinned by the
Pythagorean identity, brute force and convergence rates):

* parity: EVerr, EFerr_L2 and EFerr_E of the GPU's own eigenpairs computed
  on the device and by the oracle from the same eigenvectors, to 1e-9
  relative (the same Gauss sums in another order; a difference of squares
  is never formed, so tiny errors keep their relative accuracy) plus
  1e-22 absolute;
* Eq. Pythagorean on the GPU results: EFerr_E = EVerr + EFerr_L2;
* the paper's 1D study (Sec. 8, Fig. 12: n_e = 32, p = 3, IGA against rIGA),
  on the 12 lowest modes (N = 33 for IGA): the rIGA space contains the IGA one,
  so rIGA's eigenvalue errors are no larger mode by mode (min-max), both are
  >= 0 up to rounding (Galerkin);
* the 2D study (Figs. 13-14: diagonal modes (i, i), p = 2..5): parity and
  the identity on n_e = 64 meshes.
Only simple eigenvalues (1D, and diagonal modes in 2D) are compared: the
eigenvector of a degenerate eigenvalue is not unique.
"""
import numpy as np
import pytest

from oracle import accuracy, eigen
from paper_2009_08167_gb300.inputs import Mesh
from tests.gpu_helpers import riga_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    r = riga_ctx()
    yield r
    r.set_eig_options(slice=0, precision=0, extra=2, seed=1)
    r.close()


def _parity(mesh, ev, U, modes, g_ev, g_l2, g_e):
    o_ev, o_l2, o_e = accuracy.mode_errors(mesh.dim, mesh.ne, mesh.p, mesh.mults, ev, U, modes)
    for g, o in ((g_ev, o_ev), (g_l2, o_l2), (g_e, o_e)):
        assert np.all(np.abs(g - o) <= 1e-9 * np.abs(o) + 1e-22), (g, o)
    # Eq. Pythagorean on the GPU's numbers
    assert np.all(np.abs(g_e - (g_ev + g_l2)) <= 1e-12 + 1e-8 * g_e)


@pytest.mark.parametrize("bs", [None, 4])
def test_1d_spectrum_ne32_p3(R, bs):
    mesh = Mesh(1, 32, 3, bs, 8)
    R.set_eig_options(slice=0, extra=2, seed=3)
    R.assemble(mesh)
    k = 12
    ev, U, rs = R.eigs(k, 0.0, 1e-10)
    modes = [(i + 1,) for i in range(k)]
    g_ev, g_l2, g_e = R.eig_errors(modes)
    _parity(mesh, ev, U, modes, g_ev, g_l2, g_e)
    assert np.all(g_ev >= -1e-13)


def test_1d_riga_no_worse_than_iga(R):
    errs = {}
    for bs in (None, 4):
        mesh = Mesh(1, 32, 3, bs, 8)
        R.set_eig_options(slice=0, extra=2, seed=3)
        R.assemble(mesh)
        k = 12
        R.eigs(k, 0.0, 1e-10, vectors=False)
        errs[bs] = R.eig_errors([(i + 1,) for i in range(k)])[0]
    assert np.all(errs[4] <= errs[None] + 1e-13)


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_2d_diagonal_modes_ne64(R, p):
    mesh = Mesh(2, 64, p, 16, 8)
    lam, idx, _ = eigen.kron_sum_eigs(2, mesh.ne, p, mesh.mults, k=80, with_vectors=False)
    R.set_eig_options(slice=0, extra=2, seed=4)
    R.assemble(mesh)
    ev, U, rs = R.eigs(80, 0.0, 1e-10)
    diag = [i for i in range(80) if idx[i][0] == idx[i][1]]
    modes = [(int(idx[i][0]) + 1, int(idx[i][1]) + 1) for i in diag]
    # the first eigenpairs of the context are the ones riga_eig_errors reads:
    # compute them all and keep the diagonal ones
    all_modes = [(int(a) + 1, int(b) + 1) for a, b in idx[:80]]
    g_ev, g_l2, g_e = R.eig_errors(all_modes)
    d = np.array(diag)
    _parity(mesh, ev[d], U[:, d], modes, g_ev[d], g_l2[d], g_e[d])
    assert np.all(g_ev[d] > -1e-12)  # Galerkin: lambda_h >= lambda, up to rounding
