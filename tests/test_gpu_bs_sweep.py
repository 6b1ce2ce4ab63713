"""The rIGA blocksize sweep (Sec. 7, Figs. 6 and 9: factorization, f/b
solve and mat-vec cost against the blocksize) on a small 2D mesh: every
blocksize's DOF count follows Eq. dofs, its eigenvalues match the
Kronecker-sum oracle, and knot insertion nests the spaces (a blocksize that
divides another adds C0 lines to its mesh), so the eigenvalues fall
monotonically from IGA (bs = n_e) down to bs = 1 (Galerkin min-max)."""
import numpy as np
import pytest

from oracle import eigen
from paper_2009_08167_gb300.inputs import Mesh

pytestmark = pytest.mark.gpu


def test_bs_sweep_small_2d():
    import bench

    ne, p, k = 32, 2, 12
    rows = bench.bs_sweep(2, ne, p, k, steps=1)
    assert [r["bs"] for r in rows] == [1, 2, 4, 8, 16, 32]
    prev = None
    for r in rows:
        bs = r["bs"]
        ell = int(np.log2(ne // bs))
        n1 = ne + (2 ** ell) * (p - 1) - 1 if bs < ne else ne + p - 2
        assert r["N"] == n1 ** 2  # Eq. dofs
        mesh = Mesh(2, ne, p, None if bs == ne else bs)
        lam, _, _ = eigen.kron_sum_eigs(2, mesh.ne, p, mesh.mults, k=k, with_vectors=False)
        ev = np.array(r["evals"])
        assert np.max(np.abs(ev - lam) / lam) <= 1e-10
        assert r["pairs"] == k
        for key in ("fact_ms", "fb_ms", "mv_ms", "eigs_ms"):
            assert r[key] > 0
        if prev is not None:
            assert np.all(prev <= ev * (1 + 1e-12))  # the finer-blocked space is richer
        prev = ev
