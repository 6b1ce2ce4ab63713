"""GPU parity of the batched path: many independent problems in one forest.

Tolerances as in the single-problem parity tests: assembly 1e-13 relative to
the largest entry, solves 1e-10 relative, eigenvalues 1e-10 relative,
residuals 1e-10, inertia exact.
"""
import numpy as np
import pytest

from oracle import eigen
from paper_2009_08167_gb300.inputs import Mesh, config_c4, normal
from tests.gpu_helpers import oracle_matrices, riga_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    r = riga_ctx()
    yield r
    r.close()


def _small_batch():
    """Problems of uneven size, degree, separator spacing and coefficients,
    including a 1D and a 3D problem in the same forest."""
    meshes = [Mesh(2, 12, 2, 4, 4), Mesh(2, [9, 14], 3, 5, 6), Mesh(2, 7, 3, None), Mesh(1, 40, 2, 8, 8),
              Mesh(3, [4, 5, 3], 2, 2, 3), Mesh(2, 16, 2, 8, 8)]
    cK = [np.exp(normal(100 + b, m.n_elem, 0.5)) for b, m in enumerate(meshes)]
    cK[2] = None  # constant coefficients inside a batch with variable ones
    return meshes, cK


def _block_oracle(meshes, cK):
    return [oracle_matrices(m, c, None) if c is not None else oracle_matrices(m) for m, c in zip(meshes, cK)]


def test_batch_assembly_block_diagonal(R):
    meshes, cK = _small_batch()
    R.assemble_batch(meshes, cK)
    rp, col, kv, mv = R.get_matrices()
    r0 = 0
    e0 = 0
    for (K, M) in _block_oracle(meshes, cK):
        n = K.n
        rows = rp[r0:r0 + n + 1] - rp[r0]
        assert np.array_equal(rows, K.indptr)
        nz = K.nnz
        assert np.array_equal(col[e0:e0 + nz] - r0, K.indices)
        assert np.max(np.abs(kv[e0:e0 + nz] - K.data)) <= 1e-13 * np.abs(K.data).max()
        assert np.max(np.abs(mv[e0:e0 + nz] - M.data)) <= 1e-13 * np.abs(M.data).max()
        r0 += n
        e0 += nz
    assert r0 == rp.size - 1


def test_batch_factor_inertia_and_solve(R):
    meshes, cK = _small_batch()
    R.assemble_batch(meshes, cK)
    mats = _block_oracle(meshes, cK)
    lams = [eigen.ghep_dense(K.todense(), M.todense())[0] for K, M in mats]
    allv = np.sort(np.concatenate(lams))
    sigma = 0.5 * (allv[40] + allv[41])
    nneg = R.factor(sigma)
    assert nneg == int(sum(np.sum(l < sigma) for l in lams))  # Sylvester, summed over the forest
    rng = np.random.default_rng(9)
    N = sum(K.n for K, _ in mats)
    b = rng.normal(size=N)
    x, _ = R.solve(b)
    r0 = 0
    for (K, M) in mats:
        A = K.todense() - sigma * M.todense()
        xr = np.linalg.solve(A, b[r0:r0 + K.n])
        assert np.linalg.norm(x[r0:r0 + K.n] - xr) <= 1e-10 * np.linalg.norm(xr)
        r0 += K.n


def test_batch_eigs_small_vs_oracle(R):
    meshes, cK = _small_batch()
    R.assemble_batch(meshes, cK)
    k = 8
    ev, rs, nc = R.eigs_batch(k, 0.0, 1e-12)
    assert np.all(nc == k)
    assert np.all(rs <= 1e-10)
    for b, (K, M) in enumerate(_block_oracle(meshes, cK)):
        lam = eigen.ghep_dense(K.todense(), M.todense())[0][:k]
        assert np.max(np.abs(ev[b] - lam) / lam) <= 1e-10, b


def test_batch_eigs_shifted(R):
    """A shift inside the spectrum: the k eigenvalues above it, per problem."""
    meshes, cK = _small_batch()
    R.assemble_batch(meshes, cK)
    mats = _block_oracle(meshes, cK)
    lams = [eigen.ghep_dense(K.todense(), M.todense())[0] for K, M in mats]
    sigma = 0.5 * min(l[5] for l in lams) + 0.5 * min(l[6] for l in lams)
    k = 5
    ev, rs, nc = R.eigs_batch(k, sigma, 1e-12)
    assert np.all(nc == k)
    for b, lam in enumerate(lams):
        ref = lam[lam > sigma][:k]
        assert np.max(np.abs(ev[b] - ref) / ref) <= 1e-10, b


def _many_batch():
    """Twenty small 2D problems: a batch wide enough for the warp-per-item
    solve kernel (at least 16 trees)."""
    meshes, cK = [], []
    for b in range(20):
        ne = 6 + (7 * b) % 11
        m = Mesh(2, [ne, ne + b % 3], 2 + b % 2, 3 + b % 4, 3 + b % 5)
        meshes.append(m)
        cK.append(np.exp(normal(300 + b, m.n_elem, 0.5)))
    return meshes, cK


def test_batch_many_trees_solve_and_eigs(R):
    meshes, cK = _many_batch()
    R.assemble_batch(meshes, cK)
    mats = _block_oracle(meshes, cK)
    lams = [eigen.ghep_dense(K.todense(), M.todense())[0] for K, M in mats]
    sigma = 0.5 * (np.sort(np.concatenate(lams))[100] + np.sort(np.concatenate(lams))[101])
    assert R.factor(sigma) == int(sum(np.sum(l < sigma) for l in lams))
    N = sum(K.n for K, _ in mats)
    b = np.random.default_rng(21).normal(size=N)
    x, _ = R.solve(b)
    r0 = 0
    for (K, M) in mats:
        xr = np.linalg.solve(K.todense() - sigma * M.todense(), b[r0:r0 + K.n])
        assert np.linalg.norm(x[r0:r0 + K.n] - xr) <= 1e-10 * np.linalg.norm(xr)
        r0 += K.n
    k = 6
    ev, rs, nc = R.eigs_batch(k, 0.0, 1e-12)
    assert np.all(nc == k) and np.all(rs <= 1e-10)
    for bb, lam in enumerate(lams):
        assert np.max(np.abs(ev[bb] - lam[:k]) / lam[:k]) <= 1e-10, bb


def test_batch_errors(R):
    from paper_2009_08167_gb300.riga import RigaError, RIGA_EINVAL, RIGA_ESTATE
    meshes, cK = _small_batch()
    R.assemble_batch(meshes, cK)
    with pytest.raises(RigaError) as e:
        R.eigs(4)
    assert e.value.code == RIGA_ESTATE
    with pytest.raises(RigaError) as e:
        R.eigs_batch(44, 0.0, 1e-10)  # more pairs than the 1D problem (44 DOFs) holds
    assert e.value.code == RIGA_EINVAL
    bad = [Mesh(2, 8, 2, None), Mesh(2, 8, 9, None)]
    with pytest.raises(RigaError) as e:
        R.assemble_batch(bad)
    assert e.value.code == RIGA_EINVAL
    # a single problem afterwards replaces the batch
    m = Mesh(2, 10, 2, None)
    R.assemble(m)
    ev, _, _ = R.eigs(4, 0.0, 1e-12, vectors=False)
    K, M = oracle_matrices(m)
    lam = eigen.ghep_dense(K.todense(), M.todense())[0][:4]
    assert np.max(np.abs(ev - lam) / lam) <= 1e-10


def test_batch_c4_full(R):
    """The full 512-problem batch (20 pairs each): every pair's FP64 residual,
    completeness of the whole batch by one inertia count, and sampled problems
    against the oracle's shift-and-invert Lanczos."""
    probs = config_c4()
    meshes = [p["mesh"] for p in probs]
    cK = [np.exp(p["a"]) for p in probs]
    R.assemble_batch(meshes, cK)
    k = 20
    ev, rs, nc = R.eigs_batch(k, 0.0, 1e-10)
    assert np.all(nc == k)
    assert np.all(rs <= 1e-10)
    assert np.all(np.diff(ev, axis=1) >= 0)
    # completeness: below a shift under every problem's 20th eigenvalue, the
    # forest's inertia equals the number of returned eigenvalues
    s = 0.5 * (np.min(ev[:, k - 1]) + np.min(ev[:, k - 2]))
    cnt = int(np.sum(ev < s))
    if np.min(np.abs(ev - s)) > 1e-8 * s:
        assert R.factor(s) == cnt
    # sampled problems: the three smallest meshes
    order = np.argsort([m.ne[0] for m in meshes])[:3]
    for b in order:
        K, M = oracle_matrices(meshes[b], cK[b], None)
        lam, _, _ = eigen.lanczos_shift_invert(K, M, k, 0.0, tol=1e-12, seed=3)
        assert np.max(np.abs(ev[b] - lam) / lam) <= 1e-10, b


def test_autotune_tile_shapes_change_no_result(R):
    """riga_autotune times the factorization for each tile cut-off and keeps
    the fastest; every entry's update sums the same products in the same
    order whatever the tile shape, so the pivots are bit-identical, and the
    batch's eigenpairs still match the oracle."""
    meshes, cK = _small_batch()
    R.assemble_batch(meshes, cK)
    R.factor(0.0)
    D0 = R.get_factor()[0].copy()
    t, ms = R.autotune()
    assert t in (0, 128, 256, 512, 1024, 4096)
    assert all(m > 0.0 for m in ms)
    assert np.array_equal(R.get_factor()[0], D0)
    k = 8
    ev, rs, nc = R.eigs_batch(k, 0.0, 1e-12)
    assert np.all(nc == k)
    assert np.all(rs <= 1e-10)
    for b, (K, M) in enumerate(_block_oracle(meshes, cK)):
        lam = eigen.ghep_dense(K.todense(), M.todense())[0][:k]
        assert np.max(np.abs(ev[b] - lam) / lam) <= 1e-10, b


@pytest.mark.parametrize("prec", [1, 2], ids=["fp32", "tf32"])
def test_batch_c4_full_mixed(R, prec):
    """The 512-problem batch with low-precision fronts (FP32 FFMA, or TF32
    tensor-core Schur updates) and FP64 refinement: every pair's FP64
    residual <= 1e-10, the eigenvalues of the FP64 batch path to 1e-10
    relative, one forest inertia count, and the three smallest problems
    against the oracle's shift-and-invert Lanczos."""
    probs = config_c4()
    meshes = [p["mesh"] for p in probs]
    cK = [np.exp(p["a"]) for p in probs]
    R.assemble_batch(meshes, cK)
    k = 20
    R.set_eig_options(slice=0, precision=0, extra=2, seed=1)
    ev64, _, _ = R.eigs_batch(k, 0.0, 1e-10)
    R.set_eig_options(slice=0, precision=prec, extra=2, seed=1)
    try:
        ev, rs, nc = R.eigs_batch(k, 0.0, 1e-10)
    finally:
        R.set_eig_options(slice=0, precision=0, extra=2, seed=1)
    assert np.all(nc == k)
    assert np.all(rs <= 1e-10)
    assert np.max(np.abs(ev - ev64) / ev64) <= 1e-10
    s = 0.5 * (np.min(ev[:, k - 1]) + np.min(ev[:, k - 2]))
    cnt = int(np.sum(ev < s))
    if np.min(np.abs(ev - s)) > 1e-8 * s:
        assert R.factor(s) == cnt
    order = np.argsort([m.ne[0] for m in meshes])[:3]
    for b in order:
        K, M = oracle_matrices(meshes[b], cK[b], None)
        lam, _, _ = eigen.lanczos_shift_invert(K, M, k, 0.0, tol=1e-12, seed=3)
        assert np.max(np.abs(ev[b] - lam) / lam) <= 1e-10, b
