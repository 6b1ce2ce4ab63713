"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (from the floating-point error of each step, fp64 unit roundoff
1.1e-16): assembly 1e-13 relative to the largest entry (sums of at most
(p+1)^d quadrature products); LDL^T: the componentwise backward-error bound
|PAP^T - LDL^T| <= 1e-13 (|L||D||L^T| + |K| + |sigma||M|) for the GPU factor
and for the oracle's, and pivots and multipliers within the forward-error
bound that this backward error and the conditioning of each pivot imply
(tests.gpu_helpers.ldlt_forward_bounds, first order, times 2); solves 1e-10
relative; eigenvalues 1e-10 relative and residuals 1e-10 (the stated bar of
the FP64 path); eigenvector subspaces 1e-9 in cosine; integer outputs
(orders, inertia) exact.
"""
import numpy as np
import pytest

from oracle import adjoint, assembly, bspline, eigen, factor, symbolic
from paper_2009_08167_gb300.inputs import Mesh, normal
from tests.gpu_helpers import compare_eigvecs, ldlt_forward_bounds, oracle_matrices, riga_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    r = riga_ctx()
    yield r
    r.close()


ASM_CASES = [Mesh(2, 16, 2, None), Mesh(2, [13, 9], 3, 4, 4), Mesh(1, 33, 4, 8), Mesh(3, [5, 4, 6], 2, 2, 3),
             Mesh(2, 64, 3, 16, 8)]


@pytest.mark.parametrize("mesh", ASM_CASES, ids=[repr(m) for m in ASM_CASES])
def test_assembly_parity(R, mesh):
    R.assemble(mesh)
    rp, col, kv, mv = R.get_matrices()
    K, M = oracle_matrices(mesh)
    assert np.array_equal(rp, K.indptr) and np.array_equal(col, K.indices)
    assert np.max(np.abs(kv - K.data)) <= 1e-13 * np.abs(K.data).max()
    assert np.max(np.abs(mv - M.data)) <= 1e-13 * np.abs(M.data).max()


def test_assembly_coefficients_parity(R):
    mesh = Mesh(2, [12, 10], 3, 4, 6)
    ck = np.exp(normal(11, mesh.n_elem, 0.5))
    cm = np.exp(normal(12, mesh.n_elem, 0.25))
    R.assemble(mesh, ck, cm)
    rp, col, kv, mv = R.get_matrices()
    K, M = oracle_matrices(mesh, ck, cm)
    assert np.array_equal(rp, K.indptr) and np.array_equal(col, K.indices)
    assert np.max(np.abs(kv - K.data)) <= 1e-13 * np.abs(K.data).max()
    assert np.max(np.abs(mv - M.data)) <= 1e-13 * np.abs(M.data).max()


def _gap_shifts(lam, count):
    gaps = [i for i in range(lam.size - 1) if lam[i + 1] - lam[i] > 1e-3 * lam[i]]
    pick = [gaps[len(gaps) * j // (count + 1)] for j in range(1, count + 1)]
    return [0.5 * (lam[i] + lam[i + 1]) for i in pick]


# componentwise backward-error bar of each FP64 factorization, relative to
# |L||D||L^T| + |K| + |sigma||M|: n u with n up to a few thousand
EPS_BWD = 1e-13

FACT_CASES = [Mesh(2, 16, 2, None), Mesh(2, 24, 3, 8, 8), Mesh(3, [5, 6, 4], 2, None, 3), Mesh(1, 50, 3, 10, 8)]


@pytest.mark.parametrize("mesh", FACT_CASES, ids=[repr(m) for m in FACT_CASES])
def test_factor_and_solve_parity(R, mesh):
    factor_parity(R, mesh)


def factor_parity(R, mesh):
    """FP64 factor at sigma = 0 and two shifts in gaps against the oracle's
    dense LDL^T of the permuted matrix: inertia, pivots, L entries, the
    componentwise backward error of the GPU factor and one solve."""
    R.assemble(mesh)
    K, M = oracle_matrices(mesh)
    Kd, Md = K.todense(), M.todense()
    lam, _ = eigen.ghep_dense(Kd, Md)
    sym = R.get_symbolic()
    perm = sym["perm"]
    rng = np.random.default_rng(4)
    b = rng.normal(size=K.n)
    for sigma in [0.0] + _gap_shifts(lam, 2):
        nneg = R.factor(sigma)
        assert nneg == int(np.sum(lam < sigma))  # Sylvester inertia, exact
        A = Kd - sigma * Md
        Ap = A[np.ix_(perm, perm)]
        L, d = factor.ldlt_dense(Ap)
        D, Lptr, Lg = R.get_factor(with_L=True)
        pos = np.empty(K.n, dtype=np.int64)
        pos[perm] = np.arange(K.n)
        fp, fi = sym["front_ptr"], sym["front_idx"]
        # the GPU factors its own A = K - sigma M, whose entries differ from
        # the oracle's by rounding of K and sigma M (cancellation), so the
        # data term |K| + |sigma| |M| joins the backward-error bounds
        data = (np.abs(Kd) + abs(sigma) * np.abs(Md))[np.ix_(perm, perm)]
        # the oracle's own componentwise backward error
        Bo = (np.abs(L) * np.abs(d)[None, :]) @ np.abs(L).T + data
        assert np.max(np.abs(Ap - (L * d[None, :]) @ L.T) - EPS_BWD * Bo) <= 0.0
        # both factors are exact LDL^T of matrices within EPS_BWD B of P A P^T
        # (the GPU's bound is asserted below), so they differ by at most the
        # forward bounds of a perturbation 2 EPS_BWD B; the factor 2 covers
        # the second-order terms
        dbound, Lbound = ldlt_forward_bounds(L, d, Bo, 2 * EPS_BWD)
        assert np.all(np.abs(D - d) <= 2 * dbound)
        # L entries of each dense front (lower part of the first k columns)
        for F in range(sym["node_ptr"].size - 1):
            idx = pos[fi[fp[F]:fp[F + 1]]]
            n = idx.size
            k = sym["node_ptr"][F + 1] - sym["node_ptr"][F]
            blk = Lg[Lptr[F]:Lptr[F + 1]].reshape(k, n).T  # column-major n x k
            ref = L[np.ix_(idx, idx[:k])]
            low = np.tril(np.ones((n, k), dtype=bool), -1)
            assert np.all(np.abs(blk[low] - ref[low]) <= 2 * Lbound[np.ix_(idx, idx[:k])][low])
        # componentwise backward error of the GPU factor itself:
        # |P A P^T - L D L^T| <= c u (|L| |D| |L^T| + data), c u = EPS_BWD
        Lfull = np.eye(K.n)
        for F in range(sym["node_ptr"].size - 1):
            idx = pos[fi[fp[F]:fp[F + 1]]]
            n = idx.size
            k = sym["node_ptr"][F + 1] - sym["node_ptr"][F]
            blk = Lg[Lptr[F]:Lptr[F + 1]].reshape(k, n).T
            low = np.tril(np.ones((n, k), dtype=bool), -1)
            sub = np.zeros((n, k))
            sub[low] = blk[low]
            Lfull[np.ix_(idx, idx[:k])] += sub
        R_ = Ap - (Lfull * D[None, :]) @ Lfull.T
        bound = (np.abs(Lfull) * np.abs(D)[None, :]) @ np.abs(Lfull).T + data
        assert np.max(np.abs(R_) - EPS_BWD * bound) <= 0.0
        x, _ = R.solve(b)
        xr = np.linalg.solve(A, b)
        assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)


def test_fp32_factor_refined_solve(R):
    mesh = Mesh(2, 32, 3, 8, 8)
    R.assemble(mesh)
    K, M = oracle_matrices(mesh)
    lam, _ = eigen.ghep_dense(K.todense(), M.todense())
    sigma = _gap_shifts(lam, 1)[0]
    n64 = R.factor(sigma)
    b = np.random.default_rng(5).normal(size=K.n)
    x64, _ = R.solve(b)
    n32 = R.factor(sigma, precision=1)
    assert n32 == n64
    x32, sweeps = R.solve(b, tol=1e-13)
    A = (K.todense() - sigma * M.todense())
    assert np.linalg.norm(A @ x32 - b) <= 1e-12 * np.linalg.norm(b)
    assert np.linalg.norm(x32 - x64) <= 1e-10 * np.linalg.norm(x64)
    assert sweeps >= 2


def _check_eigs(R, mesh, k, sigma=0.0, tol=1e-10, ref=None):
    R.assemble(mesh)
    K, M = oracle_matrices(mesh)
    if ref is None:
        lam, V = eigen.ghep_dense(K.todense(), M.todense())
        above = np.nonzero(lam > sigma)[0]
        lam_all, V_all = lam[above], V[:, above]
        lam_r, V_r = lam_all[:k], V_all[:, :k]
    else:
        lam_all, V_all = ref
        lam_r, V_r = lam_all[:k], V_all[:, :k]
    ev, U, rs = R.eigs(k, sigma, tol)
    assert ev.size == k
    assert np.max(np.abs(ev - lam_r) / np.abs(lam_r)) <= 1e-10
    assert np.max(rs) <= tol
    # M-orthonormality and eigenvector subspaces
    G = U.T @ M.matvec(U)
    assert np.max(np.abs(G - np.eye(k))) <= 1e-9
    compare_eigvecs(V_r, U, M, lam_r, lam_next=lam_all[k] if lam_all.size > k else None)
    return ev, U


def test_eigs_c1(R):
    # 2D Laplace, p=2, 16x16 elements, maximum continuity, lowest 10 pairs, sigma = 0
    R.set_eig_options(slice=0, extra=2, seed=1)
    _check_eigs(R, Mesh(2, 16, 2, None), 10)


def test_eigs_riga_slicing_and_shift(R):
    R.set_eig_options(slice=8, extra=2, seed=3)
    _check_eigs(R, Mesh(2, 24, 3, 8, 8), 24)
    mesh = Mesh(2, 20, 2, 5, 6)
    K, M = oracle_matrices(mesh)
    lam, V = eigen.ghep_dense(K.todense(), M.todense())
    s = 0.5 * (lam[15] + lam[16]) if lam[16] - lam[15] > 1e-3 * lam[15] else 0.5 * (lam[16] + lam[17])
    R.set_eig_options(slice=0, extra=2, seed=4)
    _check_eigs(R, mesh, 12, sigma=s)


def test_eigs_3d_and_1d(R):
    R.set_eig_options(slice=0, extra=3, seed=5)
    _check_eigs(R, Mesh(3, [6, 6, 5], 2, 3, 4), 15)
    R.set_eig_options(slice=0, extra=2, seed=6)
    _check_eigs(R, Mesh(1, 64, 3, 16, 8), 20)


def test_eigs_rayleigh_quotient_option(R):
    """riga_set_eig_accuracy(ctx, 1): the locked eigenvalues are double-double
    Rayleigh quotients of the Ritz vectors.  Both forms meet the oracle bars;
    they differ by the rounding of sigma + 1/theta (far below 1e-12), so the
    residuals change by at most that much (r(lambda') = r(lambda) -
    (lambda' - lambda) M u)."""
    mesh = Mesh(2, 24, 3, 8, 8)
    R.set_eig_options(slice=0, extra=2, seed=7)
    ev0, _ = _check_eigs(R, mesh, 16)
    rs0 = R.eigs(16, 0.0, 1e-10, vectors=False)[2]
    R.set_eig_accuracy(1)
    try:
        ev1, _ = _check_eigs(R, mesh, 16)
        rs1 = R.eigs(16, 0.0, 1e-10, vectors=False)[2]
    finally:
        R.set_eig_accuracy(0)
    assert np.max(np.abs(ev1 - ev0) / ev0) <= 1e-12
    assert np.all(rs1 <= rs0 + 1e-12)
    R.set_eig_options(slice=0, extra=2, seed=1)


def test_eigs_fp32_factor_path(R):
    R.set_eig_options(slice=0, precision=1, extra=2, seed=7)
    _check_eigs(R, Mesh(2, 24, 3, 8, 8), 16)
    R.set_eig_options(slice=0, precision=0, extra=2, seed=1)


def test_eigs_c2_riga_full_size(R):
    # 2D Laplace p=3, 256x256 elements, C0 lines every 16 elements, 100 pairs in
    # slices of 50; the Kronecker-sum oracle gives the exact discrete spectrum
    mesh = Mesh(2, 256, 3, 16, 8)
    lam_r, idx, V_r = eigen.kron_sum_eigs(2, mesh.ne, 3, mesh.mults, k=104)
    R.set_eig_options(slice=50, extra=2, seed=11)
    R.assemble(mesh)
    ev, U, rs = R.eigs(100, 0.0, 1e-10)
    assert np.max(np.abs(ev - lam_r[:100]) / lam_r[:100]) <= 1e-10
    assert np.max(rs) <= 1e-10
    K, M = oracle_matrices(mesh)
    compare_eigvecs(V_r[:, :100], U, M, lam_r[:100], rel=1e-6, lam_next=lam_r[100])
    st = R.stats()
    assert st["n_fact"] >= 2


def test_adjoint_parity_and_homogeneity(R):
    mesh = Mesh(2, [10, 8], 2, 4, 6)
    a = normal(21, mesh.n_elem, 0.5)
    b = normal(22, mesh.n_elem, 0.25)
    R.set_eig_options(slice=0, extra=2, seed=8)
    R.assemble(mesh, np.exp(a), np.exp(b))
    k = 6
    ev, U, rs = R.eigs(k, 0.0, 1e-11)
    w = np.linspace(1.0, 2.0, k)
    ga, gb = R.eig_grad(k, w)
    K, M = oracle_matrices(mesh, np.exp(a), np.exp(b))
    lam, V = eigen.ghep_dense(K.todense(), M.todense())
    ra, rb = adjoint.eig_grad(2, mesh.ne, mesh.p, mesh.mults, np.exp(a), np.exp(b), lam[:k], V[:, :k], w)
    assert np.max(np.abs(ga - ra)) <= 1e-8 * np.abs(ra).max()
    assert np.max(np.abs(gb - rb)) <= 1e-8 * np.abs(rb).max()
    assert abs(ga.sum() - np.sum(w * ev)) <= 1e-9 * np.sum(w * ev)
    assert abs(gb.sum() + np.sum(w * ev)) <= 1e-9 * np.sum(w * ev)


def test_error_paths(R):
    from paper_2009_08167_gb300.riga import RigaError, RIGA_EINVAL, RIGA_ESTATE, Riga
    r2 = Riga(0)
    with pytest.raises(RigaError) as e:
        r2.factor(0.0)
    assert e.value.code == RIGA_ESTATE
    r2.assemble(Mesh(2, 6, 2, None))
    with pytest.raises(RigaError) as e:
        r2.eigs(10 ** 6, 0.0, 1e-10)
    assert e.value.code == RIGA_EINVAL
    with pytest.raises(RigaError):
        r2.assemble(Mesh(2, 6, 2, None), -np.ones(36))
    r2.close()


def test_spmv_parity(R):
    mesh = Mesh(3, [4, 5, 6], 2, None, 3)
    R.assemble(mesh)
    K, M = oracle_matrices(mesh)
    x = np.random.default_rng(9).normal(size=K.n)
    assert np.allclose(R.spmv(0, x), M.matvec(x), rtol=1e-13, atol=1e-15)
    assert np.allclose(R.spmv(1, x), K.matvec(x), rtol=1e-12, atol=1e-12)


def test_wait_budget_exhaustion_reports_timeout(R):
    # a zero wait budget makes the persistent solve's dependency waits give up:
    # the kernel returns, the host reports RIGA_ETIMEOUT, and the context stays
    # usable with the default budget
    from paper_2009_08167_gb300.riga import RigaError, RIGA_ETIMEOUT
    mesh = Mesh(2, 32, 3, 8, 8)
    R.assemble(mesh)
    K, M = oracle_matrices(mesh)
    R.factor(0.0)
    b = np.random.default_rng(13).normal(size=K.n)
    R.set_wait_limit(0)
    with pytest.raises(RigaError) as e:
        R.solve(b)
    assert e.value.code == RIGA_ETIMEOUT
    R.set_wait_limit(1 << 24)
    R.factor(0.0)
    x, _ = R.solve(b)
    xr = np.linalg.solve(K.todense(), b)
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)
