"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped
Kronecker term, a wrong sign, a transposed index, a wrong quadrature) fails
at least one of them.  None of these compares the oracle with itself.
"""
import os

import numpy as np
import pytest

from oracle import adjoint, assembly, bspline, eigen, factor, symbolic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")


def _golden(kind):
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            parts = line.split()
            if parts[0] == kind:
                rows.append(parts[1:])
    assert rows, kind
    return rows


# ---------------------------------------------------------------- quadrature
def test_gauss_legendre_closed_forms():
    t, w = bspline.gauss_legendre(1)
    assert np.allclose(t, [0.0]) and np.allclose(w, [2.0])
    t, w = bspline.gauss_legendre(2)
    assert np.allclose(t, [-1 / np.sqrt(3), 1 / np.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [1, 1], atol=1e-15)
    t, w = bspline.gauss_legendre(3)
    assert np.allclose(t, [-np.sqrt(0.6), 0, np.sqrt(0.6)], atol=1e-15)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


@pytest.mark.parametrize("nq", [1, 2, 3, 4, 6])
def test_gauss_legendre_exactness(nq):
    t, w = bspline.gauss_legendre(nq)
    for deg in range(2 * nq):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.sum(w * t ** deg) - exact) < 1e-14
    deg = 2 * nq
    assert abs(np.sum(w * t ** deg) - 2.0 / (deg + 1)) > 1e-6


# --------------------------------------------------------------------- basis
@pytest.mark.parametrize("p,bs", [(1, None), (2, None), (3, None), (3, 4), (2, 2)])
def test_basis_partition_of_unity_and_derivative(p, bs):
    ne = 8
    mult = bspline.riga_multiplicities(ne, p, bs) if bs else None
    knots = bspline.open_knot_vector(ne, p, mult)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, 200)
    vals, ders = bspline.basis_and_derivative(knots, p, x)
    assert np.allclose(vals.sum(axis=0), 1.0, atol=1e-14)
    assert np.all(vals >= -1e-15)
    assert np.allclose(ders.sum(axis=0), 0.0, atol=1e-12)
    # derivative against a central difference away from the knots
    eps = 1e-6
    xs = np.array([0.0625 + 0.125 * i for i in range(ne)]) + 0.01
    vp, _ = bspline.basis_and_derivative(knots, p, xs + eps)
    vm, _ = bspline.basis_and_derivative(knots, p, xs - eps)
    _, d0 = bspline.basis_and_derivative(knots, p, xs)
    assert np.allclose((vp - vm) / (2 * eps), d0, atol=1e-6)


def test_basis_linear_hat_closed_form():
    ne = 4
    knots = bspline.open_knot_vector(ne, 1)
    x = np.array([0.1, 0.3, 0.6, 0.9])
    vals, _ = bspline.basis_and_derivative(knots, 1, x)
    h = 1 / ne
    for i in range(ne + 1):
        hat = np.maximum(0, 1 - np.abs(x - i * h) / h)
        assert np.allclose(vals[i], hat, atol=1e-15)


def test_c0_dofs_interpolate():
    # at a multiplicity-p knot exactly one function is non-zero and equals 1
    for p in (2, 3, 4):
        ne, bs = 32, 8
        mult = bspline.riga_multiplicities(ne, p, bs)
        c0 = bspline.c0_dofs(ne, p, mult)
        assert len(c0) == ne // bs - 1
        # block interiors have bs + p - 2 DOFs between consecutive C0 DOFs
        assert np.all(np.diff(c0) == bs + p - 1)
        assert c0[0] == bs + p - 2


# ---------------------------------------------------------------- 1D matrices
def test_p1_matrices_closed_form():
    ne = 10
    h = 1 / ne
    K, M = bspline.matrices_1d(ne, 1)
    n = ne - 1
    Kc = (2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)) / h
    Mc = (4 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)) * h / 6
    assert np.allclose(K, Kc, atol=1e-12)
    assert np.allclose(M, Mc, atol=1e-15)


def test_p1_spectrum_closed_form():
    # sine eigenvectors of the tridiagonal pair give
    # lambda_k = (6/h^2) (1 - cos k pi h) / (2 + cos k pi h)
    ne = 40
    h = 1 / ne
    lam, _ = eigen.eig1d(ne, 1)
    k = np.arange(1, ne)
    cf = (6 / h ** 2) * (1 - np.cos(k * np.pi * h)) / (2 + np.cos(k * np.pi * h))
    assert np.max(np.abs(lam - cf) / cf) < 1e-12


@pytest.mark.parametrize("p,bs", [(2, None), (3, None), (3, 4), (4, 2)])
def test_partition_of_unity_and_neumann_kernel(p, bs):
    ne = 8
    mult = bspline.riga_multiplicities(ne, p, bs) if bs else None
    K, M = bspline.matrices_1d(ne, p, mult, dirichlet=False)
    assert abs(M.sum() - 1.0) < 1e-14  # length of (0,1)
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-11  # K 1 = 0
    assert np.allclose(K, K.T) and np.allclose(M, M.T)
    # 2D: sum M = area, K 1 = 0 with the Kronecker construction
    Kx, Mx = assembly.assemble_kron(2, [ne, ne], p, [mult, mult], dirichlet=False)
    assert abs(Mx.data.sum() - 1.0) < 1e-13
    assert np.abs(Kx.matvec(np.ones(Kx.n))).max() < 1e-10


def test_mass_integrates_polynomials():
    # M^x_ij = int B_i B_j: sum_j M_ij = int B_i, and int B_i = (t_{i+p+1}-t_i)/(p+1)
    for p, bs in [(2, None), (3, 4)]:
        ne = 8
        mult = bspline.riga_multiplicities(ne, p, bs) if bs else None
        knots = bspline.open_knot_vector(ne, p, mult)
        _, M = bspline.matrices_1d(ne, p, mult, dirichlet=False)
        n = M.shape[0]
        integ = np.array([(knots[i + p + 1] - knots[i]) / (p + 1) for i in range(n)])
        assert np.allclose(M.sum(axis=1), integ, atol=1e-15)


def test_coefficient_assembly_reduces_to_kronecker():
    for p, bs in [(2, None), (3, 4)]:
        ne = [6, 5]
        mults = [bspline.riga_multiplicities(n, p, bs) if bs else None for n in ne]
        Kk, Mk = assembly.assemble_kron(2, ne, p, mults)
        Kc, Mc = assembly.assemble_coef(2, ne, p, mults, None, None)
        assert np.array_equal(Kk.indices, Kc.indices)
        assert np.allclose(Kk.data, Kc.data, atol=1e-13)
        assert np.allclose(Mk.data, Mc.data, atol=1e-16)
        # scaling every coefficient scales the matrices
        Kc2, Mc2 = assembly.assemble_coef(2, ne, p, mults, np.full(30, 2.0), np.full(30, 3.0))
        assert np.allclose(Kc2.data, 2 * Kk.data) and np.allclose(Mc2.data, 3 * Mk.data)


def test_coefficient_assembly_area_weighted():
    rng = np.random.default_rng(3)
    ne = [4, 5]
    cm = np.exp(rng.normal(size=20))
    _, M = assembly.assemble_coef(2, ne, 2, None, None, cm, dirichlet=False)
    assert abs(M.data.sum() - np.sum(cm) / 20) < 1e-13  # sum_e exp(b_e) |e|


# -------------------------------------------------------------- counts (paper)
def test_dof_counts_eq_dofs():
    for d, ne, p, lev, val in _golden("dofs"):
        d, ne, p, lev, val = int(d), int(ne), int(p), int(lev), int(val)
        bs = ne // (2 ** lev) if lev > 0 else None
        mults = [bspline.riga_multiplicities(ne, p, bs) if bs else None] * d
        _, N = assembly.dof_count(d, [ne] * d, p, mults)
        assert N == val
        formula = (ne + p - 2) ** d if lev == 0 else (ne + 2 ** lev * (p - 1) - 1) ** d
        assert N == formula


def test_nnz_iga_eq_nonzeros():
    for d, ne, p, _, val in _golden("nnz_iga"):
        d, ne, p, val = int(d), int(ne), int(p), int(val)
        P = assembly.pattern_1d(ne, p, None, dirichlet=False)
        assert int(P.sum()) ** d == val


def test_nnz_riga_exact_and_ratio_claim():
    # exact 1D count for rIGA: 2^l [2^-l ne (2p+1) + p^2 - 1] + 1 (the printed
    # Eq. nonzeros omits the trailing +1 per direction)
    for ne, p, bs in [(64, 2, 16), (128, 3, 16), (256, 5, 16), (32, 3, 8)]:
        lev = int(np.log2(ne // bs))
        P = assembly.pattern_1d(ne, p, bspline.riga_multiplicities(ne, p, bs), dirichlet=False)
        exact = 2 ** lev * (ne // 2 ** lev * (2 * p + 1) + p * p - 1) + 1
        assert int(P.sum()) == exact
    for d, ne, p, lev, claim in _golden("ratio"):
        ne, p, lev, claim = int(ne), int(p), int(lev), float(claim)
        bs = ne // 2 ** lev
        r = 2 ** lev * (ne // 2 ** lev * (2 * p + 1) + p * p - 1) + 1
        i = ne * (2 * p + 1) + p * p
        assert abs(r / i - claim) < 0.01


# --------------------------------------------------------------- eigenvalues
def test_kronecker_sum_equals_dense_ghep():
    for d, ne, p, bs in [(2, [6, 5], 2, None), (2, [8, 8], 3, 4), (3, [3, 4, 3], 2, None)]:
        mults = [bspline.riga_multiplicities(n, p, bs) if bs else None for n in ne]
        K, M = assembly.assemble_kron(d, ne, p, mults)
        lam, V = eigen.ghep_dense(K.todense(), M.todense())
        lk, _, Vk = eigen.kron_sum_eigs(d, ne, p, mults)
        assert np.max(np.abs(lam - lk) / lk) < 1e-12
        # Kronecker eigenvectors are eigenvectors of the assembled pencil
        rho = eigen.residual_rho(K, M, lk, Vk)
        assert rho.max() < 1e-12


def test_continuum_bounds_and_convergence():
    exact = [int(v) for v in _golden("exact")[0][-1].split(",")]
    prev = None
    for ne in (8, 16, 32):
        lam, _, _ = eigen.kron_sum_eigs(2, [ne, ne], 3, k=10, with_vectors=False)
        r = lam / np.pi ** 2
        assert np.all(r >= np.array(exact) - 1e-12)  # Galerkin upper bounds
        err = np.max(r / np.array(exact) - 1)
        if prev is not None:
            assert err < prev / 8  # high-order convergence
        prev = err
    assert prev < 1e-6
    exact3 = [int(v) for v in _golden("exact")[1][-1].split(",")]
    lam, _, _ = eigen.kron_sum_eigs(3, [8, 8, 8], 2, k=10, with_vectors=False)
    assert np.all(lam / np.pi ** 2 >= np.array(exact3) - 1e-12)
    assert np.max(lam / np.pi ** 2 / np.array(exact3) - 1) < 1e-2


def test_riga_enriches_space():
    # knot insertion nests the IGA space inside the rIGA space: min-max gives
    # lambda_i(rIGA) <= lambda_i(IGA) for i <= N_IGA (Sec. 3.2)
    ne, p = 16, 3
    li, _ = eigen.eig1d(ne, p)
    lr, _ = eigen.eig1d(ne, p, bspline.riga_multiplicities(ne, p, 4))
    assert lr.size > li.size
    assert np.all(lr[:li.size] <= li * (1 + 1e-13))


# -------------------------------------------------------------------- factor
def test_ldlt_dense_reconstructs_and_inertia():
    K, M = assembly.assemble_kron(2, [6, 6], 2)
    A = K.todense()
    Mm = M.todense()
    lam, _ = eigen.ghep_dense(A, Mm)
    gaps = [i for i in range(lam.size - 1) if lam[i + 1] - lam[i] > 1e-3 * lam[i]]
    for sigma in (0.0, 0.5 * (lam[gaps[2]] + lam[gaps[2] + 1]), 0.5 * (lam[gaps[5]] + lam[gaps[5] + 1])):
        S = A - sigma * Mm
        L, d = factor.ldlt_dense(S)
        assert np.allclose(L @ np.diag(d) @ L.T, S, atol=1e-10 * np.abs(S).max())
        assert np.allclose(np.triu(L, 1), 0) and np.allclose(np.diag(L), 1)
        # Sylvester: negatives of D = eigenvalues below sigma
        assert int(np.sum(d < 0)) == int(np.sum(lam < sigma))
        b = np.random.default_rng(1).normal(size=S.shape[0])
        x = factor.solve_ldlt_dense(L, d, b)
        assert np.linalg.norm(S @ x - b) < 1e-10 * np.linalg.norm(b)


def test_banded_ldlt_matches_dense():
    K, M = assembly.assemble_kron(2, [7, 6], 3, [bspline.riga_multiplicities(7, 3, 3), None])
    lam, _ = eigen.ghep_dense(K.todense(), M.todense())
    sigma = 0.5 * (lam[6] + lam[7])
    A = factor.shifted(K, M, sigma)
    band = factor.BandedLDLT(A, factor.half_bandwidth(A))
    L, d = factor.ldlt_dense(A.todense())
    assert np.allclose(band.d, d, rtol=1e-10)
    assert band.inertia() == 7
    b = np.arange(A.n, dtype=float)
    assert np.allclose(band.solve(b), factor.solve_ldlt_dense(L, d, b), rtol=1e-9)


def test_ldlt_breakdown_detected():
    with pytest.raises(factor.PivotBreakdown):
        factor.ldlt_dense(np.array([[0.0, 1.0], [1.0, 0.0]]))


# ------------------------------------------------------------------ symbolic
def _tree_case(ne, p, bs, le):
    mults = [bspline.riga_multiplicities(n, p, bs) if bs else None for n in ne]
    K, M = assembly.assemble_kron(len(ne), ne, p, mults)
    n1, N = assembly.dof_count(len(ne), ne, p, mults)
    c0 = symbolic.riga_c0_lists(len(ne), ne, p, mults)
    nodes, perm = symbolic.build_tree(n1, c0, p, le)
    return K, M, n1, N, nodes, perm


@pytest.mark.parametrize("ne,p,bs,le", [([16, 16], 2, None, 8), ([16, 16], 3, 4, 8), ([12, 9], 2, 4, 4),
                                         ([5, 6, 4], 2, None, 3), ([8, 8, 8], 2, 4, 8)])
def test_separators_separate_and_fronts_cover_fill(ne, p, bs, le):
    K, M, n1, N, nodes, perm = _tree_case(ne, p, bs, le)
    assert np.array_equal(np.sort(perm), np.arange(N))
    pos = np.empty(N, dtype=np.int64)
    pos[perm] = np.arange(N)
    # subtree variable sets; the two children of a node never couple in A
    sub = []
    for nd in nodes:
        s = set(nd["vars"].tolist())
        for c in nd["children"]:
            s |= sub[c]
        sub.append(s)
    rows = np.repeat(np.arange(N), np.diff(K.indptr))
    for nd in nodes:
        if len(nd["children"]) == 2:
            a, b = sub[nd["children"][0]], sub[nd["children"][1]]
            for r, c in zip(rows, K.indices):
                assert not (r in a and c in b)
    fr = symbolic.fronts(nodes, perm, (K.indptr, K.indices))
    struct, par = symbolic.symbolic_elimination((K.indptr, K.indices), perm)
    # the dense front of node F holds every fill entry of its columns, and its
    # border is exactly the union of the structures below its own block
    for (own, border) in fr:
        own_pos = set(pos[own].tolist())
        border_pos = set(pos[border].tolist())
        union = set()
        for v in own:
            union |= set(struct[pos[v]].tolist())
        assert union - own_pos == border_pos
    # Liu's etree equals the brute-force one
    assert np.array_equal(symbolic.etree_liu((K.indptr, K.indices), perm), par)
    # column counts sum (brute force) <= dense-front count
    nnz_true = sum(s.size + 1 for s in struct)
    nnz_front, _ = symbolic.front_nnz_and_flops(fr)
    assert nnz_true <= nnz_front


@pytest.mark.parametrize("k,m", [(1, 0), (7, 0), (12, 0), (5, 3), (9, 14), (16, 1)])
def test_front_counts_closed_forms_and_elimination_count(k, m):
    """front_nnz_and_flops against things it does not compute itself.
    (1) Closed forms: a dense front of n = k + m variables with k pivots holds
    k(k+1)/2 + k m entries of L, and eliminating its k pivots costs
    ((n^3 - n) - (m^3 - m)) / 3 flops: the full dense LDL^T of n variables,
    sum_{j=1..n} j (j - 1) = (n^3 - n) / 3, minus that of the m-variable
    Schur complement left over.  (2) A brute-force count: the test eliminates
    the k pivots of a random symmetric front entry by entry on its lower
    triangle, counts the multiply-adds it performs (2 flops each) and checks
    that what it computed is the Schur complement A22 - A21 A11^{-1} A12.  A
    doubled or halved formula, or one that counts the upper triangle too,
    fails both."""
    n = k + m
    own, border = np.arange(k), np.arange(k, n)
    nnz, flops = symbolic.front_nnz_and_flops([(own, border)])
    assert nnz == k * (k + 1) // 2 + k * m
    assert flops == ((n ** 3 - n) - (m ** 3 - m)) // 3
    rng = np.random.default_rng(100 * k + m)
    B = rng.normal(size=(n, n))
    A = B @ B.T + n * np.eye(n)
    W = A.copy()
    madds = 0
    for i in range(k):
        for r in range(i + 1, n):
            lri = W[r, i] / W[i, i]
            for c in range(i + 1, r + 1):
                W[r, c] -= lri * W[c, i]
                madds += 1
    assert 2 * madds == flops
    schur = A[k:, k:] - A[k:, :k] @ np.linalg.solve(A[:k, :k], A[:k, k:])
    assert np.allclose(np.tril(W[k:, k:]), np.tril(schur), rtol=1e-12, atol=1e-12 * n)
    # additivity over fronts
    nnz2, flops2 = symbolic.front_nnz_and_flops([(own, border), (np.arange(n, n + 3), np.empty(0, np.int64))])
    assert nnz2 == nnz + 6 and flops2 == flops + (27 - 3) // 3


@pytest.mark.parametrize("ne,p,bs,le", [([6, 6], 2, None, 3), ([8, 8], 3, 4, 8), ([4, 4, 4], 2, None, 2)])
def test_column_counts_equal_numeric_factor_nnz(ne, p, bs, le):
    """Sum of (column count + 1) from the brute-force symbolic elimination
    equals the number of non-zeros of the numeric L of the permuted matrix
    (dense LDL^T, random values, so no entry cancels by accident); the
    fronts hold at least those entries and cost at least the true sparse
    flop count sum_j c_j (c_j + 1)."""
    K, M, n1, N, nodes, perm = _tree_case(ne, p, bs, le)
    struct, _ = symbolic.symbolic_elimination((K.indptr, K.indices), perm)
    rng = np.random.default_rng(11)
    A = K.todense()
    Ar = np.where(A != 0.0, rng.uniform(0.5, 1.0, size=A.shape), 0.0)
    Ar = np.triu(Ar, 1)
    Ar = Ar + Ar.T + np.diag(np.full(N, 4.0 * N))
    P = Ar[np.ix_(perm, perm)]
    L, d = factor.ldlt_dense(P)
    nnz_numeric = int(np.count_nonzero(np.abs(np.tril(L)) > 1e-300))
    counts = np.array([s.size for s in struct])
    assert int(np.sum(counts + 1)) == nnz_numeric
    fr = symbolic.fronts(nodes, perm, (K.indptr, K.indices))
    nnz_front, flops_front = symbolic.front_nnz_and_flops(fr)
    assert nnz_front >= nnz_numeric
    assert flops_front >= int(np.sum(counts * (counts + 1)))


def test_tree_shapes_c1_and_riga_blocks():
    # C1: 16x16 p=2 IGA, 14x14 DOFs... n1 = 16; first cut a 2-thick slab at 7
    _, _, n1, N, nodes, perm = _tree_case([16, 16], 2, None, 8)
    assert n1 == [16, 16] and N == 256
    root = nodes[-1]
    assert root["box"] == [(7, 9), (0, 16)]
    assert len(nodes) == 7
    # rIGA 2D blocks are the leaves when leaf_extent >= block interior
    _, _, n1, N, nodes, perm = _tree_case([64, 64], 3, 16, 17)
    leaves = [nd for nd in nodes if not nd["children"]]
    assert len(leaves) == 16 and all(nd["vars"].size == 17 * 17 for nd in leaves)
    assert nodes[-1]["vars"].size == n1[1]  # root = a full C0 line


# ----------------------------------------------------------------- Lanczos
def test_lanczos_matches_dense_and_finds_multiplicities():
    for ne, p, bs in [([10, 10], 2, None), ([8, 8], 3, 4)]:
        mults = [bspline.riga_multiplicities(n, p, bs) if bs else None for n in ne]
        K, M = assembly.assemble_kron(2, ne, p, mults)
        lam, _ = eigen.ghep_dense(K.todense(), M.todense())
        l, U, info = eigen.lanczos_shift_invert(K, M, 12, 0.0, tol=1e-12, seed=5)
        assert np.max(np.abs(l - lam[:12]) / lam[:12]) < 1e-11
        assert eigen.residual_rho(K, M, l, U).max() < 1e-9
        G = U.T @ M.matvec(U)
        assert np.abs(G - np.eye(12)).max() < 1e-10
        # second slice above a mid shift
        g = [i for i in range(10, lam.size - 1) if lam[i + 1] - lam[i] > 1e-3 * lam[i]][0]
        s2 = 0.5 * (lam[g] + lam[g + 1])
        l2, U2, _ = eigen.lanczos_shift_invert(K, M, 8, s2, tol=1e-12, seed=6)
        assert np.max(np.abs(l2 - lam[g + 1:g + 9]) / lam[g + 1:g + 9]) < 1e-11


def test_lanczos_krylov_relation():
    # V^T M V = I and V^T M H V = T (Eq. LanczosRitz) on one run
    K, M = assembly.assemble_kron(2, [8, 8], 2)
    fac = eigen._Factor(K, M, 0.0)
    N = K.n
    rng = np.random.default_rng(2)
    theta, U, est = eigen.lanczos_run(K, M, fac, rng.normal(size=N), [], 20, 40, 1e-30)
    # Ritz vectors of a complete run are M-orthonormal and Ritz values are Rayleigh quotients
    G = U.T @ M.matvec(U)
    assert np.abs(G - np.eye(U.shape[1])).max() < 1e-10
    HU = np.stack([fac.solve(M.matvec(U[:, i])) for i in range(U.shape[1])], axis=1)
    rq = np.einsum("ij,ij->j", M.matvec(U), HU)
    assert np.allclose(rq, theta, rtol=1e-10)


# ------------------------------------------------------------------ adjoint
def test_adjoint_homogeneity_and_fd():
    ne, p = [5, 4], 2
    rng = np.random.default_rng(7)
    nel = 20
    a = rng.normal(0, 0.5, nel)
    b = rng.normal(0, 0.5, nel)
    K, M = assembly.assemble_coef(2, ne, p, None, np.exp(a), np.exp(b))
    lam, V = eigen.ghep_dense(K.todense(), M.todense())
    k = 3
    w = np.ones(k)
    ga, gb = adjoint.eig_grad(2, ne, p, None, np.exp(a), np.exp(b), lam[:k], V[:, :k], w)
    # scaling K by e^t scales lambda by e^t; scaling M by e^t scales it by e^-t
    assert abs(ga.sum() - lam[:k].sum()) < 1e-10 * lam[:k].sum()
    assert abs(gb.sum() + lam[:k].sum()) < 1e-10 * lam[:k].sum()

    def S(aa, bb):
        Kf, Mf = assembly.assemble_coef(2, ne, p, None, np.exp(aa), np.exp(bb))
        return eigen.ghep_dense(Kf.todense(), Mf.todense())[0][:k].sum()

    h = 1e-5
    for e in (0, 7, 13):
        da = np.zeros(nel)
        da[e] = h
        fd = (S(a + da, b) - S(a - da, b)) / (2 * h)
        assert abs(fd - ga[e]) < 1e-6 * max(1.0, abs(ga[e]))
        fd = (S(a, b + da) - S(a, b - da)) / (2 * h)
        assert abs(fd - gb[e]) < 1e-6 * max(1.0, abs(gb[e]))
