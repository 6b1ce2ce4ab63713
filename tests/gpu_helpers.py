"""Shared helpers of the GPU tests: library context, oracle comparisons."""
import os

import numpy as np

from oracle import assembly, eigen, factor


def riga_ctx():
    from paper_2009_08167_gb300 import riga
    if not os.path.exists(riga.LIB_PATH):
        from paper_2009_08167_gb300.build import build
        build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return riga.Riga(0)


def oracle_matrices(mesh, coefK=None, coefM=None):
    if coefK is None and coefM is None:
        return assembly.assemble_kron(mesh.dim, mesh.ne, mesh.p, mesh.mults)
    return assembly.assemble_coef(mesh.dim, mesh.ne, mesh.p, mesh.mults, coefK, coefM)


def ldlt_forward_bounds(L, d, B, eps):
    """First-order forward-error bounds of an LDL^T factorization without
    pivoting when the factored matrix moves by |dA| <= eps B (componentwise).

    From A + dA = (L + dL)(D + dD)(L + dL)^T, the symmetric E = L^{-1} dA L^{-T}
    equals X D + dD + D X^T to first order, X = L^{-1} dL strictly lower
    triangular.  So dD = diag(E) and X_ij = E_ij / d_j (i > j), and with
    G = |L^{-1}| B |L^{-T}|:
        |dd_k| <= eps G_kk,      |dL| <= eps |L| (strict_lower(G) |D|^{-1}).
    G measures the conditioning of each pivot and multiplier; a pivot of a
    nearly singular leading block has a large G_kk / |d_k|.
    Returns (pivot bounds, dense multiplier bounds)."""
    import scipy.linalg as sla
    n = L.shape[0]
    Li = np.abs(sla.solve_triangular(L, np.eye(n), lower=True, unit_diagonal=True))
    G = Li @ B @ Li.T
    return eps * np.diag(G), eps * (np.abs(L) @ (np.tril(G, -1) / np.abs(d)[None, :]))


def clusters(lam, rel=1e-8):
    """Index groups of (nearly) equal eigenvalues."""
    groups = [[0]]
    for i in range(1, lam.size):
        if lam[i] - lam[i - 1] <= rel * abs(lam[i]):
            groups[-1].append(i)
        else:
            groups.append([i])
    return groups


def compare_eigvecs(U_ref, U, M, lam_ref, rel=1e-8, tol=1e-9, lam_next=None):
    """Eigenvectors agree as cluster subspaces: the singular values of
    U_ref^T M U over each cluster are all >= 1 - tol.  Simple eigenvalues
    reduce to |u_ref^T M u| >= 1 - tol.  A cluster cut by the end of the
    range (its next member, lam_next, lies beyond it) is skipped: the
    computed vectors span an undetermined part of that subspace."""
    MU = M.matvec(U)
    worst = 1.0
    k = lam_ref.size
    for g in clusters(lam_ref, rel):
        cut = g[-1] == k - 1 and (lam_next is None or lam_next - lam_ref[-1] <= rel * abs(lam_next))
        if cut:
            continue
        S = U_ref[:, g].T @ MU[:, g]
        s = np.linalg.svd(S, compute_uv=False)
        worst = min(worst, s.min())
    assert worst >= 1 - tol, worst
    return worst


def kron_1d_matrices(mesh):
    """Dense 1D stiffness and mass matrices (Dirichlet functions removed) per
    direction, x first: the factors of Eq. 2Dmatrix."""
    from oracle import bspline
    return [bspline.matrices_1d(mesh.ne[a], mesh.p, mesh.mults[a], True) for a in range(mesh.dim)]


def kron_apply(mats, U):
    """(A_z (x) A_y (x) A_x) U for the columns of U (x fastest); mats = [A_x, A_y(, A_z)]."""
    U = np.asarray(U)
    dims = [A.shape[1] for A in mats]
    cols = U.shape[1]
    T = U.reshape(list(reversed(dims)) + [cols])  # (n_z, n_y, n_x, cols) for 3D
    d = len(mats)
    for a, A in enumerate(mats):
        ax = d - 1 - a  # tensor axis of direction a
        T = np.moveaxis(np.tensordot(A, T, axes=([1], [ax])), 0, ax)
    return T.reshape(-1, cols)


def kron_residuals(mesh, lam, U):
    """rho_i = ||K u_i - lam_i M u_i|| / (|lam_i| ||M u_i||) with K and M
    applied through their Kronecker structure (no global matrix is built):
    K = sum_a (M (x) ... K on axis a ... (x) M), M = M (x) M (x) M."""
    one = kron_1d_matrices(mesh)
    Ks = [o[0] for o in one]
    Ms = [o[1] for o in one]
    MU = kron_apply(Ms, U)
    KU = np.zeros_like(MU)
    for a in range(mesh.dim):
        mats = [Ks[b] if b == a else Ms[b] for b in range(mesh.dim)]
        KU += kron_apply(mats, U)
    R = KU - MU * lam[None, :]
    return np.linalg.norm(R, axis=0) / (np.abs(lam) * np.linalg.norm(MU, axis=0)), MU


def compare_eigvecs_kron(mesh, V_ref, U, lam_ref, rel=1e-8, tol=1e-9, lam_next=None):
    """compare_eigvecs with M applied through its Kronecker structure."""
    one = kron_1d_matrices(mesh)

    class _KM:
        @staticmethod
        def matvec(X):
            return kron_apply([o[1] for o in one], X)

    return compare_eigvecs(V_ref, U, _KM, lam_ref, rel=rel, tol=tol, lam_next=lam_next)
