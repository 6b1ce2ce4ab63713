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
