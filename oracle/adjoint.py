"""Eigenvalue sensitivities to per-element coefficients (oracle; test infrastructure only).

Not in the paper.  For K = sum_e exp(a_e) K_e, M = sum_e exp(b_e) M_e and an
M-normalised eigenvector u of a simple eigenvalue lambda, differentiating
K u = lambda M u and u^T M u = 1 gives

    d lambda / d a_e =  exp(a_e) u_e^T K_e u_e,
    d lambda / d b_e = -lambda exp(b_e) u_e^T M_e u_e,

with u_e the element's local coefficients.  For a weighted sum
L = sum_i w_i lambda_i the gradient is the w-weighted sum of these.
Element matrices are the tensor products of the 1D element matrices of
Eq. 1Dmatrix (Eq. 2Dmatrix applied element by element).
"""
import numpy as np

from .assembly import element_index_maps


def eig_grad(dim, ne, p, mults, coefK, coefM, lam, U, weights):
    """Return (grad_a, grad_b) of sum_i weights[i] * lam[i] with respect to
    a_e and b_e (``coefK[e] = exp(a_e)``, ``coefM[e] = exp(b_e)``)."""
    maps = element_index_maps(dim, ne, p, mults)
    nd = [int(m[2].max()) + 1 for m in maps]
    nel = int(np.prod(ne))
    ga = np.zeros(nel)
    gb = np.zeros(nel)
    q = p + 1
    for e in range(nel):
        ei = []
        rem = e
        for a in range(dim):
            ei.append(rem % ne[a])
            rem //= ne[a]
        Ke_list = [maps[a][0][ei[a]] for a in range(dim)]
        Me_list = [maps[a][1][ei[a]] for a in range(dim)]
        idx_list = [maps[a][2][ei[a]] for a in range(dim)]
        Mloc = np.ones((1, 1))
        for a in reversed(range(dim)):
            Mloc = np.kron(Mloc, Me_list[a])
        Kloc = np.zeros((q ** dim, q ** dim))
        for s in range(dim):
            T = np.ones((1, 1))
            for a in reversed(range(dim)):
                T = np.kron(T, Ke_list[a] if a == s else Me_list[a])
            Kloc += T
        gl = np.zeros(1, dtype=np.int64)
        valid = np.ones(1, dtype=bool)
        for a in reversed(range(dim)):
            ia = idx_list[a]
            mul = int(np.prod(nd[:a])) if a > 0 else 1
            gl = (gl[:, None] + (ia[None, :] * mul)).ravel()
            valid = (valid[:, None] & (ia[None, :] >= 0)).ravel()
        ue = np.zeros((q ** dim, U.shape[1]))
        ue[valid] = U[gl[valid]]
        qk = np.einsum("ai,ab,bi->i", ue, Kloc, ue)
        qm = np.einsum("ai,ab,bi->i", ue, Mloc, ue)
        ga[e] = coefK[e] * np.sum(weights * qk)
        gb[e] = -coefM[e] * np.sum(weights * lam * qm)
    return ga, gb
