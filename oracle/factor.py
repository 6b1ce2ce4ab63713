"""LDL^T of the shifted matrix A = K - sigma M (oracle; test infrastructure only).

Sec. 4.2 factors the spectral-transformation matrix and, in the Remark on
inertia, reads the number of eigenvalues below sigma off the negative
entries of D (Sylvester's law of inertia).  The paper writes L L^T in Sec.
4.2 but LDL^T in that Remark; LDL^T is used (A is indefinite once sigma
exceeds the smallest eigenvalue).  1x1 pivots, no pivoting: the
factorization of a given order is unique when it exists, which is what
makes the GPU factor comparable entry by entry.
"""
import numpy as np


class PivotBreakdown(Exception):
    pass


def ldlt_dense(A, rel_tol=1e-300):
    """Dense LDL^T without pivoting, column by column from the definition
    d_j = a_jj - sum_{k<j} L_jk^2 d_k,
    L_ij = (a_ij - sum_{k<j} L_ik d_k L_jk) / d_j.
    Returns (L unit lower triangular, d)."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    L = np.eye(n)
    d = np.zeros(n)
    scale = np.abs(A).max() if n else 1.0
    for j in range(n):
        w = L[j, :j] * d[:j]
        d[j] = A[j, j] - L[j, :j] @ w
        if not np.isfinite(d[j]) or abs(d[j]) <= rel_tol * scale:
            raise PivotBreakdown(j)
        if j + 1 < n:
            L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ w) / d[j]
    return L, d


def solve_ldlt_dense(L, d, b):
    """x = (L D L^T)^{-1} b by forward substitution, diagonal scaling and
    back substitution."""
    n = L.shape[0]
    y = np.array(b, dtype=np.float64)
    for i in range(n):
        y[i] -= L[i, :i] @ y[:i]
    y = y / d if y.ndim == 1 else y / d[:, None]
    for i in reversed(range(n)):
        y[i] -= L[i + 1:, i] @ y[i + 1:]
    return y


class BandedLDLT:
    """LDL^T of a symmetric banded matrix in its natural order.

    Storage: ``band[j, t] = L[j+t, j]`` for t = 1..bw and ``d[j]``.  The
    right-looking update after pivot j subtracts d_j l l^T from the next bw x bw
    lower triangle.  Half-bandwidth bw = n1 p + p in the x-fastest numbering
    of a tensor-product B-spline space (n1 DOFs in the fastest direction).
    """

    def __init__(self, csr_A, bw):
        n = csr_A.n
        self.n = n
        self.bw = bw
        B = np.zeros((n + bw + 1, bw + 1))
        rows = np.repeat(np.arange(n), np.diff(csr_A.indptr))
        cols = csr_A.indices
        low = rows >= cols
        assert np.all(rows - cols <= bw)
        B[cols[low], rows[low] - cols[low]] = csr_A.data[low]
        self.d = np.zeros(n)
        r_idx, c_idx = np.triu_indices(bw)  # r <= c
        scale = np.abs(csr_A.data).max()
        for j in range(n):
            dj = B[j, 0]
            if not np.isfinite(dj) or abs(dj) <= 1e-300 * scale:
                raise PivotBreakdown(j)
            self.d[j] = dj
            col = B[j, 1:].copy()  # A[j+1..j+bw, j]
            l = col / dj
            B[j, 1:] = l
            # trailing update: A[j+1+c, j+1+r] -= dj l_r l_c for r <= c
            B[j + 1 + r_idx, c_idx - r_idx] -= dj * l[r_idx] * l[c_idx]
        self.band = B[:n]

    def inertia(self):
        return int(np.sum(self.d < 0))

    def solve(self, b):
        n, bw = self.n, self.bw
        y = np.array(b, dtype=np.float64)
        L = self.band
        for j in range(n):
            hi = min(n, j + bw + 1)
            y[j + 1:hi] -= L[j, 1:hi - j] * y[j]
        y /= self.d
        for j in reversed(range(n)):
            hi = min(n, j + bw + 1)
            y[j] -= L[j, 1:hi - j] @ y[j + 1:hi]
        return y


def half_bandwidth(csr):
    rows = np.repeat(np.arange(csr.n), np.diff(csr.indptr))
    return int(np.max(np.abs(rows - csr.indices)))


def shifted(K, M, sigma):
    """CSR of K - sigma M (same pattern)."""
    from .assembly import Csr
    assert np.array_equal(K.indices, M.indices)
    return Csr(K.indptr, K.indices, K.data - sigma * M.data, K.n)


def inertia_dense(A):
    """Number of negative pivots of the dense LDL^T of A (Remark on inertia)."""
    _, d = ldlt_dense(A)
    return int(np.sum(d < 0))
