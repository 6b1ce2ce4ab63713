"""Assembly of the d-dimensional stiffness K and mass M (oracle; test infrastructure only).

Constant coefficients: Kronecker construction of Eq. 2Dmatrix (Sec. 3.1.1).
Per-element coefficients K = sum_e exp(a_e) K_e, M = sum_e exp(b_e) M_e:
not in the paper; element matrices are tensor products of the 1D element
matrices of Eq. 1Dmatrix.  Global DOF index is x-fastest: i + n_x*(j + n_y*k).
Sparse matrices are plain (indptr, indices, data) CSR triples built with
numpy sorting; dense forms are used for small cases.
"""
import numpy as np

from . import bspline


class Csr:
    """Minimal CSR container (rows sorted, columns sorted within a row)."""

    def __init__(self, indptr, indices, data, n):
        self.indptr = np.asarray(indptr, dtype=np.int64)
        self.indices = np.asarray(indices, dtype=np.int64)
        self.data = np.asarray(data, dtype=np.float64)
        self.n = int(n)

    @property
    def nnz(self):
        return int(self.indices.size)

    def matvec(self, x):
        x = np.asarray(x, dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.indptr))
        prod = self.data[:, None] * x[self.indices].reshape(self.nnz, -1)
        out = np.zeros((self.n, prod.shape[1]))
        np.add.at(out, rows, prod)
        return out.reshape((self.n,) + x.shape[1:])

    def todense(self):
        A = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.indptr))
        np.add.at(A, (rows, self.indices), self.data)
        return A

    def get(self, r, c):
        lo, hi = self.indptr[r], self.indptr[r + 1]
        k = np.searchsorted(self.indices[lo:hi], c)
        if k < hi - lo and self.indices[lo + k] == c:
            return self.data[lo + k]
        return 0.0


def coo_to_csr(rows, cols, vals, n):
    """Sum duplicate (row, col) entries and return a CSR matrix."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    vals = vals[order]
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start) if vals.size else vals
    r = uniq // n
    c = uniq % n
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(indptr, r + 1, 1)
    indptr = np.cumsum(indptr)
    return Csr(indptr, c, summed, n)


def dense_to_csr(A, pattern=None):
    """CSR of a dense matrix keeping the entries where ``pattern`` is True
    (default: non-zeros)."""
    if pattern is None:
        pattern = A != 0.0
    r, c = np.nonzero(pattern)
    return coo_to_csr(r, c, A[r, c], A.shape[0])


def kron_csr(mats):
    """Kronecker product mats[0] (x) mats[1] (x) ... of dense banded 1D matrices,
    returned as CSR over the structurally non-zero pattern of each factor.
    The first factor is the slowest index (Eq. 2Dmatrix ordering)."""
    entries = []
    for A, P in mats:
        r, c = np.nonzero(P)
        entries.append((r, c, A[r, c], A.shape[0]))
    rows = np.zeros(1, dtype=np.int64)
    cols = np.zeros(1, dtype=np.int64)
    vals = np.ones(1)
    n = 1
    for r, c, v, m in entries:
        rows = (rows[:, None] * m + r[None, :]).ravel()
        cols = (cols[:, None] * m + c[None, :]).ravel()
        vals = (vals[:, None] * v[None, :]).ravel()
        n *= m
    return coo_to_csr(rows, cols, vals, n)


def pattern_1d(ne, p, mult=None, dirichlet=True):
    """Structural pattern of the 1D matrices: B_i and B_j interact iff their
    supports share an element (Fig. 3)."""
    _, _, idx = bspline.element_matrices_1d(ne, p, mult, dirichlet)
    n = int(idx.max()) + 1
    P = np.zeros((n, n), dtype=bool)
    for e in range(ne):
        g = idx[e][idx[e] >= 0]
        P[np.ix_(g, g)] = True
    return P


def assemble_kron(dim, ne, p, mults=None, dirichlet=True):
    """K and M by the Kronecker formulas of Eq. 2Dmatrix (CSR over the
    structural pattern).

    2D: K = M^y (x) K^x + K^y (x) M^x, M = M^y (x) M^x; 3D analogous.
    ``ne`` and ``mults`` are per direction (x first).
    """
    if mults is None:
        mults = [None] * dim
    K1, M1, P1 = [], [], []
    for a in range(dim):
        K, M = bspline.matrices_1d(ne[a], p, mults[a], dirichlet)
        K1.append(K)
        M1.append(M)
        P1.append(pattern_1d(ne[a], p, mults[a], dirichlet))
    # factors listed slowest first: z, y, x
    order = list(range(dim))[::-1]
    Mtot = kron_csr([(M1[a], P1[a]) for a in order])
    Kparts = []
    for s in range(dim):
        fac = [(K1[a], P1[a]) if a == s else (M1[a], P1[a]) for a in order]
        Kparts.append(kron_csr(fac))
    data = sum(kp.data for kp in Kparts)
    for kp in Kparts:
        assert np.array_equal(kp.indices, Mtot.indices)
    Ktot = Csr(Mtot.indptr, Mtot.indices, data, Mtot.n)
    return Ktot, Mtot


def element_index_maps(dim, ne, p, mults=None, dirichlet=True):
    """Per direction: element-local 1D matrices and global index maps."""
    if mults is None:
        mults = [None] * dim
    return [bspline.element_matrices_1d(ne[a], p, mults[a], dirichlet) for a in range(dim)]


def assemble_coef(dim, ne, p, mults, coefK, coefM, dirichlet=True):
    """K = sum_e exp(a_e) K_e and M = sum_e exp(b_e) M_e, with
    ``coefK[e] = exp(a_e)`` and ``coefM[e] = exp(b_e)`` given directly
    (None = 1).  Element index e is x-fastest.  The element matrices are
    tensor products of the 1D element matrices: in 2D
    K_e = M^y_e (x) K^x_e + K^y_e (x) M^x_e, M_e = M^y_e (x) M^x_e.
    Returns CSR K, M on the union pattern of all element contributions.
    """
    maps = element_index_maps(dim, ne, p, mults, dirichlet)
    nd = [int(m[2].max()) + 1 for m in maps]
    nel = int(np.prod(ne))
    if coefK is None:
        coefK = np.ones(nel)
    if coefM is None:
        coefM = np.ones(nel)
    rows, cols, kv, mv = [], [], [], []
    q = p + 1
    for e in range(nel):
        ei = []
        rem = e
        for a in range(dim):
            ei.append(rem % ne[a])
            rem //= ne[a]
        # local tensor-product matrices, slowest direction first
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
        # local -> global (x fastest); -1 marks a Dirichlet-removed function
        gl = np.zeros(1, dtype=np.int64)
        valid = np.ones(1, dtype=bool)
        for a in reversed(range(dim)):
            ia = idx_list[a]
            mul = int(np.prod(nd[:a])) if a > 0 else 1
            gl = (gl[:, None] + (ia[None, :] * mul)).ravel()
            valid = (valid[:, None] & (ia[None, :] >= 0)).ravel()
        sel = np.nonzero(valid)[0]
        gsel = gl[sel]
        rr = np.repeat(gsel, sel.size)
        cc = np.tile(gsel, sel.size)
        rows.append(rr)
        cols.append(cc)
        kv.append(coefK[e] * Kloc[np.ix_(sel, sel)].ravel())
        mv.append(coefM[e] * Mloc[np.ix_(sel, sel)].ravel())
    n = int(np.prod(nd))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    K = coo_to_csr(rows, cols, np.concatenate(kv), n)
    M = coo_to_csr(rows, cols, np.concatenate(mv), n)
    assert np.array_equal(K.indices, M.indices)
    return K, M


def dof_count(dim, ne, p, mults=None, dirichlet=True):
    """Number of DOFs per direction and in total (Eq. dofs for uniform meshes)."""
    if mults is None:
        mults = [None] * dim
    n1 = []
    for a in range(dim):
        knots = bspline.open_knot_vector(ne[a], p, mults[a])
        n = bspline.n_functions(knots, p)
        n1.append(n - 2 if dirichlet else n)
    return n1, int(np.prod(n1))
