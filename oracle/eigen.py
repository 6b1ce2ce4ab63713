"""Generalized Hermitian eigenproblem K u = lambda M u (oracle; test infrastructure only).

* ``ghep_dense``: the plain definition, for small N: M = R R^T, then the
  symmetric eigenproblem of R^{-1} K R^{-T} (Sec. 4.1 describes this
  reduction as the fragile alternative the shift-and-invert approach avoids;
  for the small, well-conditioned test matrices it is exact to rounding).
* ``kron_sum_eigs``: for constant coefficients K and M are Kronecker sums /
  products of 1D matrices (Eq. 2Dmatrix), so every eigenvalue is
  mu^x_i + mu^y_j (+ mu^z_k) and every eigenvector v^y_j (x) v^x_i, with
  (mu, v) the 1D generalized eigenpairs.  Exact up to rounding.
* ``lanczos_shift_invert``: the paper's method: Lanczos on
  H = (K - sigma M)^{-1} M in the M-inner product (Eq. Lanczos,
  Eq. LanczosAlphaBeta), full reorthogonalization against all stored
  vectors (Sec. 4.2), Rayleigh-Ritz on T_m (Eq. RitzValues) and
  lambda = sigma + 1/theta; converged vectors are locked and the process is
  restarted from a fresh start vector M-orthogonal to them until the inertia
  count (Remark on inertia) confirms nothing is missing.
"""
import numpy as np

from . import bspline
from .factor import BandedLDLT, half_bandwidth, shifted, ldlt_dense, solve_ldlt_dense


def ghep_dense(K, M):
    """All eigenpairs of the dense GHEP, ascending, M-orthonormal vectors."""
    K = np.asarray(K, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    R = np.linalg.cholesky(M)
    Ri = np.linalg.inv(R)
    C = Ri @ K @ Ri.T
    C = 0.5 * (C + C.T)
    lam, W = np.linalg.eigh(C)
    V = Ri.T @ W
    return lam, V


def eig1d(ne, p, mult=None, dirichlet=True):
    """Generalized eigenpairs of the 1D pair (K^x, M^x) of Eq. 1Dmatrix."""
    K, M = bspline.matrices_1d(ne, p, mult, dirichlet)
    return ghep_dense(K, M)


def kron_sum_eigs(dim, ne, p, mults=None, k=None, with_vectors=True):
    """Lowest k eigenpairs of the constant-coefficient d-dimensional problem
    from 1D eigenpairs (Eq. 2Dmatrix).  Returns (lam, index tuples, vecs):
    index tuples (i_x, i_y[, i_z]) identify the 1D factors; vecs are
    M-normalised, x fastest.  Ties are ordered by the index tuple."""
    if mults is None:
        mults = [None] * dim
    one = [eig1d(ne[a], p, mults[a]) for a in range(dim)]
    grids = np.meshgrid(*[np.arange(o[0].size) for o in one], indexing="ij")
    idx = np.stack([g.ravel() for g in grids], axis=1)
    lam = np.zeros(idx.shape[0])
    for a in range(dim):
        lam += one[a][0][idx[:, a]]
    order = np.lexsort(tuple(idx[:, a] for a in reversed(range(dim))) + (lam,))
    if k is not None:
        order = order[:k]
    lam = lam[order]
    idx = idx[order]
    vecs = None
    if with_vectors:
        cols = []
        for t in idx:
            v = np.ones(1)
            for a in reversed(range(dim)):
                v = np.kron(v, one[a][1][:, t[a]])
            cols.append(v)
        vecs = np.stack(cols, axis=1)
    return lam, idx, vecs


def residual_rho(K, M, lam, U):
    """rho_i = ||K u_i - lam_i M u_i||_2 / (|lam_i| ||M u_i||_2) (a reading:
    the paper does not state SLEPc's residual)."""
    KU = K.matvec(U) if hasattr(K, "matvec") else K @ U
    MU = M.matvec(U) if hasattr(M, "matvec") else M @ U
    R = KU - MU * lam[None, :]
    return np.linalg.norm(R, axis=0) / (np.abs(lam) * np.linalg.norm(MU, axis=0))


class _Factor:
    """A^{-1} application and inertia for A = K - sigma M: dense LDL^T for
    small N, banded LDL^T in natural order otherwise."""

    def __init__(self, K, M, sigma):
        self.sigma = sigma
        A = shifted(K, M, sigma)
        if A.n <= 1500:
            self.L, self.d = ldlt_dense(A.todense())
            self.band = None
        else:
            self.band = BandedLDLT(A, half_bandwidth(A))
            self.d = self.band.d

    def solve(self, b):
        if self.band is None:
            return solve_ldlt_dense(self.L, self.d, b)
        return self.band.solve(b)

    def inertia(self):
        return int(np.sum(self.d < 0))


def _m_dot(M, x, y):
    return float(x @ M.matvec(y))


def lanczos_run(K, M, fac, v1, locked, m_max, want, tol, check_every=10):
    """One Lanczos run on H = A^{-1} M from v1 (Eq. LanczosAlphaBeta) with
    full reorthogonalization against the run's own vectors and the locked
    vectors (two Gram-Schmidt passes).  Stops when the ``want`` largest
    positive theta have residual estimate |beta_{m+1} w_m| <= tol |theta|, or
    at m_max steps.  Returns (theta, Ritz vectors, estimates) sorted by
    decreasing theta."""
    N = v1.size
    Y = np.stack(locked, axis=1) if locked else np.zeros((N, 0))
    MY = M.matvec(Y) if Y.shape[1] else Y
    V = np.zeros((N, m_max + 1))
    MV = np.zeros((N, m_max + 1))
    alpha = np.zeros(m_max)
    beta = np.zeros(m_max + 1)
    v = v1.copy()
    for _ in range(2):
        if Y.shape[1]:
            v -= Y @ (MY.T @ v)
    Mv = M.matvec(v)
    nv = np.sqrt(v @ Mv)
    V[:, 0] = v / nv
    MV[:, 0] = Mv / nv
    m = 0
    for j in range(m_max):
        w = fac.solve(MV[:, j])
        alpha[j] = MV[:, j] @ w
        w -= alpha[j] * V[:, j]
        if j > 0:
            w -= beta[j] * V[:, j - 1]
        for _ in range(2):
            w -= V[:, :j + 1] @ (MV[:, :j + 1].T @ w)
            if Y.shape[1]:
                w -= Y @ (MY.T @ w)
        Mw = M.matvec(w)
        beta[j + 1] = np.sqrt(max(w @ Mw, 0.0))
        m = j + 1
        if beta[j + 1] == 0.0:
            break
        V[:, j + 1] = w / beta[j + 1]
        MV[:, j + 1] = Mw / beta[j + 1]
        if m % check_every == 0 or m == m_max:
            T = np.diag(alpha[:m]) + np.diag(beta[1:m], 1) + np.diag(beta[1:m], -1)
            theta, W = np.linalg.eigh(T)
            est = np.abs(beta[m] * W[m - 1, :])
            pos = np.nonzero(theta > 0)[0][::-1]
            top = pos[:want]
            if top.size >= want and np.all(est[top] <= tol * np.abs(theta[top])):
                break
    T = np.diag(alpha[:m]) + np.diag(beta[1:m], 1) + np.diag(beta[1:m], -1)
    theta, W = np.linalg.eigh(T)
    est = np.abs(beta[m] * W[m - 1, :])
    order = np.argsort(-theta)
    U = V[:, :m] @ W[:, order]
    return theta[order], U, est[order]


def lanczos_shift_invert(K, M, k, sigma=0.0, tol=1e-12, seed=1, m_max=None, max_restarts=20, extra=2):
    """The k smallest eigenvalues lambda > sigma and M-normalised vectors by
    shift-and-invert Lanczos with locking and restarts (Sec. 4.1-4.2), with
    completeness confirmed by Sylvester inertia (Remark on inertia).

    ``extra`` additional pairs are computed so that the check shift sigma'
    can sit in the gap after the k-th eigenvalue.  Returns (lam, U, info).
    """
    rng = np.random.default_rng(seed)
    N = K.n
    fac = _Factor(K, M, sigma)
    nu0 = fac.inertia()
    want = k + extra
    if m_max is None:
        m_max = min(N - 1, max(3 * want, want + 40))
    locked_l, locked_u = [], []
    runs = 0
    for runs in range(1, max_restarts + 1):
        v1 = rng.standard_normal(N)
        theta, U, est = lanczos_run(K, M, fac, v1, locked_u, m_max, want - len(locked_l), tol)
        for t, u, e in zip(theta, U.T, est):
            if t > 0 and e <= tol * abs(t) and len(locked_l) < want:
                u = u / np.sqrt(_m_dot(M, u, u))
                locked_l.append(sigma + 1.0 / t)
                locked_u.append(u)
        if len(locked_l) >= want:
            lam = np.array(locked_l)
            order = np.argsort(lam)
            lam = lam[order]
            # completeness: eigenvalues in (sigma, sigma') by inertia
            sp = 0.5 * (lam[k - 1] + lam[k])
            nu1 = _Factor(K, M, sp).inertia()
            found = int(np.sum(lam < sp))
            if nu1 - nu0 == found:
                U = np.stack([locked_u[i] for i in order[:k]], axis=1)
                return lam[:k], U, {"runs": runs, "inertia": (nu0, nu1), "check_shift": sp}
            # something missing below sp: keep the smallest ones and go on
            keep = order[:found]
            locked_l = [locked_l[i] for i in keep]
            locked_u = [locked_u[i] for i in keep]
    raise RuntimeError("lanczos_shift_invert: no convergence")
