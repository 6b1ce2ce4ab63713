"""Host Rayleigh-Ritz of block Lanczos (riga_band_eig): eigenpairs of
symmetric band matrices against numpy's dense symmetric eigensolver, with
exact multiplicities included.  No GPU."""
import os

import numpy as np
import pytest

from paper_2009_08167_gb300 import riga


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(riga.LIB_PATH):
        from paper_2009_08167_gb300.build import build
        build()


def _band(n, b, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, n))
    A = A + A.T
    for i in range(n):
        for j in range(n):
            if abs(i - j) > b:
                A[i, j] = 0.0
    return A


@pytest.mark.parametrize("n,b", [(1, 1), (7, 1), (40, 2), (120, 4), (203, 6), (64, 63)])
def test_band_eig_vs_dense(n, b):
    T = _band(n, b, 10 * n + b)
    which = sorted(set(range(0, n, max(1, n // 17))) | {n - 1})
    theta, S = riga.band_eig(T, b, which)
    ref = np.linalg.eigvalsh(T)
    scale = np.abs(ref).max()
    assert np.max(np.abs(theta - ref)) <= 1e-12 * scale
    R = T @ S - S * theta[which]
    assert np.max(np.abs(R)) <= 1e-11 * scale
    assert np.max(np.abs(S.T @ S - np.eye(len(which)))) <= 1e-10


def test_band_eig_multiplicity():
    # block Lanczos can produce exact multiplicities: two copies of one band
    # matrix interleaved (a permutation of a block-diagonal matrix keeps the
    # band when the copies alternate) give every eigenvalue twice
    n0, b0 = 30, 2
    T0 = _band(n0, b0, 3)
    n = 2 * n0
    T = np.zeros((n, n))
    for i in range(n0):
        for j in range(n0):
            T[2 * i, 2 * j] = T0[i, j]
            T[2 * i + 1, 2 * j + 1] = T0[i, j]
    b = 2 * b0
    which = list(range(n))
    theta, S = riga.band_eig(T, b, which)
    ref = np.sort(np.concatenate([np.linalg.eigvalsh(T0)] * 2))
    scale = np.abs(ref).max()
    assert np.max(np.abs(theta - ref)) <= 1e-12 * scale
    assert np.max(np.abs(T @ S - S * theta)) <= 1e-11 * scale
    assert np.max(np.abs(S.T @ S - np.eye(n))) <= 1e-10


@pytest.mark.parametrize("n,b", [(30, 2), (97, 4), (160, 4)])
def test_band_eig_last_rows(n, b):
    T = _band(n, b, 77 + n)
    theta, _, Z = riga.band_eig(T, b, (), last_rows=b)
    lam, V = np.linalg.eigh(T)
    assert np.max(np.abs(theta - lam)) <= 1e-12 * np.abs(lam).max()
    # eigenvectors are determined up to sign (the spectrum is simple here)
    ref = V[n - b:, :]
    sgn = np.sign(np.sum(ref * Z, axis=0))
    assert np.max(np.abs(Z - ref * sgn)) <= 1e-10


@pytest.mark.parametrize("scale", [1e-200, 1e-150, 1.0, 1e150, 1e200])
def test_band_eig_extreme_scales(scale):
    """The rotations' norms are scaled where squares would leave the double
    range: eigenvalues of s T are s times those of T (to rounding) for s far
    from 1, and the last rows of the eigenvectors do not depend on s."""
    n, b = 90, 2
    T = _band(n, b, 7)
    th1, _ = riga.band_eig(T, b, [])
    ths, _ = riga.band_eig(scale * T, b, [])
    ref = np.linalg.eigvalsh(T)
    assert np.all(np.isfinite(ths))
    assert np.max(np.abs(ths / scale - ref)) <= 1e-12 * np.abs(ref).max()
    assert np.max(np.abs(th1 - ref)) <= 1e-12 * np.abs(ref).max()


def test_band_eig_rejects_bad_arguments():
    """riga_band_eig's documented RIGA_EINVAL cases, through the C ABI."""
    import ctypes
    lib = riga.load_library()
    n, b = 6, 2
    T = np.asfortranarray(_band(n, b, 3))
    theta = np.zeros(n)
    S = np.zeros((n, 2), order="F")
    Z = np.zeros((2, n), order="F")
    P = ctypes.c_void_p

    def call(nn, bb, which, r, t=T, th=theta, s=S, z=Z):
        wh = np.ascontiguousarray(which, dtype=np.int32)
        return lib.riga_band_eig(nn, bb, t.ctypes.data_as(P) if t is not None else None,
                                 th.ctypes.data_as(P) if th is not None else None, int(wh.size),
                                 wh.ctypes.data_as(P) if wh.size else None, s.ctypes.data_as(P) if s is not None else None,
                                 r, z.ctypes.data_as(P) if z is not None else None)

    assert call(n, b, [0, 5], 2) == riga.RIGA_OK
    assert call(0, b, [], 0) == riga.RIGA_EINVAL          # n < 1
    assert call(n, -1, [], 0) == riga.RIGA_EINVAL         # negative bandwidth
    assert call(n, b, [0, 6], 0) == riga.RIGA_EINVAL      # index out of range
    assert call(n, b, [-1], 0) == riga.RIGA_EINVAL
    assert call(n, b, [], n + 1) == riga.RIGA_EINVAL      # more last rows than rows
    assert call(n, b, [], 2, z=None) == riga.RIGA_EINVAL  # rows asked, no output
    assert call(n, b, [], 0, t=None) == riga.RIGA_EINVAL
    assert call(n, b, [1], 0, s=None) == riga.RIGA_EINVAL  # vectors asked, no output


def _tridiag(d, e):
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


@pytest.mark.parametrize("case", ["random250", "wilkinson21", "split", "graded", "constant"])
def test_tridiagonal_qr_cases(case):
    """The tridiagonal Rayleigh-Ritz step (implicit QR, bulge chasing) on the
    shapes Lanczos produces and on the classical hard cases: Wilkinson's
    W21+ (pairs of eigenvalues equal to 1e-14 relative), a matrix that
    splits into independent blocks (zero couplings), a strongly graded one,
    and a constant-diagonal one (every shift exact at the start)."""
    rng = np.random.default_rng(5)
    if case == "random250":
        d, e = rng.normal(size=250), rng.normal(size=249)
    elif case == "wilkinson21":
        d, e = np.abs(np.arange(-10, 11)).astype(float), np.ones(20)
    elif case == "split":
        d, e = rng.normal(size=60), rng.normal(size=59)
        e[[9, 10, 30, 58]] = 0.0
    elif case == "graded":
        d = 10.0 ** (-np.arange(40) / 3.0)
        e = 0.3 * np.sqrt(d[:-1] * d[1:])
    else:
        d, e = np.full(50, 2.0), np.ones(49)
    T = _tridiag(d, e)
    n = len(d)
    theta, S = riga.band_eig(T, 1, list(range(n)))
    ref = np.linalg.eigvalsh(T)
    scale = np.abs(ref).max()
    assert np.max(np.abs(theta - ref)) <= 1e-13 * scale * max(1.0, n / 50)
    assert np.max(np.abs(T @ S - S * theta)) <= 1e-12 * scale * max(1.0, n / 50)
    assert np.max(np.abs(S.T @ S - np.eye(n))) <= 1e-11


@pytest.mark.parametrize("case", ["dense60", "arrow_tridiag", "repeated"])
def test_dense_symmetric_eig(case):
    """riga_sym_eig (Householder tridiagonalization + implicit QR) against
    numpy on a random dense matrix, on the arrowhead-plus-tridiagonal shape
    of a thick-restarted Lanczos projection, and on a matrix with an exactly
    repeated eigenvalue."""
    rng = np.random.default_rng(13)
    if case == "dense60":
        A = rng.normal(size=(60, 60))
        A = A + A.T
    elif case == "arrow_tridiag":
        c, n = 25, 90
        A = np.zeros((n, n))
        A[np.arange(c), np.arange(c)] = np.sort(rng.normal(size=c))
        A[:c, c] = A[c, :c] = 0.3 * rng.normal(size=c)
        d = rng.normal(size=n - c)
        e = np.abs(rng.normal(size=n - c - 1))
        A[c:, c:] = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    else:
        Qm, _ = np.linalg.qr(rng.normal(size=(40, 40)))
        lam = np.concatenate([np.full(5, 2.0), rng.normal(size=35)])
        A = (Qm * lam) @ Qm.T
        A = 0.5 * (A + A.T)
    theta, Z = riga.sym_eig(A)
    ref = np.linalg.eigvalsh(A)
    scale = np.abs(ref).max()
    assert np.max(np.abs(theta - ref)) <= 1e-13 * scale * A.shape[0] / 10
    assert np.max(np.abs(A @ Z - Z * theta)) <= 1e-13 * scale * A.shape[0] / 10
    assert np.max(np.abs(Z.T @ Z - np.eye(A.shape[0]))) <= 1e-12


def test_band_eigvecs_threads_deterministic_with_clusters():
    """Many wanted vectors on a large band matrix (the case that splits the
    clusters of Ritz values over host threads): two calls agree bit for bit,
    the vectors are eigenvectors and orthonormal, including inside exact
    double eigenvalues (two interleaved copies of one band matrix)."""
    n0, b0 = 110, 2
    T0 = _band(n0, b0, 19)
    n, b = 2 * n0, 2 * b0
    T = np.zeros((n, n))
    T[0::2, 0::2] = T0
    T[1::2, 1::2] = T0
    which = list(range(n - 96, n))
    th1, S1 = riga.band_eig(T, b, which)
    th2, S2 = riga.band_eig(T, b, which)
    assert np.array_equal(th1, th2) and np.array_equal(S1, S2)
    scale = np.abs(th1).max()
    assert np.max(np.abs(T @ S1 - S1 * th1[which])) <= 1e-11 * scale
    assert np.max(np.abs(S1.T @ S1 - np.eye(len(which)))) <= 1e-10
