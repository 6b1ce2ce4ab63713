"""Eigenvalue and eigenfunction errors of discrete eigenpairs against the exact
Laplace eigenpairs of the unit interval, square or cube (oracle; test
infrastructure only: imported by tests/ alone).

Sec. 2, Eq. exact: lambda = pi^2 (i^2 + j^2 [+ k^2]) and
u = 2^{d/2} sin(i pi x) sin(j pi y) [sin(k pi z)] (1D: sqrt(2) sin(i pi x)),
mode indices from 1.
Sec. 2, Eq. eigerrors: EVerr = (lambda_h - lambda) / lambda,
EFerr_L2 = ||u_h - u||^2 and EFerr_E = a(u_h - u, u_h - u) / lambda, with
u_h L2-normalised (M-normalised coefficients) and its sign taken so that
(u_h, u) >= 0.  Eq. Pythagorean states EFerr_E = EVerr + EFerr_L2 whenever
lambda_h is the Rayleigh quotient of u_h; the tests use that as a pin.

The integrals are Gauss-Legendre sums with nq points per element (default
p + 6; u_h is a piecewise polynomial of degree p and u a product of sines),
the fields evaluated on the tensor grid of the 1D points from the 1D basis
tables (Cox-de Boor, oracle/bspline.py).
"""
import numpy as np

from . import bspline


def _tables(ne, p, mult, nq):
    """1D quadrature points and weights on [0,1], and the values and
    derivatives of the B-splines that survive the Dirichlet conditions (the
    first and last function dropped) at those points."""
    knots = bspline.open_knot_vector(ne, p, mult)
    x, w = bspline.quadrature_points(ne, nq)
    vals, ders = bspline.basis_and_derivative(knots, p, x.ravel())
    return x.ravel(), w.ravel(), vals[1:-1], ders[1:-1]


def _field(tabs, coeff):
    """Values and gradient of u_h = sum c_I prod_a B_{I_a}(x_a) on the tensor
    grid of quadrature points.  coeff has one axis per direction, the x axis
    last (the global numbering is x fastest); the results have the same axis
    order over quadrature points."""
    dim = len(tabs)
    # tables in axis order (z, y, x) / (y, x) / (x)
    order = list(reversed(range(dim)))
    B = [tabs[a][2] for a in order]
    D = [tabs[a][3] for a in order]
    letters = "abc"[:dim]
    out = "".join(chr(ord("p") + t) for t in range(dim))
    spec_in = letters + "," + ",".join(letters[t] + out[t] for t in range(dim))
    val = np.einsum(spec_in + "->" + out, coeff, *B)
    grad = []
    for a in range(dim):  # derivative along the axis at position t of the coeff array
        t = order.index(a)
        mats = [D[s] if s == t else B[s] for s in range(dim)]
        grad.append(np.einsum(spec_in + "->" + out, coeff, *mats))
    return val, grad


def _exact(tabs, mode):
    """Exact eigenfunction and gradient on the same grid (axis order as in
    _field)."""
    dim = len(tabs)
    order = list(reversed(range(dim)))
    xs = [tabs[a][0] for a in order]
    ks = [mode[a] for a in order]
    amp = 2.0 ** (dim / 2.0)
    s = [np.sin(k * np.pi * x) for k, x in zip(ks, xs)]
    c = [k * np.pi * np.cos(k * np.pi * x) for k, x in zip(ks, xs)]

    def outer(fs):
        r = fs[0]
        for f in fs[1:]:
            r = np.multiply.outer(r, f)
        return r

    val = amp * outer(s)
    grad = []
    for a in range(dim):
        t = order.index(a)
        grad.append(amp * outer([c[q] if q == t else s[q] for q in range(dim)]))
    return val, grad


def mode_errors(dim, ne, p, mults, lam_h, u_h, modes, nq=None):
    """EVerr, EFerr_L2 and EFerr_E (Eq. eigerrors) of discrete eigenpairs.

    dim: 1, 2 or 3; ne: elements per side (int, or one per direction);
    mults: per-direction interior knot multiplicities (None = maximum
    continuity); lam_h[c] and the M-normalised coefficient column u_h[:, c]
    (x fastest, Dirichlet functions removed) are compared with the exact mode
    of index tuple modes[c] (1-based).  Returns three arrays."""
    if np.isscalar(ne):
        ne = [int(ne)] * dim
    if mults is None:
        mults = [None] * dim
    nq = nq if nq is not None else p + 6
    tabs = [_tables(ne[a], p, mults[a], nq) for a in range(dim)]
    wts = [tabs[a][1] for a in reversed(range(dim))]
    W = wts[0]
    for wv in wts[1:]:
        W = np.multiply.outer(W, wv)
    shape = tuple(tabs[a][2].shape[0] for a in reversed(range(dim)))
    u_h = np.atleast_2d(np.asarray(u_h, dtype=np.float64).T).T
    lam_h = np.atleast_1d(np.asarray(lam_h, dtype=np.float64))
    ev, efl, efe = [], [], []
    for c in range(u_h.shape[1]):
        mode = tuple(int(m) for m in modes[c])
        lam_e = np.pi ** 2 * float(sum(m * m for m in mode))
        vh, gh = _field(tabs, u_h[:, c].reshape(shape))
        ve, ge = _exact(tabs, mode)
        sgn = 1.0 if np.sum(W * vh * ve) >= 0.0 else -1.0
        l2 = np.sum(W * (sgn * vh - ve) ** 2)
        en = sum(np.sum(W * (sgn * gh[a] - ge[a]) ** 2) for a in range(dim))
        ev.append((lam_h[c] - lam_e) / lam_e)
        efl.append(l2)
        efe.append(en / lam_e)
    return np.array(ev), np.array(efl), np.array(efe)
