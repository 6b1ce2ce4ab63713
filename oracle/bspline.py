"""B-spline spaces on [0,1] for IGA and refined IGA (oracle; test infrastructure only).

Sec. 3.1 (Eq. U, Eq. N, Eq. 1Dmatrix) and Sec. 3.2 (knot insertion up to
multiplicity p at the C0 separators).
"""
import numpy as np


def open_knot_vector(ne, p, mult=None):
    """Open uniform knot vector on [0,1] with ``ne`` elements (Eq. U).

    The end knots are repeated p+1 times; interior knot i/ne (i=1..ne-1) is
    repeated ``mult[i-1]`` times (1 = maximum continuity C^{p-1}; p = C0, the
    rIGA separator of Sec. 3.2).
    """
    if mult is None:
        mult = [1] * (ne - 1)
    assert len(mult) == ne - 1
    knots = [0.0] * (p + 1)
    for i in range(1, ne):
        assert 1 <= mult[i - 1] <= p
        knots += [i / ne] * int(mult[i - 1])
    knots += [1.0] * (p + 1)
    return np.array(knots, dtype=np.float64)


def riga_multiplicities(ne, p, bs):
    """Interior knot multiplicities of rIGA with blocks of ``bs`` elements:
    knots at multiples of bs are raised to multiplicity p (Sec. 3.2, Fig. 2).
    ``bs >= ne`` gives IGA (all ones)."""
    return [p if (bs > 0 and i % bs == 0) else 1 for i in range(1, ne)]


def n_functions(knots, p):
    """Number of B-splines of degree p on the knot vector."""
    return len(knots) - p - 1


def basis_and_derivative(knots, p, x):
    """Values and first derivatives of ALL B-splines B_{i,p} at points x.

    Straight from the Cox-de Boor recursion (Eq. N) with the 0/0 := 0
    convention, degree by degree.  The derivative uses the textbook relation
    B'_{i,p} = p B_{i,p-1}/(xi_{i+p}-xi_i) - p B_{i+1,p-1}/(xi_{i+p+1}-xi_{i+1}).
    Points must lie in [0,1); the half-open spans of Eq. N are used as written.
    Returns (vals, ders), each of shape (n_functions, len(x)).
    """
    knots = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(knots) - 1
    B = np.zeros((m, x.size))
    for i in range(m):
        B[i] = ((knots[i] <= x) & (x < knots[i + 1])).astype(np.float64)
    prev = B
    for d in range(1, p + 1):
        cur = np.zeros((m - d, x.size))
        for i in range(m - d):
            den1 = knots[i + d] - knots[i]
            den2 = knots[i + d + 1] - knots[i + 1]
            if den1 > 0:
                cur[i] += (x - knots[i]) / den1 * prev[i]
            if den2 > 0:
                cur[i] += (knots[i + d + 1] - x) / den2 * prev[i + 1]
        if d == p:
            lower = prev  # degree p-1
        prev = cur
    vals = prev
    ders = np.zeros_like(vals)
    if p == 0:
        return vals, ders
    for i in range(m - p):
        den1 = knots[i + p] - knots[i]
        den2 = knots[i + p + 1] - knots[i + 1]
        if den1 > 0:
            ders[i] += p / den1 * lower[i]
        if den2 > 0:
            ders[i] -= p / den2 * lower[i + 1]
    return vals, ders


def gauss_legendre(nq):
    """Gauss-Legendre nodes and weights on [-1,1] by Newton's method on the
    Legendre polynomial P_nq, evaluated by its three-term recurrence."""
    nodes = np.zeros(nq)
    weights = np.zeros(nq)
    for i in range(nq):
        t = np.cos(np.pi * (i + 0.75) / (nq + 0.5))
        for _ in range(100):
            p0, p1 = 1.0, t
            if nq == 0:
                break
            if nq == 1:
                pn, pm = p1, p0
            else:
                for j in range(1, nq):
                    p0, p1 = p1, ((2 * j + 1) * t * p1 - j * p0) / (j + 1)
                pn, pm = p1, p0
            dp = nq * (t * pn - pm) / (t * t - 1.0)
            dt = pn / dp
            t -= dt
            if abs(dt) < 1e-16:
                break
        # final derivative at the converged node
        p0, p1 = 1.0, t
        for j in range(1, nq):
            p0, p1 = p1, ((2 * j + 1) * t * p1 - j * p0) / (j + 1)
        dp = nq * (t * p1 - p0) / (t * t - 1.0)
        nodes[i] = t
        weights[i] = 2.0 / ((1.0 - t * t) * dp * dp)
    order = np.argsort(nodes)
    return nodes[order], weights[order]


def quadrature_points(ne, nq):
    """Per-element Gauss points and weights on the uniform mesh of [0,1]:
    arrays of shape (ne, nq).  The rule has p+1 points per element (a
    reading: the paper does not state its quadrature)."""
    t, w = gauss_legendre(nq)
    h = 1.0 / ne
    e = np.arange(ne)[:, None]
    x = (e + (t[None, :] + 1.0) / 2.0) * h
    wx = np.broadcast_to(w[None, :] * h / 2.0, (ne, nq)).copy()
    return x, wx


def matrices_1d(ne, p, mult=None, dirichlet=True):
    """1D stiffness K^x_ij = int B'_i B'_j and mass M^x_ij = int B_i B_j
    (Eq. 1Dmatrix) as dense arrays, integrated element by element with p+1
    Gauss points.  ``dirichlet`` drops the first and last function (the only
    ones non-zero at x=0 and x=1), consistent with Eq. dofs."""
    knots = open_knot_vector(ne, p, mult)
    x, w = quadrature_points(ne, p + 1)
    vals, ders = basis_and_derivative(knots, p, x.ravel())
    w = w.ravel()
    K = (ders * w[None, :]) @ ders.T
    M = (vals * w[None, :]) @ vals.T
    if dirichlet:
        K = K[1:-1, 1:-1]
        M = M[1:-1, 1:-1]
    return K, M


def element_matrices_1d(ne, p, mult=None, dirichlet=True):
    """Element-local 1D matrices and their global function indices.

    Returns (Ke, Me, idx): Ke, Me of shape (ne, p+1, p+1) hold
    int_e B'_a B'_b and int_e B_a B_b over the p+1 functions that are
    non-zero on element e; idx (ne, p+1) gives their global indices after
    Dirichlet removal (-1 for a removed boundary function).
    """
    knots = open_knot_vector(ne, p, mult)
    nf = n_functions(knots, p)
    x, w = quadrature_points(ne, p + 1)
    Ke = np.zeros((ne, p + 1, p + 1))
    Me = np.zeros((ne, p + 1, p + 1))
    idx = np.zeros((ne, p + 1), dtype=np.int64)
    for e in range(ne):
        vals, ders = basis_and_derivative(knots, p, x[e])
        nz = [i for i in range(nf) if np.any(vals[i] != 0.0) or np.any(ders[i] != 0.0)]
        # the p+1 functions whose support covers element e
        lo = [i for i in range(nf) if knots[i] <= x[e, 0] < knots[i + p + 1]]
        assert len(lo) == p + 1 and set(nz) <= set(lo)
        V = vals[lo]
        D = ders[lo]
        Ke[e] = (D * w[e][None, :]) @ D.T
        Me[e] = (V * w[e][None, :]) @ V.T
        g = np.array(lo, dtype=np.int64)
        if dirichlet:
            g = g - 1
            g[(g < 0) | (g >= nf - 2)] = -1
        idx[e] = g
    return Ke, Me, idx


def c0_dofs(ne, p, mult=None, dirichlet=True):
    """Indices of the interpolatory (C0) functions at interior knots of
    multiplicity p: the rIGA separator DOFs of Sec. 3.2 (Fig. 3).

    For a knot first stored at position s of the knot vector with multiplicity
    p, the function B_{s-1} has that knot p times inside its support and is
    the only one non-zero there.  Found here by evaluating the basis at the
    knot: exactly one function is non-zero at a C0 knot.
    """
    knots = open_knot_vector(ne, p, mult)
    nf = n_functions(knots, p)
    if mult is None:
        mult = [1] * (ne - 1)
    out = []
    for i in range(1, ne):
        if mult[i - 1] == p:
            t = i / ne
            vals, _ = basis_and_derivative(knots, p, [t])
            nz = np.nonzero(np.abs(vals[:, 0]) > 1e-14)[0]
            assert len(nz) == 1 and abs(vals[nz[0], 0] - 1.0) < 1e-12
            g = int(nz[0])
            if dirichlet:
                g -= 1
            out.append(g)
    return out
