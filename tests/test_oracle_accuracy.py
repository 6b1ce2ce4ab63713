"""Pins of the oracle's eigenvalue / eigenfunction error module
(oracle/accuracy.py, Eq. eigerrors), none of which compares it with itself:

* Eq. Pythagorean: EFerr_E = EVerr + EFerr_L2 for every M-normalised discrete
  eigenpair (lambda_h its Rayleigh quotient); a wrong basis derivative, sign,
  weight or mode amplitude breaks it.  The three terms are sums at the scale
  ||u||^2 = a(u, u)/lambda = 1, so rounding leaves about 1e-15 absolute: the
  bar is 1e-12 absolute plus 1e-9 relative.  The identity holds for any
  scaling of the exact mode (the amplitude terms cancel), so the amplitude
  is pinned by the next two items.
* Brute force: the L2 and energy errors of a 1D mode recomputed by composite
  Simpson sums on 80,000 subintervals (the knots on the grid), with the
  discrete field evaluated point by point.
* Convergence: for the first mode EVerr = O(h^{2p}) and EFerr_L2 = O(h^{2p+2})
  (halving h divides them by about 2^{2p} and 2^{2p+2}).
"""
import numpy as np
import pytest

from oracle import accuracy, bspline, eigen


def _modes_1d(ne, p, mult):
    lam, V = eigen.eig1d(ne, p, mult)
    return lam, V


@pytest.mark.parametrize("p,bs", [(2, None), (3, None), (3, 4), (2, 8)])
def test_pythagorean_identity_1d(p, bs):
    ne = 16
    mult = bspline.riga_multiplicities(ne, p, bs) if bs else None
    lam, V = _modes_1d(ne, p, mult)
    n = lam.size // 2
    ev, efl, efe = accuracy.mode_errors(1, ne, p, [mult], lam[:n], V[:, :n], [(i + 1,) for i in range(n)])
    assert np.all(ev > -1e-14)  # Galerkin: lambda_h >= lambda
    assert np.all(np.abs(efe - (ev + efl)) <= 1e-12 + 1e-9 * efe)


def test_pythagorean_identity_2d_kronecker_modes():
    ne, p = 12, 2
    lam, idx, vecs = eigen.kron_sum_eigs(2, [ne, ne], p, None, k=12)
    modes = [tuple(int(t) + 1 for t in row) for row in idx]
    ev, efl, efe = accuracy.mode_errors(2, ne, p, None, lam, vecs, modes)
    assert np.all(np.abs(efe - (ev + efl)) <= 1e-12 + 1e-9 * efe)
    # the 2D eigenvalue error of mode (i, j) is the weighted sum of the 1D ones
    lam1, _ = eigen.eig1d(ne, p)
    for c, (i, j) in enumerate(modes):
        lam_e = np.pi ** 2 * (i * i + j * j)
        assert abs(ev[c] - (lam1[i - 1] + lam1[j - 1] - lam_e) / lam_e) <= 1e-12


def _simpson_errors(ne, p, coeff, mode, nsub=80000):
    knots = bspline.open_knot_vector(ne, p)
    x = np.linspace(0.0, 1.0, nsub + 1)
    xe = np.minimum(x, 1.0 - 1e-15)  # the half-open spans of Eq. N at x = 1
    vals, ders = bspline.basis_and_derivative(knots, p, xe)
    uh = coeff @ vals[1:-1]
    duh = coeff @ ders[1:-1]
    ue = np.sqrt(2.0) * np.sin(mode * np.pi * x)
    due = np.sqrt(2.0) * mode * np.pi * np.cos(mode * np.pi * x)
    if np.sum(uh * ue) < 0:
        uh, duh = -uh, -duh
    w = np.ones(nsub + 1)
    w[1:-1:2] = 4.0
    w[2:-1:2] = 2.0
    w *= (1.0 / nsub) / 3.0
    return np.sum(w * (uh - ue) ** 2), np.sum(w * (duh - due) ** 2) / (np.pi ** 2 * mode * mode)


@pytest.mark.parametrize("p", [1, 2])
def test_errors_against_composite_simpson(p):
    ne = 8
    lam, V = _modes_1d(ne, p, None)
    modes = [1, 2, 5]
    ev, efl, efe = accuracy.mode_errors(1, ne, p, None, lam[[m - 1 for m in modes]], V[:, [m - 1 for m in modes]],
                                        [(m,) for m in modes])
    for c, m in enumerate(modes):
        l2, en = _simpson_errors(ne, p, V[:, m - 1], m)
        assert abs(efl[c] - l2) <= 1e-9 * max(l2, 1e-12) + 1e-15
        assert abs(efe[c] - en) <= 1e-9 * max(en, 1e-12) + 1e-15


@pytest.mark.parametrize("p", [2, 3])
def test_first_mode_convergence_rates(p):
    res = []
    for ne in (8, 16):
        lam, V = _modes_1d(ne, p, None)
        ev, efl, _ = accuracy.mode_errors(1, ne, p, None, lam[:1], V[:, :1], [(1,)])
        res.append((ev[0], efl[0]))
    r_ev = res[0][0] / res[1][0]
    r_l2 = res[0][1] / res[1][1]
    assert 0.7 * 2 ** (2 * p) <= r_ev <= 1.3 * 2 ** (2 * p)
    assert 0.7 * 2 ** (2 * p + 2) <= r_l2 <= 1.3 * 2 ** (2 * p + 2)
