"""CPU pins of the forward-error bounds that the GPU factor-parity tests use.

tests.gpu_helpers.ldlt_forward_bounds turns a componentwise backward error
|dA| <= eps B of an LDL^T factorization without pivoting into first-order
bounds on each pivot and multiplier.  Here the oracle's own factorization of
perturbed matrices checks both directions: every perturbation within eps B
stays inside the bounds (times the factor 2 the GPU tests allow), and the
pivot bound is attained to first order by the perturbation that aligns every
term's sign, so a dropped absolute value, a transposed inverse or a missing
entry of B fails.
"""
import numpy as np
import pytest

from oracle import eigen, factor
from paper_2009_08167_gb300.inputs import Mesh
from tests.gpu_helpers import ldlt_forward_bounds, oracle_matrices

CASES = [(Mesh(2, 16, 2, None), 0), (Mesh(2, 16, 2, None), 1), (Mesh(3, [5, 6, 4], 2, None, 3), 1)]


def _matrix(mesh, which):
    """P-free K - sigma M at sigma = 0 (which 0) or in a gap a third of the
    way up the spectrum (which 1), with its backward-error scale B."""
    K, M = oracle_matrices(mesh)
    Kd, Md = K.todense(), M.todense()
    sigma = 0.0
    if which:
        lam, _ = eigen.ghep_dense(Kd, Md)
        gaps = [i for i in range(lam.size - 1) if lam[i + 1] - lam[i] > 1e-3 * lam[i]]
        i = gaps[len(gaps) // 3]
        sigma = 0.5 * (lam[i] + lam[i + 1])
    A = Kd - sigma * Md
    L, d = factor.ldlt_dense(A)
    B = (np.abs(L) * np.abs(d)[None, :]) @ np.abs(L).T + np.abs(Kd) + abs(sigma) * np.abs(Md)
    return A, L, d, B


@pytest.mark.parametrize("case", CASES, ids=[f"{m!r}-{w}" for m, w in CASES])
def test_random_perturbations_stay_inside(case):
    mesh, which = case
    A, L, d, B = _matrix(mesh, which)
    eps = 1e-13
    dbound, Lbound = ldlt_forward_bounds(L, d, B, eps)
    rng = np.random.default_rng(11)
    low = np.tril(np.ones(L.shape, dtype=bool), -1)
    worst_d = worst_L = 0.0
    for _ in range(3):
        E = rng.uniform(-1.0, 1.0, size=A.shape)
        E = np.triu(E) + np.triu(E, 1).T
        L2, d2 = factor.ldlt_dense(A + eps * B * E)
        assert np.all(np.abs(d2 - d) <= 2 * dbound)
        assert np.all(np.abs(L2 - L)[low] <= 2 * Lbound[low])
        worst_d = max(worst_d, np.max(np.abs(d2 - d) / dbound))
        nz = low & (Lbound > 0)
        worst_L = max(worst_L, np.max(np.abs(L2 - L)[nz] / Lbound[nz]))
    # not vacuous: random perturbations reach a good part of the bounds
    assert worst_d > 0.3 and worst_L > 0.3


@pytest.mark.parametrize("case", CASES, ids=[f"{m!r}-{w}" for m, w in CASES])
def test_sign_aligned_perturbation_attains_pivot_bound(case):
    mesh, which = case
    A, L, d, B = _matrix(mesh, which)
    n = A.shape[0]
    Li = np.linalg.inv(L)
    eps = 1e-14
    dbound, _ = ldlt_forward_bounds(L, d, B, eps)
    # for pivot k, dd_k = sum_ab Li_ka dA_ab Li_kb to first order; the
    # symmetric choice dA_ab = eps B_ab sign(Li_ka Li_kb) makes every term
    # positive, so dd_k = eps G_kk
    for k in [n // 3, n // 2, n - 1, int(np.argmax(dbound / np.abs(d)))]:
        s = np.sign(np.outer(Li[k], Li[k]))
        _, d2 = factor.ldlt_dense(A + eps * B * s)
        assert abs((d2[k] - d[k]) / dbound[k] - 1.0) < 1e-2
