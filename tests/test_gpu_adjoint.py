"""Eigenvalue adjoint through torch.autograd on the 128x128 p=3 rIGA mesh
(C0 lines every 16 elements) with random per-element coefficients
exp(a_e), exp(b_e), a, b ~ N(0, 0.25^2): gradient of the sum of the lowest 20
eigenvalues against central finite differences (step 1e-6) at 64 seeded
coordinates, and Euler homogeneity (scaling K by e^t scales every eigenvalue
by e^t, scaling M by e^t by e^-t)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_c5_gradient_fd_and_homogeneity():
    import torch

    from paper_2009_08167_gb300.autograd import eigvals
    from paper_2009_08167_gb300.inputs import config_c5, splitmix64
    from tests.gpu_helpers import riga_ctx

    cfg = config_c5()
    mesh, k = cfg["mesh"], cfg["k"]
    dev = torch.device("cuda", 0)
    R = riga_ctx()
    R.set_eig_options(slice=0, extra=4, seed=5)
    # central differences at step 1e-6 turn an eigenvalue noise delta into
    # delta / 1e-6: the eigenvalues are taken as double-double Rayleigh
    # quotients (sigma + 1/theta carries about 1e-15 relative, which alone
    # puts the difference quotient at the 1e-5 bar)
    R.set_eig_accuracy(1)
    a = torch.tensor(cfg["a"], dtype=torch.float64, device=dev, requires_grad=True)
    b = torch.tensor(cfg["b"], dtype=torch.float64, device=dev, requires_grad=True)
    lam = eigvals(a, b, R, mesh, k, tol=1e-12)
    S = lam.sum()
    S.backward()
    ga = a.grad.cpu().numpy()
    gb = b.grad.cpu().numpy()
    s = float(S.item())
    # Euler homogeneity
    assert abs(ga.sum() - s) <= 1e-9 * s
    assert abs(gb.sum() + s) <= 1e-9 * s
    # central differences at 64 seeded coordinates (32 in a, 32 in b)
    ne = mesh.n_elem
    pick = (splitmix64(0xC5F, 64) % np.uint64(ne)).astype(np.int64)
    h = 1e-6

    def total(av, bv):
        with torch.no_grad():
            return float(eigvals(av, bv, R, mesh, k, tol=1e-12).sum().item())

    fd, an = [], []
    for j, e in enumerate(pick):
        which_a = j < 32
        base_a = a.detach().clone()
        base_b = b.detach().clone()
        if which_a:
            ap, am = base_a.clone(), base_a.clone()
            ap[e] += h
            am[e] -= h
            fd.append((total(ap, base_b) - total(am, base_b)) / (2 * h))
            an.append(ga[e])
        else:
            bp, bm = base_b.clone(), base_b.clone()
            bp[e] += h
            bm[e] -= h
            fd.append((total(base_a, bp) - total(base_a, bm)) / (2 * h))
            an.append(gb[e])
    fd = np.array(fd)
    an = np.array(an)
    assert np.linalg.norm(an - fd) <= 1e-5 * np.linalg.norm(fd)
    # per coordinate, with a floor for the finite-difference noise
    assert np.all(np.abs(an - fd) <= 1e-4 * np.abs(fd) + 1e-5 * np.abs(np.concatenate([ga, gb])).max())
    R.close()


def test_assemble_log_matches_exponentiated_coefficients():
    """riga_assemble_log(a, b) (exponentials taken on the device) gives the
    matrices of riga_assemble(exp(a), exp(b)) up to the rounding of exp, on
    host and on device inputs; all-zero logs give the constant-coefficient
    (Kronecker) matrices."""
    import torch

    from paper_2009_08167_gb300.inputs import Mesh
    from tests.gpu_helpers import riga_ctx

    mesh = Mesh(2, 24, 3, 8, 8)
    rng = np.random.default_rng(41)
    a = 0.25 * rng.normal(size=mesh.n_elem)
    b = 0.25 * rng.normal(size=mesh.n_elem)
    R = riga_ctx()
    R.assemble(mesh, np.exp(a), np.exp(b))
    _, _, K0, M0 = R.get_matrices()
    R.assemble(mesh, a, b, log=True)
    _, _, K1, M1 = R.get_matrices()
    assert np.allclose(K1, K0, rtol=1e-14, atol=0) and np.allclose(M1, M0, rtol=1e-14, atol=0)
    dev = torch.device("cuda", 0)
    R.assemble(mesh, torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev), log=True)
    _, _, K2, M2 = R.get_matrices()
    assert np.array_equal(K2, K1) and np.array_equal(M2, M1)
    R.assemble(mesh, np.zeros(mesh.n_elem), np.zeros(mesh.n_elem), log=True)
    _, _, K3, M3 = R.get_matrices()
    R.assemble(mesh)
    _, _, K4, M4 = R.get_matrices()
    assert np.allclose(K3, K4, rtol=1e-13, atol=1e-14 * np.abs(K4).max())
    assert np.allclose(M3, M4, rtol=1e-13, atol=1e-14 * np.abs(M4).max())
    R.close()
