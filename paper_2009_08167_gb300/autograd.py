"""torch.autograd wrapper of the eigenvalue adjoint (riga_eig_grad).

EigVals(a, b) returns the k smallest eigenvalues of K(a) u = lambda M(b) u,
K(a) = sum_e exp(a_e) K_e, M(b) = sum_e exp(b_e) M_e, as a differentiable
function of the per-element log-coefficients a and b.  The forward pass is
riga_assemble_log (log-coefficients in, exponentials
taken in the library) + riga_eigs; the backward pass is riga_eig_grad with the
incoming dL/dlambda as weights (simple eigenvalues, or symmetric functions of
complete degenerate groups).  Marshalling only: the work runs in the library.
"""
import torch

from .riga import Riga


class _EigVals(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, b, solver, mesh, k, tol, sigma):
        la = a.detach().to(torch.float64).contiguous()
        lb = b.detach().to(torch.float64).contiguous()
        solver.assemble(mesh, la, lb, log=True)  # the library exponentiates
        ev, _, rs = solver.eigs(k, sigma, tol, vectors=False, device_out=a.is_cuda)
        ctx.solver = solver
        ctx.k = k
        ev = ev if torch.is_tensor(ev) else torch.from_numpy(ev)
        return ev.to(a.device)

    @staticmethod
    def backward(ctx, grad_lam):
        w = grad_lam.detach().to(torch.float64).contiguous()
        ga, gb = ctx.solver.eig_grad(ctx.k, w)
        return ga, gb, None, None, None, None, None


def eigvals(a, b, solver: Riga, mesh, k, tol=1e-10, sigma=0.0):
    """k smallest eigenvalues above sigma, differentiable in a and b (1D tensors
    of length n_elem, float64; CUDA tensors keep everything on the device)."""
    return _EigVals.apply(a, b, solver, mesh, k, tol, sigma)
