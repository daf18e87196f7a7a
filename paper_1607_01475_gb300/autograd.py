"""Differentiable PSD solve for PyTorch.

``psd_solve_autograd(f, s, ...)`` returns the solution u of the fourth-order
problem N_h[u] = f (Sec. 5.3) for a CUDA float64 tensor f and a scalar s
(float or 0-d tensor); gradients flow to f and s through the library's
adjoint solve (psd_adjoint: conjugate gradients on the symmetric Jacobian
with the FFT preconditioner, by the implicit function theorem at the
converged solution, so no forward iterates are stored).  Argument
marshalling only: every step runs in libpsd.so.
"""

import torch

from ._lib import PSD_FP64, Solver

_cache = {}


def _solver(shape, h, p, s, eps, precision, tol, max_iter):
    key = (tuple(shape), h, p, s, eps, precision, tol, max_iter, torch.cuda.current_device())
    sol = _cache.get(key)
    if sol is None:
        if len(_cache) > 16:
            _cache.clear()
        sol = Solver(4, shape, h, p, s, eps, 0.0, precision=precision, tol=tol, max_iter=max_iter)
        _cache[key] = sol
    return sol


class PSDSolve(torch.autograd.Function):
    """u = PSD solution of N_h[u] = f for parameters (h, p, s, eps)."""

    @staticmethod
    def forward(ctx, f, s, h, p, eps, u0, precision, tol, max_iter, adj_tol):
        sval = float(s)
        sol = _solver(f.shape, h, p, sval, eps, precision, tol, max_iter)
        u = (u0.detach().clone() if u0 is not None else torch.zeros_like(f)).contiguous()
        sol.solve(f.detach().contiguous(), u)
        ctx.save_for_backward(u)
        ctx.params = (h, p, sval, eps, precision, tol, max_iter, adj_tol, torch.is_tensor(s))
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        h, p, sval, eps, precision, tol, max_iter, adj_tol, s_is_tensor = ctx.params
        sol = _solver(u.shape, h, p, sval, eps, precision, tol, max_iter)
        gu = grad_u.detach().contiguous().to(torch.float64)
        gf = torch.empty_like(gu)
        gs, _ = sol.adjoint(u, gu, gf, tol_rel=adj_tol)
        grad_s = torch.tensor(gs, dtype=torch.float64, device=u.device) if s_is_tensor else None
        return gf, grad_s, None, None, None, None, None, None, None, None


def psd_solve_autograd(f, s, h, p=4.0, eps=0.1, u0=None, precision=PSD_FP64, tol=1e-12, max_iter=20000,
                       adj_tol=1e-12):
    return PSDSolve.apply(f, s, h, p, eps, u0, precision, tol, max_iter, adj_tol)
