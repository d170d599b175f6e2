"""torch.autograd wrappers of the estimator (marshalling only; every step runs in libfm).

field_map_cost(omega, fm)
    Psi(omega) of Eq. 5 as a differentiable scalar; backward multiplies the incoming
    gradient by grad Psi (Eq. 8) from the gradient kernel.
field_map_solve(y, beta, fm, smap, te, mask, niter, ...)
    The NCG-MLS-IC field map w^ as a differentiable function of the images y and the
    weight beta.  Backward applies the implicit function theorem at w^ (the solve is
    assumed converged: grad Psi(w^) = 0): one IC(0)-preconditioned CG solve with the true
    Hessian gives lambda, then dl/dbeta = -lambda' C'C w^ and dl/dy = -(d grad Phi/dy)'
    lambda (fm_adjoint_solve, fm_implicit_grad).
"""
from __future__ import annotations

import torch


class _CostFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, omega, fm):
        cost, g, _ = fm.cost_grad(omega.detach().contiguous(), want_curv=False)
        ctx.save_for_backward(g)
        return torch.tensor(cost, dtype=torch.float64, device=omega.device)

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        return gout.to(g.dtype) * g, None


def field_map_cost(omega, fm):
    """Differentiable Psi(omega) for the data last given to fm.set_data."""
    return _CostFn.apply(omega, fm)


class _SolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, beta, fm, smap, te, mask, niter, omega0, tol, maxiter):
        yd = y.detach().contiguous()
        fm.set_data(yd, smap, te, mask, float(beta))
        w, _ = fm.solve(omega0, niter=niter, want_history=False)
        ctx.fm = fm
        ctx.args = (smap, te, mask, float(beta), tol, maxiter)
        ctx.beta_like = (beta.dtype, beta.device)
        ctx.save_for_backward(yd, w)
        ctx.stats = {}
        return w

    @staticmethod
    def backward(ctx, gw):
        fm = ctx.fm
        yd, w = ctx.saved_tensors
        smap, te, mask, beta, tol, maxiter = ctx.args
        if fm.data[0] is not yd or fm.data[4] != beta:  # the context holds other data now
            fm.set_data(yd, smap, te, mask, beta)
        b = gw.to(w.dtype).contiguous()
        lam, it, rr = fm.adjoint_solve(w, b, tol=tol, maxiter=maxiter)
        fm.last_adjoint = {"iterations": it, "relres": rr}
        need_y, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        dy, db = fm.implicit_grad(w, lam, yd, smap, want_dy=need_y, want_dbeta=need_b)
        gb = torch.tensor(db, dtype=ctx.beta_like[0], device=ctx.beta_like[1]) if need_b else None
        return dy, gb, None, None, None, None, None, None, None, None


def field_map_solve(y, beta, fm, smap, te, mask=None, niter=100, omega0=None, tol=None, maxiter=1000):
    """Differentiable converged field map.  y: complex images (fm's precision), beta: a
    float or a 0-dim floating tensor (a float becomes a CPU float64 tensor)."""
    if not torch.is_tensor(beta):
        beta = torch.tensor(float(beta), dtype=torch.float64)
    return _SolveFn.apply(y, beta, fm, smap, te, mask, niter, omega0, tol, maxiter)
