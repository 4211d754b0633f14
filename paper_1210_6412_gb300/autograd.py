"""torch.autograd.Function for parametric chains: theta -> P(theta) -> x_init.

P_e = softmax over the out-edges of each state of theta[class_e] + offset_e.  The
forward pass builds P and solves for Pr(init |= <> GS) through the CUDA library; the
backward pass solves the adjoint system (I - A)^T y = e_init there, forms
d x_init / d P_e = y_s x_{s'}, and applies the softmax chain rule per class.  All of
it runs in libreach.so; this module only moves tensors.
"""
from __future__ import annotations

import torch

from . import (REACH_PROB01, Solver, reach_param_grad_theta, reach_param_probs)


class ReachProb(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, rowptr, col, cls, offset, goal, init, method="jacobi", eps=1e-13,
                max_iter=1_000_000, mode=REACH_PROB01, adj_eps=1e-14, adj_method="jacobi"):
        n = rowptr.numel() - 1
        m = col.numel()
        theta = theta.detach().contiguous()
        p = torch.empty(m, dtype=torch.float64, device=theta.device)
        reach_param_probs(rowptr, cls, offset, theta, p)
        solver = Solver(n, rowptr, col, p, goal, mode=mode)
        x = torch.empty(n, dtype=torch.float64, device=theta.device)
        solver.solve(method, eps=eps, max_iter=max_iter, out=x)
        ctx.solver = solver
        ctx.init = int(init)
        ctx.adj = (adj_eps, max_iter, adj_method)
        ctx.n_classes = theta.numel()
        ctx.save_for_backward(rowptr, cls, p)
        return x[int(init)].clone()

    @staticmethod
    def backward(ctx, grad_out):
        rowptr, cls, p = ctx.saved_tensors
        g_p = torch.empty_like(p)
        ctx.solver.grad(ctx.init, eps=ctx.adj[0], max_iter=ctx.adj[1], out=g_p, method=ctx.adj[2])
        g_theta = torch.empty(ctx.n_classes, dtype=torch.float64, device=p.device)
        reach_param_grad_theta(rowptr, cls, p, g_p, ctx.n_classes, g_theta)
        ctx.solver.close()
        return (grad_out * g_theta,) + (None,) * 12


def reach_prob(theta, rowptr, col, cls, offset, goal, init, **kw):
    """Pr(init |= <> GS) of the chain with probabilities softmax(theta[cls] + offset).

    Keywords: method (forward solver), eps, max_iter, mode, adj_eps and adj_method (the
    adjoint solver: "jacobi" or "bicgstab").
    """
    return ReachProb.apply(theta, rowptr, col, cls, offset, goal, init,
                           kw.get("method", "jacobi"), kw.get("eps", 1e-13),
                           kw.get("max_iter", 1_000_000), kw.get("mode", REACH_PROB01),
                           kw.get("adj_eps", 1e-14), kw.get("adj_method", "jacobi"))
