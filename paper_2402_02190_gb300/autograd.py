"""The CPRA relaxed loss as a differentiable PyTorch function.

``cpra_loss(solver, theta, emb, gamma)`` returns the scalar relaxed loss
R(theta, h^0) of Eq. CPRA-loss-function-GNN (-penalty / -variation) for the
two-layer GCN of App. C.1 on the solver's graph.  Forward and backward run
in the library's CUDA kernels (``cpra_forward`` / ``cpra_backward``): the
backward is the hand-written adjoint, not autograd through PyTorch ops.
PyTorch only provides the tensors and orders the library's stream against
the caller's.
"""
from __future__ import annotations

import torch

from . import cpra


class CPRALossFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, emb, solver, gamma):
        if theta.dtype != torch.float32 or emb.dtype != torch.float32:
            raise TypeError("theta and emb must be float32")
        theta = theta.contiguous()
        emb = emb.contiguous()
        terms = torch.empty(3 * solver.S + 2, dtype=torch.float32, device=theta.device)
        cur = torch.cuda.current_stream()
        solver.stream.wait_stream(cur)   # inputs produced on the caller's stream
        cpra.cpra_forward(solver.ctx, theta, emb, float(gamma), terms)
        for t in (theta, emb, terms):    # used on the library stream
            t.record_stream(solver.stream)
        cur.wait_stream(solver.stream)
        ctx.solver = solver
        ctx.shapes = (theta.shape, emb.shape)
        ctx.device = theta.device
        R = terms[3 * solver.S + 1].clone()
        parts = terms[: 3 * solver.S + 1].clone()
        ctx.mark_non_differentiable(parts)
        return R, parts

    @staticmethod
    def backward(ctx, grad_R, grad_terms):
        if grad_terms is not None and torch.count_nonzero(grad_terms).item() != 0:
            raise RuntimeError("only the total loss R is differentiable")
        solver = ctx.solver
        scale = float(grad_R) if grad_R is not None else 0.0
        g_theta = torch.empty(ctx.shapes[0], dtype=torch.float32, device=ctx.device)
        g_emb = torch.empty(ctx.shapes[1], dtype=torch.float32, device=ctx.device)
        cur = torch.cuda.current_stream()
        solver.stream.wait_stream(cur)
        cpra.cpra_backward(solver.ctx, scale, g_theta, g_emb)
        cur.wait_stream(solver.stream)
        g_theta.record_stream(solver.stream)
        g_emb.record_stream(solver.stream)
        return g_theta, g_emb, None, None


def cpra_loss(solver, theta, emb, gamma: float):
    """Returns (R, terms): R is differentiable with respect to theta and emb;
    terms holds cost_s, pen_s, ann_s per shot and Psi."""
    return CPRALossFunction.apply(theta, emb, solver, gamma)
