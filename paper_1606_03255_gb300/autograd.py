"""torch.autograd support for the Fourier-Laplace transform f = C(w) c.

Forward: fl_execute (Algorithm 2).  Backward, for an upstream gradient
G = dL/dRe f + i dL/dIm f (PyTorch's convention for complex tensors):

* grad c = C^* G                     -- fl_adjoint, the adjoint transform;
* grad w_j = G_j * conj(f'(w_j)),    f'(w) = sum_k (2 pi i k) c_k e^{2 pi i k w}
                                      -- fl_grad_w, the k-weighted transform with
                                      the product fused into its last kernel.

f' is recomputed in the backward pass instead of being stored (the band grids
of one transform are several GB at N = 2^20), and nothing of the forward but
c, the plan and its nodes is kept.

Nodes are an (M, 2) float64 tensor of (Re w, Im w); their gradient is returned
in the same layout ((d/d Re w, d/d Im w) = (Re, Im) of the complex gradient).
"""
from __future__ import annotations

import torch

from . import fl


class FourierLaplaceFunction(torch.autograd.Function):
    """f = C(w) c through an existing plan whose nodes are `nodes`."""

    @staticmethod
    def forward(ctx, c, nodes, plan):
        ctx.plan = plan
        ctx.save_for_backward(c)
        return plan.execute(c.contiguous())

    @staticmethod
    def backward(ctx, grad_f):
        (c,) = ctx.saved_tensors
        plan = ctx.plan
        g = grad_f.contiguous().to(plan.cdtype)
        grad_c = plan.adjoint(g) if ctx.needs_input_grad[0] else None
        grad_w = None
        if ctx.needs_input_grad[1]:
            gw = plan.grad_w(c.contiguous(), g)
            grad_w = torch.view_as_real(gw).to(torch.float64)
        return grad_c, grad_w, None


class FourierLaplace(torch.nn.Module):
    """f = sum_k c_k exp(2 pi i k w_j) with autograd in c and in the nodes w.

    The plan (banding and sorting of the nodes, tables) is rebuilt when the
    node tensor changes (new storage or an in-place update) and reused
    otherwise.
    """

    def __init__(self, N: int, eps: float = 1e-6, precision: str = "fp32", q: int = 0):
        super().__init__()
        self.N = int(N)
        self.eps = float(eps)
        self.precision = precision
        self.q = int(q)
        self._plan = None
        self._key = None

    def plan_for(self, nodes: torch.Tensor) -> fl.Plan:
        key = (nodes.data_ptr(), nodes._version, tuple(nodes.shape), nodes.device)
        if self._plan is None or key != self._key:
            if self._plan is not None:
                self._plan.close()
            self._plan = fl.Plan(self.N, nodes.detach(), self.eps, precision=self.precision,
                                 q=self.q)
            self._key = key
        return self._plan

    def forward(self, c: torch.Tensor, nodes: torch.Tensor) -> torch.Tensor:
        if nodes.dtype != torch.float64 or nodes.dim() != 2 or nodes.shape[1] != 2:
            raise TypeError("nodes must be a float64 tensor of shape (M, 2): (Re w, Im w)")
        plan = self.plan_for(nodes)
        return FourierLaplaceFunction.apply(c, nodes, plan)


def fourier_laplace(c: torch.Tensor, nodes: torch.Tensor, eps: float = 1e-6,
                    precision: str = "fp32", q: int = 0) -> torch.Tensor:
    """One-shot differentiable transform (plans on every call)."""
    plan = fl.Plan(c.numel(), nodes.detach(), eps, precision=precision, q=q)
    return FourierLaplaceFunction.apply(c, nodes, plan)
