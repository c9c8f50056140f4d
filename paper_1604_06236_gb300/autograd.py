"""Differentiable type-5 and type-4 inverses (torch.autograd.Function).

Forward: plan on the nodes, then the non-iterative inverse (Secs. III, IV).
Backward, with G_{q,m} = e^{j 2 pi m t_q} (Eq. 48) and the type-4 matrix G^H
(Eq. 47) — the type-4/5 duality of Sec. VI:
  * type-5, S = G^{-1} f:  grad_f = G^{-H} grad_S, computed by the type-4
    inverse; grad_x from the derivative type-2 of S (library kernels);
  * type-4, a = G^{-H} A:  grad_A = G^{-1} grad_a, computed by the type-5
    inverse; grad_x from the derivative type-2 of grad_A.
The plan (node geometry, kernel samples, weights) is rebuilt from the saved
nodes in the backward pass instead of being kept alive between the passes.

Nodes x: float64 tensor of shape (N,) shared by every right-hand side, or
(B, N) with one node set per instance (data then (B, N)).
"""
import torch

from . import FP32, FP64, Plan

__all__ = ["inv5", "inv4"]


def _plans(x, tol, prec):
    xd = x.detach()
    if xd.dim() == 1:
        return [Plan(xd, tol=tol, prec=prec)]
    return [Plan(xd[i], tol=tol, prec=prec) for i in range(xd.shape[0])]


def _split(t, x):
    """Per-plan slices of a (..., N) tensor: all rows for shared nodes, row i for instance i."""
    if x.dim() == 1:
        return [t]
    return [t[i] for i in range(x.shape[0])]


class _Inverse(torch.autograd.Function):
    @staticmethod
    def forward(ctx, data, x, kind, tol, prec):
        plans = _plans(x, tol, prec)
        outs = []
        for pl, d in zip(plans, _split(data, x)):
            outs.append(pl.inv5(d) if kind == 5 else pl.inv4(d))
            pl.close()
        out = outs[0] if x.dim() == 1 else torch.stack(outs)
        ctx.save_for_backward(x, out)
        ctx.kind, ctx.tol, ctx.prec = kind, tol, prec
        return out

    @staticmethod
    def backward(ctx, g):
        x, out = ctx.saved_tensors
        need_data, need_x = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        plans = _plans(x, ctx.tol, ctx.prec)
        g = g.contiguous().to(out.dtype)
        gd, gx = [], []
        for pl, gi, oi in zip(plans, _split(g, x), _split(out, x)):
            # the dual inverse carries the gradient back to the data
            gdi = pl.inv4(gi) if ctx.kind == 5 else pl.inv5(gi)
            gd.append(gdi)
            if need_x:
                gx.append(pl.inv5_grad_nodes(gdi, oi) if ctx.kind == 5 else pl.inv4_grad_nodes(gdi, oi))
            pl.close()
        grad_data = (gd[0] if x.dim() == 1 else torch.stack(gd)) if need_data else None
        grad_x = None
        if need_x:
            grad_x = (gx[0] if x.dim() == 1 else torch.stack(gx)).to(x.dtype)
        return grad_data, grad_x, None, None, None


def inv5(f, x, tol=None, prec=FP32):
    """Type-5 inverse S from samples f at nodes x (radians), differentiable in f and x."""
    return _Inverse.apply(f, x, 5, tol, prec)


def inv4(A, x, tol=None, prec=FP32):
    """Type-4 inverse a from spectral samples A, differentiable in A and x."""
    return _Inverse.apply(A, x, 4, tol, prec)
