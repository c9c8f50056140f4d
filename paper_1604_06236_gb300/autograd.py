"""Differentiable type-5 and type-4 inverses (torch.autograd.Function).

Forward: plan on the nodes, then the non-iterative inverse (Secs. III, IV).
Backward, with G_{q,m} = e^{j 2 pi m t_q} (Eq. 48) and the type-4 matrix G^H
(Eq. 47) — the type-4/5 duality of Sec. VI:
  * type-5, S = G^{-1} f:  grad_f = G^{-H} grad_S, computed by the type-4
    inverse; grad_x from the derivative type-2 of S (library kernels);
  * type-4, a = G^{-H} A:  grad_A = G^{-1} grad_a, computed by the type-5
    inverse; grad_x from the derivative type-2 of grad_A.
Between the passes only the kernel samples K_q (Eq. 29) and the derivative
samples L'(z_p) (Sec. III-D) are kept, 32 bytes per node (Plan.save); the
backward pass restores each plan from them and the saved nodes, recomputing
the spreading geometry (exact turns, cell sort, extended node list), the
node phases and the weights instead of storing them, and skipping the plan's
log-kernel type-1, FFTs and type-2.

Plans are made with the deferred coincident-node check: all of a pass's
plans and transforms are queued before the host waits for the checks.  With
one node set per instance the instances are spread over a few CUDA streams
(each instance's plan and transforms stay on one stream, ordered after the
caller's stream and joined back into it), so that the plans, whose stages
are latency-bound at one right-hand side, overlap.

Nodes x: float64 tensor of shape (N,) shared by every right-hand side, or
(B, N) with one node set per instance (data then (B, N)).
"""
import torch

from . import DEFER_CHECK, FP32, FP64, Plan

__all__ = ["inv5", "inv4"]


def _node_sets(x):
    xd = x.detach()
    return [xd] if xd.dim() == 1 else [xd[i] for i in range(xd.shape[0])]


def _split(t, x):
    """Per-plan slices of a (..., N) tensor: all rows for shared nodes, row i for instance i."""
    if x.dim() == 1:
        return [t]
    return [t[i] for i in range(x.shape[0])]


_STREAMS = {}
_NSTREAMS = 8


def _lanes(device, count):
    """The caller's stream alone for one instance, else a pool of side
    streams of this device, each ordered after the caller's stream."""
    main = torch.cuda.current_stream(device)
    if count <= 1:
        return main, [main]
    pool = _STREAMS.get(device.index)
    if pool is None:
        pool = _STREAMS[device.index] = [torch.cuda.Stream(device) for _ in range(_NSTREAMS)]
    lanes = pool[:min(count, len(pool))]
    for s in lanes:
        s.wait_stream(main)
    return main, lanes


def _join(main, lanes, tensors):
    """Order the caller's stream after the side streams; tensors made on a
    side stream are marked as used by the caller's stream."""
    for s in lanes:
        if s is not main:
            main.wait_stream(s)
    for t in tensors:
        t.record_stream(main)


def _finish(plans):
    """Wait for the plans' coincident-node checks, then release them."""
    try:
        for pl in plans:
            pl.check()
    finally:
        for pl in plans:
            pl.close()


class _Inverse(torch.autograd.Function):
    @staticmethod
    def forward(ctx, data, x, kind, tol, prec):
        plans, outs, saved = [], [], []
        sets = _node_sets(x)
        main, lanes = _lanes(x.device, len(sets))
        try:
            for i, (xi, d) in enumerate(zip(sets, _split(data, x))):
                s = lanes[i % len(lanes)]
                with torch.cuda.stream(s):
                    pl = Plan(xi, tol=tol, prec=prec | DEFER_CHECK, stream=s)
                    plans.append(pl)
                    outs.append(pl.inv5(d, stream=s) if kind == 5 else pl.inv4(d, stream=s))
                    saved.append(pl.save(stream=s))
        finally:
            _join(main, lanes, outs + [t for K, D, _ in saved for t in (K, D)])
            _finish(plans)
        out = outs[0] if x.dim() == 1 else torch.stack(outs)
        ctx.save_for_backward(x, out, *[t for K, D, _ in saved for t in (K, D)])
        ctx.params = [p for _, _, p in saved]
        ctx.kind, ctx.tol, ctx.prec = kind, plans[0].tol, prec
        return out

    @staticmethod
    def backward(ctx, g):
        x, out, *kd = ctx.saved_tensors
        need_data, need_x = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        g = g.contiguous().to(out.dtype)
        gd, gx, plans = [], [], []
        sets = _node_sets(x)
        main, lanes = _lanes(x.device, len(sets))
        try:
            for i, (xi, gi, oi) in enumerate(zip(sets, _split(g, x), _split(out, x))):
                s = lanes[i % len(lanes)]
                with torch.cuda.stream(s):
                    pl = Plan(xi, tol=ctx.tol, prec=ctx.prec | DEFER_CHECK, stream=s,
                              saved=(kd[2 * i], kd[2 * i + 1], ctx.params[i]))
                    plans.append(pl)
                    # the dual inverse carries the gradient back to the data
                    gdi = pl.inv4(gi, stream=s) if ctx.kind == 5 else pl.inv5(gi, stream=s)
                    gd.append(gdi)
                    if need_x:
                        gx.append(pl.inv5_grad_nodes(gdi, oi, stream=s) if ctx.kind == 5
                                  else pl.inv4_grad_nodes(gdi, oi, stream=s))
        finally:
            _join(main, lanes, gd + gx)
            _finish(plans)
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
