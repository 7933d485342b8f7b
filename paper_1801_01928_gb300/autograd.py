"""torch.autograd.Function wrappers over the hand-written forward and adjoint entry points.

    completion_loss(X, idx, y)   1/2 sum_t (X(i_t) - y_t)^2, paper Section 1 (completion) with
                                 the adjoint of Section 3.2; one fused pass computes the loss
                                 and its core gradient when a gradient is needed
    gram(A, B)                   G_ab = <A_a, B_b>, paper Section 4 ('gram') and Section 3.1
    project_sum(U, V, Z, c)      tangent coordinates of P_X(sum_j c_j Z_j), paper Section 3.2,
                                 differentiated w.r.t. the Z cores and c with X held fixed

Every forward and backward is one call into libt3f; the only arithmetic done here is the
chain-rule scaling of a cotangent that is not exactly one (a scalar times a gradient
array). The differentiable argument of each wrapper is the packed core buffer `TT.data`.
"""
from __future__ import annotations

import torch

from . import _binding as B


def _meta(t: B.TT):
    return (t.n, t.ranks, t.batch, t.m)


def _scaled(g: torch.Tensor, s: torch.Tensor, like: torch.Tensor) -> torch.Tensor:
    if s.numel() == 1 and float(s) == 1.0:
        out = g
    else:
        out = g * s.to(g.dtype)
    return out.to(like.dtype)


class _CompletionLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, data, meta, idx, y):
        X = B.TT(data.detach(), *meta)
        if ctx.needs_input_grad[0]:
            dX, loss = B.gather_backward(X, idx, y=y, want_loss=True)
            ctx.save_for_backward(dX.data)
        else:
            _, loss = B.gather(X, idx, y=y, want_vals=False, want_loss=True)
        return loss.reshape(())

    @staticmethod
    def backward(ctx, gl):
        (g,) = ctx.saved_tensors
        return _scaled(g, gl, g), None, None, None


class _Gram(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a_data, b_data, a_meta, b_meta, math):
        A = B.TT(a_data.detach(), *a_meta)
        Bt = B.TT(b_data.detach(), *b_meta)
        ctx.save_for_backward(a_data, b_data)
        ctx.meta = (a_meta, b_meta)
        ctx.math = math
        return B.gram(A, Bt, math=math)

    @staticmethod
    def backward(ctx, dG):
        a_data, b_data = ctx.saved_tensors
        a_meta, b_meta = ctx.meta
        A = B.TT(a_data.detach(), *a_meta)
        Bt = B.TT(b_data.detach(), *b_meta)
        need_a, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        dA, dB = B.gram_backward(A, Bt, dG, need_A=need_a, need_B=need_b, math=ctx.math)
        return (dA.data.to(a_data.dtype) if need_a else None,
                dB.data.to(b_data.dtype) if need_b else None, None, None, None)


class _ProjectSum(torch.autograd.Function):
    @staticmethod
    def forward(ctx, z_data, c, U, V, z_meta):
        Z = B.TT(z_data.detach(), *z_meta)
        dU = B.project_sum(U, V, Z, c.detach())
        ctx.save_for_backward(z_data, c)
        ctx.UV = (U, V)
        ctx.z_meta = z_meta
        return dU.data

    @staticmethod
    def backward(ctx, g):
        z_data, c = ctx.saved_tensors
        U, V = ctx.UV
        Z = B.TT(z_data.detach(), *ctx.z_meta)
        gbar = B.TT(g.contiguous().to(torch.float32), U.n, U.ranks, U.batch, None)
        need_z, need_c = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        dZ, dc = B.project_sum_backward(U, V, Z, c.detach(), gbar, need_Z=need_z, need_c=need_c)
        return (dZ.data.to(z_data.dtype) if need_z else None,
                dc.to(c.dtype) if need_c else None, None, None, None)


def completion_loss(X: B.TT, idx: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """FP64 scalar 1/2 sum (X(i_t) - y_t)^2; differentiable w.r.t. X.data."""
    if X.batch != 1:
        raise ValueError("completion_loss takes one TT (batch 1)")
    return _CompletionLoss.apply(X.data, _meta(X), idx, y)


def gram(A: B.TT, Bt: B.TT, math: str = "fp32") -> torch.Tensor:
    """FP32 [A.batch, B.batch] Gram matrix; differentiable w.r.t. A.data and B.data. math
    "tf32" / "bf16" runs the forward and the adjoint on the tensor cores."""
    return _Gram.apply(A.data, Bt.data, _meta(A), _meta(Bt), math)


def project_sum(U: B.TT, V: B.TT, Z: B.TT, c: torch.Tensor) -> B.TT:
    """Tangent coordinates dU (a TT with U's shape) of P_X(sum_j c_j Z_j); its .data is
    differentiable w.r.t. Z.data and c."""
    out = _ProjectSum.apply(Z.data, c, U, V, _meta(Z))
    return B.TT(out, U.n, U.ranks, U.batch, None)
