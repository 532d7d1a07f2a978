"""torch.autograd.Function wrappers of the hand-written forward and backward kernels.

``SimplexEncodingFunction`` (and the same class for the grid comparator) returns the
encoding of ``x`` from ``tables`` and, in backward, the table gradient computed by
``sxe_encode_bwd`` (Sec. 5 e) and, when ``x`` requires it, the input gradient dL/dx
computed by ``sxe_encode_bwd_input``.
``MlpFunction`` wraps ``sxe_mlp_fwd`` / ``sxe_mlp_bwd`` and returns dL/din and dL/dW.
"""
from __future__ import annotations

import torch

from .api import Encoder, Mlp


class EncodingFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, tables: torch.Tensor, encoder: Encoder):
        x = x.contiguous()
        out = encoder.encode_fwd(x, tables.contiguous())
        ctx.save_for_backward(x, tables)
        ctx.encoder = encoder
        ctx.tables_dtype = tables.dtype
        return out

    @staticmethod
    def backward(ctx, dout: torch.Tensor):
        x, tables = ctx.saved_tensors
        enc = ctx.encoder
        dout = dout.to(torch.float32).contiguous()
        grad = None
        if ctx.needs_input_grad[1]:
            grad = torch.zeros(enc.table_shape(), dtype=torch.float32, device=x.device)
            enc.encode_bwd(x, dout, grad)
            grad = grad.to(ctx.tables_dtype)
        dx = enc.encode_bwd_input(x, tables.contiguous(), dout) if ctx.needs_input_grad[0] else None
        return dx, grad, None


class MlpFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, W: torch.Tensor, mlp: Mlp):
        x = x.contiguous()
        y = mlp.mlp_fwd(W, x)
        ctx.save_for_backward(x, W)
        ctx.mlp = mlp
        return y

    @staticmethod
    def backward(ctx, dy: torch.Tensor):
        x, W = ctx.saved_tensors
        mlp = ctx.mlp
        dW = torch.zeros((mlp.n_params,), dtype=torch.float32, device=x.device)
        din = torch.empty((x.shape[0], mlp.n_in), dtype=torch.float32, device=x.device)
        mlp.mlp_bwd(W, x, dy.to(torch.float32).contiguous(), dW, din=din)
        return din.to(x.dtype), dW.to(W.dtype), None


def encode(x, tables, encoder: Encoder):
    return EncodingFunction.apply(x, tables, encoder)


def mlp_apply(x, W, mlp: Mlp):
    return MlpFunction.apply(x, W, mlp)
