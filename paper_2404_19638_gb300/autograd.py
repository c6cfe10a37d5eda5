"""Differentiation through the SDDMM / SpMM adjoint pair (Sec. 3.2).

Both operations take or output two dense vectors per nonzero, and each one's
gradient is the other one:

  SpMM   C = S B            dB = S^T dC  (SpMM^T via the transpose plan)
                            ds_e = <dC_i, b_j>  (an SDDMM with unit values)
  SDDMM  c_e = s_e<a_i,b_j>  dA = (S.g) B  (SpMM with values s*g)
                            dB = (S.g)^T A  (SpMM^T with values s*g)
                            ds_e = g_e <a_i, b_j>  (SDDMM with values g)

Every backward step is one of the library's kernels; gradients of BF16 / F16
factors are written in the factor's dtype by the kernel itself (FP32
accumulation inside).  The pattern S is not differentiated; its values are.
"""
from __future__ import annotations

import torch

from . import ops
from .sparse import CSR


def _vals_or_none(v):
    return v if (v is not None and v.numel() > 0) else None


class SDDMMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, S: CSR, vals, A, B):
        ctx.S = S
        ctx.save_for_backward(vals, A, B)
        return ops.sddmm(S, A, B, _vals_or_none(vals), use_default_vals=False)

    @staticmethod
    def backward(ctx, g):
        vals, A, B = ctx.saved_tensors
        S = ctx.S
        g = g.contiguous().float()
        v = _vals_or_none(vals)
        dvals = dA = dB = None
        if ctx.needs_input_grad[1]:
            dvals = ops.sddmm(S, A, B, g, use_default_vals=False)
        if ctx.needs_input_grad[2]:
            dA = ops.spmm(S, B, v, g, out_dtype=A.dtype, use_default_vals=False)
        if ctx.needs_input_grad[3]:
            dB = ops.spmm_t(S, A, v, g, out_dtype=B.dtype, use_default_vals=False)
        return None, dvals, dA, dB


class SpMMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, S: CSR, vals, B):
        ctx.S = S
        ctx.save_for_backward(vals, B)
        return ops.spmm(S, B, _vals_or_none(vals), use_default_vals=False)

    @staticmethod
    def backward(ctx, dC):
        vals, B = ctx.saved_tensors
        S = ctx.S
        dC = dC.contiguous().float()
        dvals = dB = None
        if ctx.needs_input_grad[1]:
            dvals = ops.sddmm(S, dC, B, use_default_vals=False)
        if ctx.needs_input_grad[2]:
            dB = ops.spmm_t(S, dC, _vals_or_none(vals), out_dtype=B.dtype, use_default_vals=False)
        return None, dvals, dB


def sddmm(S: CSR, A, B, vals=None):
    """Differentiable SDDMM; ``vals`` None means all ones (not differentiated)."""
    if vals is None:
        vals = torch.empty(0, dtype=torch.float32, device=S.device)
    return SDDMMFunction.apply(S, vals, A, B)


def spmm(S: CSR, B, vals=None):
    """Differentiable SpMM (FP32 output)."""
    if vals is None:
        vals = torch.empty(0, dtype=torch.float32, device=S.device)
    return SpMMFunction.apply(S, vals, B)


class GNNLayerFunction(torch.autograd.Function):
    """Y = SpMM(S_e, H) with e = SDDMM(S, H, H): an attention-style graph layer.

    Backward accumulates the three contributions to dH in FP32 inside the
    kernels (accumulate mode) and writes H's dtype once:
      dE_e = <dY_i, h_j>;  dH = (S.dE) H + (S.dE)^T H + S_e^T dY.
    """

    @staticmethod
    def forward(ctx, S: CSR, vals, H):
        v = _vals_or_none(vals)
        e = ops.sddmm(S, H, H, v, use_default_vals=False)
        Y = ops.spmm(S, H, e, use_default_vals=False)
        ctx.S = S
        ctx.save_for_backward(vals, H, e)
        return Y

    @staticmethod
    def backward(ctx, dY):
        vals, H, e = ctx.saved_tensors
        S = ctx.S
        dY = dY.contiguous().float()
        v = _vals_or_none(vals)
        dE = ops.sddmm(S, dY, H, use_default_vals=False)
        acc = ops.spmm(S, H, v, dE, use_default_vals=False)
        ops.spmm_t(S, H, v, dE, out=acc, accumulate=True, use_default_vals=False)
        ops.spmm_t(S, dY, e, out=acc, accumulate=True, use_default_vals=False)
        dH = acc if H.dtype == torch.float32 else ops.cast(acc, H.dtype)
        return None, None, dH


def gnn_layer(S: CSR, H, vals=None):
    if vals is None:
        vals = torch.empty(0, dtype=torch.float32, device=S.device)
    return GNNLayerFunction.apply(S, vals, H)


__all__ = ["SDDMMFunction", "SpMMFunction", "GNNLayerFunction", "sddmm", "spmm", "gnn_layer"]
