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
from .binding import SpkError
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


def _dw_per_head(S, dY, B, dw, heads, Kh):
    for h in range(heads):
        c0 = h * Kh
        ops.sddmm(S, dY[:, c0:c0 + Kh], B[:, c0:c0 + Kh], out=dw[h], use_default_vals=False)


class FusedMMFunction(torch.autograd.Function):
    """Differentiable FusedMM: per head h, e = scale * s * <A_i, B_j>,
    w = e or its row softmax, Y_i = sum_j w_ij B_j.

    Backward (chain rule, per head; dw_ij = <dY_i, B_j>):
      g = dw, or w * (dw - rowdot_i) with softmax, rowdot_i = sum_j w_ij dw_ij
          = <dY_i, Y_i> (read from the saved output)
      c = scale * s * g;  dA = C B;  dB = C^T A + W^T dY  (C, W: S's pattern
      holding c, w)
    Steps: dw by one multi-head SDDMM (FP32 operands; one SDDMM per head
    otherwise, or where no multi-head kernel covers K), the row term and score gradient
    kernels (c folds in the sparse values, so every SpMM takes one value
    array per head), then dA = one multi-head SpMM (c per head) and
    dB = two multi-head SpMM^T (c with A, then w with dY added), each one
    pass over the pattern for all heads, in FP32.  The sparse values are not
    differentiated.
    """

    @staticmethod
    def forward(ctx, S: CSR, vals, A, B, heads: int, scale: float, softmax: bool):
        v = _vals_or_none(vals)
        Y, scores, lse = ops.fusedmm(S, A, B, v, heads=heads, scale=scale, softmax=softmax, want_scores=True,
                                     want_lse=softmax, use_default_vals=False)
        ctx.S, ctx.heads, ctx.scale, ctx.softmax = S, heads, scale, softmax
        ctx.save_for_backward(vals, A, B, Y, scores, lse if softmax else scores[:0])
        return Y

    @staticmethod
    def backward(ctx, dY):
        vals, A, B, Y, scores, lse = ctx.saved_tensors
        S, heads, scale, softmax = ctx.S, ctx.heads, ctx.scale, ctx.softmax
        dY = dY.contiguous().float()
        v = _vals_or_none(vals)
        K = A.size(1)
        Kh = K // heads
        w = ops.fused_weights(S, scores, lse, heads, softmax) if softmax else scores
        dw = torch.empty_like(scores)
        if B.dtype == torch.float32 and heads > 1:
            try:                                   # all heads in one pass over the pattern
                ops.sddmm_mh(S, dY, B, heads, out=dw)
            except SpkError as err:                # no multi-head kernel for this K: one SDDMM per head
                if err.code != "SPK_ERR_UNSUPPORTED":
                    raise
                _dw_per_head(S, dY, B, dw, heads, Kh)
        else:
            _dw_per_head(S, dY, B, dw, heads, Kh)
        R = ops.fused_rowdot(dY, Y, heads) if softmax else None
        c = ops.fused_score_grad(S, w, dw, R, heads, softmax, scale, v)
        dA = dB = None
        if ctx.needs_input_grad[2]:
            dA = ops.spmm_mh(S, B, c, heads)
            if A.dtype != torch.float32:
                dA = ops.cast(dA, A.dtype)
        if ctx.needs_input_grad[3]:
            dB = ops.spmm_t_mh(S, A, c, heads)
            ops.spmm_t_mh(S, dY, w, heads, out=dB, accumulate=True)
            if B.dtype != torch.float32:
                dB = ops.cast(dB, B.dtype)
        return None, None, dA, dB, None, None, None


def fusedmm(S: CSR, A, B, vals=None, *, heads: int = 1, scale: float = 1.0, softmax: bool = False):
    """Differentiable FusedMM (FP32 output M x K); ``vals`` None means all ones."""
    if vals is None:
        vals = torch.empty(0, dtype=torch.float32, device=S.device)
    return FusedMMFunction.apply(S, vals, A, B, int(heads), float(scale), bool(softmax))


__all__ = ["SDDMMFunction", "SpMMFunction", "GNNLayerFunction", "FusedMMFunction", "sddmm", "spmm", "gnn_layer",
           "fusedmm"]
