"""The compute entry points: SDDMM (Eq. 1), SpMM (Eq. 2), SpMM^T, and the
precision kernels, as thin wrappers over libspk (argument marshalling only;
every step runs in the library's CUDA kernels)."""
from __future__ import annotations

import ctypes

import torch

from .binding import SPK_BF16, SPK_E4M3, SPK_F16, SPK_F32, Tune, check, lib
from .sparse import CSR, TensorCorePlan, TransposePlan, _stream

_DT = {torch.float32: SPK_F32, torch.bfloat16: SPK_BF16, torch.float16: SPK_F16,
       torch.float8_e4m3fn: SPK_E4M3, torch.uint8: SPK_E4M3}
_OUT_DT = {torch.float32: SPK_F32, torch.bfloat16: SPK_BF16, torch.float16: SPK_F16}


def _dense(X: torch.Tensor, name: str, device) -> tuple[int, int]:
    if X.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    if X.device != device:
        raise ValueError(f"{name} is on {X.device}, the pattern on {device}")
    if X.dtype not in _DT:
        raise TypeError(f"{name}: unsupported dtype {X.dtype}")
    if X.stride(1) != 1 and X.size(1) > 1:
        raise ValueError(f"{name} must be row-major with unit column stride")
    ld = X.stride(0) if X.size(0) > 1 else max(X.size(1), 1)
    return _DT[X.dtype], ld


def _vals(v, S, name):
    if v is None:
        return None
    if v.dtype != torch.float32 or v.device != S.device or v.numel() != S.nnz:
        raise ValueError(f"{name} must be a float32 tensor of length nnz on the pattern's device")
    return v.contiguous()


def _ptr(t):
    return None if t is None else t.data_ptr()


def _tune(t):
    t = Tune.make(t)
    return None if t is None else ctypes.byref(t)


def _scale(s, n, name, device):
    if s is None:
        return None
    if s.dtype != torch.float32 or s.numel() != n or s.device != device:
        raise ValueError(f"{name} must be float32 with one entry per row")
    return s.contiguous()


def sddmm(S: CSR, A: torch.Tensor, B: torch.Tensor, vals=None, vals2=None, *, a_scale=None, b_scale=None,
          out: torch.Tensor | None = None, tune=None, use_default_vals: bool = True) -> torch.Tensor:
    """out_e = s_e * <A[i,:], B[j,:]> for every stored e = (i, j).  FP32, length nnz."""
    if vals is None and use_default_vals:
        vals = S.vals
    dta, lda = _dense(A, "A", S.device)
    dtb, ldb = _dense(B, "B", S.device)
    if A.size(0) != S.M or B.size(0) != S.N or A.size(1) != B.size(1):
        raise ValueError(f"shapes: S {S.M}x{S.N}, A {tuple(A.shape)}, B {tuple(B.shape)}")
    K = A.size(1)
    if out is None:
        out = torch.empty(S.nnz, dtype=torch.float32, device=S.device)
    vals, vals2 = _vals(vals, S, "vals"), _vals(vals2, S, "vals2")
    a_scale = _scale(a_scale, S.M, "a_scale", S.device)
    b_scale = _scale(b_scale, S.N, "b_scale", S.device)
    check(lib().spk_sddmm(S.handle, _ptr(vals), _ptr(vals2), dta, A.data_ptr(), lda, _ptr(a_scale), dtb,
                          B.data_ptr(), ldb, _ptr(b_scale), K, out.data_ptr(), _tune(tune), _stream(S.device)),
          "spk_sddmm")
    return out


def sddmm_mh(S: CSR, A: torch.Tensor, B: torch.Tensor, heads: int, vals=None, *,
             out: torch.Tensor | None = None) -> torch.Tensor:
    """Per head h (equal slices of K): out[h, e] = s_e * <A[i, head h], B[j, head h]>,
    heads x nnz FP32, one pass over the pattern for all heads (vals None: ones).
    Raises SpkError where no multi-head kernel covers K (use sddmm per slice)."""
    dta, lda = _dense(A, "A", S.device)
    dtb, ldb = _dense(B, "B", S.device)
    if dta != dtb:
        raise TypeError("A and B must have the same dtype")
    if A.size(0) != S.M or B.size(0) != S.N or A.size(1) != B.size(1):
        raise ValueError("A must be M x K and B N x K")
    K = A.size(1)
    if out is None:
        out = torch.empty((heads, S.nnz), dtype=torch.float32, device=S.device)
    if out.dtype != torch.float32 or tuple(out.shape) != (heads, S.nnz) or not out.is_contiguous():
        raise ValueError("out must be a contiguous heads x nnz float32 tensor")
    vals = _vals(vals, S, "vals")
    check(lib().spk_sddmm_mh(S.handle, _ptr(vals), int(heads), dta, A.data_ptr(), lda, B.data_ptr(), ldb, K,
                             out.data_ptr(), _stream(S.device)), "spk_sddmm_mh")
    return out


def spmm(S: CSR, B: torch.Tensor, vals=None, vals2=None, *, b_scale=None, out: torch.Tensor | None = None,
         out_dtype=torch.float32, accumulate: bool = False, tune=None, use_default_vals: bool = True) -> torch.Tensor:
    """C = S B (or C += S B with accumulate=True).  C is M x K."""
    if vals is None and use_default_vals:
        vals = S.vals
    dtb, ldb = _dense(B, "B", S.device)
    if B.size(0) != S.N:
        raise ValueError(f"B has {B.size(0)} rows, S has {S.N} columns")
    K = B.size(1)
    if out is None:
        if accumulate:
            raise ValueError("accumulate needs an output tensor")
        out = torch.empty((S.M, K), dtype=out_dtype, device=S.device)
    dtc, ldc = _dense(out, "out", S.device)
    if out.dtype not in _OUT_DT or out.shape != (S.M, K):
        raise ValueError("out must be M x K in float32, bfloat16 or float16")
    vals, vals2 = _vals(vals, S, "vals"), _vals(vals2, S, "vals2")
    b_scale = _scale(b_scale, S.N, "b_scale", S.device)
    t = Tune.make(tune)
    ws = S.workspace(K) if (S.has_schedule and (t is None or t.variant != 1)) else None
    check(lib().spk_spmm(S.handle, _ptr(vals), _ptr(vals2), dtb, B.data_ptr(), ldb, _ptr(b_scale), K, dtc,
                         out.data_ptr(), ldc, int(accumulate), _ptr(ws), 0 if ws is None else ws.numel(),
                         None if t is None else ctypes.byref(t), _stream(S.device)), "spk_spmm")
    return out


def spmm_t(S: CSR, Y: torch.Tensor, vals=None, vals2=None, *, y_scale=None, out: torch.Tensor | None = None,
           out_dtype=torch.float32, accumulate: bool = False, tune=None, plan: TransposePlan | None = None,
           use_default_vals: bool = True) -> torch.Tensor:
    """X = S^T Y (N x K) through the transpose plan of S (built on first use)."""
    if vals is None and use_default_vals:
        vals = S.vals
    P = plan or S.transpose_plan()
    dty, ldy = _dense(Y, "Y", S.device)
    if Y.size(0) != S.M:
        raise ValueError(f"Y has {Y.size(0)} rows, S has {S.M} rows")
    K = Y.size(1)
    if out is None:
        if accumulate:
            raise ValueError("accumulate needs an output tensor")
        out = torch.empty((S.N, K), dtype=out_dtype, device=S.device)
    dtx, ldx = _dense(out, "out", S.device)
    if out.dtype not in _OUT_DT or out.shape != (S.N, K):
        raise ValueError("out must be N x K in float32, bfloat16 or float16")
    vals, vals2 = _vals(vals, S, "vals"), _vals(vals2, S, "vals2")
    y_scale = _scale(y_scale, S.M, "y_scale", S.device)
    t = Tune.make(tune)
    ws = P.workspace(K)
    check(lib().spk_spmm_t(P.handle, _ptr(vals), _ptr(vals2), dty, Y.data_ptr(), ldy, _ptr(y_scale), K, dtx,
                           out.data_ptr(), ldx, int(accumulate), _ptr(ws), 0 if ws is None else ws.numel(),
                           None if t is None else ctypes.byref(t), _stream(S.device)), "spk_spmm_t")
    return out


def _head_vals(vals: torch.Tensor, S: CSR, heads: int) -> torch.Tensor:
    if vals.dtype != torch.float32 or vals.device != S.device or vals.dim() != 2 or vals.shape != (heads, S.nnz) \
            or vals.stride(1) != 1:
        raise ValueError("vals must be float32, heads x nnz, rows contiguous, on the pattern's device")
    return vals


def spmm_mh(S: CSR, B: torch.Tensor, vals: torch.Tensor, heads: int, *, out: torch.Tensor | None = None,
            accumulate: bool = False) -> torch.Tensor:
    """C[:, head h] = S_h B[:, head h] with the values of head h in vals[h]
    (heads x nnz): one pass over the pattern for all heads.  FP32 output."""
    dtb, ldb = _dense(B, "B", S.device)
    if B.size(0) != S.N:
        raise ValueError(f"B has {B.size(0)} rows, S has {S.N} columns")
    K = B.size(1)
    vals = _head_vals(vals, S, heads)
    if out is None:
        if accumulate:
            raise ValueError("accumulate needs an output tensor")
        out = torch.empty((S.M, K), dtype=torch.float32, device=S.device)
    _, ldc = _dense(out, "out", S.device)
    if out.dtype != torch.float32 or out.shape != (S.M, K):
        raise ValueError("out must be M x K float32")
    ws = S.workspace(K) if S.has_schedule else None
    check(lib().spk_spmm_mh(S.handle, vals.data_ptr(), vals.stride(0), int(heads), dtb, B.data_ptr(), ldb, K,
                            out.data_ptr(), ldc, int(accumulate), _ptr(ws), 0 if ws is None else ws.numel(),
                            _stream(S.device)), "spk_spmm_mh")
    return out


def spmm_t_mh(S: CSR, Y: torch.Tensor, vals: torch.Tensor, heads: int, *, out: torch.Tensor | None = None,
              accumulate: bool = False, plan: TransposePlan | None = None) -> torch.Tensor:
    """X[:, head h] = S_h^T Y[:, head h] with the values of head h in vals[h]
    (heads x nnz), through the transpose plan.  FP32 output."""
    P = plan or S.transpose_plan()
    dty, ldy = _dense(Y, "Y", S.device)
    if Y.size(0) != S.M:
        raise ValueError(f"Y has {Y.size(0)} rows, S has {S.M} rows")
    K = Y.size(1)
    vals = _head_vals(vals, S, heads)
    if out is None:
        if accumulate:
            raise ValueError("accumulate needs an output tensor")
        out = torch.empty((S.N, K), dtype=torch.float32, device=S.device)
    _, ldx = _dense(out, "out", S.device)
    if out.dtype != torch.float32 or out.shape != (S.N, K):
        raise ValueError("out must be N x K float32")
    n = ctypes.c_size_t()
    check(lib().spk_spmm_t_mh_workspace_size(P.handle, K, int(heads), ctypes.byref(n)), "spk_spmm_t_mh_workspace_size")
    ws = P.mh_workspace(n.value)
    check(lib().spk_spmm_t_mh(P.handle, vals.data_ptr(), vals.stride(0), int(heads), dty, Y.data_ptr(), ldy, K,
                              out.data_ptr(), ldx, int(accumulate), ws.data_ptr(), ws.numel(), _stream(S.device)),
          "spk_spmm_t_mh")
    return out


def fusedmm(S: CSR, A: torch.Tensor, B: torch.Tensor, vals=None, *, heads: int = 1, scale: float = 1.0,
            softmax: bool = False, want_scores: bool = False, want_lse: bool = False,
            out: torch.Tensor | None = None, tune=None, use_default_vals: bool = True):
    """FusedMM: SDDMM cascaded into SpMM on B, per head of ``heads`` equal
    slices of K, optionally with row-softmax weights:
    Y[i, h] = sum_j w_h(i, j) B[j, h],  w = scale * s * <A_i, B_j>  (or its
    row softmax).  Returns (Y, scores or None, lse or None); scores is
    heads x nnz, lse is M x heads (softmax only)."""
    if vals is None and use_default_vals:
        vals = S.vals
    dta, lda = _dense(A, "A", S.device)
    dtb, ldb = _dense(B, "B", S.device)
    if dta != dtb:
        raise TypeError("A and B must have the same dtype")
    if A.size(0) != S.M or B.size(0) != S.N or A.size(1) != B.size(1):
        raise ValueError("A must be M x K and B N x K")
    K = A.size(1)
    if out is None:
        out = torch.empty((S.M, K), dtype=torch.float32, device=S.device)
    if out.dtype != torch.float32 or out.shape != (S.M, K):
        raise ValueError("out must be M x K float32")
    _, ldy = _dense(out, "out", S.device)
    vals = _vals(vals, S, "vals")
    scores = torch.empty((heads, S.nnz), dtype=torch.float32, device=S.device) if want_scores else None
    lse = torch.empty((S.M, heads), dtype=torch.float32, device=S.device) if (want_lse and softmax) else None
    ws = S.fused_workspace(K, heads)
    check(lib().spk_fusedmm(S.handle, _ptr(vals), float(scale), int(bool(softmax)), dta, A.data_ptr(), lda,
                            B.data_ptr(), ldb, K, int(heads), out.data_ptr(), ldy, _ptr(scores), _ptr(lse),
                            _ptr(ws), 0 if ws is None else ws.numel(), _tune(tune), _stream(S.device)), "spk_fusedmm")
    return out, scores, lse


def _f32(t, shape, name, device):
    """A float32 tensor of the given shape on the pattern's device, or raise
    (no host pointer ever reaches a kernel)."""
    if t is None or t.dtype != torch.float32 or tuple(t.shape) != tuple(shape) or t.device != device:
        raise ValueError(f"{name} must be a float32 tensor of shape {tuple(shape)} on {device}")
    return t.contiguous()


def fused_weights(S: CSR, scores: torch.Tensor, lse, heads: int, softmax: bool) -> torch.Tensor:
    """Per-entry weights of a FusedMM forward: the scores, or exp(score - lse[row])
    with softmax.  heads x nnz FP32."""
    scores = _f32(scores, (heads, S.nnz), "scores", S.device)
    lse = _f32(lse, (S.M, heads), "lse", S.device) if softmax else None
    w = torch.empty_like(scores)
    check(lib().spk_fused_weights(S.handle, int(heads), int(bool(softmax)), scores.data_ptr(), _ptr(lse),
                                  w.data_ptr(), _stream(S.device)), "spk_fused_weights")
    return w


def fused_rowdot(dY: torch.Tensor, Y: torch.Tensor, heads: int) -> torch.Tensor:
    """rowdot[i, h] = <dY_i, Y_i> over head h's columns.  M x heads FP32."""
    if dY.dtype != torch.float32 or Y.dtype != torch.float32 or dY.shape != Y.shape or dY.dim() != 2:
        raise ValueError("dY and Y must be M x K float32 of one shape")
    if not dY.is_cuda or Y.device != dY.device:
        raise ValueError("dY and Y must be CUDA tensors on one device")
    _, lddy = _dense(dY, "dY", dY.device)
    _, ldy = _dense(Y, "Y", dY.device)
    M, K = Y.shape
    R = torch.empty((M, heads), dtype=torch.float32, device=Y.device)
    check(lib().spk_fused_rowdot(M, K, int(heads), dY.data_ptr(), lddy, Y.data_ptr(), ldy, R.data_ptr(),
                                 _stream(Y.device)), "spk_fused_rowdot")
    return R


def fused_score_grad(S: CSR, w: torch.Tensor, dw: torch.Tensor, rowdot, heads: int, softmax: bool,
                     scale: float, vals=None) -> torch.Tensor:
    """Gradient w.r.t. the unscaled dot products <A_i, B_j>: scale * s * dw, or
    scale * s * w * (dw - rowdot[row]) with softmax (s = vals, None = ones).
    heads x nnz FP32."""
    dw = _f32(dw, (heads, S.nnz), "dw", S.device)
    w = _f32(w, (heads, S.nnz), "w", S.device) if softmax else None
    rowdot = _f32(rowdot, (S.M, heads), "rowdot", S.device) if softmax else None
    vals = _vals(vals, S, "vals")
    de = torch.empty_like(dw)
    check(lib().spk_fused_score_grad(S.handle, int(heads), int(bool(softmax)), float(scale), _ptr(vals), _ptr(w),
                                     dw.data_ptr(), _ptr(rowdot), de.data_ptr(), _stream(S.device)),
          "spk_fused_score_grad")
    return de


def cast(x: torch.Tensor, dtype) -> torch.Tensor:
    """Round-to-nearest-even cast of an FP32 tensor to bfloat16 / float16."""
    if x.dtype != torch.float32 or not x.is_cuda:
        raise TypeError("cast expects a float32 CUDA tensor")
    if dtype not in (torch.bfloat16, torch.float16):
        raise TypeError("cast target must be bfloat16 or float16")
    x = x.contiguous()
    out = torch.empty(x.shape, dtype=dtype, device=x.device)
    check(lib().spk_cast(x.data_ptr(), x.numel(), _DT[dtype], out.data_ptr(), _stream(x.device)), "spk_cast")
    return out


def quantize_e4m3_rows(X: torch.Tensor):
    """Per-row E4M3 codes (torch.float8_e4m3fn) and FP32 scales (amax/448)."""
    if X.dtype != torch.float32 or X.dim() != 2 or not X.is_cuda:
        raise TypeError("quantize_e4m3_rows expects a 2-D float32 CUDA tensor")
    X = X.contiguous()
    M, K = X.shape
    Q = torch.empty((M, K), dtype=torch.float8_e4m3fn, device=X.device)
    scales = torch.empty(M, dtype=torch.float32, device=X.device)
    check(lib().spk_quantize_e4m3_rows(X.data_ptr(), M, K, K, Q.data_ptr(), K, scales.data_ptr(),
                                       _stream(X.device)), "spk_quantize_e4m3_rows")
    return Q, scales


__all__ = ["sddmm", "spmm", "spmm_t", "fusedmm", "fused_weights", "fused_rowdot", "fused_score_grad", "cast",
           "quantize_e4m3_rows"]


def tc_sddmm(P: TensorCorePlan, A: torch.Tensor, B: torch.Tensor, vals=None, *, out: torch.Tensor | None = None,
             tune=None, use_default_vals: bool = True) -> torch.Tensor:
    """SDDMM (Eq. 1) with the plan's dense tiles on the tensor cores and the
    remaining entries on the gather kernels.  A, B BF16."""
    S = P.S
    if vals is None and use_default_vals:
        vals = S.vals
    dta, lda = _dense(A, "A", S.device)
    dtb, ldb = _dense(B, "B", S.device)
    if A.size(0) != S.M or B.size(0) != S.N or A.size(1) != B.size(1):
        raise ValueError(f"shapes: S {S.M}x{S.N}, A {tuple(A.shape)}, B {tuple(B.shape)}")
    if dta != dtb:
        raise TypeError("A and B must have the same dtype")
    if out is None:
        out = torch.empty(S.nnz, dtype=torch.float32, device=S.device)
    vals = _vals(vals, S, "vals")
    ws = P.workspace()
    check(lib().spk_tc_sddmm(P.handle, _ptr(vals), dta, A.data_ptr(), lda, B.data_ptr(), ldb, A.size(1),
                             out.data_ptr(), _ptr(ws), 0 if ws is None else ws.numel(), _tune(tune),
                             _stream(S.device)), "spk_tc_sddmm")
    return out
