"""FP64 CPU oracle for SDDMM / SpMM (Sec. 3.2, Eq. 1 and Eq. 2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_2404_19638_gb300``) never imports it, and this package
never imports the product path: the two share no code.

The arithmetic lives in ``oracle.c`` (plain loops, double accumulation).  This
wrapper only marshals numpy arrays and composes the primitives into the
gradients of Sec. 3.2's adjoint pair, written out from their closed forms.

Dense operands are passed as numpy arrays whose dtype names the format:
float32 -> FP32, float64 -> FP64, ``uint16`` + ``fmt='bf16'|'f16'`` -> 16-bit
patterns, ``uint8`` -> E4M3 codes (with optional per-row float32 scales).
Sparse values are taken in float64 (float32 inputs convert exactly).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FMT = {"f32": 0, "bf16": 1, "f16": 2, "e4m3": 3, "f64": 4}

_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.oracle_decode_bf16.restype = ctypes.c_double
            L.oracle_decode_f16.restype = ctypes.c_double
            L.oracle_decode_e4m3.restype = ctypes.c_double
            for f in (L.oracle_decode_bf16, L.oracle_decode_f16, L.oracle_decode_e4m3):
                f.argtypes = [ctypes.c_uint32]
            for f in (L.oracle_encode_bf16, L.oracle_encode_f16, L.oracle_encode_e4m3):
                f.restype = ctypes.c_uint32
                f.argtypes = [ctypes.c_float]
            L.oracle_encode_array.argtypes = [ctypes.c_int, _i64, _p, _p]
            L.oracle_quantize_e4m3_rows.argtypes = [_i64, _i64, _p, _i64, _p, _i64, _p]
            L.oracle_sddmm.argtypes = [_i64, _i64, _i64, _p, _p, _p, _p, ctypes.c_int,
                                       ctypes.c_int, _p, _i64, _p, ctypes.c_int, _p, _i64, _p,
                                       _i64, _p, _p]
            L.oracle_spmm.argtypes = [_i64, _i64, _i64, _p, _p, _p, _p, ctypes.c_int,
                                      ctypes.c_int, _p, _i64, _p, _i64, _p, _p]
            L.oracle_spmm_t.argtypes = [_i64, _i64, _i64, _p, _p, _p, _p, ctypes.c_int,
                                        ctypes.c_int, _p, _i64, _p, _i64, _p, _p]
            L.oracle_fusedmm.argtypes = [_i64, _i64, _i64, _i64, _p, _p, _p, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, _p, _i64, ctypes.c_int, _p, _i64,
                                         _i64, _p, _p, _p, _p]
            L.oracle_transpose.argtypes = [_i64, _i64, _p, _p, _p, _p, _p]
            L.oracle_merge_path.argtypes = [_i64, _p, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
            L.oracle_rcm.argtypes = [_i64, _p, _p, _p]
            L.oracle_coo_to_csr.argtypes = [_i64, _i64, _i64, _p, _p, _p, ctypes.c_int, _p, _p, _p,
                                            ctypes.POINTER(_i64)]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def _dense(X, fmt):
    """Contiguous operand + format code; 2-D with leading dimension = row length."""
    if fmt is None:
        fmt = {np.dtype(np.float32): "f32", np.dtype(np.uint8): "e4m3",
               np.dtype(np.float64): "f64"}.get(X.dtype)
        if fmt is None:
            raise ValueError("16-bit operands need fmt='bf16' or 'f16'")
    want = {"f32": np.float32, "bf16": np.uint16, "f16": np.uint16, "e4m3": np.uint8,
            "f64": np.float64}[fmt]
    X = np.ascontiguousarray(X, dtype=want)
    if X.ndim != 2:
        raise ValueError("dense operand must be 2-D")
    return X, FMT[fmt]


def _rows(rows):
    return None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)


# ----------------------------------------------------------------------------
# Formats
# ----------------------------------------------------------------------------

_LUT: dict = {}


def decode_table(fmt: str) -> np.ndarray:
    """Value of every code of a format, from the C decoder (cached)."""
    if fmt not in _LUT:
        f = {"bf16": lib().oracle_decode_bf16, "f16": lib().oracle_decode_f16,
             "e4m3": lib().oracle_decode_e4m3}[fmt]
        n = 256 if fmt == "e4m3" else 65536
        _LUT[fmt] = np.array([f(c) for c in range(n)], dtype=np.float64)
    return _LUT[fmt]


def decode(codes, fmt: str) -> np.ndarray:
    return decode_table(fmt)[np.asarray(codes).astype(np.int64)]


def encode(x, fmt: str) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint8 if fmt == "e4m3" else np.uint16)
    lib().oracle_encode_array(FMT[fmt], x.size, _ptr(x), _ptr(out))
    return out


def quantize_e4m3_rows(X):
    """Per-row E4M3 codes and scales (scale = amax/448, 1 for an all-zero row)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    M, K = X.shape
    codes = np.empty((M, K), dtype=np.uint8)
    scales = np.empty(M, dtype=np.float32)
    lib().oracle_quantize_e4m3_rows(M, K, _ptr(X), K, _ptr(codes), K, _ptr(scales))
    return codes, scales


def dequantize(X, fmt: str | None = None, scale=None) -> np.ndarray:
    """Dense operand -> float64 values (what the oracle multiplies)."""
    X, code = _dense(X, fmt)
    if code in (0, 4):
        out = X.astype(np.float64)
    else:
        name = [k for k, v in FMT.items() if v == code][0]
        out = decode(X, name)
    if scale is not None:
        out = out * np.asarray(scale, dtype=np.float64)[:, None]
    return out


# ----------------------------------------------------------------------------
# Kernels
# ----------------------------------------------------------------------------

def sddmm(rowptr, colidx, A, B, vals=None, vals2=None, rows=None, *, fmt_a=None, fmt_b=None,
          a_scale=None, b_scale=None, absmode=False, N=None) -> np.ndarray:
    """Eq. 1.  Returns a float64 array of length nnz; entries of rows not listed
    in ``rows`` are NaN."""
    rowptr = _c(rowptr, np.int32); colidx = _c(colidx, np.int32)
    A, fa = _dense(A, fmt_a); B, fb = _dense(B, fmt_b)
    M, K = A.shape[0], A.shape[1]
    if B.shape[1] != K:
        raise ValueError("A and B must have the same number of columns")
    N = B.shape[0] if N is None else N
    out = np.full(colidx.size, np.nan)
    rows = _rows(rows)
    rc = lib().oracle_sddmm(M, N, K, _ptr(rowptr), _ptr(colidx), _ptr(_c(vals, np.float64)),
                            _ptr(_c(vals2, np.float64)), int(absmode), fa, _ptr(A), K,
                            _ptr(_c(a_scale, np.float32)), fb, _ptr(B), K, _ptr(_c(b_scale, np.float32)),
                            0 if rows is None else rows.size, _ptr(rows), _ptr(out))
    if rc:
        raise ValueError(f"oracle_sddmm: bad input ({rc})")
    return out


def spmm(rowptr, colidx, B, vals=None, vals2=None, rows=None, *, fmt_b=None, b_scale=None,
         absmode=False) -> np.ndarray:
    """Eq. 2.  Returns float64 (len(rows) or M) x K."""
    rowptr = _c(rowptr, np.int32); colidx = _c(colidx, np.int32)
    B, fb = _dense(B, fmt_b)
    M = rowptr.size - 1
    N, K = B.shape
    rows = _rows(rows)
    out = np.empty((M if rows is None else rows.size, K))
    rc = lib().oracle_spmm(M, N, K, _ptr(rowptr), _ptr(colidx), _ptr(_c(vals, np.float64)),
                           _ptr(_c(vals2, np.float64)), int(absmode), fb, _ptr(B), K,
                           _ptr(_c(b_scale, np.float32)), 0 if rows is None else rows.size,
                           _ptr(rows), _ptr(out))
    if rc:
        raise ValueError(f"oracle_spmm: bad input ({rc})")
    return out


def spmm_t(rowptr, colidx, N, Y, vals=None, vals2=None, cols=None, *, fmt_y=None, y_scale=None,
           absmode=False) -> np.ndarray:
    """S^T Y.  Returns float64 (len(cols) or N) x K."""
    rowptr = _c(rowptr, np.int32); colidx = _c(colidx, np.int32)
    Y, fy = _dense(Y, fmt_y)
    M, K = Y.shape
    if rowptr.size - 1 != M:
        raise ValueError("Y must have M rows")
    cols = _rows(cols)
    out = np.empty((N if cols is None else cols.size, K))
    rc = lib().oracle_spmm_t(M, N, K, _ptr(rowptr), _ptr(colidx), _ptr(_c(vals, np.float64)),
                             _ptr(_c(vals2, np.float64)), int(absmode), fy, _ptr(Y), K,
                             _ptr(_c(y_scale, np.float32)), 0 if cols is None else cols.size,
                             _ptr(cols), _ptr(out))
    if rc:
        raise ValueError(f"oracle_spmm_t: bad input ({rc})")
    return out


def fusedmm(rowptr, colidx, A, B, vals=None, *, heads=1, scale=1.0, softmax=False, rows=None, fmt_a=None,
            fmt_b=None, absmode=False, N=None):
    """SDDMM cascaded into SpMM (Sec. 2), per head, optional row softmax.
    Returns (Y float64 (len(rows) or M) x K, scores float64 heads x nnz (NaN
    outside the rows computed), lse float64 (len(rows) or M) x heads)."""
    rowptr = _c(rowptr, np.int32); colidx = _c(colidx, np.int32)
    A, fa = _dense(A, fmt_a); B, fb = _dense(B, fmt_b)
    M, K = A.shape
    if B.shape[1] != K:
        raise ValueError("A and B must have the same number of columns")
    N = B.shape[0] if N is None else N
    rows = _rows(rows)
    count = M if rows is None else rows.size
    Y = np.empty((count, K))
    scores = np.full((heads, colidx.size), np.nan)
    lse = np.empty((count, heads))
    rc = lib().oracle_fusedmm(M, N, K, int(heads), _ptr(rowptr), _ptr(colidx), _ptr(_c(vals, np.float64)),
                              float(scale), int(bool(softmax)), int(absmode), fa, _ptr(A), K, fb, _ptr(B), K,
                              0 if rows is None else rows.size, _ptr(rows), _ptr(Y), _ptr(scores), _ptr(lse))
    if rc:
        raise ValueError(f"oracle_fusedmm: bad input ({rc})")
    return Y, scores, lse


def transpose(rowptr, colidx, N):
    """Stable CSR -> CSC: (colptr, rowidx, perm)."""
    rowptr = _c(rowptr, np.int32); colidx = _c(colidx, np.int32)
    M = rowptr.size - 1
    colptr = np.empty(N + 1, np.int32)
    rowidx = np.empty(colidx.size, np.int32)
    perm = np.empty(colidx.size, np.int32)
    rc = lib().oracle_transpose(M, N, _ptr(rowptr), _ptr(colidx), _ptr(colptr), _ptr(rowidx), _ptr(perm))
    if rc:
        raise ValueError(f"oracle_transpose: bad input ({rc})")
    return colptr, rowidx, perm


def coo_to_csr(rows, cols, M: int, N: int, vals=None, dedup: int = 1):
    """COO -> CSR ordered by (row, column), ties in input order; dedup 0 keeps
    every entry, 1 the first of each repeated (row, column), 2 one entry with
    the repeats' values summed.  Returns (rowptr, colidx, vals float64 or
    None)."""
    rows = _c(rows, np.int32); cols = _c(cols, np.int32)
    nnz = rows.size
    rowptr = np.empty(M + 1, np.int32)
    colidx = np.empty(nnz, np.int32)
    out_v = np.empty(nnz) if vals is not None else None
    n = _i64(0)
    rc = lib().oracle_coo_to_csr(M, N, nnz, _ptr(rows), _ptr(cols), _ptr(_c(vals, np.float64)), int(dedup),
                                 _ptr(rowptr), _ptr(colidx), _ptr(out_v), ctypes.byref(n))
    if rc:
        raise ValueError(f"oracle_coo_to_csr: bad input ({rc})")
    k = n.value
    return rowptr, colidx[:k].copy(), None if out_v is None else out_v[:k].copy()


def rcm(rowptr, colidx):
    """Reverse Cuthill-McKee order of a square pattern: perm[p] = the row placed
    at position p (ties by (degree, index), components from the unvisited
    vertex of smallest (degree, index))."""
    rowptr = _c(rowptr, np.int32); colidx = _c(colidx, np.int32)
    M = rowptr.size - 1
    perm = np.empty(M, np.int32)
    rc = lib().oracle_rcm(M, _ptr(rowptr), _ptr(colidx), _ptr(perm))
    if rc:
        raise ValueError(f"oracle_rcm: bad input ({rc})")
    return perm


def row_order(rowptr, colidx, N: int, kind: str):
    """Row relabelling by a stable sort: "degree" (most nonzeros first) or
    "leading" (smallest column first; rows without entries last).  Ties keep
    the original order.  perm[p] = the row placed at position p."""
    rowptr = np.asarray(rowptr, np.int64)
    deg = np.diff(rowptr)
    M = deg.size
    if kind == "degree":
        key = -deg
    elif kind == "leading":
        key = np.full(M, N, np.int64)
        for i in range(M):
            if deg[i]:
                key[i] = int(np.min(np.asarray(colidx)[rowptr[i]:rowptr[i + 1]]))
    else:
        raise ValueError(kind)
    return np.argsort(key, kind="stable").astype(np.int32)


def merge_path(rowptr, d: int):
    """(rows finished, nonzeros consumed) after d steps of the merge path."""
    rowptr = _c(rowptr, np.int32)
    r, e = _i64(0), _i64(0)
    lib().oracle_merge_path(rowptr.size - 1, _ptr(rowptr), int(d), ctypes.byref(r), ctypes.byref(e))
    return r.value, e.value


# ----------------------------------------------------------------------------
# Gradients of the adjoint pair (Sec. 3.2), closed forms over the primitives
# ----------------------------------------------------------------------------

def sddmm_grads(rowptr, colidx, A, B, vals, G, **fmt):
    """L = sum_e G_e * SDDMM(S,A,B)_e.
    dA = (S.G) B,  dB = (S.G)^T A,  ds_e = G_e <a_i, b_j>."""
    N = B.shape[0]
    dA = spmm(rowptr, colidx, B, vals, G, fmt_b=fmt.get("fmt_b"))
    dB = spmm_t(rowptr, colidx, N, A, vals, G, fmt_y=fmt.get("fmt_a"))
    ds = sddmm(rowptr, colidx, A, B, G, None, fmt_a=fmt.get("fmt_a"), fmt_b=fmt.get("fmt_b"))
    return dA, dB, ds


def spmm_grads(rowptr, colidx, B, vals, dY, **fmt):
    """L = sum G.SpMM(S,B) with G = dY.  dB = S^T dY,  ds_e = <dY_i, b_j>."""
    N = B.shape[0]
    dB = spmm_t(rowptr, colidx, N, dY, vals)
    ds = sddmm(rowptr, colidx, dY, B, None, None, fmt_b=fmt.get("fmt_b"))
    return dB, ds


def gnn_forward(rowptr, colidx, H, vals=None, fmt=None):
    """e = SDDMM(S, H, H); Y = SpMM(S_e, H) with the values of S_e = e."""
    e = sddmm(rowptr, colidx, H, H, vals, None, fmt_a=fmt, fmt_b=fmt)
    Y = spmm(rowptr, colidx, H, e, None, fmt_b=fmt)
    return e, Y


def gnn_grad(rowptr, colidx, H, dY, vals=None, fmt=None):
    """dH of L = sum dY . Y for the layer above:
    dE_e = <dY_i, h_j>;  dH = (S.dE) H + (S.dE)^T H + S_e^T dY."""
    N = H.shape[0]
    e = sddmm(rowptr, colidx, H, H, vals, None, fmt_a=fmt, fmt_b=fmt)
    dE = sddmm(rowptr, colidx, dY, H, None, None, fmt_b=fmt)
    g1 = spmm(rowptr, colidx, H, vals, dE, fmt_b=fmt)
    g2 = spmm_t(rowptr, colidx, N, H, vals, dE, fmt_y=fmt)
    g3 = spmm_t(rowptr, colidx, N, dY, e)
    return g1 + g2 + g3


def fusedmm_grad(rowptr, colidx, A, B, dY, vals=None, *, heads=1, scale=1.0, softmax=False, fmt=None,
                 absmode=False):
    """dA, dB of L = sum dY . Y for Y = fusedmm(S, A, B) (Sec. 2's SDDMM -> SpMM
    cascade), by the chain rule per head h over columns h*K/heads.. :
      e = scale s <a_i, b_j>,  w = e or softmax_j(e),  Y_i = sum_j w_ij b_j
      dw_ij = <dY_i, b_j>;  g = dw, or w (dw - sum_j' w_ij' dw_ij') with softmax
      c = scale g;  dA = (S.c) B;  dB = (S.c)^T A + W^T dY.
    The weights come from this oracle's own FusedMM forward (scores, lse).

    absmode=True returns the denominators of the componentwise error metric
    instead: the same chain rule over the magnitudes of every term,
      |dw|~ = sum_k |dY_ik||b_jk|,  |g|~ = |dw|~, or
      |w|~ (|dw|~ + sum_j' |w_ij'|~ |dw_ij'|~) with softmax,
      dA~ = sum_j |scale s_ij| |g_ij|~ |b_j|,
      dB~ = sum_i |scale s_ij| |g_ij|~ |a_i| + sum_i |w_ij|~ |dY_i|,
    where a softmax weight's magnitude is |w| (1 + |e|~) with
    |e|~ = |scale| sum_k |s_ij a_ik b_jk|: a weight exp(e - lse) carries the
    absolute rounding error of its exponent as a relative error.  Cancelling
    sums (softmax score gradients sum to zero over a row) thus get the
    magnitude of their terms, not of their result."""
    if absmode:
        return _fusedmm_grad_den(rowptr, colidx, A, B, dY, vals, heads=heads, scale=scale, softmax=softmax, fmt=fmt)
    rowptr = _c(rowptr, np.int32); colidx = _c(colidx, np.int32)
    M, K = A.shape
    N = B.shape[0]
    Kh = K // heads
    rows = np.repeat(np.arange(M), np.diff(rowptr))
    dY = np.asarray(dY, np.float64)
    _, scores, lse = fusedmm(rowptr, colidx, A, B, vals, heads=heads, scale=scale, softmax=softmax,
                             fmt_a=fmt, fmt_b=fmt)
    dA = np.zeros((M, K))
    dB = np.zeros((N, K))
    for h in range(heads):
        sl = slice(h * Kh, (h + 1) * Kh)
        w = np.exp(scores[h] - lse[rows, h]) if softmax else scores[h]
        dw = sddmm(rowptr, colidx, dY[:, sl], B[:, sl], None, None, fmt_b=fmt)
        if softmax:
            rowsum = np.bincount(rows, weights=w * dw, minlength=M)
            g = w * (dw - rowsum[rows])
        else:
            g = dw
        c = scale * g
        dA[:, sl] = spmm(rowptr, colidx, B[:, sl], vals, c, fmt_b=fmt)
        dB[:, sl] = spmm_t(rowptr, colidx, N, A[:, sl], vals, c, fmt_y=fmt) + spmm_t(rowptr, colidx, N, dY[:, sl], w)
    return dA, dB


def _fusedmm_grad_den(rowptr, colidx, A, B, dY, vals=None, *, heads=1, scale=1.0, softmax=False, fmt=None):
    """Componentwise denominators of fusedmm_grad (see its absmode)."""
    rowptr = _c(rowptr, np.int32); colidx = _c(colidx, np.int32)
    M, K = A.shape
    N = B.shape[0]
    Kh = K // heads
    rows = np.repeat(np.arange(M), np.diff(rowptr))
    dY = np.asarray(dY, np.float64)
    _, scores, lse = fusedmm(rowptr, colidx, A, B, vals, heads=heads, scale=scale, softmax=softmax,
                             fmt_a=fmt, fmt_b=fmt)
    dA = np.zeros((M, K))
    dB = np.zeros((N, K))
    for h in range(heads):
        sl = slice(h * Kh, (h + 1) * Kh)
        e_abs = abs(scale) * sddmm(rowptr, colidx, A[:, sl], B[:, sl], vals, None, fmt_a=fmt, fmt_b=fmt,
                                   absmode=True)
        w = np.exp(scores[h] - lse[rows, h]) * (1.0 + e_abs) if softmax else np.abs(scores[h])
        dw = sddmm(rowptr, colidx, dY[:, sl], B[:, sl], None, None, fmt_b=fmt, absmode=True)
        if softmax:
            rowsum = np.bincount(rows, weights=w * dw, minlength=M)
            g = w * (dw + rowsum[rows])
        else:
            g = dw
        c = abs(scale) * g
        dA[:, sl] = spmm(rowptr, colidx, B[:, sl], vals, c, fmt_b=fmt, absmode=True)
        dB[:, sl] = (spmm_t(rowptr, colidx, N, A[:, sl], vals, c, fmt_y=fmt, absmode=True)
                     + spmm_t(rowptr, colidx, N, dY[:, sl], w, absmode=True))
    return dA, dB
