"""Sparse pattern handles: CSR pattern + balanced schedule + transpose plan.

PyTorch provides the device memory (the library never allocates): the
schedule, the transpose plan and SpMM carry workspaces are ``torch.uint8``
CUDA tensors owned by these objects.  All pattern-dependent setup happens
once (Sec. 5.1: the pattern is fixed while the values change).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from .binding import SpkError, check, lib

DEFAULT_CHUNK_WORK = 512


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _buffer(nbytes: int, device) -> torch.Tensor:
    # the caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _as_i32(x, device) -> torch.Tensor:
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32))
    x = x.to(device=device, dtype=torch.int32)
    return x.contiguous()


DEDUP = {"keep": 0, "first": 1, "sum": 2}


def coo_to_csr(rows, cols, shape, vals=None, *, dedup: str = "first", device="cuda"):
    """Coordinates -> CSR on the device (spk_coo_to_csr): entries ordered by
    (row, column), ties in input order; repeated (row, column) entries kept
    ("keep"), reduced to the first ("first") or summed ("sum").  Returns
    (rowptr, colidx, vals or None) as device tensors."""
    device = torch.device(device)
    if device.type == "cuda" and device.index is None:
        device = torch.device("cuda", torch.cuda.current_device())
    M, N = int(shape[0]), int(shape[1])
    r = _as_i32(rows, device)
    c = _as_i32(cols, device)
    if r.numel() != c.numel():
        raise ValueError("rows and cols must have the same length")
    n = int(r.numel())
    v = None if vals is None else torch.as_tensor(vals, dtype=torch.float32).to(device).contiguous()
    tb = ctypes.c_size_t()
    check(lib().spk_coo_to_csr_size(M, N, n, ctypes.byref(tb)), "spk_coo_to_csr_size")
    temp = _buffer(tb.value, device)
    rowptr = torch.empty(M + 1, dtype=torch.int32, device=device)
    colidx = torch.empty(max(n, 1), dtype=torch.int32, device=device)
    vout = None if v is None else torch.empty(max(n, 1), dtype=torch.float32, device=device)
    nout = ctypes.c_int64()
    with torch.cuda.device(device):
        check(lib().spk_coo_to_csr(M, N, n, r.data_ptr() if n else None, c.data_ptr() if n else None,
                                   None if v is None else v.data_ptr(), DEDUP[dedup], rowptr.data_ptr(),
                                   colidx.data_ptr(), None if vout is None else vout.data_ptr(), ctypes.byref(nout),
                                   temp.data_ptr(), temp.numel(), _stream(device)), "spk_coo_to_csr")
    k = nout.value
    return rowptr, colidx[:k].clone(), None if vout is None else vout[:k].clone()


class CSR:
    """Pattern of an M x N sparse matrix S (Sec. 3.1), optionally with values.

    ``rowptr``/``colidx`` are int32 (numpy or torch); they are moved to
    ``device`` once.  ``vals`` (FP32, length nnz, or None for all ones) is the
    default value array of calls that do not pass their own.
    """

    def __init__(self, rowptr, colidx, shape, vals=None, *, device="cuda", schedule: bool = True,
                 chunk_work: int = DEFAULT_CHUNK_WORK):
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.M, self.N = int(shape[0]), int(shape[1])
        self.rowptr = _as_i32(rowptr, self.device)
        self.colidx = _as_i32(colidx, self.device)
        if self.rowptr.numel() != self.M + 1:
            raise ValueError("rowptr must have M + 1 entries")
        self.nnz = int(self.colidx.numel())
        self.vals = None if vals is None else torch.as_tensor(vals, dtype=torch.float32).to(self.device).contiguous()
        self._h = ctypes.c_void_p()
        check(lib().spk_csr_create(ctypes.byref(self._h), self.M, self.N, self.nnz, self.rowptr.data_ptr(),
                                   self.colidx.data_ptr() if self.nnz else None), "spk_csr_create")
        self._sched = None
        self._ws = {}
        self._tplan = None
        if schedule:
            self.build_schedule(chunk_work)

    @classmethod
    def from_coo(cls, rows, cols, shape, vals=None, *, dedup: str = "first", device="cuda", **kw) -> "CSR":
        """A pattern (and values) given by coordinates, converted on the device."""
        rp, ci, v = coo_to_csr(rows, cols, shape, vals, dedup=dedup, device=device)
        return cls(rp, ci, shape, v, device=device, **kw)

    # ---------------------------------------------------------------- setup
    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def build_schedule(self, chunk_work: int = DEFAULT_CHUNK_WORK) -> None:
        nbytes = ctypes.c_size_t()
        check(lib().spk_schedule_size(self._h, int(chunk_work), ctypes.byref(nbytes)), "spk_schedule_size")
        storage = _buffer(nbytes.value, self.device)
        with torch.cuda.device(self.device):
            check(lib().spk_schedule_build(self._h, int(chunk_work), storage.data_ptr(), storage.numel(),
                                           _stream(self.device)), "spk_schedule_build")
        self._sched = storage
        self._ws.clear()

    @property
    def has_schedule(self) -> bool:
        return self._sched is not None

    def schedule_info(self) -> dict:
        nc, npc, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        check(lib().spk_schedule_info(self._h, ctypes.byref(nc), ctypes.byref(npc), ctypes.byref(w)),
              "spk_schedule_info")
        return {"nchunks": nc.value, "npieces": npc.value, "chunk_work": w.value}

    def schedule_bounds(self) -> torch.Tensor:
        """(nchunks + 1) x 2 int32 boundaries (row, nonzero) of the schedule."""
        n = self.schedule_info()["nchunks"] + 1
        out = torch.empty((n, 2), dtype=torch.int32, device=self.device)
        check(lib().spk_schedule_bounds(self._h, out.data_ptr(), _stream(self.device)), "spk_schedule_bounds")
        return out

    def merge_path_points(self, W: int, n: int) -> torch.Tensor:
        """Raw merge-path split points at diagonals 0, W, ..., n*W (clamped)."""
        out = torch.empty((n + 1, 2), dtype=torch.int32, device=self.device)
        check(lib().spk_merge_path_points(self._h, int(W), int(n), out.data_ptr(), _stream(self.device)),
              "spk_merge_path_points")
        return out

    def validate(self) -> dict:
        """Device check of the CSR invariants; synchronises."""
        rep = torch.empty(4, dtype=torch.int32, device=self.device)
        check(lib().spk_csr_validate(self._h, rep.data_ptr(), _stream(self.device)), "spk_csr_validate")
        r = rep.cpu().tolist()
        return {"error": r[0], "first_bad": r[1], "bad_count": r[2], "unsorted": bool(r[3])}

    def workspace(self, K: int) -> torch.Tensor | None:
        """Carry workspace of an SpMM with K columns (cached per K)."""
        nbytes = ctypes.c_size_t()
        check(lib().spk_spmm_workspace_size(self._h, int(K), ctypes.byref(nbytes)), "spk_spmm_workspace_size")
        if nbytes.value == 0:
            return None
        ws = self._ws.get(K)
        if ws is None or ws.numel() < nbytes.value:
            ws = _buffer(nbytes.value, self.device)
            self._ws[K] = ws
        return ws

    def fused_workspace(self, K: int, heads: int) -> torch.Tensor | None:
        """Carry workspace of a FusedMM with K columns in `heads` heads (cached)."""
        nbytes = ctypes.c_size_t()
        check(lib().spk_fusedmm_workspace_size(self._h, int(K), int(heads), ctypes.byref(nbytes)),
              "spk_fusedmm_workspace_size")
        if nbytes.value == 0:
            return None
        key = ("fused", K, heads)
        ws = self._ws.get(key)
        if ws is None or ws.numel() < nbytes.value:
            ws = _buffer(nbytes.value, self.device)
            self._ws[key] = ws
        return ws

    def transpose_plan(self, chunk_work: int | None = None) -> "TransposePlan":
        """The transpose plan of S: the attached one when ``chunk_work`` is None
        (built with the default chunk size on first use), else one of that
        chunk size (rebuilt and attached if the attached one differs)."""
        if self._tplan is None or (chunk_work is not None and self._tplan.chunk_work != chunk_work):
            self._tplan = TransposePlan(self, DEFAULT_CHUNK_WORK if chunk_work is None else chunk_work)
        return self._tplan

    def tune_default(self, op: int, dtype_code: int, K: int) -> dict:
        from .binding import Tune
        t = Tune()
        check(lib().spk_tune_default(self._h, int(op), int(dtype_code), int(K), ctypes.byref(t)), "spk_tune_default")
        return t.as_dict()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().spk_csr_destroy(h)
            except Exception:
                pass
            self._h = None

    def __repr__(self):
        return f"CSR(M={self.M}, N={self.N}, nnz={self.nnz}, schedule={self.has_schedule})"


class TransposePlan:
    """CSC of S (the CSR of S^T) with the slot permutation, built on the device."""

    def __init__(self, S: CSR, chunk_work: int = DEFAULT_CHUNK_WORK):
        self.S = S
        self.chunk_work = chunk_work
        self.M, self.N, self.nnz = S.M, S.N, S.nnz
        st, tmp = ctypes.c_size_t(), ctypes.c_size_t()
        check(lib().spk_tplan_size(S.handle, int(chunk_work), ctypes.byref(st), ctypes.byref(tmp)), "spk_tplan_size")
        self._storage = _buffer(st.value, S.device)
        temp = _buffer(tmp.value, S.device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(S.device):
            check(lib().spk_tplan_build(S.handle, int(chunk_work), self._storage.data_ptr(), self._storage.numel(),
                                        temp.data_ptr(), temp.numel(), ctypes.byref(self._h), _stream(S.device)),
                  "spk_tplan_build")
        del temp
        self._ws = {}

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def arrays(self):
        """(colptr, rowidx, perm) as int32 CUDA tensors (views of the plan storage)."""
        cp, ri, pm = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        check(lib().spk_tplan_arrays(self._h, ctypes.byref(cp), ctypes.byref(ri), ctypes.byref(pm)),
              "spk_tplan_arrays")
        base = self._storage.data_ptr()

        def view(ptr, n):
            off = ptr.value - base
            return self._storage[off:off + 4 * n].view(torch.int32)

        return view(cp, self.N + 1), view(ri, self.nnz), view(pm, self.nnz)

    def mh_workspace(self, nbytes: int) -> torch.Tensor:
        """Workspace of a multi-head S^T Y (cached, grown on demand)."""
        ws = self._ws.get("mh")
        if ws is None or ws.numel() < nbytes:
            ws = _buffer(nbytes, self.S.device)
            self._ws["mh"] = ws
        return ws

    def workspace(self, K: int) -> torch.Tensor | None:
        nbytes = ctypes.c_size_t()
        check(lib().spk_spmm_t_workspace_size(self._h, int(K), ctypes.byref(nbytes)), "spk_spmm_t_workspace_size")
        if nbytes.value == 0:
            return None
        ws = self._ws.get(K)
        if ws is None or ws.numel() < nbytes.value:
            ws = _buffer(nbytes.value, self.S.device)
            self._ws[K] = ws
        return ws

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().spk_tplan_destroy(h)
            except Exception:
                pass
            self._h = None


__all__ = ["CSR", "TransposePlan", "SpkError", "DEFAULT_CHUNK_WORK"]


ORDERS = {"degree": 1, "leading": 2, "rcm": 3}
_DT = {torch.float32: 0, torch.bfloat16: 1, torch.float16: 2, torch.uint8: 3}


class Reordering:
    """Row relabelling of a pattern for locality (spk_reorder_rows,
    spk_permute_pattern): ``perm[p]`` is the original row placed at position
    p; ``S`` is the relabelled pattern (same column ids) carrying the values
    in its slot order; ``emap[e']`` is the original slot of each of its entries.

    With A' = gather_rows(A), SDDMM(S', A', B) = gather_values(SDDMM(S, A, B))
    and SpMM(S', B) = gather_rows(SpMM(S, B)); scatter_values / scatter_rows
    map results back to the original indices."""

    def __init__(self, S: CSR, order: str = "rcm", *, chunk_work: int = DEFAULT_CHUNK_WORK):
        self.order = order
        self.M, self.N, self.nnz = S.M, S.N, S.nnz
        self.device = S.device
        tb = ctypes.c_size_t()
        check(lib().spk_reorder_size(S.handle, ctypes.byref(tb)), "spk_reorder_size")
        temp = _buffer(tb.value, S.device)
        self.perm = torch.empty(max(S.M, 1), dtype=torch.int32, device=S.device)[:S.M]
        with torch.cuda.device(S.device):
            check(lib().spk_reorder_rows(S.handle, ORDERS[order], self.perm.data_ptr() if S.M else None,
                                         temp.data_ptr(), temp.numel(), _stream(S.device)), "spk_reorder_rows")
            rp = torch.empty(S.M + 1, dtype=torch.int32, device=S.device)
            ci = torch.empty(max(S.nnz, 1), dtype=torch.int32, device=S.device)
            self.emap = torch.empty(max(S.nnz, 1), dtype=torch.int32, device=S.device)
            check(lib().spk_permute_pattern(S.handle, self.perm.data_ptr() if S.M else None, rp.data_ptr(),
                                            ci.data_ptr(), self.emap.data_ptr(), temp.data_ptr(), temp.numel(),
                                            _stream(S.device)), "spk_permute_pattern")
        self.emap = self.emap[:S.nnz]
        vals = None if S.vals is None else self.gather_values(S.vals)
        self.S = CSR(rp, ci[:S.nnz], (S.M, S.N), vals, device=S.device, chunk_work=chunk_work)

    def _rows(self, X: torch.Tensor, scatter: int) -> torch.Tensor:
        if X.dim() != 2 or X.size(0) != self.M or X.stride(1) != 1 or X.device != self.device:
            raise ValueError("expected an M x K row-major CUDA tensor")
        Y = torch.empty((self.M, X.size(1)), dtype=X.dtype, device=X.device)
        check(lib().spk_permute_rows(X.data_ptr(), X.stride(0), _DT[X.dtype], self.M, X.size(1),
                                     self.perm.data_ptr() if self.M else None, scatter, Y.data_ptr(), Y.stride(0),
                                     _stream(X.device)), "spk_permute_rows")
        return Y

    def gather_rows(self, X: torch.Tensor) -> torch.Tensor:
        """X'[p] = X[perm[p]] (an M-row operand or result into the new order)."""
        return self._rows(X, 0)

    def scatter_rows(self, Xp: torch.Tensor) -> torch.Tensor:
        """X[perm[p]] = X'[p] (back to the original row order)."""
        return self._rows(Xp, 1)

    def _vals(self, x: torch.Tensor, scatter: int) -> torch.Tensor:
        if x.dtype != torch.float32 or x.numel() != self.nnz or x.device != self.device:
            raise ValueError("expected nnz FP32 values on the pattern's device")
        x = x.contiguous()
        y = torch.empty_like(x)
        check(lib().spk_permute_values(x.data_ptr(), self.emap.data_ptr() if self.nnz else None, self.nnz, scatter,
                                       y.data_ptr(), _stream(x.device)), "spk_permute_values")
        return y

    def gather_values(self, x: torch.Tensor) -> torch.Tensor:
        """Per-entry values of S into the slot order of S'."""
        return self._vals(x, 0)

    def scatter_values(self, xp: torch.Tensor) -> torch.Tensor:
        """Per-entry results on S' back to the slot order of S."""
        return self._vals(xp, 1)


class TensorCorePlan:
    """Dense 128 x 64 tiles of a pattern for the tensor cores, and the rest
    (spk_tc_plan_build): tiles holding at least ``threshold`` entries run as
    dense contractions, every other entry on the gather kernels."""

    def __init__(self, S: CSR, threshold: int = 1024, *, chunk_work: int = DEFAULT_CHUNK_WORK):
        self.S = S
        self.M, self.N, self.nnz = S.M, S.N, S.nnz
        st, tmp = ctypes.c_size_t(), ctypes.c_size_t()
        check(lib().spk_tc_plan_size(S.handle, int(threshold), int(chunk_work), ctypes.byref(st), ctypes.byref(tmp)),
              "spk_tc_plan_size")
        self._storage = _buffer(st.value, S.device)
        temp = _buffer(tmp.value, S.device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(S.device):
            check(lib().spk_tc_plan_build(S.handle, int(threshold), int(chunk_work), self._storage.data_ptr(),
                                          self._storage.numel(), temp.data_ptr(), temp.numel(), ctypes.byref(self._h),
                                          _stream(S.device)), "spk_tc_plan_build")
        del temp
        self._ws = None

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def info(self) -> dict:
        t, d, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(lib().spk_tc_plan_info(self._h, ctypes.byref(t), ctypes.byref(d), ctypes.byref(r)), "spk_tc_plan_info")
        return {"tiles": t.value, "dense_nnz": d.value, "rest_nnz": r.value}

    def arrays(self) -> dict:
        """Device views: tiles (T x 4), dense-entry slots, the remainder's
        rowptr / colidx / slots, and the status word."""
        ptrs = [ctypes.c_void_p() for _ in range(6)]
        check(lib().spk_tc_plan_arrays(self._h, *[ctypes.byref(p) for p in ptrs]), "spk_tc_plan_arrays")
        base = self._storage.data_ptr()
        inf = self.info()

        def view(ptr, n):
            off = ptr.value - base
            return self._storage[off:off + 4 * n].view(torch.int32)

        return {"tiles": view(ptrs[0], 4 * inf["tiles"]).view(-1, 4), "ent_slot": view(ptrs[1], inf["dense_nnz"]),
                "rest_rowptr": view(ptrs[2], self.M + 1), "rest_colidx": view(ptrs[3], inf["rest_nnz"]),
                "rest_emap": view(ptrs[4], inf["rest_nnz"]), "status": view(ptrs[5], 1)}

    def workspace(self) -> torch.Tensor | None:
        n = ctypes.c_size_t()
        check(lib().spk_tc_sddmm_workspace_size(self._h, ctypes.byref(n)), "spk_tc_sddmm_workspace_size")
        if n.value == 0:
            return None
        if self._ws is None or self._ws.numel() < n.value:
            self._ws = _buffer(n.value, self.S.device)
        return self._ws

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().spk_tc_plan_destroy(h)
            except Exception:
                pass
            self._h = None
