"""Batched persistent launch of many independent SDDMM / SpMM problems.

One ``spk_batch_run`` is a single kernel launch over all (item, chunk) work
units, so the whole batch can be captured once in a CUDA graph and replayed.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from .binding import BatchItem, SPK_BF16, SPK_F32, Tune, check, lib
from .sparse import CSR, _buffer, _stream

OP_SDDMM, OP_SPMM = 0, 1


@dataclass
class Item:
    op: int                      # OP_SDDMM or OP_SPMM
    S: CSR                       # needs a schedule
    B: torch.Tensor              # N x K, float32 or bfloat16
    out: torch.Tensor            # SDDMM: float32[nnz]; SpMM: float32 M x K
    A: torch.Tensor | None = None
    vals: torch.Tensor | None = None
    tune: dict | None = None


class Batch:
    def __init__(self, items: list[Item], device=None):
        if not items:
            raise ValueError("empty batch")
        self.items = items
        self.device = items[0].S.device if device is None else torch.device(device)
        self._tunes = []
        arr = (BatchItem * len(items))()
        for k, it in enumerate(items):
            dt = {torch.float32: SPK_F32, torch.bfloat16: SPK_BF16}.get(it.B.dtype)
            if dt is None:
                raise TypeError("batched operands must be float32 or bfloat16")
            K = it.B.size(1)
            t = Tune.make(it.tune)
            self._tunes.append(t)
            vals = it.vals if it.vals is not None else it.S.vals
            arr[k] = BatchItem(op=it.op, S=it.S.handle.value, vals=None if vals is None else vals.data_ptr(), dt=dt,
                               A=None if it.A is None else it.A.data_ptr(),
                               lda=0 if it.A is None else it.A.stride(0), B=it.B.data_ptr(), ldb=it.B.stride(0),
                               K=K, out=it.out.data_ptr(), ldc=it.out.stride(0) if it.op == OP_SPMM else 0,
                               tune=None if t is None else ctypes.pointer(t))
        self._arr = arr
        self._h = ctypes.c_void_p()
        self._create()

    def _create(self) -> None:
        """(Re)build the native work list from the items' current schedules."""
        self._destroy()
        nbytes = ctypes.c_size_t()
        check(lib().spk_batch_size(self._arr, len(self.items), ctypes.byref(nbytes)), "spk_batch_size")
        self._storage = _buffer(nbytes.value, self.device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(lib().spk_batch_create(self._arr, len(self.items), self._storage.data_ptr(), self._storage.numel(),
                                         ctypes.byref(self._h), _stream(self.device)), "spk_batch_create")
        self._graph = None

    def _destroy(self) -> None:
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().spk_batch_destroy(h)
        self._h = None

    def autotune(self, chunk_works=(64, 128, 256, 512), reps: int = 3) -> dict:
        """Pick the balanced-schedule chunk size of the whole batch by timing
        one persistent launch per candidate (CUDA events, median of reps);
        every item's schedule is rebuilt with the winner.  Returns
        {"chunk_work": W, "ms": {W: median ms}}."""
        patterns = []
        for it in self.items:
            if all(it.S is not p for p in patterns):
                patterns.append(it.S)
        times = {}
        for W in chunk_works:
            for S in patterns:
                S.build_schedule(W)
            self._create()
            self.run()
            torch.cuda.synchronize(self.device)
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                self.run()
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            times[W] = sorted(ts)[len(ts) // 2]
        best = min(times, key=times.get)
        for S in patterns:
            S.build_schedule(best)
        self._create()
        return {"chunk_work": best, "ms": times}

    def info(self) -> dict:
        units, ctas = ctypes.c_int64(), ctypes.c_int32()
        check(lib().spk_batch_info(self._h, ctypes.byref(units), ctypes.byref(ctas)), "spk_batch_info")
        return {"work_units": units.value, "ctas": ctas.value}

    def run(self) -> None:
        """One persistent launch on the current stream."""
        check(lib().spk_batch_run(self._h, _stream(self.device)), "spk_batch_run")

    def capture(self) -> "torch.cuda.CUDAGraph":
        """Capture one run in a CUDA graph (once); ``replay()`` then relaunches it."""
        if self._graph is None:
            self.run()                                   # warm-up outside capture
            torch.cuda.synchronize(self.device)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self.run()
            self._graph = g
        return self._graph

    def replay(self) -> None:
        self.capture().replay()

    def __del__(self):
        try:
            self._destroy()
        except Exception:
            pass


__all__ = ["Batch", "Item", "OP_SDDMM", "OP_SPMM"]
