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
            if getattr(self, "_regs", 0):
                check(lib().spk_batch_set_registers(self._h, self._regs), "spk_batch_set_registers")
        self._graph = None

    def _destroy(self) -> None:
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().spk_batch_destroy(h)
        self._h = None

    def set_registers(self, regs: int) -> None:
        """Kernel build of later runs: 80 or 96 registers per thread, or 0 for
        the one creation chose (a captured graph is dropped)."""
        check(lib().spk_batch_set_registers(self._h, int(regs)), "spk_batch_set_registers")
        self._regs = int(regs)
        self._graph = None

    def set_item_tune(self, k: int, tune) -> None:
        """Shape of item k for the next rebuild (None = default by K)."""
        t = Tune.make(tune)
        self._tunes[k] = t
        self._arr[k].tune = None if t is None else ctypes.pointer(t)

    def _time(self, reps: int) -> float:
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
        return sorted(ts)[len(ts) // 2]

    def _patterns(self) -> list:
        patterns = []
        for it in self.items:
            if all(it.S is not p for p in patterns):
                patterns.append(it.S)
        return patterns

    def autotune(self, chunk_works=(64, 128, 256, 512), reps: int = 3, per_item: bool = False,
                 min_gain: float = 0.01) -> dict:
        """Pick schedules and shapes by timing whole persistent launches (CUDA
        events, median of reps).

        First one balanced-schedule chunk size for every pattern.  With
        per_item, then, one pass of coordinate descent over per-item choices,
        each kept only if the whole launch gets at least min_gain faster:
        the chunk size of each group of patterns of similar size (nonzeros
        within a factor of 4), largest patterns first; the shape (group
        lanes, vectors per lane, nonzeros per batch; spk_batch_shapes) of
        each class of items of one op, K and dtype; the kernel's register
        budget (80 or 96).  Returns {"chunk_work": W, "ms": {W: ms}} plus,
        with per_item, "chunk_work_by_nnz", "shapes", "registers", "ms_final"
        and "trials" (whole launches timed after the first stage, each
        reps + 1 runs; the count depends only on the items and chunk_works)."""
        patterns = self._patterns()
        times = {}
        for W in chunk_works:
            for S in patterns:
                S.build_schedule(W)
            self._create()
            times[W] = self._time(reps)
        best = min(times, key=times.get)
        for S in patterns:
            S.build_schedule(best)
        self._create()
        res = {"chunk_work": best, "ms": times}
        if not per_item:
            return res
        from .binding import batch_shapes
        cur = times[best]
        trials = 0

        # chunk size per group of patterns of similar size, largest first
        groups = {}
        for S in patterns:
            groups.setdefault(max(S.nnz, 1).bit_length() // 2, []).append(S)
        chunk_by_group = {}
        for key in sorted(groups, reverse=True):
            chosen = best
            for W in [w for w in sorted(set(chunk_works) | {1024}) if w != best]:
                for S in groups[key]:
                    S.build_schedule(W)
                self._create()
                t = self._time(reps)
                trials += 1
                if t < cur * (1.0 - min_gain):
                    cur, chosen = t, W
            for S in groups[key]:
                S.build_schedule(chosen)
            chunk_by_group[key] = chosen
        self._create()

        # shape per (op, K, dtype) class
        classes = {}
        for k, it in enumerate(self.items):
            classes.setdefault((it.op, it.B.size(1), it.B.dtype), []).append(k)
        shapes = {}
        for (op, K, dt), ks in sorted(classes.items(), key=lambda kv: (kv[0][0], kv[0][1], str(kv[0][2]))):
            nvec = K // (4 if dt == torch.float32 else 8)
            start = [self._tunes[k] for k in ks]
            t0 = start[0]
            now = ((t0.group_lanes, t0.vecs_per_lane, t0.unroll) if t0 is not None and t0.group_lanes
                   else (4 if nvec <= 4 else (8 if nvec <= 8 else 16), 1, 4))
            chosen = None
            for G, NV, U in batch_shapes(op):
                if G * NV < nvec or (G, NV, U) == now:
                    continue
                for k in ks:
                    self.set_item_tune(k, {"group_lanes": G, "vecs_per_lane": NV, "unroll": U})
                self._create()
                t = self._time(reps)
                trials += 1
                if t < cur * (1.0 - min_gain):
                    cur, chosen = t, (G, NV, U)
                for k, t0 in zip(ks, start):
                    self.set_item_tune(k, t0)
            if chosen is not None:
                for k in ks:
                    self.set_item_tune(k, {"group_lanes": chosen[0], "vecs_per_lane": chosen[1], "unroll": chosen[2]})
            shapes[f"{'sddmm' if op == 0 else 'spmm'} K={K} {str(dt)[6:]}"] = chosen
        self._create()

        # register budget of the kernel build
        regs = 0
        for r in (80, 96):
            self.set_registers(r)
            t = self._time(reps)
            trials += 1
            if t < cur * (1.0 - min_gain):
                cur, regs = t, r
        self.set_registers(regs)
        res.update({"chunk_work_by_nnz": {f"nnz < 4^{key + 1}": w for key, w in sorted(chunk_by_group.items())},
                    "shapes": shapes, "registers": regs or "default", "ms_final": cur, "trials": trials})
        return res

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
