"""Autotuner for the kernel schedule of one sparse pattern.

The fastest lane-group shape (lanes per dense row, 16-byte vectors per lane,
nonzeros in flight), CTA size and balanced-schedule chunk size depend on the
degree distribution of S, on K and on the dtype.  Following the paper's
"set up once, run many times" structure (Sec. 5.1: the pattern is fixed while
values change), the tuner times a small set of candidates once per
(pattern, op, dtype, K) with CUDA events on the current stream, keeps the
winner, and caches it in a JSON file keyed by a signature of the pattern's
shape and degree histogram.

    tuner = Autotuner()                     # cache: $SPK_AUTOTUNE_CACHE or ~/.cache/spk/autotune.json
    best = tuner.tune(S, "sddmm", A, B)     # rebuilds S's schedule with the best chunk size
    spk.sddmm(S, A, B, tune=best["tune"])
"""
from __future__ import annotations

import hashlib
import json
import os
import threading

import numpy as np
import torch

from . import ops
from .binding import SpkError
from .sparse import CSR

_VEC = {torch.float32: 4, torch.bfloat16: 8, torch.float16: 8, torch.float8_e4m3fn: 16, torch.uint8: 16}


def pattern_signature(rowptr: np.ndarray, M: int, N: int) -> str:
    """Shape, nnz and the log2-binned row-degree histogram, hashed."""
    deg = np.diff(np.asarray(rowptr, dtype=np.int64))
    bins = np.bincount(np.floor(np.log2(np.maximum(deg, 1))).astype(np.int64) + (deg > 0), minlength=34)
    h = hashlib.sha1()
    h.update(np.asarray([M, N, int(deg.sum()), int(deg.max(initial=0))], dtype=np.int64).tobytes())
    h.update(bins.astype(np.int64).tobytes())
    return h.hexdigest()[:20]


def candidate_shapes(K: int, dtype) -> list[tuple[int, int, int]]:
    """Compiled (G, NV, U) shapes that cover a row of K elements in one block
    without more than half the lanes idle."""
    vec = _VEC.get(dtype, 4)
    nvec = max(1, K // vec) if K % vec == 0 else K
    from .binding import compiled_shapes
    out = []
    for (G, NV, U) in sorted(compiled_shapes()):
        cover = G * NV
        if cover >= nvec and cover <= max(4, 2 * nvec):
            out.append((G, NV, U))
    return out or [(32, 4, 4)]


class Autotuner:
    def __init__(self, cache_path: str | None = None, chunk_works=(256, 512, 1024), threads=(128, 256),
                 reps: int = 5):
        self.path = cache_path or os.environ.get("SPK_AUTOTUNE_CACHE") or os.path.join(
            os.path.expanduser("~"), ".cache", "spk", "autotune.json")
        self.chunk_works = tuple(chunk_works)
        self.threads = tuple(threads)
        self.reps = reps
        self._lock = threading.Lock()
        self._cache = self._load()

    def _load(self) -> dict:
        try:
            with open(self.path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}

    def _save(self) -> None:
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            tmp = self.path + f".{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(self._cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except OSError:
            pass

    @staticmethod
    def key(S: CSR, op: str, dtype, K: int) -> str:
        sig = pattern_signature(S.rowptr.cpu().numpy(), S.M, S.N)
        return f"{sig}|{op}|{str(dtype).replace('torch.', '')}|{K}"

    def lookup(self, S: CSR, op: str, dtype, K: int) -> dict | None:
        return self._cache.get(self.key(S, op, dtype, K))

    @staticmethod
    def _attach(S: CSR, op: str, W: int) -> None:
        """Give S the schedule (SDDMM, SpMM) or transpose plan (S^T Y) of chunk size W."""
        if op == "spmm_t":
            S.transpose_plan(W)
        elif not S.has_schedule or S.schedule_info()["chunk_work"] != W:
            S.build_schedule(W)

    def _time(self, fn) -> float:
        fn()
        torch.cuda.synchronize(self._dev)
        ts = []
        for _ in range(self.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    def tune(self, S: CSR, op: str, A: torch.Tensor | None, B: torch.Tensor, force: bool = False) -> dict:
        """Best {"tune": {...}, "chunk_work": W, "ms": t} for op in {"sddmm",
        "spmm", "spmm_t"}; S ends with the winning schedule (or, for
        "spmm_t", transpose plan) attached.  For "spmm_t", B is the M x K
        operand Y of S^T Y and A is unused."""
        if op not in ("sddmm", "spmm", "spmm_t"):
            raise ValueError("op must be sddmm, spmm or spmm_t")
        self._dev = S.device
        K = B.size(1)
        dtype = B.dtype
        k = self.key(S, op, dtype, K)
        with self._lock:
            hit = None if force else self._cache.get(k)
        if hit is not None:
            self._attach(S, op, hit["chunk_work"])
            return hit
        if op == "sddmm":
            out = torch.empty(S.nnz, dtype=torch.float32, device=S.device)
            run = lambda t: ops.sddmm(S, A, B, out=out, tune=t)
        elif op == "spmm":
            out = torch.empty((S.M, K), dtype=torch.float32, device=S.device)
            run = lambda t: ops.spmm(S, B, out=out, tune=t)
        else:                                    # B is the M x K operand Y of S^T Y
            out = torch.empty((S.N, K), dtype=torch.float32, device=S.device)
            run = lambda t: ops.spmm_t(S, B, out=out, tune=t, plan=S.transpose_plan())
        best = None
        for W in self.chunk_works:
            self._attach(S, op, W)
            for (G, NV, U) in candidate_shapes(K, dtype):
                # shared-memory ring (2 or 4 slots), then the register path at each CTA size
                cands = [{"variant": 2, "stages": st} for st in (2, 4)]
                cands += [{"variant": 3, "cta_threads": thr} for thr in self.threads]
                for c in cands:
                    t = {"group_lanes": G, "vecs_per_lane": NV, "unroll": U, **c}
                    try:
                        ms = self._time(lambda: run(t))
                    except SpkError:
                        continue
                    if best is None or ms < best["ms"]:
                        best = {"tune": t, "chunk_work": W, "ms": ms}
        # the row-split variant, for patterns without long rows
        for (G, NV, U) in candidate_shapes(K, dtype)[:2]:
            t = {"variant": 1, "group_lanes": G, "vecs_per_lane": NV, "unroll": U, "cta_threads": self.threads[0]}
            try:
                ms = self._time(lambda: run(t))
            except SpkError:
                continue
            if best is not None and ms < best["ms"]:
                best = {"tune": t, "chunk_work": best["chunk_work"], "ms": ms}
        if best is None:
            raise RuntimeError("no candidate kernel ran")
        self._attach(S, op, best["chunk_work"])
        with self._lock:
            self._cache[k] = best
            self._save()
        return best


__all__ = ["Autotuner", "pattern_signature", "candidate_shapes"]
