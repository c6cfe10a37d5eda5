"""ctypes binding of libspk (include/spk.h): argument marshalling only.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2404_19638_gb300._build``); there is no fallback path, so a
missing library raises immediately.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

_i32, _i64, _sz, _vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p
_P = ctypes.POINTER

SPK_F32, SPK_BF16, SPK_F16, SPK_E4M3 = 0, 1, 2, 3

STATUS = {0: "SPK_OK", 1: "SPK_ERR_ARG", 2: "SPK_ERR_SHAPE", 3: "SPK_ERR_INDEX", 4: "SPK_ERR_DTYPE",
          5: "SPK_ERR_WORKSPACE", 6: "SPK_ERR_CUDA", 7: "SPK_ERR_TIMEOUT", 8: "SPK_ERR_UNSUPPORTED",
          9: "SPK_ERR_STATE"}


class SpkError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        self.code = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.code}: {message}")


class Tune(ctypes.Structure):
    """spk_tune: 0 fields mean the library default."""
    _fields_ = [("variant", _i32), ("group_lanes", _i32), ("vecs_per_lane", _i32), ("unroll", _i32),
                ("cta_threads", _i32), ("stages", _i32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}

    @classmethod
    def make(cls, t) -> "Tune | None":
        if t is None or isinstance(t, Tune):
            return t
        return cls(**{k: int(v) for k, v in dict(t).items()})


class BatchItem(ctypes.Structure):
    _fields_ = [("op", _i32), ("S", _vp), ("vals", _vp), ("dt", ctypes.c_int), ("A", _vp), ("lda", _i64),
                ("B", _vp), ("ldb", _i64), ("K", _i32), ("out", _vp), ("ldc", _i64), ("tune", _P(Tune))]


_PROTOS = {
    "spk_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "spk_last_error": (ctypes.c_char_p, []),
    "spk_version": (_i32, []),
    "spk_shapes": (_i32, [_vp, _i32]),
    "spk_batch_shapes": (_i32, [_i32, _vp, _i32]),
    "spk_batch_set_registers": (ctypes.c_int, [_vp, _i32]),
    "spk_tune_default": (ctypes.c_int, [_vp, _i32, ctypes.c_int, _i32, _P(Tune)]),
    "spk_csr_create": (ctypes.c_int, [_P(_vp), _i64, _i64, _i64, _vp, _vp]),
    "spk_csr_destroy": (ctypes.c_int, [_vp]),
    "spk_csr_validate": (ctypes.c_int, [_vp, _vp, _vp]),
    "spk_coo_to_csr_size": (ctypes.c_int, [_i64, _i64, _i64, _P(_sz)]),
    "spk_coo_to_csr": (ctypes.c_int, [_i64, _i64, _i64, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _P(_i64), _vp, _sz, _vp]),
    "spk_reorder_size": (ctypes.c_int, [_vp, _P(_sz)]),
    "spk_reorder_rows": (ctypes.c_int, [_vp, _i32, _vp, _vp, _sz, _vp]),
    "spk_permute_pattern": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "spk_permute_rows": (ctypes.c_int, [_vp, _i64, ctypes.c_int, _i64, _i32, _vp, _i32, _vp, _i64, _vp]),
    "spk_permute_values": (ctypes.c_int, [_vp, _vp, _i64, _i32, _vp, _vp]),
    "spk_schedule_size": (ctypes.c_int, [_vp, _i32, _P(_sz)]),
    "spk_schedule_build": (ctypes.c_int, [_vp, _i32, _vp, _sz, _vp]),
    "spk_schedule_info": (ctypes.c_int, [_vp, _P(_i64), _P(_i64), _P(_i32)]),
    "spk_schedule_bounds": (ctypes.c_int, [_vp, _vp, _vp]),
    "spk_merge_path_points": (ctypes.c_int, [_vp, _i32, _i64, _vp, _vp]),
    "spk_spmm_workspace_size": (ctypes.c_int, [_vp, _i32, _P(_sz)]),
    "spk_sddmm_mh": (ctypes.c_int, [_vp, _vp, _i32, ctypes.c_int, _vp, _i64, _vp, _i64, _i32, _vp, _vp]),
    "spk_sddmm": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _i64, _vp, ctypes.c_int, _vp, _i64, _vp, _i32,
                                 _vp, _P(Tune), _vp]),
    "spk_spmm": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _i64, _vp, _i32, ctypes.c_int, _vp, _i64, _i32,
                                _vp, _sz, _P(Tune), _vp]),
    "spk_spmm_mh": (ctypes.c_int, [_vp, _vp, _i64, _i32, ctypes.c_int, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _sz,
                                   _vp]),
    "spk_spmm_t_mh_workspace_size": (ctypes.c_int, [_vp, _i32, _i32, _P(_sz)]),
    "spk_spmm_t_mh": (ctypes.c_int, [_vp, _vp, _i64, _i32, ctypes.c_int, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _sz,
                                     _vp]),
    "spk_spmm_static": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _i64, _vp, _i32, ctypes.c_int, _vp, _i64,
                                       _i32, _P(Tune), _vp]),
    "spk_fusedmm_workspace_size": (ctypes.c_int, [_vp, _i32, _i32, _P(_sz)]),
    "spk_fusedmm": (ctypes.c_int, [_vp, _vp, ctypes.c_float, _i32, ctypes.c_int, _vp, _i64, _vp, _i64, _i32, _i32,
                                   _vp, _i64, _vp, _vp, _vp, _sz, _P(Tune), _vp]),
    "spk_fused_weights": (ctypes.c_int, [_vp, _i32, _i32, _vp, _vp, _vp, _vp]),
    "spk_fused_rowdot": (ctypes.c_int, [_i64, _i32, _i32, _vp, _i64, _vp, _i64, _vp, _vp]),
    "spk_fused_score_grad": (ctypes.c_int, [_vp, _i32, _i32, ctypes.c_float, _vp, _vp, _vp, _vp, _vp, _vp]),
    "spk_tc_plan_size": (ctypes.c_int, [_vp, _i32, _i32, _P(_sz), _P(_sz)]),
    "spk_tc_plan_build": (ctypes.c_int, [_vp, _i32, _i32, _vp, _sz, _vp, _sz, _P(_vp), _vp]),
    "spk_tc_plan_info": (ctypes.c_int, [_vp, _P(_i64), _P(_i64), _P(_i64)]),
    "spk_tc_plan_arrays": (ctypes.c_int, [_vp, _P(_vp), _P(_vp), _P(_vp), _P(_vp), _P(_vp), _P(_vp)]),
    "spk_tc_plan_destroy": (ctypes.c_int, [_vp]),
    "spk_tc_sddmm_workspace_size": (ctypes.c_int, [_vp, _P(_sz)]),
    "spk_tc_sddmm": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _i64, _vp, _i64, _i32, _vp, _vp, _sz, _P(Tune), _vp]),
    "spk_tc_sddmm_unarmed": (ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _i32, _vp, _vp]),
    "spk_tplan_size": (ctypes.c_int, [_vp, _i32, _P(_sz), _P(_sz)]),
    "spk_tplan_build": (ctypes.c_int, [_vp, _i32, _vp, _sz, _vp, _sz, _P(_vp), _vp]),
    "spk_tplan_arrays": (ctypes.c_int, [_vp, _P(_vp), _P(_vp), _P(_vp)]),
    "spk_tplan_destroy": (ctypes.c_int, [_vp]),
    "spk_spmm_t_workspace_size": (ctypes.c_int, [_vp, _i32, _P(_sz)]),
    "spk_spmm_t": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _i64, _vp, _i32, ctypes.c_int, _vp, _i64, _i32,
                                  _vp, _sz, _P(Tune), _vp]),
    "spk_cast": (ctypes.c_int, [_vp, _i64, ctypes.c_int, _vp, _vp]),
    "spk_quantize_e4m3_rows": (ctypes.c_int, [_vp, _i64, _i64, _i64, _vp, _i64, _vp, _vp]),
    "spk_batch_size": (ctypes.c_int, [_P(BatchItem), _i32, _P(_sz)]),
    "spk_batch_create": (ctypes.c_int, [_P(BatchItem), _i32, _vp, _sz, _P(_vp), _vp]),
    "spk_batch_run": (ctypes.c_int, [_vp, _vp]),
    "spk_batch_info": (ctypes.c_int, [_vp, _P(_i64), _P(_i32)]),
    "spk_batch_destroy": (ctypes.c_int, [_vp]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libspk (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libspk.so not found at {path}: build it first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            import torch  # noqa: F401  (loads the CUDA runtime libspk links against)
            L = ctypes.CDLL(path)
            for name, (res, args) in _PROTOS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != 0:
        msg = lib().spk_last_error()
        raise SpkError(status, where, msg.decode() if msg else "")


def batch_shapes(op: int) -> list[tuple[int, int, int]]:
    """(group_lanes, vecs_per_lane, unroll) shapes the batched launch offers
    for op (0 SDDMM, 1 SpMM)."""
    n = lib().spk_batch_shapes(op, None, 0)
    buf = (ctypes.c_int32 * (3 * max(n, 1)))()
    lib().spk_batch_shapes(op, buf, n)
    return [(buf[3 * i], buf[3 * i + 1], buf[3 * i + 2]) for i in range(n)]


def compiled_shapes() -> list[tuple[int, int, int]]:
    """(group_lanes, vecs_per_lane, unroll) shapes compiled into libspk."""
    n = lib().spk_shapes(None, 0)
    buf = (ctypes.c_int32 * (3 * n))()
    lib().spk_shapes(buf, n)
    return [(buf[3 * i], buf[3 * i + 1], buf[3 * i + 2]) for i in range(n)]
