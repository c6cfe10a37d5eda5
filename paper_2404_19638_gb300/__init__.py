"""GB300-native local SDDMM / SpMM (the Compute phase of SpComm3D, Sec. 6.1).

    S = CSR(rowptr, colidx, (M, N), vals)        # pattern + balanced schedule
    S = CSR.from_coo(rows, cols, (M, N), vals)   # the same from coordinates (sorted on the device)
    R = Reordering(S, "rcm")                      # row relabelling for locality: R.S, R.gather_rows(A), ...
    T = TensorCorePlan(S); out = tc_sddmm(T, A16, B16)   # dense 128 x 64 tiles on the tensor cores (BF16)
    out = sddmm(S, A, B)                          # Eq. 1, FP32 per nonzero
    C = spmm(S, B)                                # Eq. 2
    X = spmm_t(S, Y)                              # S^T Y via the transpose plan
    Y, _, _ = fusedmm(S, A, B, heads=4, softmax=True)   # SDDMM -> (softmax) -> SpMM in one kernel

All arithmetic runs in libspk's CUDA kernels for sm_103a (include/spk.h);
PyTorch supplies device memory and streams.  There is no CPU fallback: the
first call raises if libspk.so was not built.
"""
from .binding import SpkError, Tune, library_path
from .sparse import CSR, TransposePlan, DEFAULT_CHUNK_WORK, coo_to_csr, Reordering, TensorCorePlan
from .ops import sddmm, spmm, spmm_t, fusedmm, cast, quantize_e4m3_rows, tc_sddmm
from . import autograd
from .batch import Batch, Item, OP_SDDMM, OP_SPMM
from .autotune import Autotuner

__all__ = ["CSR", "TransposePlan", "sddmm", "spmm", "spmm_t", "fusedmm", "cast", "quantize_e4m3_rows", "autograd",
           "Batch", "Item", "OP_SDDMM", "OP_SPMM", "Autotuner", "SpkError", "Tune", "library_path", "DEFAULT_CHUNK_WORK",
           "coo_to_csr", "Reordering", "TensorCorePlan", "tc_sddmm"]
