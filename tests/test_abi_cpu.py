"""The C ABI on the host: the library loads, exports every function declared in
include/spk.h, and rejects bad arguments before touching the GPU (none of
these calls launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2404_19638_gb300 import _build, binding
    if not os.path.exists(_build.LIB):
        _build.build()
    return binding.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "spk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spk_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_and_version(L):
    assert L.spk_version() >= 10000
    assert L.spk_status_string(0) == b"ok"
    assert L.spk_status_string(5).startswith(b"workspace")


def _handle(L, M=10, N=8, nnz=20):
    h = ctypes.c_void_p()
    # device pointers are only stored, never dereferenced, by spk_csr_create
    assert L.spk_csr_create(ctypes.byref(h), M, N, nnz, 4096, 8192) == 0
    return h


def test_csr_create_rejects_bad_arguments(L):
    h = ctypes.c_void_p()
    assert L.spk_csr_create(None, 1, 1, 0, 4096, None) == 1
    assert L.spk_csr_create(ctypes.byref(h), -1, 1, 0, 4096, None) == 1
    assert L.spk_csr_create(ctypes.byref(h), 1, 1, 0, None, None) == 1
    assert L.spk_csr_create(ctypes.byref(h), 4, 0, 3, 4096, 8192) == 2      # nonzeros without columns
    assert L.spk_csr_create(ctypes.byref(h), 1 << 31, 1, 0, 4096, None) == 8
    assert b"int32" in L.spk_last_error()
    assert L.spk_csr_create(ctypes.byref(h), 4, 4, 3, 4096, None) == 1       # colidx NULL with nnz > 0


def test_compute_calls_reject_bad_arguments(L):
    from paper_2404_19638_gb300.binding import Tune
    h = _handle(L)
    sddmm = lambda *a: L.spk_sddmm(h, None, None, *a)
    # dtype pair, K, leading dimensions, E4M3 scales
    assert sddmm(1, 4096, 16, None, 0, 4096, 16, None, 16, 4096, None, None) == 4
    assert sddmm(0, 4096, 16, None, 0, 4096, 16, None, 0, 4096, None, None) == 2
    assert sddmm(0, 4096, 8, None, 0, 4096, 16, None, 16, 4096, None, None) == 2
    big = 1 << 30                                                           # rows of 4 GiB in FP32
    assert sddmm(0, 4096, 16, None, 0, 4096, big, None, 16, 4096, None, None) == 2
    assert sddmm(0, 4096, big, None, 0, 4096, 16, None, 16, 4096, None, None) == 2
    assert b"4 GiB" in L.spk_last_error()
    assert sddmm(3, 4096, 16, None, 3, 4096, 16, None, 16, 4096, None, None) == 1
    assert sddmm(0, None, 16, None, 0, 4096, 16, None, 16, 4096, None, None) == 1
    # balanced variant without a schedule
    t = Tune(variant=2)
    assert sddmm(0, 4096, 16, None, 0, 4096, 16, None, 16, 4096, ctypes.byref(t), None) == 9
    # shape not compiled
    t = Tune(variant=1, group_lanes=2, vecs_per_lane=1, unroll=4)
    assert sddmm(0, 4096, 16, None, 0, 4096, 16, None, 16, 4096, ctypes.byref(t), None) == 8
    spmm = lambda *a: L.spk_spmm(h, None, None, *a)
    assert spmm(0, 4096, 16, None, 16, 3, 8192, 16, 0, None, 0, None, None) == 4     # E4M3 output
    assert spmm(0, 4096, 16, None, 16, 0, 8192, 16, 2, None, 0, None, None) == 1     # accumulate flag
    assert spmm(0, 4096, 16, None, 16, 0, 8192, 8, 0, None, 0, None, None) == 2      # ldc < K
    assert spmm(0, 4096, 1 << 30, None, 16, 0, 8192, 16, 0, None, 0, None, None) == 2  # 4 GiB rows of B
    assert spmm(0, 4096, 16, None, 16, 0, None, 16, 0, None, 0, None, None) == 1     # C NULL
    assert L.spk_spmm(None, None, None, 0, 4096, 16, None, 16, 0, 8192, 16, 0, None, 0, None, None) == 1
    L.spk_csr_destroy(h)


def test_schedule_and_plan_sizes_on_host(L):
    h = _handle(L, M=1000, N=500, nnz=7000)
    n = ctypes.c_size_t()
    assert L.spk_schedule_size(h, 0, ctypes.byref(n)) == 0 and n.value > 7000 * 4
    assert L.spk_schedule_size(h, 16, ctypes.byref(n)) == 1              # chunk_work too small
    assert L.spk_schedule_build(h, 512, None, 0, None) == 5              # no storage
    assert L.spk_schedule_build(h, 512, 4096 + 8, 1 << 30, None) == 5    # misaligned storage
    st, tmp = ctypes.c_size_t(), ctypes.c_size_t()
    assert L.spk_tplan_size(h, 0, ctypes.byref(st), ctypes.byref(tmp)) == 0
    assert st.value >= (501 + 2 * 7000) * 4 and tmp.value >= 4 * 7000 * 4
    p = ctypes.c_void_p()
    assert L.spk_tplan_build(h, 0, None, 0, None, 0, ctypes.byref(p), None) == 5
    assert L.spk_schedule_info(h, None, None, None) == 9                 # nothing attached yet
    L.spk_csr_destroy(h)


def test_precision_calls_reject_bad_arguments(L):
    assert L.spk_cast(4096, 10, 0, 8192, None) == 4                      # F32 is not a cast target
    assert L.spk_cast(None, 10, 1, 8192, None) == 1
    assert L.spk_quantize_e4m3_rows(4096, 4, 8, 4, 8192, 8, 12288, None) == 2


def test_batch_rejects_bad_items(L):
    from paper_2404_19638_gb300.binding import BatchItem
    h = _handle(L)
    n = ctypes.c_size_t()
    arr = (BatchItem * 1)()
    arr[0] = BatchItem(op=1, S=h.value, vals=None, dt=0, A=None, lda=0, B=4096, ldb=16, K=16, out=8192, ldc=16)
    assert L.spk_batch_size(arr, 1, ctypes.byref(n)) == 9                # no schedule attached
    arr[0].op = 5
    assert L.spk_batch_size(arr, 1, ctypes.byref(n)) == 1
    assert L.spk_batch_size(arr, 0, ctypes.byref(n)) == 1
    L.spk_csr_destroy(h)


def test_python_binding_raises_with_message(L):
    from paper_2404_19638_gb300.binding import SpkError, check
    h = ctypes.c_void_p()
    with pytest.raises(SpkError) as ei:
        check(L.spk_csr_create(ctypes.byref(h), -3, 1, 0, 4096, None), "spk_csr_create")
    assert ei.value.code == "SPK_ERR_ARG" and "negative" in str(ei.value)


def test_fused_backward_steps_reject_bad_arguments(L):
    h = _handle(L)
    assert L.spk_fused_weights(h, 2, 1, 4096, 8192, 12288, None) == 9        # no schedule: needs the COO rows
    assert L.spk_fused_weights(h, 0, 0, 4096, None, 12288, None) == 1        # heads < 1
    assert L.spk_fused_weights(h, 1, 2, 4096, None, 12288, None) == 1        # softmax flag not 0/1
    assert L.spk_fused_score_grad(h, 2, 1, 1.0, None, 4096, 8192, 12288, 16384, None) == 9
    assert L.spk_fused_score_grad(h, 70000, 0, 1.0, None, None, 8192, None, 16384, None) == 1   # heads > 65535
    assert L.spk_fused_rowdot(10, 12, 5, 4096, 12, 8192, 12, 12288, None) == 2   # K not a multiple of heads
    assert L.spk_fused_rowdot(10, 12, 3, 4096, 8, 8192, 12, 12288, None) == 2    # row stride below K
    assert L.spk_fused_rowdot(10, 12, 3, None, 12, 8192, 12, 12288, None) == 1
    assert L.spk_fused_rowdot(0, 12, 3, None, 12, None, 12, None, None) == 0     # empty: nothing to do
    L.spk_csr_destroy(h)


def test_python_wrappers_reject_host_tensors():
    """Host tensors never reach a kernel: the wrappers raise first."""
    import torch
    from paper_2404_19638_gb300 import ops
    X = torch.zeros((4, 8), dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA"):
        ops.fused_rowdot(X, X, 2)
    with pytest.raises(TypeError):
        ops.cast(X, torch.bfloat16)
    with pytest.raises(TypeError):
        ops.quantize_e4m3_rows(X)


def test_batch_shape_lists_and_register_choice(L):
    """The batched shapes per op (host only) and the register-budget call's
    argument checks."""
    from paper_2404_19638_gb300.binding import batch_shapes
    sd, sp = batch_shapes(0), batch_shapes(1)
    assert sd and sp and batch_shapes(2) == []
    assert all(U in (4, 8) and G in (4, 8, 16) and NV == 1 for G, NV, U in sd + sp)
    assert set(sd) <= set(sp)                                             # SpMM adds 8-nonzero batches
    assert any(U == 8 for _, _, U in sp)
    buf = (ctypes.c_int32 * 3)()
    assert L.spk_batch_shapes(1, buf, 1) == len(sp) and tuple(buf) == sp[0]
    assert L.spk_batch_set_registers(None, 80) == 1                      # NULL handle


def test_sddmm_heads_rejects_bad_arguments(L):
    """spk_sddmm_mh checks its arguments on the host before any launch."""
    h = _handle(L)
    mh = lambda heads, dt, K, lda=64, ldb=64: L.spk_sddmm_mh(h, None, heads, dt, 4096, lda, 8192, ldb, K, 12288, None)
    assert mh(4, 2, 64) == 4                                             # F16 not offered
    assert mh(3, 0, 64) == 2                                             # K not a multiple of heads
    assert mh(4, 0, 64, lda=32) == 2                                     # leading dimension < K
    assert mh(4, 0, 64, ldb=1 << 30) == 2                                # rows of 4 GiB
    assert mh(4, 0, 64) == 9                                             # no schedule attached
    assert L.spk_sddmm_mh(None, None, 4, 0, 4096, 64, 8192, 64, 64, 12288, None) == 1
    L.spk_csr_destroy(h)
