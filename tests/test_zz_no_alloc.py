"""spk_spmm_static, the SpMM entry point that allocates nothing, called
through the C ABI.  It exists for callers that cannot call cudaMalloc (code
inside a host process that owns the device memory pool, or a loop where an
allocation's implicit synchronisation is not allowed): its split-row carry
slots live in the library's own static device array instead of a caller
workspace.  Every result is checked element by element against the FP64
oracle, and against spk_spmm with a caller workspace on the same inputs, on
two calls in a row.  Kept in a file of its own, collected last, so that it
runs both alone in a fresh process and after every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, comp_err, edge_pattern

pytestmark = pytest.mark.gpu
SCRATCH_BYTES = 4 << 20          # SPK_STATIC_SCRATCH_BYTES in include/spk.h
F32, BF16 = 0, 1


@pytest.fixture(scope="module")
def spk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2404_19638_gb300 as m
    return m


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dt(B):
    return BF16 if B.dtype == torch.bfloat16 else F32


def _spmm(L, S, vals, B, C, ws, acc=0, tune=None):
    return L.spk_spmm(S.handle, vals.data_ptr(), None, _dt(B), B.data_ptr(), B.stride(0), None, B.size(1), F32,
                      C.data_ptr(), C.stride(0), acc, ws.data_ptr(), ws.numel(), tune, _stream())


def _spmm_static(L, S, vals, B, C, acc=0, tune=None):
    return L.spk_spmm_static(S.handle, vals.data_ptr(), None, _dt(B), B.data_ptr(), B.stride(0), None, B.size(1),
                             F32, C.data_ptr(), C.stride(0), acc, tune, _stream())


def _oracle(rp, ci, B, vals, C0=None):
    """Oracle result and componentwise denominator of C0 + S B (C0 = None: S B)."""
    vals = vals.cpu().numpy()
    if B.dtype == torch.bfloat16:
        Bq = B.view(torch.int16).cpu().numpy().view(np.uint16)
        ref = oracle.spmm(rp, ci, Bq, vals, fmt_b="bf16")
        den = oracle.spmm(rp, ci, Bq, vals, fmt_b="bf16", absmode=True)
    else:
        Bn = B.cpu().numpy()
        ref = oracle.spmm(rp, ci, Bn, vals)
        den = oracle.spmm(rp, ci, Bn, vals, absmode=True)
    if C0 is not None:
        c0 = C0.cpu().numpy().astype(np.float64)
        ref, den = ref + c0, den + np.abs(c0)
    return ref, den


@pytest.mark.parametrize("K,dtype,acc", [(64, torch.float32, 0), (24, torch.float32, 0), (9, torch.float32, 0),
                                         (64, torch.bfloat16, 0), (32, torch.float32, 1)])
def test_static_scratch_matches_oracle_and_workspace_entry_point(spk, K, dtype, acc):
    from paper_2404_19638_gb300.binding import lib
    L = lib()
    M, N = 2000, 1500
    rp, ci = edge_pattern(M, N, seed=11, long_row=4000)
    S = spk.CSR(rp, ci, (M, N), device="cuda", chunk_work=64)
    npieces = S.schedule_info()["npieces"]
    assert npieces > 0 and npieces * K * 4 <= SCRATCH_BYTES
    ws = S.workspace(K)
    g = np.random.default_rng(K + 7 * acc)
    runs = []
    for call in range(2):                      # two calls in a row, different inputs
        vals = torch.from_numpy(g.uniform(-1, 1, ci.size).astype(np.float32)).cuda()
        B = torch.from_numpy(g.standard_normal((N, K)).astype(np.float32)).cuda().to(dtype)
        C0 = torch.from_numpy(g.standard_normal((M, K)).astype(np.float32)).cuda() if acc else None
        C_ws = C0.clone() if acc else torch.full((M, K), float("nan"), device="cuda")
        C_st = C0.clone() if acc else torch.full((M, K), float("nan"), device="cuda")
        assert _spmm(L, S, vals, B, C_ws, ws, acc) == 0, L.spk_last_error()
        assert _spmm_static(L, S, vals, B, C_st, acc) == 0, L.spk_last_error()
        runs.append((vals, B, C0, C_ws, C_st))
    torch.cuda.synchronize()
    for vals, B, C0, C_ws, C_st in runs:
        ref, den = _oracle(rp, ci, B, vals, C0)
        assert comp_err(C_st.cpu().numpy(), ref, den) <= TOL
        assert comp_err(C_st.cpu().numpy(), C_ws.cpu().numpy(), den) <= TOL
    # back to back on the stream with no synchronisation in between
    if not acc:
        vals, B, _, C_ws, _ = runs[0]
        C1 = torch.full((M, K), float("nan"), device="cuda")
        C2 = torch.full((M, K), float("nan"), device="cuda")
        assert _spmm_static(L, S, vals, B, C1) == 0 and _spmm_static(L, S, vals, B, C2) == 0
        torch.cuda.synchronize()
        ref, den = _oracle(rp, ci, B, vals)
        for C in (C1, C2):
            assert comp_err(C.cpu().numpy(), ref, den) <= TOL
            assert comp_err(C.cpu().numpy(), C_ws.cpu().numpy(), den) <= TOL


def test_static_scratch_rejects_oversize(spk):
    from paper_2404_19638_gb300.binding import lib, Tune
    L = lib()
    M, N = 400, 300
    rp, ci = edge_pattern(M, N, seed=12, long_row=3000)
    S = spk.CSR(rp, ci, (M, N), device="cuda", chunk_work=32)
    npieces = S.schedule_info()["npieces"]
    K = SCRATCH_BYTES // (4 * npieces) + 4      # just above the limit
    assert npieces * K * 4 > SCRATCH_BYTES
    vals = torch.from_numpy(np.random.default_rng(3).uniform(-1, 1, ci.size).astype(np.float32)).cuda()
    B = torch.from_numpy(np.random.default_rng(4).standard_normal((N, K)).astype(np.float32)).cuda()
    C = torch.zeros((M, K), device="cuda")
    assert _spmm_static(L, S, vals, B, C) == 5                     # SPK_ERR_WORKSPACE, before any launch
    assert b"scratch" in L.spk_last_error()
    # the row-split kernel uses no carry slots: the same K is accepted there
    row_split = Tune(variant=1)
    assert _spmm_static(L, S, vals, B, C, tune=ctypes.byref(row_split)) == 0, L.spk_last_error()
    torch.cuda.synchronize()
    ref, den = _oracle(rp, ci, B, vals)
    assert comp_err(C.cpu().numpy(), ref, den) <= TOL
