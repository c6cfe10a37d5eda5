"""spk_spmm_static, the SpMM entry point that allocates nothing (its carry
slots live in the library's static device scratch), called through the C ABI
and checked against spk_spmm with a caller workspace on the same inputs.
Kept in a file of its own, collected last, so that it runs both alone in a
fresh process and after every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, comp_err, edge_pattern

pytestmark = pytest.mark.gpu
SCRATCH_BYTES = 4 << 20          # SPK_STATIC_SCRATCH_BYTES in include/spk.h


@pytest.fixture(scope="module")
def spk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2404_19638_gb300 as m
    return m


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _spmm(L, S, vals, B, C, ws):
    return L.spk_spmm(S.handle, vals.data_ptr(), None, 0, B.data_ptr(), B.stride(0), None, B.size(1), 0,
                      C.data_ptr(), C.stride(0), 0, ws.data_ptr(), ws.numel(), None, _stream())


def _spmm_static(L, S, vals, B, C):
    return L.spk_spmm_static(S.handle, vals.data_ptr(), None, 0, B.data_ptr(), B.stride(0), None, B.size(1), 0,
                             C.data_ptr(), C.stride(0), 0, None, _stream())


@pytest.mark.parametrize("K", [64, 24])
def test_static_scratch_matches_workspace_entry_point(spk, K):
    from paper_2404_19638_gb300.binding import lib
    L = lib()
    M, N = 2000, 1500
    rp, ci = edge_pattern(M, N, seed=11, long_row=4000)
    S = spk.CSR(rp, ci, (M, N), device="cuda", chunk_work=64)
    npieces = S.schedule_info()["npieces"]
    assert npieces > 0 and npieces * K * 4 <= SCRATCH_BYTES
    ws = S.workspace(K)
    g = np.random.default_rng(K)
    runs = []
    for call in range(2):                      # two calls in a row, different inputs
        vals = torch.from_numpy(g.uniform(-1, 1, ci.size).astype(np.float32)).cuda()
        B = torch.from_numpy(g.standard_normal((N, K)).astype(np.float32)).cuda()
        C_ws = torch.full((M, K), float("nan"), device="cuda")
        C_st = torch.full((M, K), float("nan"), device="cuda")
        assert _spmm(L, S, vals, B, C_ws, ws) == 0
        assert _spmm_static(L, S, vals, B, C_st) == 0, L.spk_last_error()
        runs.append((vals, B, C_ws, C_st))
    torch.cuda.synchronize()
    for vals, B, C_ws, C_st in runs:
        den = oracle.spmm(rp, ci, B.cpu().numpy(), vals.cpu().numpy(), absmode=True)
        assert comp_err(C_st.cpu().numpy(), C_ws.cpu().numpy(), den) <= TOL
    # back to back on the stream with no synchronisation in between
    vals, B, C_ws, _ = runs[0]
    C1 = torch.full((M, K), float("nan"), device="cuda")
    C2 = torch.full((M, K), float("nan"), device="cuda")
    assert _spmm_static(L, S, vals, B, C1) == 0 and _spmm_static(L, S, vals, B, C2) == 0
    torch.cuda.synchronize()
    den = oracle.spmm(rp, ci, B.cpu().numpy(), vals.cpu().numpy(), absmode=True)
    assert comp_err(C1.cpu().numpy(), C_ws.cpu().numpy(), den) <= TOL
    assert comp_err(C2.cpu().numpy(), C_ws.cpu().numpy(), den) <= TOL


def test_static_scratch_rejects_oversize(spk):
    from paper_2404_19638_gb300.binding import lib
    L = lib()
    M, N = 400, 300
    rp, ci = edge_pattern(M, N, seed=12, long_row=3000)
    S = spk.CSR(rp, ci, (M, N), device="cuda", chunk_work=32)
    npieces = S.schedule_info()["npieces"]
    K = SCRATCH_BYTES // (4 * npieces) + 4      # just above the limit
    assert npieces * K * 4 > SCRATCH_BYTES
    vals = torch.ones(ci.size, device="cuda")
    B = torch.zeros((N, K), device="cuda")
    C = torch.zeros((M, K), device="cuda")
    assert _spmm_static(L, S, vals, B, C) == 5                     # SPK_ERR_WORKSPACE, before any launch
    assert b"scratch" in L.spk_last_error()
