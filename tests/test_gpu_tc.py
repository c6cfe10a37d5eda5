"""Dense row-panel tiles on the tensor cores (tcgen05): the plan's tiles,
entries and remainder against a direct count of the pattern, and SDDMM
(Eq. 1) through the plan — dense tiles on the tensor cores, the rest on the
gather kernels — element by element against the oracle on the BF16 inputs
(the kernel-accuracy gate, FP32 accumulation), across K, ragged last panels
and column tiles, unaligned blocks, values or none, and thresholds that take
every tile or none."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import TOL, comp_err

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def spk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2404_19638_gb300 as m
    return m


def _tiles_by_count(rp, ci, threshold):
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    key = (rows // 128).astype(np.int64) * (1 << 32) + ci // 64
    uk, cnt = np.unique(key, return_counts=True)
    dense = uk[cnt >= threshold]
    return {(int(k >> 32), int(k & 0xffffffff)): int(c) for k, c in zip(uk, cnt) if c >= threshold}, \
        np.isin(key, dense)


@pytest.mark.parametrize("M,N,blocks,aligned,threshold", [(1000, 900, 12, True, 1024), (1000, 900, 12, False, 600),
                                                          (517, 389, 6, True, 1), (700, 500, 4, True, 100000 // 13)])
def test_plan_matches_direct_count(spk, M, N, blocks, aligned, threshold):
    threshold = min(threshold, 8192)
    rp, ci = synth.dense_blocks(M, N, blocks, 0.3, 5, seed=M + blocks, aligned=aligned)
    S = spk.CSR(rp, ci, (M, N), device=DEV)
    P = spk.TensorCorePlan(S, threshold)
    exp, isdense = _tiles_by_count(rp, ci, threshold)
    info = P.info()
    assert info["tiles"] == len(exp) and info["dense_nnz"] == int(isdense.sum())
    assert info["rest_nnz"] == ci.size - int(isdense.sum())
    arr = P.arrays()
    tiles = arr["tiles"].cpu().numpy()
    got = {(int(t[0]), int(t[1])): int(t[3]) for t in tiles}
    assert got == exp
    slots = arr["ent_slot"].cpu().numpy()
    assert np.array_equal(np.sort(slots), np.flatnonzero(isdense))
    # the remainder: the other entries of every row, in order
    rest = np.flatnonzero(~isdense)
    rows = np.repeat(np.arange(M), np.diff(rp))
    assert np.array_equal(arr["rest_emap"].cpu().numpy(), rest)
    assert np.array_equal(arr["rest_colidx"].cpu().numpy(), ci[rest])
    assert np.array_equal(arr["rest_rowptr"].cpu().numpy(),
                          np.searchsorted(rows[rest], np.arange(M + 1), side="left").astype(np.int32))


@pytest.mark.parametrize("K", [16, 64, 128, 256])
@pytest.mark.parametrize("with_vals", [True, False])
def test_tc_sddmm_matches_oracle(spk, K, with_vals):
    M, N = 1100, 950                       # ragged last panel (1100 = 8 x 128 + 76) and column tile
    rp, ci = synth.dense_blocks(M, N, 14, 0.4, 6, seed=K, aligned=True)
    rp2, ci2 = synth.dense_blocks(M, N, 5, 0.5, 0, seed=K + 1, aligned=False)
    rows = np.concatenate([np.repeat(np.arange(M), np.diff(rp)), np.repeat(np.arange(M), np.diff(rp2))])
    rp, ci = synth.csr_from_coo(rows, np.concatenate([ci, ci2]), M, N)
    g = np.random.default_rng(K)
    vals = g.uniform(-1, 1, ci.size).astype(np.float32) if with_vals else None
    S = spk.CSR(rp, ci, (M, N), None if vals is None else torch.from_numpy(vals), device=DEV)
    P = spk.TensorCorePlan(S, 512)
    assert P.info()["tiles"] >= 10 and P.info()["rest_nnz"] > 0
    A = torch.from_numpy(g.standard_normal((M, K)).astype(np.float32)).to(DEV).to(torch.bfloat16)
    B = torch.from_numpy(g.standard_normal((N, K)).astype(np.float32)).to(DEV).to(torch.bfloat16)
    out = spk.tc_sddmm(P, A, B).cpu().numpy()
    Aq = A.view(torch.int16).cpu().numpy().view(np.uint16)
    Bq = B.view(torch.int16).cpu().numpy().view(np.uint16)
    ref = oracle.sddmm(rp, ci, Aq, Bq, vals, fmt_a="bf16", fmt_b="bf16")
    den = oracle.sddmm(rp, ci, Aq, Bq, vals, fmt_a="bf16", fmt_b="bf16", absmode=True)
    assert comp_err(out, ref, den) <= TOL
    assert int(P.arrays()["status"].cpu()[0]) == 0
    # the gather kernels on the whole pattern agree within the same tolerance
    plain = spk.sddmm(S, A, B).cpu().numpy()
    assert comp_err(out, plain, den) <= 2 * TOL


@pytest.mark.parametrize("threshold", [1, 8192])
def test_tc_sddmm_all_tiles_or_none(spk, threshold):
    """threshold 1: every nonempty tile on the tensor cores, no remainder;
    8192: only completely full tiles (none here), everything on the gather kernels."""
    M, N, K = 640, 320, 64
    rp, ci = synth.dense_blocks(M, N, 3, 0.6, 9, seed=5)
    g = np.random.default_rng(9)
    vals = g.uniform(-1, 1, ci.size).astype(np.float32)
    S = spk.CSR(rp, ci, (M, N), torch.from_numpy(vals), device=DEV)
    P = spk.TensorCorePlan(S, threshold)
    info = P.info()
    assert (info["rest_nnz"] == 0) if threshold == 1 else (info["tiles"] == 0)
    A = torch.from_numpy(g.standard_normal((M, K)).astype(np.float32)).to(DEV).to(torch.bfloat16)
    B = torch.from_numpy(g.standard_normal((N, K)).astype(np.float32)).to(DEV).to(torch.bfloat16)
    out = spk.tc_sddmm(P, A, B).cpu().numpy()
    Aq = A.view(torch.int16).cpu().numpy().view(np.uint16)
    Bq = B.view(torch.int16).cpu().numpy().view(np.uint16)
    assert comp_err(out, oracle.sddmm(rp, ci, Aq, Bq, vals, fmt_a="bf16", fmt_b="bf16"),
                    oracle.sddmm(rp, ci, Aq, Bq, vals, fmt_a="bf16", fmt_b="bf16", absmode=True)) <= TOL


def test_tensor_core_wait_limit_reports_status(spk):
    """The kernel's waits on the tensor core's barrier are bounded: with no MMA
    issued (an internal entry point) every wait runs out, the kernel records
    the status, frees its tensor memory and returns without touching the
    output — no fault, no hang — and the library still computes correctly."""
    import ctypes
    from paper_2404_19638_gb300.binding import lib
    M, N, K = 384, 256, 64
    rp, ci = synth.dense_blocks(M, N, 2, 0.9, 3, seed=17)
    g = np.random.default_rng(17)
    S = spk.CSR(rp, ci, (M, N), device=DEV)
    P = spk.TensorCorePlan(S, 2048)
    assert P.info()["tiles"] >= 1
    A = torch.from_numpy(g.standard_normal((M, K)).astype(np.float32)).to(DEV).to(torch.bfloat16)
    B = torch.from_numpy(g.standard_normal((N, K)).astype(np.float32)).to(DEV).to(torch.bfloat16)
    out = torch.full((ci.size,), 7.0, device=DEV)
    L = lib()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.spk_tc_sddmm_unarmed(P.handle, A.data_ptr(), K, B.data_ptr(), K, K, out.data_ptr(), st) == 0
    torch.cuda.synchronize()
    assert int(P.arrays()["status"].cpu()[0]) == 1
    assert torch.all(out == 7.0)
    # the context is intact: a normal call gives the oracle's result
    P.arrays()["status"].zero_()
    got = spk.tc_sddmm(P, A, B).cpu().numpy()
    Aq = A.view(torch.int16).cpu().numpy().view(np.uint16)
    Bq = B.view(torch.int16).cpu().numpy().view(np.uint16)
    assert comp_err(got, oracle.sddmm(rp, ci, Aq, Bq, None, fmt_a="bf16", fmt_b="bf16"),
                    oracle.sddmm(rp, ci, Aq, Bq, None, fmt_a="bf16", fmt_b="bf16", absmode=True)) <= TOL
    assert int(P.arrays()["status"].cpu()[0]) == 0
