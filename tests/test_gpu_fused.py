"""FusedMM (SDDMM cascaded into SpMM, per head, optional row softmax) on the
GPU against the oracle: outputs, scores and row log-sum-exp, split rows,
empty rows, heads, dtypes, determinism."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, comp_err, edge_pattern

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def spk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2404_19638_gb300 as m
    return m


def _case(M, N, K, seed, long_row=2500):
    rp, ci = edge_pattern(M, N, seed, long_row=long_row)
    g = np.random.default_rng(seed)
    vals = g.uniform(0.5, 1.5, ci.size).astype(np.float32)
    A = g.standard_normal((M, K)).astype(np.float32)
    B = g.standard_normal((N, K)).astype(np.float32)
    return rp, ci, vals, A, B


def _check(spk, rp, ci, vals, A, B, heads, softmax, dt, W, seed_note="", tune=None):
    M, K = A.shape
    N = B.shape[0]
    scale = 1.0 / np.sqrt(K // heads)
    S = spk.CSR(rp, ci, (M, N), torch.from_numpy(vals), device=DEV, chunk_work=W)
    if dt == torch.float32:
        tA, tB = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
        Aq, Bq, fmt = A, B, None
    else:
        tA = spk.cast(torch.from_numpy(A).to(DEV), dt)
        tB = spk.cast(torch.from_numpy(B).to(DEV), dt)
        fmt = "bf16" if dt == torch.bfloat16 else "f16"
        Aq = tA.view(torch.int16).cpu().numpy().view(np.uint16)
        Bq = tB.view(torch.int16).cpu().numpy().view(np.uint16)
    Y, sc, lse = spk.fusedmm(S, tA, tB, heads=heads, scale=scale, softmax=softmax, want_scores=True, want_lse=True,
                             tune=tune)
    Yr, scr, lser = oracle.fusedmm(rp, ci, Aq, Bq, vals, heads=heads, scale=scale, softmax=softmax,
                                   fmt_a=fmt, fmt_b=fmt)
    Ya, _, _ = oracle.fusedmm(rp, ci, Aq, Bq, vals, heads=heads, scale=scale, softmax=softmax, fmt_a=fmt, fmt_b=fmt,
                              absmode=True)
    assert comp_err(Y.cpu().numpy(), Yr, Ya) <= TOL, seed_note
    # scores: each is one head's SDDMM, scaled
    D = K // heads
    for h in range(heads):
        den = np.abs(scale) * oracle.sddmm(rp, ci, Aq[:, h * D:(h + 1) * D], Bq[:, h * D:(h + 1) * D], vals,
                                           fmt_a=fmt, fmt_b=fmt, absmode=True)
        assert comp_err(sc[h].cpu().numpy(), scr[h], den) <= TOL, seed_note
    if softmax:
        got = lse.cpu().numpy()
        fin = np.isfinite(lser)
        assert np.array_equal(np.isfinite(got), fin)
        assert np.max(np.abs(got[fin] - lser[fin]) / (1.0 + np.abs(lser[fin])), initial=0.0) <= 1e-5
    # deterministic (split rows are merged in a fixed order)
    Y2, sc2, _ = spk.fusedmm(S, tA, tB, heads=heads, scale=scale, softmax=softmax, want_scores=True, tune=tune)
    assert torch.equal(Y, Y2) and torch.equal(sc, sc2)
    return S


@pytest.mark.parametrize("K,heads", [(16, 1), (16, 4), (32, 2), (64, 1), (64, 4), (128, 2), (256, 1)])
@pytest.mark.parametrize("softmax", [False, True])
def test_fused_f32(spk, K, heads, softmax):
    rp, ci, vals, A, B = _case(600, 450, K, seed=K + heads)
    _check(spk, rp, ci, vals, A, B, heads, softmax, torch.float32, W=128, seed_note=f"K={K} H={heads}")


@pytest.mark.parametrize("shape", [(4, 1, 4), (8, 1, 4), (16, 1, 4), (32, 1, 8), (32, 2, 4), (8, 2, 4), (4, 2, 4)])
def test_fused_head_per_grid_row(spk, shape):
    """The kernel with one head per grid row (used for rows of more than 32
    vectors, or when a shape is asked for)."""
    G, NV, U = shape
    K = 4 * G * NV
    for heads in (1, 2):
        rp, ci, vals, A, B = _case(400, 350, K * heads, seed=G + NV + heads)
        _check(spk, rp, ci, vals, A, B, heads, heads == 2, torch.float32, W=64,
               tune={"group_lanes": G, "vecs_per_lane": NV, "unroll": U})


def _lane_splits():
    """(dtype, vectors a lane, K, heads) whose rows split into a compiled lane
    width: 4-32 lanes (at most 16 with two vectors a lane), whole heads per lane."""
    out = []
    for dt in (torch.float32, torch.bfloat16):
        vecn = 4 if dt == torch.float32 else 8
        for nv_lane in (1, 2):
            for K, heads in ((32, 1), (64, 2), (64, 4), (128, 4)):
                nv = K // vecn
                G = nv // nv_lane
                if nv % nv_lane == 0 and G in (4, 8, 16, 32) and not (nv_lane == 2 and G == 32) and G % heads == 0:
                    name = f"{'f32' if dt == torch.float32 else 'bf16'}-nv{nv_lane}-K{K}-h{heads}"
                    out.append(pytest.param(dt, nv_lane, K, heads, id=name))
    return out


@pytest.mark.parametrize("dt,nv_lane,K,heads", _lane_splits())
def test_fused_all_heads_vectors_per_lane(spk, dt, nv_lane, K, heads):
    """The all-heads kernel with one or two adjacent 16-byte vectors a lane
    (tune.vecs_per_lane alone), with and without softmax, split rows included."""
    rp, ci, vals, A, B = _case(500, 420, K, seed=5 * K + heads + nv_lane)
    for softmax in (False, True):
        _check(spk, rp, ci, vals, A, B, heads, softmax, dt, W=64, tune={"vecs_per_lane": nv_lane})


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("K,heads", [(64, 1), (64, 8), (128, 2)])
def test_fused_low_precision(spk, dt, K, heads):
    rp, ci, vals, A, B = _case(500, 400, K, seed=3 * K + heads)
    for softmax in (False, True):
        _check(spk, rp, ci, vals, A, B, heads, softmax, dt, W=96)


@pytest.mark.parametrize("W", [32, 64, 512, 4096])
def test_fused_split_rows(spk, W):
    """Long rows cut into many pieces: the softmax merge of the pieces."""
    rp, ci, vals, A, B = _case(300, 30000, 32, seed=W, long_row=20000)
    S = _check(spk, rp, ci, vals, A, B, 2, True, torch.float32, W=W)
    if W <= 512:
        assert S.schedule_info()["npieces"] > 0


def test_fused_edges(spk):
    K = 16
    # nnz = 0: Y = 0, lse = -inf
    rp = np.zeros(41, np.int32); ci = np.zeros(0, np.int32)
    S = spk.CSR(rp, ci, (40, 30), device=DEV, chunk_work=32)
    A = torch.randn(40, K, device=DEV); B = torch.randn(30, K, device=DEV)
    Y, sc, lse = spk.fusedmm(S, A, B, heads=2, softmax=True, want_scores=True, want_lse=True)
    assert torch.count_nonzero(Y) == 0 and torch.all(torch.isneginf(lse)) and sc.numel() == 0
    # one nonzero per row with softmax: Y = the neighbour's row exactly
    M, N = 64, 50
    g = np.random.default_rng(8)
    ci = g.integers(0, N, M).astype(np.int32)
    rp = np.arange(M + 1, dtype=np.int32)
    S = spk.CSR(rp, ci, (M, N), device=DEV, chunk_work=32)
    A = torch.randn(M, K, device=DEV); B = torch.randn(N, K, device=DEV)
    Y, _, _ = spk.fusedmm(S, A, B, softmax=True)
    assert torch.equal(Y, B[torch.from_numpy(ci).long().to(DEV)])
    # unsupported head width is rejected before any launch
    with pytest.raises(spk.SpkError):
        spk.fusedmm(S, A, B, heads=8)          # dh = 2 floats: not a 16-byte vector
