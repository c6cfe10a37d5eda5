"""Differentiable FusedMM on the GPU against the oracle's finite-difference
pinned chain rule: the three elementwise kernels of the backward one by one,
then dA and dB end to end for FP32 and BF16 factors, with and without the row
softmax, one and several heads; every output componentwise."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, comp_err, edge_pattern, row_of

pytestmark = pytest.mark.gpu
DEV = "cuda"

# End-to-end gradients, componentwise like every other output: each entry of
# dA / dB is compared with the oracle's chain rule relative to the sum of the
# magnitudes of the terms that form it (oracle.fusedmm_grad with absmode: the
# same chain rule over |A|, |B|, |dY|, |w|, |dw|, the softmax row term as
# sum |w| |dw|, and a softmax weight's magnitude widened by its exponent's).
# Softmax score gradients sum to zero over a row, so an entry can cancel far
# below its terms; the denominator does not cancel.  FP32: 1e-5.  BF16 dH =
# dA + dB: each written in BF16 and summed in BF16, three roundings of at
# most 2^-8 of quantities bounded by the denominator, two of them disjoint.
GRAD_TOL = TOL
GRAD_TOL_16 = 2 * 2.0 ** -8 + TOL
# The normwise check below is kept as a second, coarser view.
NORM_TOL = 1e-4


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
    A = (0.5 * g.standard_normal((M, K))).astype(np.float32)
    B = (0.5 * g.standard_normal((N, K))).astype(np.float32)
    dY = g.standard_normal((M, K)).astype(np.float32)
    return rp, ci, vals, A, B, dY


def _normwise(got, ref):
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(np.asarray(got, np.float64) - ref)) / max(np.max(np.abs(ref)), 1e-300))


def test_weights_kernel(spk):
    rp, ci, vals, A, B, _ = _case(500, 400, 24, seed=1)
    S = spk.CSR(rp, ci, (500, 400), device=DEV)
    _, sc, lse = oracle.fusedmm(rp, ci, A, B, vals, heads=3, scale=0.5, softmax=True)
    sc32, lse32 = sc.astype(np.float32), lse.astype(np.float32)
    w = spk.ops.fused_weights(S, torch.from_numpy(sc32).to(DEV), torch.from_numpy(lse32).to(DEV), 3, True)
    rows = row_of(rp)
    ref = np.exp(sc32.astype(np.float64) - lse32.astype(np.float64)[rows].T)
    # exp of an exactly representable FP32 difference: a few ulps of the result
    # plus one rounding of the difference, scaled by the exponent's argument
    den = ref * (1.0 + np.abs(sc32.astype(np.float64) - lse32.astype(np.float64)[rows].T))
    assert comp_err(w.cpu().numpy(), ref, den) <= TOL
    # without softmax the weights are the scores themselves
    w0 = spk.ops.fused_weights(S, torch.from_numpy(sc32).to(DEV), None, 3, False)
    assert np.array_equal(w0.cpu().numpy(), sc32)


def test_rowdot_kernel(spk):
    g = np.random.default_rng(2)
    # 16-byte path (head width a multiple of 4) and scalar path (3, 5, 9 columns)
    for (M, K, heads) in [(1, 4, 1), (333, 96, 3), (1000, 64, 4), (77, 40, 5), (50, 9, 3), (64, 25, 5), (5, 9, 1)]:
        dY = g.standard_normal((M, K)).astype(np.float32)
        Y = g.standard_normal((M, K)).astype(np.float32)
        R = spk.ops.fused_rowdot(torch.from_numpy(dY).to(DEV), torch.from_numpy(Y).to(DEV), heads).cpu().numpy()
        Kh = K // heads
        p = dY.astype(np.float64) * Y.astype(np.float64)
        ref = p.reshape(M, heads, Kh).sum(axis=2)
        den = np.abs(p).reshape(M, heads, Kh).sum(axis=2)
        assert comp_err(R, ref, den) <= TOL
    # a strided dY (a column block of a wider tensor)
    W = torch.from_numpy(g.standard_normal((50, 64)).astype(np.float32)).to(DEV)
    Y = torch.from_numpy(g.standard_normal((50, 32)).astype(np.float32)).to(DEV)
    R = spk.ops.fused_rowdot(W[:, 16:48], Y, 2).cpu().numpy()
    p = W[:, 16:48].double().cpu().numpy() * Y.double().cpu().numpy()
    assert comp_err(R, p.reshape(50, 2, 16).sum(2), np.abs(p).reshape(50, 2, 16).sum(2)) <= TOL
    # a 4-byte-aligned column offset falls back to scalar loads
    R = spk.ops.fused_rowdot(W[:, 1:13], Y[:, :12], 3).cpu().numpy()
    p = W[:, 1:13].double().cpu().numpy() * Y[:, :12].double().cpu().numpy()
    assert comp_err(R, p.reshape(50, 3, 4).sum(2), np.abs(p).reshape(50, 3, 4).sum(2)) <= TOL
    # M = 0 is a no-op
    E = torch.empty((0, 8), device=DEV)
    assert spk.ops.fused_rowdot(E, E, 2).shape == (0, 2)


@pytest.mark.parametrize("softmax", [False, True])
def test_score_grad_kernel(spk, softmax):
    rp, ci, _, _, _, _ = _case(400, 300, 8, seed=3)
    S = spk.CSR(rp, ci, (400, 300), device=DEV)
    g = np.random.default_rng(4)
    heads, nnz = 2, ci.size
    w = g.uniform(0, 1, (heads, nnz)).astype(np.float32)
    dw = g.standard_normal((heads, nnz)).astype(np.float32)
    R = g.standard_normal((400, heads)).astype(np.float32)
    s = g.uniform(-2, 2, nnz).astype(np.float32)
    rows = row_of(rp)
    w64, dw64, R64 = w.astype(np.float64), dw.astype(np.float64), R.astype(np.float64)[rows].T
    for vals in (None, s):
        de = spk.ops.fused_score_grad(S, torch.from_numpy(w).to(DEV), torch.from_numpy(dw).to(DEV),
                                      torch.from_numpy(R).to(DEV), heads, softmax, 0.3,
                                      None if vals is None else torch.from_numpy(vals).to(DEV)).cpu().numpy()
        s64 = 1.0 if vals is None else vals.astype(np.float64)
        if softmax:
            ref = 0.3 * s64 * w64 * (dw64 - R64)
            den = np.abs(0.3 * s64) * w64 * (np.abs(dw64) + np.abs(R64))
        else:
            ref = 0.3 * s64 * dw64
            den = np.abs(ref)
        assert comp_err(de, ref, den) <= TOL


@pytest.mark.parametrize("heads,softmax", [(1, False), (1, True), (2, True), (4, True), (4, False), (3, True)])
def test_fusedmm_grad_f32(spk, heads, softmax):
    # heads 2 and 4 take the multi-head dw SDDMM; 3 heads (K = 48) have no
    # multi-head kernel and take one SDDMM per head
    M, N, K = 600, 450, 16 * heads
    rp, ci, vals, A, B, dY = _case(M, N, K, seed=10 + heads + 5 * softmax)
    scale = 1.0 / np.sqrt(K // heads)
    S = spk.CSR(rp, ci, (M, N), torch.from_numpy(vals), device=DEV)
    tA = torch.from_numpy(A).to(DEV).requires_grad_()
    tB = torch.from_numpy(B).to(DEV).requires_grad_()
    Y = spk.autograd.fusedmm(S, tA, tB, S.vals, heads=heads, scale=scale, softmax=softmax)
    Yr, _, _ = oracle.fusedmm(rp, ci, A, B, vals, heads=heads, scale=scale, softmax=softmax)
    Ya, _, _ = oracle.fusedmm(rp, ci, A, B, vals, heads=heads, scale=scale, softmax=softmax, absmode=True)
    assert comp_err(Y.detach().cpu().numpy(), Yr, Ya) <= TOL
    Y.backward(torch.from_numpy(dY).to(DEV))
    dA, dB = oracle.fusedmm_grad(rp, ci, A, B, dY, vals, heads=heads, scale=scale, softmax=softmax)
    dA_den, dB_den = oracle.fusedmm_grad(rp, ci, A, B, dY, vals, heads=heads, scale=scale, softmax=softmax,
                                         absmode=True)
    assert comp_err(tA.grad.cpu().numpy(), dA, dA_den) <= GRAD_TOL
    assert comp_err(tB.grad.cpu().numpy(), dB, dB_den) <= GRAD_TOL
    assert _normwise(tA.grad.cpu().numpy(), dA) <= NORM_TOL
    assert _normwise(tB.grad.cpu().numpy(), dB) <= NORM_TOL
    empty = np.flatnonzero(np.diff(rp) == 0)
    assert np.all(tA.grad.cpu().numpy()[empty] == 0.0)


@pytest.mark.parametrize("softmax", [False, True])
def test_fusedmm_grad_bf16_shared_operand(spk, softmax):
    """A = B = H in BF16 (a square pattern): dH = dA + dB, each written in BF16."""
    M, K, heads = 500, 32, 2
    rp, ci, vals, H, _, dY = _case(M, M, K, seed=21 + softmax)
    S = spk.CSR(rp, ci, (M, M), torch.from_numpy(vals), device=DEV)
    tH = spk.cast(torch.from_numpy(H).to(DEV), torch.bfloat16).requires_grad_()
    Hq = tH.detach().view(torch.int16).cpu().numpy().view(np.uint16)
    Y = spk.autograd.fusedmm(S, tH, tH, S.vals, heads=heads, scale=0.25, softmax=softmax)
    Y.backward(torch.from_numpy(dY).to(DEV))
    dA, dB = oracle.fusedmm_grad(rp, ci, Hq, Hq, dY, vals, heads=heads, scale=0.25, softmax=softmax, fmt="bf16")
    dA_den, dB_den = oracle.fusedmm_grad(rp, ci, Hq, Hq, dY, vals, heads=heads, scale=0.25, softmax=softmax,
                                         fmt="bf16", absmode=True)
    assert tH.grad.dtype == torch.bfloat16
    assert comp_err(tH.grad.float().cpu().numpy(), dA + dB, dA_den + dB_den) <= GRAD_TOL_16
    assert _normwise(tH.grad.float().cpu().numpy(), dA + dB) <= 2 * (2.0 ** -8 + NORM_TOL)


def test_fusedmm_grad_matches_unfused_composition(spk):
    """Without softmax, FusedMM is SpMM(S_e, B) with e = scale * SDDMM(S, A, B):
    the fused layer's gradients equal those of the composed primitives."""
    M, N, K = 400, 380, 32
    rp, ci, vals, A, B, dY = _case(M, N, K, seed=31)
    S = spk.CSR(rp, ci, (M, N), torch.from_numpy(vals), device=DEV)
    a1 = torch.from_numpy(A).to(DEV).requires_grad_(); b1 = torch.from_numpy(B).to(DEV).requires_grad_()
    spk.autograd.fusedmm(S, a1, b1, S.vals, scale=0.5).backward(torch.from_numpy(dY).to(DEV))
    a2 = torch.from_numpy(A).to(DEV).requires_grad_(); b2 = torch.from_numpy(B).to(DEV).requires_grad_()
    e = spk.autograd.sddmm(S, a2, b2, S.vals * 0.5)
    spk.autograd.spmm(S, b2, e).backward(torch.from_numpy(dY).to(DEV))
    dA_den, dB_den = oracle.fusedmm_grad(rp, ci, A, B, dY, vals, scale=0.5, absmode=True)
    dA, dB = oracle.fusedmm_grad(rp, ci, A, B, dY, vals, scale=0.5)
    for x, y, ref, den in ((a1.grad, a2.grad, dA, dA_den), (b1.grad, b2.grad, dB, dB_den)):
        # both against the oracle, and to each other at twice that
        assert comp_err(x.cpu().numpy(), ref, den) <= GRAD_TOL
        assert comp_err(y.cpu().numpy(), ref, den) <= GRAD_TOL
        assert comp_err(x.cpu().numpy(), y.double().cpu().numpy(), den) <= 2 * GRAD_TOL
        assert _normwise(x.cpu().numpy(), y.double().cpu().numpy()) <= NORM_TOL


@pytest.mark.parametrize("heads,K,dt", [(4, 64, torch.float32), (2, 32, torch.float32), (3, 24, torch.float32),
                                        (4, 128, torch.float32), (4, 64, torch.bfloat16), (8, 256, torch.float32)])
def test_multi_head_spmm_and_spmm_t(spk, heads, K, dt):
    """One pass for all heads: C[:, head h] = S_h B[:, head h] and
    X[:, head h] = S_h^T Y[:, head h], each head with its own values, against
    the oracle head by head (componentwise, FP32 accumulation)."""
    M, N = 700, 520
    rp, ci = edge_pattern(M, N, seed=61 + heads + K, long_row=2200)
    g = np.random.default_rng(K + heads)
    S = spk.CSR(rp, ci, (M, N), device=DEV, chunk_work=128)
    V = g.uniform(-1, 1, (heads, ci.size)).astype(np.float32)
    B = g.standard_normal((N, K)).astype(np.float32)
    Y = g.standard_normal((M, K)).astype(np.float32)
    tB = torch.from_numpy(B).to(DEV).to(dt)
    tY = torch.from_numpy(Y).to(DEV).to(dt)
    tV = torch.from_numpy(V).to(DEV)
    C = spk.ops.spmm_mh(S, tB, tV, heads).cpu().numpy()
    X = spk.ops.spmm_t_mh(S, tY, tV, heads).cpu().numpy()
    if dt == torch.bfloat16:
        Bo, Yo, kb, ky = (tB.view(torch.int16).cpu().numpy().view(np.uint16),
                          tY.view(torch.int16).cpu().numpy().view(np.uint16), {"fmt_b": "bf16"}, {"fmt_y": "bf16"})
    else:
        Bo, Yo, kb, ky = B, Y, {}, {}
    Kh = K // heads
    for h in range(heads):
        sl = slice(h * Kh, (h + 1) * Kh)
        Bh, Yh = np.ascontiguousarray(Bo[:, sl]), np.ascontiguousarray(Yo[:, sl])
        assert comp_err(C[:, sl], oracle.spmm(rp, ci, Bh, V[h], **kb),
                        oracle.spmm(rp, ci, Bh, V[h], absmode=True, **kb)) <= TOL
        assert comp_err(X[:, sl], oracle.spmm_t(rp, ci, N, Yh, V[h], **ky),
                        oracle.spmm_t(rp, ci, N, Yh, V[h], absmode=True, **ky)) <= TOL
    # accumulate mode adds onto the output
    base = torch.from_numpy(g.standard_normal((M, K)).astype(np.float32)).to(DEV)
    acc = base.clone()
    spk.ops.spmm_mh(S, tB, tV, heads, out=acc, accumulate=True)
    np.testing.assert_allclose(acc.cpu().numpy(), base.cpu().numpy() + C, rtol=1e-6, atol=1e-5)


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("K,heads", [(64, 2), (64, 4), (64, 8), (128, 4), (32, 2), (128, 8)])
def test_sddmm_heads_one_pass(spk, dt, K, heads):
    """SDDMM in heads (spk_sddmm_mh): each head's slice against the oracle's
    SDDMM of that slice at the component-wise gate, with and without values,
    split rows included; where no multi-head kernel covers K the call is
    refused with SpkError and nothing else."""
    from paper_2404_19638_gb300 import ops
    rp, ci = edge_pattern(700, 600, 5 * K + heads, long_row=2500)
    g = np.random.default_rng(K + heads)
    vals = g.uniform(-1, 1, ci.size).astype(np.float32)
    S = spk.CSR(rp, ci, (700, 600), torch.from_numpy(vals), device=DEV, chunk_work=64)
    A = torch.from_numpy(g.standard_normal((700, K)).astype(np.float32)).to(DEV)
    B = torch.from_numpy(g.standard_normal((600, K)).astype(np.float32)).to(DEV)
    fmt = None
    if dt == torch.bfloat16:
        A, B = spk.cast(A, dt), spk.cast(B, dt)
        fmt = "bf16"
    Aq = A.float().cpu().numpy() if fmt is None else A.view(torch.int16).cpu().numpy().view(np.uint16)
    Bq = B.float().cpu().numpy() if fmt is None else B.view(torch.int16).cpu().numpy().view(np.uint16)
    vecn = 4 if dt == torch.float32 else 8
    covered = (dt == torch.float32 and K in (32, 64, 128)) or (dt == torch.bfloat16 and K in (64, 128))
    if not covered or (K // heads) % vecn:
        with pytest.raises(spk.SpkError):
            ops.sddmm_mh(S, A, B, heads)
        return
    dh = K // heads
    for v in (None, S.vals):
        got = ops.sddmm_mh(S, A, B, heads, vals=v).cpu().numpy()
        vv = None if v is None else vals
        for h in range(heads):
            ref = oracle.sddmm(rp, ci, Aq[:, h * dh:(h + 1) * dh], Bq[:, h * dh:(h + 1) * dh], vv, fmt_a=fmt, fmt_b=fmt)
            den = oracle.sddmm(rp, ci, Aq[:, h * dh:(h + 1) * dh], Bq[:, h * dh:(h + 1) * dh], vv, fmt_a=fmt,
                               fmt_b=fmt, absmode=True)
            assert comp_err(got[h], ref, den) <= TOL, (K, heads, h)
