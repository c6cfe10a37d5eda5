"""Pins for the FP64 oracle, against things other than the oracle itself.

Each check is chosen so that a plausible slip in ``oracle/oracle.c`` (a dropped
scale, a swapped index, a transposed operand, a wrong tie rule) fails it:
  * a hand-worked example (tests/golden/worked_3x4.json),
  * dense brute force with numpy's FP64 matmul (Sec. 3.2, Eq. 1 and Eq. 2),
  * the adjoint identity  sum SDDMM(S,A,B) = sum A.SpMM(S,B) = trace(A^T S B),
  * exact integer arithmetic in pure Python on tiny inputs,
  * special cases (identity, permutation, all-ones, K = 1, nnz = 0),
  * library routines for the formats (torch bfloat16 / float8, numpy float16)
    and for the transpose (scipy CSR -> CSC),
  * an explicitly materialised merge for the merge-path split,
  * finite differences for the closed-form gradients.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense(rowptr, colidx, vals, M, N):
    S = np.zeros((M, N))
    for i in range(M):
        for e in range(rowptr[i], rowptr[i + 1]):
            S[i, colidx[e]] += 1.0 if vals is None else vals[e]
    return S


def random_case(M, N, K, density, seed, empty_rows=True):
    g = np.random.default_rng(seed)
    mask = g.random((M, N)) < density
    if empty_rows and M > 3:
        mask[1] = False
        mask[M - 1] = False
    rows, cols = np.nonzero(mask)
    rp, ci = synth.csr_from_coo(rows, cols, M, N)
    vals = g.uniform(-1, 1, ci.size).astype(np.float32)
    A = g.standard_normal((M, K)).astype(np.float32)
    B = g.standard_normal((N, K)).astype(np.float32)
    return rp, ci, vals, A, B


# ----------------------------------------------------------------------------
# Hand-worked example
# ----------------------------------------------------------------------------

def test_worked_example():
    w = json.load(open(os.path.join(GOLDEN, "worked_3x4.json")))
    rp = np.array(w["rowptr"], np.int32); ci = np.array(w["colidx"], np.int32)
    vals = np.array(w["vals"]); A = np.array(w["A"], np.float32); B = np.array(w["B"], np.float32)
    assert np.array_equal(oracle.sddmm(rp, ci, A, B, vals), w["sddmm"])
    assert np.array_equal(oracle.spmm(rp, ci, B, vals), w["spmm"])
    assert np.array_equal(oracle.spmm_t(rp, ci, w["N"], A, vals), w["spmm_t_of_A"])
    assert oracle.sddmm(rp, ci, A, B, vals).sum() == w["adjoint_sum"]


# ----------------------------------------------------------------------------
# Brute force against dense FP64 matmul
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("M,N,K", [(17, 23, 1), (40, 31, 8), (33, 64, 24), (64, 40, 65)])
def test_sddmm_dense_bruteforce(M, N, K):
    rp, ci, vals, A, B = random_case(M, N, K, 0.2, seed=M * N + K)
    got = oracle.sddmm(rp, ci, A, B, vals)
    full = A.astype(np.float64) @ B.astype(np.float64).T
    rows = np.repeat(np.arange(M), np.diff(rp))
    want = vals.astype(np.float64) * full[rows, ci]
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("M,N,K", [(17, 23, 1), (40, 31, 8), (33, 64, 24), (64, 40, 65)])
def test_spmm_dense_bruteforce(M, N, K):
    rp, ci, vals, A, B = random_case(M, N, K, 0.2, seed=M + N + K)
    got = oracle.spmm(rp, ci, B, vals)
    want = dense(rp, ci, vals, M, N) @ B.astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
    # sampled rows give the same rows
    rows = np.array([M - 1, 0, 5])
    np.testing.assert_allclose(oracle.spmm(rp, ci, B, vals, rows=rows), want[rows], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("M,N,K", [(17, 23, 3), (40, 31, 16)])
def test_spmm_t_dense_bruteforce(M, N, K):
    rp, ci, vals, A, B = random_case(M, N, K, 0.25, seed=7 * M + N)
    Y = A
    got = oracle.spmm_t(rp, ci, N, Y, vals)
    want = dense(rp, ci, vals, M, N).T @ Y.astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
    cols = np.array([N - 1, 2, 0])
    np.testing.assert_allclose(oracle.spmm_t(rp, ci, N, Y, vals, cols=cols), want[cols], rtol=1e-13, atol=1e-13)


def test_absmode_is_sum_of_magnitudes():
    M, N, K = 20, 30, 6
    rp, ci, vals, A, B = random_case(M, N, K, 0.3, seed=3)
    Aa, Ba = np.abs(A.astype(np.float64)), np.abs(B.astype(np.float64))
    rows = np.repeat(np.arange(M), np.diff(rp))
    want = np.abs(vals) * (Aa @ Ba.T)[rows, ci]
    np.testing.assert_allclose(oracle.sddmm(rp, ci, A, B, vals, absmode=True), want, rtol=1e-13)
    want2 = np.abs(dense(rp, ci, vals, M, N)) @ Ba
    np.testing.assert_allclose(oracle.spmm(rp, ci, B, vals, absmode=True), want2, rtol=1e-13)


# ----------------------------------------------------------------------------
# Adjoint identity and exact integer arithmetic
# ----------------------------------------------------------------------------

def test_adjoint_identity():
    M, N, K = 50, 70, 12
    rp, ci, vals, A, B = random_case(M, N, K, 0.15, seed=11)
    s1 = oracle.sddmm(rp, ci, A, B, vals).sum()
    s2 = (A.astype(np.float64) * oracle.spmm(rp, ci, B, vals)).sum()
    s3 = np.trace(A.astype(np.float64).T @ dense(rp, ci, vals, M, N) @ B.astype(np.float64))
    s4 = (B.astype(np.float64) * oracle.spmm_t(rp, ci, N, A, vals)).sum()
    assert abs(s1 - s2) < 1e-10 and abs(s1 - s3) < 1e-10 and abs(s1 - s4) < 1e-10


def test_integer_exact_against_python_ints():
    g = np.random.default_rng(5)
    M, N, K = 9, 11, 5
    mask = g.random((M, N)) < 0.4
    rows, cols = np.nonzero(mask)
    rp, ci = synth.csr_from_coo(rows, cols, M, N)
    vals = g.integers(-3, 4, ci.size)
    A = g.integers(-3, 4, (M, K)); B = g.integers(-3, 4, (N, K))
    got = oracle.sddmm(rp, ci, A.astype(np.float32), B.astype(np.float32), vals)
    gotC = oracle.spmm(rp, ci, B.astype(np.float32), vals)
    for i in range(M):
        Ci = [0] * K
        for e in range(rp[i], rp[i + 1]):
            j = int(ci[e])
            dot = sum(int(A[i, k]) * int(B[j, k]) for k in range(K))
            assert got[e] == int(vals[e]) * dot
            for k in range(K):
                Ci[k] += int(vals[e]) * int(B[j, k])
        assert list(gotC[i]) == Ci


# ----------------------------------------------------------------------------
# Special cases
# ----------------------------------------------------------------------------

def test_identity_permutation_allones_k1_empty():
    g = np.random.default_rng(2)
    n, K = 16, 4
    A = g.standard_normal((n, K)).astype(np.float32)
    B = g.standard_normal((n, K)).astype(np.float32)
    # S = I: SDDMM = rowwise <a_i, b_i>, SpMM = B
    rp = np.arange(n + 1, dtype=np.int32); ci = np.arange(n, dtype=np.int32)
    np.testing.assert_allclose(oracle.sddmm(rp, ci, A, B), (A.astype(np.float64) * B).sum(1), rtol=1e-14)
    assert np.array_equal(oracle.spmm(rp, ci, B), B.astype(np.float64))
    # permutation: SpMM permutes the rows of B
    p = g.permutation(n).astype(np.int32)
    assert np.array_equal(oracle.spmm(rp, p, B), B[p].astype(np.float64))
    # all-ones dense S: SDDMM = the full product, SpMM = column sums of B
    m = 5
    rp1 = (np.arange(m + 1) * n).astype(np.int32); ci1 = np.tile(np.arange(n, dtype=np.int32), m)
    full = A[:m].astype(np.float64) @ B.astype(np.float64).T
    np.testing.assert_allclose(oracle.sddmm(rp1, ci1, A[:m], B), full.reshape(-1), rtol=1e-13)
    np.testing.assert_allclose(oracle.spmm(rp1, ci1, B), np.tile(B.astype(np.float64).sum(0), (m, 1)), rtol=1e-13)
    # K = 1: masked outer product
    a1, b1 = A[:, :1], B[:, :1]
    rows = np.repeat(np.arange(m), n)
    np.testing.assert_allclose(oracle.sddmm(rp1, ci1, a1[:m], b1), a1[rows, 0].astype(np.float64) * b1[ci1, 0], rtol=1e-15)
    # nnz = 0: SpMM writes zeros, SDDMM writes nothing
    rp0 = np.zeros(n + 1, np.int32); ci0 = np.zeros(0, np.int32)
    assert np.array_equal(oracle.spmm(rp0, ci0, B), np.zeros((n, K)))
    assert oracle.sddmm(rp0, ci0, A, B).size == 0


def test_duplicates_sum():
    # duplicates in a row are independent entries: SpMM sums them
    rp = np.array([0, 3], np.int32); ci = np.array([1, 1, 0], np.int32)
    B = np.array([[1.0, 2.0], [3.0, 4.0]], np.float32)
    vals = np.array([1.0, 2.0, -1.0])
    assert np.array_equal(oracle.spmm(rp, ci, B, vals), [[8.0, 10.0]])


# ----------------------------------------------------------------------------
# Number formats
# ----------------------------------------------------------------------------

def test_e4m3_published_points():
    pts = json.load(open(os.path.join(GOLDEN, "e4m3_points.json")))
    for p in pts["points"]:
        assert oracle.decode([p["code"]], "e4m3")[0] == p["value"], p
    for c in pts["nan_codes"]:
        assert np.isnan(oracle.decode([c], "e4m3")[0])


def test_e4m3_table_closed_form():
    tab = oracle.decode_table("e4m3")
    for q in range(256):
        s, e, m = q >> 7, (q >> 3) & 15, q & 7
        if e == 15 and m == 7:
            assert np.isnan(tab[q]); continue
        v = (m / 8) * 2.0 ** -6 if e == 0 else (1 + m / 8) * 2.0 ** (e - 7)
        assert tab[q] == (-v if s else v)


def test_e4m3_encoder_against_torch_and_rules():
    torch = pytest.importorskip("torch")
    tab = oracle.decode_table("e4m3")
    finite = [q for q in range(256) if not np.isnan(tab[q])]
    # every representable value encodes to itself (both zeros keep their sign)
    vals = np.array([tab[q] for q in finite], np.float32)
    assert np.array_equal(oracle.encode(vals, "e4m3"), np.array(finite, np.uint8))
    # random in-range values: torch's RNE float8_e4m3fn cast (a library routine)
    g = np.random.default_rng(0)
    x = np.concatenate([g.uniform(-448, 448, 20000), g.standard_normal(20000),
                        g.standard_normal(5000) * 1e-3]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(oracle.encode(x, "e4m3"), want)
    # midpoints tie to the even code; saturation to 448 past the top
    mid = np.float32((tab[56] + tab[57]) / 2)      # between 1.0 and 1.125 -> 1.0 (even)
    assert oracle.encode([mid], "e4m3")[0] == 56
    mid = np.float32((tab[57] + tab[58]) / 2)      # between 1.125 and 1.25 -> 1.25 (even)
    assert oracle.encode([mid], "e4m3")[0] == 58
    assert list(oracle.encode(np.array([449.0, 1e6, -500.0], np.float32), "e4m3")) == [126, 126, 254]


def test_bf16_f16_encoders_against_libraries():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(1)
    x = np.concatenate([g.standard_normal(50000) * 10.0 ** g.integers(-30, 30, 50000),
                        [0.0, -0.0, 1.0, 65504.0, 65520.0, 1e-8, 3.3961e38, 3.4e38]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(oracle.encode(x, "bf16"), want)
    with np.errstate(over="ignore"):                 # values past 65520 are meant to round to inf
        want16 = x.astype(np.float16).view(np.uint16)
    assert np.array_equal(oracle.encode(x, "f16"), want16)
    # decoders agree with the library casts on every code
    codes = np.arange(65536, dtype=np.uint16)
    tb = oracle.decode_table("bf16"); th = oracle.decode_table("f16")
    lb = torch.from_numpy(codes.view(np.int16)).view(torch.bfloat16).double().numpy()
    lh = codes.view(np.float16).astype(np.float64)
    assert np.array_equal(np.isnan(tb), np.isnan(lb)) and np.array_equal(tb[~np.isnan(tb)], lb[~np.isnan(lb)])
    assert np.array_equal(np.isnan(th), np.isnan(lh)) and np.array_equal(th[~np.isnan(th)], lh[~np.isnan(lh)])


def test_quantize_e4m3_rows_rules():
    g = np.random.default_rng(4)
    X = g.standard_normal((64, 40)).astype(np.float32)
    X[3] = 0.0
    codes, scales = oracle.quantize_e4m3_rows(X)
    amax = np.abs(X).max(1)
    assert scales[3] == 1.0 and np.all(codes[3] == 0)
    nz = amax > 0
    assert np.array_equal(scales[nz], (amax[nz] / np.float32(448.0)).astype(np.float32))
    # the largest-magnitude element of each row maps to +-448
    arg = np.abs(X).argmax(1)
    top = codes[np.arange(64), arg]
    assert np.all((top[nz] & 0x7F) == 126)
    # dequantised values are within half an E4M3 step (relative 2^-4) of x
    deq = oracle.dequantize(codes, "e4m3", scales)
    big = np.abs(X) > scales[:, None] * 2.0 ** -6
    rel = np.abs(deq - X)[big] / np.abs(X)[big]
    assert rel.max() <= 2.0 ** -4 + 1e-7
    # same as encoding x / scale element by element
    q = (X / scales[:, None]).astype(np.float32)
    assert np.array_equal(codes, oracle.encode(q, "e4m3"))


def test_low_precision_operands_use_dequantised_values():
    M, N, K = 12, 15, 16
    rp, ci, vals, A, B = random_case(M, N, K, 0.3, seed=8)
    qa, sa = oracle.quantize_e4m3_rows(A); qb, sb = oracle.quantize_e4m3_rows(B)
    got = oracle.sddmm(rp, ci, qa, qb, vals, a_scale=sa, b_scale=sb)
    want = oracle.sddmm(rp, ci, oracle.dequantize(qa, "e4m3", sa), oracle.dequantize(qb, "e4m3", sb), vals)
    np.testing.assert_allclose(got, want, rtol=1e-14)
    hb = oracle.encode(B, "bf16")
    np.testing.assert_allclose(oracle.spmm(rp, ci, hb, vals, fmt_b="bf16"),
                               oracle.spmm(rp, ci, oracle.dequantize(hb, "bf16"), vals), rtol=1e-14)


# ----------------------------------------------------------------------------
# Transpose and merge path
# ----------------------------------------------------------------------------

def test_transpose_against_scipy_and_involution():
    sp = pytest.importorskip("scipy.sparse")
    M, N = 60, 45
    rp, ci, vals, _, _ = random_case(M, N, 1, 0.1, seed=9)
    colptr, rowidx, perm = oracle.transpose(rp, ci, N)
    S = sp.csr_matrix((np.arange(ci.size, dtype=np.int64), ci, rp), shape=(M, N))
    T = S.tocsc()
    assert np.array_equal(colptr, T.indptr) and np.array_equal(rowidx, T.indices)
    assert np.array_equal(perm, T.data)
    # rows inside a column ascend (stability), and transposing twice gives S back
    for j in range(N):
        assert np.all(np.diff(rowidx[colptr[j]:colptr[j + 1]]) > 0)
    rp2, ci2, perm2 = oracle.transpose(colptr, rowidx, M)
    assert np.array_equal(rp2, rp) and np.array_equal(ci2, ci)
    assert np.array_equal(perm[perm2], np.arange(ci.size))


def test_merge_path_against_materialised_merge():
    for seed in range(4):
        g = np.random.default_rng(seed)
        M = 40
        deg = g.integers(0, 6, M); deg[g.integers(0, M, 5)] = 0
        rp = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
        nnz = int(rp[-1])
        # materialise the merge: row-end r has key rowptr[r+1] and sorts before
        # the nonzero with the same index (type 0 before type 1)
        items = sorted([(int(rp[r + 1]), 0) for r in range(M)] + [(e, 1) for e in range(nnz)])
        for d in range(M + nnz + 1):
            r = sum(1 for it in items[:d] if it[1] == 0)
            assert oracle.merge_path(rp, d) == (r, d - r)


# ----------------------------------------------------------------------------
# Gradients: closed forms against central finite differences (FP64)
# ----------------------------------------------------------------------------

def _fd(f, x, v, h=1e-6):
    return (f(x + h * v) - f(x - h * v)) / (2 * h)


def test_sddmm_and_spmm_gradients_fd():
    M, N, K = 25, 30, 8
    rp, ci, vals, A, B = random_case(M, N, K, 0.2, seed=12)
    A = A.astype(np.float64); B = B.astype(np.float64); vals = vals.astype(np.float64)
    g = np.random.default_rng(13)
    G = g.standard_normal(ci.size)
    dA, dB, ds = oracle.sddmm_grads(rp, ci, A, B, vals, G)
    L = lambda A_, B_, s_: (G * oracle.sddmm(rp, ci, A_, B_, s_)).sum()
    for _ in range(3):
        VA, VB, Vs = g.standard_normal(A.shape), g.standard_normal(B.shape), g.standard_normal(vals.shape)
        assert abs(_fd(lambda t: L(t, B, vals), A, VA) - (dA * VA).sum()) < 1e-6
        assert abs(_fd(lambda t: L(A, t, vals), B, VB) - (dB * VB).sum()) < 1e-6
        assert abs(_fd(lambda t: L(A, B, t), vals, Vs) - (ds * Vs).sum()) < 1e-6
    dY = g.standard_normal((M, K))
    dB2, ds2 = oracle.spmm_grads(rp, ci, B, vals, dY)
    L2 = lambda B_, s_: (dY * oracle.spmm(rp, ci, B_, s_)).sum()
    VB, Vs = g.standard_normal(B.shape), g.standard_normal(vals.shape)
    assert abs(_fd(lambda t: L2(t, vals), B, VB) - (dB2 * VB).sum()) < 1e-6
    assert abs(_fd(lambda t: L2(B, t), vals, Vs) - (ds2 * Vs).sum()) < 1e-6


def test_gnn_gradient_fd_scale12():
    """The differentiation workload's check: R-MAT scale 12 copy, K = 8."""
    P = synth.small_rmat(scale=12, edge_factor=8, K=8, seed=0)
    H = P.A.astype(np.float64)
    g = np.random.default_rng(1)
    dY = g.standard_normal(H.shape)
    dH = oracle.gnn_grad(P.rowptr, P.colidx, H, dY)
    L = lambda H_: (dY * oracle.gnn_forward(P.rowptr, P.colidx, H_)[1]).sum()
    for _ in range(3):
        V = g.standard_normal(H.shape)
        fd = _fd(L, H, V)
        an = (dH * V).sum()
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
    # a few single coordinates, including one in the heaviest row
    heavy = int(np.argmax(np.diff(P.rowptr)))
    for (i, k) in [(heavy, 0), (0, 3), (P.M - 1, 7)]:
        V = np.zeros_like(H); V[i, k] = 1.0
        assert abs(_fd(L, H, V) - dH[i, k]) <= 1e-6 * max(1.0, abs(dH[i, k]))


# ----------------------------------------------------------------------------
# FusedMM (SDDMM cascaded into SpMM, per head, optional row softmax)
# ----------------------------------------------------------------------------

def _dense_fused(rp, ci, vals, A, B, heads, scale, softmax):
    """Dense FP64 reference: masked score matrix per head, masked row softmax."""
    M, K = A.shape
    N = B.shape[0]
    D = K // heads
    S = dense(rp, ci, vals, M, N)
    mask = dense(rp, ci, None, M, N) > 0
    Y = np.zeros((M, K))
    lse = np.full((M, heads), -np.inf)
    for h in range(heads):
        sl = slice(h * D, (h + 1) * D)
        E = scale * S * (A[:, sl].astype(np.float64) @ B[:, sl].astype(np.float64).T)
        if softmax:
            Em = np.where(mask, E, -np.inf)
            m = Em.max(axis=1, keepdims=True)
            P = np.where(mask, np.exp(Em - np.where(np.isfinite(m), m, 0.0)), 0.0)
            l = P.sum(axis=1, keepdims=True)
            W = np.divide(P, l, out=np.zeros_like(P), where=l > 0)
            nz = mask.any(axis=1)
            lse[nz, h] = m[nz, 0] + np.log(l[nz, 0])
        else:
            W = np.where(mask, E, 0.0)
        Y[:, sl] = W @ B[:, sl].astype(np.float64)
    return Y, lse


@pytest.mark.parametrize("heads,softmax", [(1, False), (2, False), (1, True), (4, True)])
def test_fusedmm_dense_bruteforce(heads, softmax):
    M, N, K = 37, 29, 16
    rp, ci, vals, A, B = random_case(M, N, K, 0.3, seed=heads * 10 + softmax)
    Y, scores, lse = oracle.fusedmm(rp, ci, A, B, vals, heads=heads, scale=0.7, softmax=softmax)
    Yd, lsed = _dense_fused(rp, ci, vals, A, B, heads, 0.7, softmax)
    np.testing.assert_allclose(Y, Yd, rtol=1e-12, atol=1e-12)
    if softmax:
        np.testing.assert_allclose(lse, lsed, rtol=1e-12, atol=1e-12)
    # scores are the SDDMM of each head's slice, scaled
    D = K // heads
    for h in range(heads):
        sd = oracle.sddmm(rp, ci, A[:, h * D:(h + 1) * D], B[:, h * D:(h + 1) * D], vals)
        np.testing.assert_allclose(scores[h], 0.7 * sd, rtol=1e-13, atol=1e-13)
    rows = np.array([M - 1, 3, 0])
    Ys, _, ls = oracle.fusedmm(rp, ci, A, B, vals, heads=heads, scale=0.7, softmax=softmax, rows=rows)
    np.testing.assert_allclose(Ys, Y[rows], rtol=1e-14, atol=1e-14)


def test_fusedmm_softmax_closed_forms():
    g = np.random.default_rng(3)
    N, K = 12, 8
    B = g.standard_normal((N, K)).astype(np.float32)
    # one nonzero per row: weight 1, Y = that B row, lse = its score
    rp = np.arange(5, dtype=np.int32)
    ci = np.array([3, 0, 11, 3], np.int32)
    A = g.standard_normal((4, K)).astype(np.float32)
    Y, sc, lse = oracle.fusedmm(rp, ci, A, B, softmax=True)
    np.testing.assert_array_equal(Y, B[ci].astype(np.float64))
    np.testing.assert_allclose(lse[:, 0], sc[0], rtol=0, atol=1e-15)
    # all scores equal (A = 0): uniform weights, Y = mean of the row's B rows, lse = log(degree)
    rp2 = np.array([0, 3, 3, 7], np.int32)
    ci2 = np.array([1, 4, 9, 0, 2, 5, 11], np.int32)
    Y2, _, lse2 = oracle.fusedmm(rp2, ci2, np.zeros((3, K), np.float32), B, softmax=True)
    np.testing.assert_allclose(Y2[0], B[[1, 4, 9]].astype(np.float64).mean(0), rtol=1e-14, atol=1e-14)
    np.testing.assert_array_equal(Y2[1], np.zeros(K))
    np.testing.assert_allclose(Y2[2], B[[0, 2, 5, 11]].astype(np.float64).mean(0), rtol=1e-14, atol=1e-14)
    assert lse2[1, 0] == -np.inf and abs(lse2[0, 0] - np.log(3)) < 1e-15 and abs(lse2[2, 0] - np.log(4)) < 1e-15
    # one score above the others by 1000 (no overflow): weight 1 on it
    Bo = np.eye(N, K, dtype=np.float32)
    Ao = np.zeros((1, K), np.float32); Ao[0, 5] = 1000.0
    rp3 = np.array([0, 4], np.int32); ci3 = np.array([2, 5, 6, 7], np.int32)
    Y3, _, lse3 = oracle.fusedmm(rp3, ci3, Ao, Bo, softmax=True)
    np.testing.assert_array_equal(Y3[0], Bo[5].astype(np.float64))
    assert abs(lse3[0, 0] - 1000.0) < 1e-12
    # a duplicated entry counts twice: two equal copies of one column share the weight
    rp4 = np.array([0, 2], np.int32); ci4 = np.array([7, 7], np.int32)
    Y4, _, lse4 = oracle.fusedmm(rp4, ci4, A[:1], B, softmax=True)
    np.testing.assert_allclose(Y4[0], B[7].astype(np.float64), rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(lse4[0, 0], float(np.dot(A[0].astype(np.float64), B[7])) + np.log(2.0), rtol=1e-14)


def test_fusedmm_plain_is_spmm_of_scores_and_absmode():
    M, N, K = 30, 25, 12
    rp, ci, vals, A, B = random_case(M, N, K, 0.3, seed=5)
    Y, sc, _ = oracle.fusedmm(rp, ci, A, B, vals, heads=3, scale=-1.5)
    D = K // 3
    Yabs, _, _ = oracle.fusedmm(rp, ci, A, B, vals, heads=3, scale=-1.5, absmode=True)
    for h in range(3):
        sl = slice(h * D, (h + 1) * D)
        np.testing.assert_allclose(Y[:, sl], dense(rp, ci, sc[h], M, N) @ B[:, sl].astype(np.float64),
                                   rtol=1e-12, atol=1e-12)
        # denominator: |scale s| sum|a b| times |b|
        ab = 1.5 * np.abs(vals.astype(np.float64)) * (np.abs(A[:, sl].astype(np.float64)) @ np.abs(B[:, sl].astype(np.float64)).T)[
            np.repeat(np.arange(M), np.diff(rp)), ci]
        np.testing.assert_allclose(Yabs[:, sl], dense(rp, ci, ab, M, N) @ np.abs(B[:, sl].astype(np.float64)),
                                   rtol=1e-12, atol=1e-12)
    assert np.all(Yabs >= np.abs(Y) - 1e-12)


@pytest.mark.parametrize("heads,softmax", [(1, False), (2, True), (3, True), (3, False)])
def test_fusedmm_gradient_fd(heads, softmax):
    """The FusedMM backward's chain rule against central finite differences
    of the oracle's own forward (a dropped softmax row term, a missing W^T dY
    contribution or a wrong head slice moves the directional derivative)."""
    M, N, K = 14, 11, 6 * heads
    rp, ci, vals, A, B = random_case(M, N, K, 0.35, seed=40 + heads)
    A = A.astype(np.float64) * 0.5; B = B.astype(np.float64) * 0.5; vals = vals.astype(np.float64)
    g = np.random.default_rng(41)
    dY = g.standard_normal((M, K))
    kw = dict(heads=heads, scale=0.8, softmax=softmax)
    dA, dB = oracle.fusedmm_grad(rp, ci, A, B, dY, vals, **kw)
    L = lambda A_, B_: (dY * oracle.fusedmm(rp, ci, A_, B_, vals, **kw)[0]).sum()
    for _ in range(3):
        VA, VB = g.standard_normal(A.shape), g.standard_normal(B.shape)
        fa, fb = _fd(lambda t: L(t, B), A, VA), _fd(lambda t: L(A, t), B, VB)
        assert abs(fa - (dA * VA).sum()) <= 1e-6 * max(1.0, abs(fa))
        assert abs(fb - (dB * VB).sum()) <= 1e-6 * max(1.0, abs(fb))
    # rows with no entries get no gradient in A
    empty = np.flatnonzero(np.diff(rp) == 0)
    assert empty.size and np.all(dA[empty] == 0.0)


def test_fusedmm_gradient_softmax_rows_sum_to_zero_in_scores():
    """With softmax, a shift of every score in a row leaves Y unchanged: the
    score gradient of each row sums to zero, i.e. for A = B = 0 directions
    that only shift scores the derivative vanishes (checked through dA along
    a_i itself when all b_j in the row are equal)."""
    M, N, K = 4, 5, 3
    rp = np.array([0, 3, 3, 5, 7], np.int32)
    ci = np.array([0, 2, 4, 1, 3, 0, 4], np.int32)
    A = np.random.default_rng(3).standard_normal((M, K))
    B = np.tile(np.array([[0.3, -0.2, 0.5]]), (N, 1))      # all b_j equal
    dY = np.random.default_rng(4).standard_normal((M, K))
    dA, _ = oracle.fusedmm_grad(rp, ci, A, B, dY, softmax=True)
    # scores in a row are equal, weights uniform, and a change of a_i shifts
    # every score of the row by the same amount: Y does not move
    np.testing.assert_allclose(dA, 0.0, atol=1e-14)


@pytest.mark.parametrize("heads,softmax", [(1, False), (2, True), (3, True)])
def test_fusedmm_gradient_against_dense_autograd(heads, softmax):
    """The oracle's FusedMM chain rule against reverse-mode differentiation of
    a dense masked formulation (torch autograd, FP64), to rounding."""
    import torch
    M, N, K = 17, 13, 4 * heads
    rp, ci, vals, A, B = random_case(M, N, K, 0.3, seed=60 + heads)
    g = np.random.default_rng(61)
    dY = g.standard_normal((M, K))
    scale = 0.7
    dA, dB = oracle.fusedmm_grad(rp, ci, A, B, dY, vals, heads=heads, scale=scale, softmax=softmax)
    S = torch.from_numpy(dense(rp, ci, vals.astype(np.float64), M, N))
    mask = torch.from_numpy(dense(rp, ci, None, M, N) > 0)
    tA = torch.from_numpy(A.astype(np.float64)).requires_grad_()
    tB = torch.from_numpy(B.astype(np.float64)).requires_grad_()
    D = K // heads
    parts = []
    for h in range(heads):
        Ah, Bh = tA[:, h * D:(h + 1) * D], tB[:, h * D:(h + 1) * D]
        E = scale * S * (Ah @ Bh.T)
        if softmax:
            W = torch.softmax(E.masked_fill(~mask, float("-inf")), dim=1)
            W = torch.where(mask, W, torch.zeros_like(W))          # empty rows: no weights
        else:
            W = torch.where(mask, E, torch.zeros_like(E))
        parts.append(W @ Bh)
    Y = torch.cat(parts, dim=1)
    gA, gB = torch.autograd.grad((torch.from_numpy(dY) * Y).sum(), (tA, tB))
    np.testing.assert_allclose(dA, gA.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(dB, gB.numpy(), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("heads,softmax", [(1, False), (2, False), (1, True), (3, True)])
def test_fusedmm_gradient_denominators(heads, softmax):
    """The componentwise denominators of the FusedMM gradient (the chain rule
    over magnitudes) against a dense masked formulation of the same magnitudes,
    and two properties that hold for any input: they bound |dA|, |dB|, and with
    every factor nonnegative and no softmax (no cancellation) they equal them."""
    M, N, K = 15, 12, 4 * heads
    rp, ci, vals, A, B = random_case(M, N, K, 0.3, seed=70 + heads + 3 * softmax)
    A = A.astype(np.float64); B = B.astype(np.float64); vals = vals.astype(np.float64)
    dY = np.random.default_rng(71).standard_normal((M, K))
    scale = -0.6
    kw = dict(heads=heads, scale=scale, softmax=softmax)
    dA, dB = oracle.fusedmm_grad(rp, ci, A, B, dY, vals, **kw)
    dA_den, dB_den = oracle.fusedmm_grad(rp, ci, A, B, dY, vals, absmode=True, **kw)
    assert np.all(dA_den >= np.abs(dA) * (1 - 1e-12)) and np.all(dB_den >= np.abs(dB) * (1 - 1e-12))
    # dense masked magnitudes, written out per head
    S_abs = np.abs(dense(rp, ci, vals, M, N))
    mask = dense(rp, ci, None, M, N) > 0
    D = K // heads
    eA, eB = np.zeros((M, K)), np.zeros((N, K))
    for h in range(heads):
        sl = slice(h * D, (h + 1) * D)
        Ah, Bh, dYh = A[:, sl], B[:, sl], dY[:, sl]
        E = scale * dense(rp, ci, vals, M, N) * (Ah @ Bh.T)
        if softmax:
            Em = np.where(mask, E, -np.inf)
            mx = np.max(Em, axis=1, keepdims=True)
            P = np.where(mask, np.exp(Em - np.where(np.isfinite(mx), mx, 0.0)), 0.0)
            tot = P.sum(axis=1, keepdims=True)
            W = np.where(tot > 0, P / np.where(tot > 0, tot, 1.0), 0.0)
            W = W * (1.0 + abs(scale) * S_abs * (np.abs(Ah) @ np.abs(Bh).T))
        else:
            W = np.where(mask, np.abs(E), 0.0)
        dw = np.where(mask, np.abs(dYh) @ np.abs(Bh).T, 0.0)
        g = W * (dw + (W * dw).sum(axis=1, keepdims=True)) if softmax else dw
        C = abs(scale) * S_abs * g
        eA[:, sl] = C @ np.abs(Bh)
        eB[:, sl] = C.T @ np.abs(Ah) + W.T @ np.abs(dYh)
    np.testing.assert_allclose(dA_den, eA, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(dB_den, eB, rtol=1e-12, atol=1e-14)
    if not softmax:
        # nonnegative factors and a positive scale: nothing cancels
        Ap, Bp, dYp, vp = np.abs(A), np.abs(B), np.abs(dY), np.abs(vals)
        kp = dict(heads=heads, scale=0.6, softmax=False)
        pA, pB = oracle.fusedmm_grad(rp, ci, Ap, Bp, dYp, vp, **kp)
        qA, qB = oracle.fusedmm_grad(rp, ci, Ap, Bp, dYp, vp, absmode=True, **kp)
        np.testing.assert_allclose(qA, pA, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(qB, pB, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("dedup", [0, 1, 2])
def test_coo_to_csr_against_numpy(dedup):
    """COO -> CSR against numpy's stable lexsort (order by row, then column,
    ties in input order), np.unique for the repeats, and np.add.at for their
    summed values; the de-duplicated pattern equals the generators' CSR."""
    g = np.random.default_rng(90 + dedup)
    M, N, n = 57, 43, 900
    rows = g.integers(0, M, n).astype(np.int32)
    cols = g.integers(0, N, n).astype(np.int32)
    rows[:40] = rows[40:80]; cols[:40] = cols[40:80]            # plenty of repeats
    rows[5] = M - 1; cols[5] = N - 1
    vals = g.uniform(-1, 1, n)
    rp, ci, v = oracle.coo_to_csr(rows, cols, M, N, vals, dedup)
    order = np.lexsort((np.arange(n), cols, rows))
    r_s, c_s, v_s = rows[order], cols[order], vals[order]
    if dedup == 0:
        exp_r, exp_c, exp_v = r_s, c_s, v_s
    else:
        first = np.ones(n, bool)
        first[1:] = (r_s[1:] != r_s[:-1]) | (c_s[1:] != c_s[:-1])
        exp_r, exp_c = r_s[first], c_s[first]
        if dedup == 1:
            exp_v = v_s[first]
        else:
            exp_v = np.zeros(first.sum())
            np.add.at(exp_v, np.cumsum(first) - 1, v_s)
        srp, sci = synth.csr_from_coo(rows, cols, M, N)
        assert np.array_equal(srp, rp) and np.array_equal(sci, ci)
    assert np.array_equal(ci, exp_c)
    assert np.array_equal(rp, np.searchsorted(exp_r, np.arange(M + 1), side="left").astype(np.int32))
    np.testing.assert_allclose(v, exp_v, rtol=1e-14, atol=1e-15)
    # empty input and an index out of range
    rp0, ci0, _ = oracle.coo_to_csr(np.zeros(0, np.int32), np.zeros(0, np.int32), 3, 2, None, dedup)
    assert np.array_equal(rp0, [0, 0, 0, 0]) and ci0.size == 0
    with pytest.raises(ValueError):
        oracle.coo_to_csr(np.array([0], np.int32), np.array([N], np.int32), M, N, None, dedup)


def test_row_orders_and_rcm_properties():
    """Row relabellings: the stable sorts by their definitions, and reverse
    Cuthill-McKee by what it is for — bandwidth 1 on a relabelled path, the
    grid width on a relabelled grid, each component contiguous, the reversed
    order ending at a vertex of smallest degree."""
    g = np.random.default_rng(81)
    rp, ci = synth.csr_from_coo(g.integers(0, 40, 300), g.integers(0, 55, 300), 40, 55)
    deg = np.diff(rp)
    p = oracle.row_order(rp, ci, 55, "degree")
    assert sorted(p.tolist()) == list(range(40)) and np.all(np.diff(deg[p]) <= 0)
    for a, b in zip(p[:-1], p[1:]):
        assert deg[a] > deg[b] or a < b                       # ties in the original order
    q = oracle.row_order(rp, ci, 55, "leading")
    lead = np.array([ci[rp[i]:rp[i + 1]].min() if deg[i] else 55 for i in range(40)])
    assert np.all(np.diff(lead[q]) >= 0)

    def relabelled(edges, n, seed):
        lab = np.random.default_rng(seed).permutation(n)
        r = np.concatenate([lab[edges[:, 0]], lab[edges[:, 1]]])
        c = np.concatenate([lab[edges[:, 1]], lab[edges[:, 0]]])
        return synth.csr_from_coo(r, c, n, n)

    def bandwidth(rp, ci, perm):
        inv = np.empty_like(perm); inv[perm] = np.arange(perm.size)
        rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
        return int(np.max(np.abs(inv[rows] - inv[ci])))

    path = np.array([[i, i + 1] for i in range(59)])
    rp, ci = relabelled(path, 60, 1)
    perm = oracle.rcm(rp, ci)
    assert sorted(perm.tolist()) == list(range(60)) and bandwidth(rp, ci, perm) == 1
    w = 9
    grid = np.array([[r * w + c, r * w + c + 1] for r in range(12) for c in range(w - 1)]
                    + [[r * w + c, (r + 1) * w + c] for r in range(11) for c in range(w)])
    rp, ci = relabelled(grid, 12 * w, 2)
    perm = oracle.rcm(rp, ci)
    assert bandwidth(rp, ci, perm) <= w + 1
    # two components (a path and a triangle) and an isolated vertex
    edges = np.array([[0, 1], [1, 2], [2, 3], [4, 5], [5, 6], [6, 4]])
    rp, ci = relabelled(edges, 8, 3)
    perm = oracle.rcm(rp, ci)
    comp = {}
    lab = np.random.default_rng(3).permutation(8)
    for v in range(8):
        comp[lab[v]] = 0 if v < 4 else (1 if v < 7 else 2)
    seq = [comp[v] for v in perm]
    assert len([k for k in range(1, 8) if seq[k] != seq[k - 1]]) == 2      # each component contiguous
    deg = np.diff(rp)
    assert deg[perm[-1]] == deg.min()
