"""CUDA path vs the FP64 oracle, element by element, at sizes the oracle
finishes in seconds (several chunks, ragged tails, empty rows, long rows)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import TOL, TOL_BF16_X, comp_err, edge_pattern, row_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2404_19638_gb300 as m
    return m


DEV = "cuda"


def _case(M, N, K, seed, long_row=0, dtype=np.float32):
    rp, ci = edge_pattern(M, N, seed, long_row=long_row)
    g = np.random.default_rng(seed + 100)
    vals = g.uniform(-1, 1, ci.size).astype(np.float32)
    A = g.standard_normal((M, K)).astype(dtype)
    B = g.standard_normal((N, K)).astype(dtype)
    return rp, ci, vals, A, B


SHAPES = [(4, 1, 4), (8, 1, 8), (16, 1, 8), (32, 1, 8), (8, 2, 8), (16, 2, 8), (32, 2, 4), (4, 2, 4), (32, 4, 4), (8, 4, 4),
          (16, 1, 4), (8, 2, 4), (8, 1, 4)]


@pytest.mark.parametrize("K", [1, 3, 8, 24, 32, 40, 64, 128, 136])
@pytest.mark.parametrize("variant", [1, 2, 3, "stages4"])
def test_sddmm_spmm_f32_k_sweep(spk, K, variant):
    M, N = 700, 500
    rp, ci, vals, A, B = _case(M, N, K, seed=K, long_row=3000)
    S = spk.CSR(rp, ci, (M, N), torch.from_numpy(vals), device=DEV, chunk_work=128)
    tA, tB = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    tune = {"variant": 2, "stages": 4} if variant == "stages4" else {"variant": variant}
    out = spk.sddmm(S, tA, tB, tune=tune).cpu().numpy()
    C = spk.spmm(S, tB, tune=tune).cpu().numpy()
    X = spk.spmm_t(S, tA, tune=tune).cpu().numpy()
    assert comp_err(out, oracle.sddmm(rp, ci, A, B, vals), oracle.sddmm(rp, ci, A, B, vals, absmode=True)) <= TOL
    assert comp_err(C, oracle.spmm(rp, ci, B, vals), oracle.spmm(rp, ci, B, vals, absmode=True)) <= TOL
    assert comp_err(X, oracle.spmm_t(rp, ci, N, A, vals), oracle.spmm_t(rp, ci, N, A, vals, absmode=True)) <= TOL


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("K", [16, 64])
def test_all_compiled_shapes(spk, shape, K):
    M, N = 600, 450
    rp, ci, vals, A, B = _case(M, N, K, seed=7 * K + shape[0], long_row=2500)
    S = spk.CSR(rp, ci, (M, N), torch.from_numpy(vals), device=DEV, chunk_work=96)
    tA, tB = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    G, NV, U = shape
    got = {}
    for variant, stages in ((1, 0), (2, 2), (2, 4), (3, 0)):
        tune = {"variant": variant, "group_lanes": G, "vecs_per_lane": NV, "unroll": U, "stages": stages}
        out = spk.sddmm(S, tA, tB, tune=tune).cpu().numpy()
        C = spk.spmm(S, tB, tune=tune).cpu().numpy()
        assert comp_err(out, oracle.sddmm(rp, ci, A, B, vals), oracle.sddmm(rp, ci, A, B, vals, absmode=True)) <= TOL
        assert comp_err(C, oracle.spmm(rp, ci, B, vals), oracle.spmm(rp, ci, B, vals, absmode=True)) <= TOL
        got[(variant, stages)] = (out, C)
    # shared-memory staging changes where gathered rows wait, not the arithmetic
    for k in ((2, 4), (3, 0)):
        assert np.array_equal(got[(2, 2)][0], got[k][0]) and np.array_equal(got[(2, 2)][1], got[k][1])


@pytest.mark.parametrize("W", [32, 64, 512, 4096])
def test_chunk_work_sweep_and_split_rows(spk, W):
    M, N, K = 900, 30000, 32
    rp, ci, vals, A, B = _case(M, N, K, seed=W, long_row=20000)
    S = spk.CSR(rp, ci, (M, N), torch.from_numpy(vals), device=DEV, chunk_work=W)
    info = S.schedule_info()
    if W <= 512:
        assert info["npieces"] > 0        # the long row is split
    tB = torch.from_numpy(B).to(DEV)
    C = spk.spmm(S, tB).cpu().numpy()
    assert comp_err(C, oracle.spmm(rp, ci, B, vals), oracle.spmm(rp, ci, B, vals, absmode=True)) <= TOL
    # deterministic: the split rows are combined in a fixed order
    C2 = spk.spmm(S, tB).cpu().numpy()
    assert np.array_equal(C, C2)
    # accumulate mode adds onto C
    base = torch.from_numpy(A).to(DEV)
    Cacc = base.clone()
    spk.spmm(S, tB, out=Cacc, accumulate=True)
    np.testing.assert_allclose(Cacc.cpu().numpy(), base.cpu().numpy() + C, rtol=1e-6, atol=1e-5)


def test_schedule_invariants_and_merge_path(spk):
    M, N = 1000, 800
    rp, ci = edge_pattern(M, N, 3, long_row=5000)
    S = spk.CSR(rp, ci, (M, N), device=DEV, chunk_work=100)
    W = 100
    n = (M + ci.size + W - 1) // W
    raw = S.merge_path_points(W, n).cpu().numpy()
    for c in range(0, n + 1, 7):
        d = min(c * W, M + ci.size)
        assert tuple(raw[c]) == oracle.merge_path(rp, d)
    assert tuple(raw[n]) == oracle.merge_path(rp, M + ci.size)
    b = S.schedule_bounds().cpu().numpy()
    assert tuple(b[0]) == (0, 0) and tuple(b[-1]) == (M, ci.size)
    assert np.all(np.diff(b[:, 0]) >= 0) and np.all(np.diff(b[:, 1]) >= 0)
    deg = np.diff(rp)
    for r, e in b[:-1]:
        assert rp[r] <= e
        if e > rp[r]:                     # a cut inside a row only happens in a long row
            assert deg[r] > W and e < rp[r + 1]


def test_transpose_plan_matches_oracle(spk):
    M, N = 1200, 5000
    rp, ci = edge_pattern(M, N, 4, long_row=7000)
    S = spk.CSR(rp, ci, (M, N), device=DEV)
    colptr, rowidx, perm = (t.cpu().numpy() for t in S.transpose_plan().arrays())
    oc, orow, operm = oracle.transpose(rp, ci, N)
    assert np.array_equal(colptr, oc) and np.array_equal(rowidx, orow) and np.array_equal(perm, operm)


def test_transpose_plan_many_columns(spk):
    # more than 2^16 columns: three radix passes
    M, N = 3000, 300000
    g = np.random.default_rng(5)
    rows = g.integers(0, M, 200000); cols = g.integers(0, N, 200000)
    rp, ci = synth.csr_from_coo(rows, cols, M, N)
    S = spk.CSR(rp, ci, (M, N), device=DEV)
    colptr, rowidx, perm = (t.cpu().numpy() for t in S.transpose_plan().arrays())
    oc, orow, operm = oracle.transpose(rp, ci, N)
    assert np.array_equal(colptr, oc) and np.array_equal(rowidx, orow) and np.array_equal(perm, operm)


@pytest.mark.parametrize("dt", ["bf16", "f16"])
def test_low_precision_inputs(spk, dt):
    M, N, K = 800, 600, 64
    rp, ci, vals, A, B = _case(M, N, K, seed=11, long_row=4000)
    S = spk.CSR(rp, ci, (M, N), torch.from_numpy(vals), device=DEV, chunk_work=256)
    tdt = torch.bfloat16 if dt == "bf16" else torch.float16
    tA = spk.cast(torch.from_numpy(A).to(DEV), tdt)
    tB = spk.cast(torch.from_numpy(B).to(DEV), tdt)
    qA, qB = oracle.encode(A, dt), oracle.encode(B, dt)
    # the GPU cast is the oracle's round-to-nearest-even encoding, bit for bit
    assert np.array_equal(tA.view(torch.int16).cpu().numpy().view(np.uint16), qA)
    assert np.array_equal(tB.view(torch.int16).cpu().numpy().view(np.uint16), qB)
    out = spk.sddmm(S, tA, tB).cpu().numpy()
    C = spk.spmm(S, tB).cpu().numpy()
    # kernel accuracy: against the oracle on the dequantised inputs (O_q)
    assert comp_err(out, oracle.sddmm(rp, ci, qA, qB, vals, fmt_a=dt, fmt_b=dt),
                    oracle.sddmm(rp, ci, qA, qB, vals, fmt_a=dt, fmt_b=dt, absmode=True)) <= TOL
    assert comp_err(C, oracle.spmm(rp, ci, qB, vals, fmt_b=dt),
                    oracle.spmm(rp, ci, qB, vals, fmt_b=dt, absmode=True)) <= TOL
    # end-to-end precision: against the oracle on the original FP32 inputs (O_x)
    assert comp_err(out, oracle.sddmm(rp, ci, A, B, vals), oracle.sddmm(rp, ci, A, B, vals, absmode=True)) <= TOL_BF16_X
    assert comp_err(C, oracle.spmm(rp, ci, B, vals), oracle.spmm(rp, ci, B, vals, absmode=True)) <= TOL_BF16_X
    # BF16 / F16 SpMM output, and the mixed F32 x BF16 SDDMM used by backward passes
    C16 = spk.spmm(S, tB, out_dtype=tdt).float().cpu().numpy()
    assert np.array_equal(C16, torch.from_numpy(C).to(tdt).float().numpy()) or \
        comp_err(C16, C, np.abs(C) + 1e-30) <= 2 ** -7
    mix = spk.sddmm(S, torch.from_numpy(A).to(DEV), tB).cpu().numpy()
    assert comp_err(mix, oracle.sddmm(rp, ci, A, qB, vals, fmt_b=dt),
                    oracle.sddmm(rp, ci, A, qB, vals, fmt_b=dt, absmode=True)) <= TOL


def test_e4m3_quantised_inputs(spk):
    M, N, K = 700, 500, 64
    rp, ci, vals, A, B = _case(M, N, K, seed=12, long_row=3000)
    A[5] = 0.0                                   # an all-zero row: scale 1
    S = spk.CSR(rp, ci, (M, N), torch.from_numpy(vals), device=DEV, chunk_work=256)
    qA, sA = spk.quantize_e4m3_rows(torch.from_numpy(A).to(DEV))
    qB, sB = spk.quantize_e4m3_rows(torch.from_numpy(B).to(DEV))
    oA, osA = oracle.quantize_e4m3_rows(A)
    oB, osB = oracle.quantize_e4m3_rows(B)
    assert np.array_equal(qA.view(torch.uint8).cpu().numpy(), oA) and np.array_equal(sA.cpu().numpy(), osA)
    assert np.array_equal(qB.view(torch.uint8).cpu().numpy(), oB) and np.array_equal(sB.cpu().numpy(), osB)
    out = spk.sddmm(S, qA, qB, a_scale=sA, b_scale=sB).cpu().numpy()
    C = spk.spmm(S, qB, b_scale=sB).cpu().numpy()
    assert comp_err(out, oracle.sddmm(rp, ci, oA, oB, vals, a_scale=osA, b_scale=osB),
                    oracle.sddmm(rp, ci, oA, oB, vals, a_scale=osA, b_scale=osB, absmode=True)) <= TOL
    assert comp_err(C, oracle.spmm(rp, ci, oB, vals, b_scale=osB),
                    oracle.spmm(rp, ci, oB, vals, b_scale=osB, absmode=True)) <= TOL
    # against the FP32 inputs: E4M3 rounding (3 mantissa bits) dominates
    ex = comp_err(out, oracle.sddmm(rp, ci, A, B, vals), oracle.sddmm(rp, ci, A, B, vals, absmode=True))
    assert ex <= 0.13


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_integer_inputs_bitwise(spk, dt):
    """Small integers keep every partial sum exact in FP32: results must equal
    the oracle's exactly, whatever the summation order."""
    M, N, K = 500, 400, 32
    rp, ci = edge_pattern(M, N, 21, long_row=3000)
    g = np.random.default_rng(21)
    vals = g.integers(-3, 4, ci.size).astype(np.float32)
    A = g.integers(-3, 4, (M, K)).astype(np.float32)
    B = g.integers(-3, 4, (N, K)).astype(np.float32)
    S = spk.CSR(rp, ci, (M, N), torch.from_numpy(vals), device=DEV, chunk_work=64)
    tA, tB = torch.from_numpy(A).to(DEV).to(dt), torch.from_numpy(B).to(DEV).to(dt)
    for variant in (1, 2, 3):
        out = spk.sddmm(S, tA, tB, tune={"variant": variant}).cpu().numpy()
        C = spk.spmm(S, tB, tune={"variant": variant}).cpu().numpy()
        X = spk.spmm_t(S, tA, tune={"variant": variant}).cpu().numpy()
        assert np.array_equal(out, oracle.sddmm(rp, ci, A, B, vals))
        assert np.array_equal(C, oracle.spmm(rp, ci, B, vals))
        assert np.array_equal(X, oracle.spmm_t(rp, ci, N, A, vals))


def test_degenerate_cases(spk):
    K = 16
    # nnz = 0: SpMM writes zeros, SDDMM writes nothing
    M, N = 50, 40
    rp = np.zeros(M + 1, np.int32); ci = np.zeros(0, np.int32)
    S = spk.CSR(rp, ci, (M, N), device=DEV)
    B = torch.randn(N, K, device=DEV)
    C = torch.full((M, K), 7.0, device=DEV)
    spk.spmm(S, B, out=C)
    assert torch.count_nonzero(C).item() == 0
    assert spk.sddmm(S, torch.randn(M, K, device=DEV), B).numel() == 0
    # identity: SDDMM = rowwise dots, SpMM = B
    n = 300
    rp = np.arange(n + 1, dtype=np.int32); ci = np.arange(n, dtype=np.int32)
    S = spk.CSR(rp, ci, (n, n), device=DEV)
    A = torch.randn(n, K, device=DEV); B = torch.randn(n, K, device=DEV)
    assert torch.equal(spk.spmm(S, B), B)
    torch.testing.assert_close(spk.sddmm(S, A, B), (A.double() * B.double()).sum(1).float(), rtol=1e-6, atol=1e-6)
    # one row holding every column (dense row), and a single long row of 2^20 nonzeros
    for cnt, ncols in [(4096, 4096), (1 << 20, 1 << 20)]:
        rp = np.array([0, cnt], np.int32); ci = np.arange(cnt, dtype=np.int32)
        g = np.random.default_rng(cnt)
        vals = g.uniform(-1, 1, cnt).astype(np.float32)
        Bn = g.standard_normal((ncols, K)).astype(np.float32)
        An = g.standard_normal((1, K)).astype(np.float32)
        S = spk.CSR(rp, ci, (1, ncols), torch.from_numpy(vals), device=DEV)
        C = spk.spmm(S, torch.from_numpy(Bn).to(DEV)).cpu().numpy()
        assert comp_err(C, oracle.spmm(rp, ci, Bn, vals), oracle.spmm(rp, ci, Bn, vals, absmode=True)) <= TOL
        out = spk.sddmm(S, torch.from_numpy(An).to(DEV), torch.from_numpy(Bn).to(DEV)).cpu().numpy()
        assert comp_err(out, oracle.sddmm(rp, ci, An, Bn, vals), oracle.sddmm(rp, ci, An, Bn, vals, absmode=True)) <= TOL


def test_strided_operands_use_scalar_path(spk):
    M, N, K = 300, 200, 12
    rp, ci, vals, A, B = _case(M, N, 20, seed=31, long_row=800)
    S = spk.CSR(rp, ci, (M, N), torch.from_numpy(vals), device=DEV, chunk_work=64)
    tA = torch.from_numpy(A).to(DEV)[:, 1:1 + K]      # misaligned, ld = 20
    tB = torch.from_numpy(B).to(DEV)[:, 3:3 + K]
    out = spk.sddmm(S, tA, tB).cpu().numpy()
    C = spk.spmm(S, tB).cpu().numpy()
    a, b = A[:, 1:1 + K].copy(), B[:, 3:3 + K].copy()
    assert comp_err(out, oracle.sddmm(rp, ci, a, b, vals), oracle.sddmm(rp, ci, a, b, vals, absmode=True)) <= TOL
    assert comp_err(C, oracle.spmm(rp, ci, b, vals), oracle.spmm(rp, ci, b, vals, absmode=True)) <= TOL


def test_validate_kernel(spk):
    M, N = 100, 50
    rp, ci = edge_pattern(M, N, 9)
    S = spk.CSR(rp, ci, (M, N), device=DEV, schedule=False)
    rep = S.validate()
    assert rep["error"] == 0 and rep["bad_count"] == 0 and not rep["unsorted"]
    bad = ci.copy(); bad[3] = N + 5
    rep = spk.CSR(rp, bad, (M, N), device=DEV, schedule=False).validate()
    assert rep["error"] == 4 and rep["first_bad"] == 3
    rp2 = rp.copy(); rp2[-1] = rp2[-1] - 1
    rep = spk.CSR(rp2, ci, (M, N), device=DEV, schedule=False).validate()
    assert rep["error"] != 0
    uns = ci.copy()
    r = int(np.argmax(np.diff(rp)))
    uns[rp[r]], uns[rp[r] + 1] = uns[rp[r] + 1], uns[rp[r]]
    assert spk.CSR(rp, uns, (M, N), device=DEV, schedule=False).validate()["unsorted"]


def test_duplicates_are_independent_entries(spk):
    rp = np.array([0, 3, 3], np.int32); ci = np.array([1, 1, 0], np.int32)
    vals = np.array([1.0, 2.0, -1.0], np.float32)
    B = np.array([[1.0, 2.0, 3.0, 4.0], [3.0, 4.0, 5.0, 6.0]], np.float32)
    S = spk.CSR(rp, ci, (2, 2), torch.from_numpy(vals), device=DEV)
    C = spk.spmm(S, torch.from_numpy(B).to(DEV)).cpu().numpy()
    assert np.array_equal(C, oracle.spmm(rp, ci, B, vals))


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("K", [16, 32, 64, 128])
def test_spmm_16bit_lane_layouts(spk, dt, K):
    """16-bit SpMM: 16-byte lane vectors, or 8-byte vectors over twice the
    lanes when a 16-byte layout would leave half the group idle; both give the
    same bits as the register path (each output element accumulates its
    nonzeros in the same order)."""
    M, N = 500, 420
    rp, ci, vals, A, B = _case(M, N, K, seed=K + 11, long_row=2500)
    S = spk.CSR(rp, ci, (M, N), torch.from_numpy(vals), device=DEV, chunk_work=96)
    tB = spk.cast(torch.from_numpy(B).to(DEV), dt)
    fmt = "bf16" if dt == torch.bfloat16 else "f16"
    Bq = tB.view(torch.int16).cpu().numpy().view(np.uint16)
    ref = oracle.spmm(rp, ci, Bq, vals, fmt_b=fmt)
    den = oracle.spmm(rp, ci, Bq, vals, fmt_b=fmt, absmode=True)
    base = spk.spmm(S, tB, tune={"variant": 3}).cpu().numpy()
    assert comp_err(base, ref, den) <= TOL
    for shape in [(4, 1, 4), (8, 1, 4), (16, 1, 8), (32, 1, 8), (4, 2, 4), (8, 2, 4)]:
        G, NV, U = shape
        got = spk.spmm(S, tB, tune={"variant": 2, "group_lanes": G, "vecs_per_lane": NV, "unroll": U}).cpu().numpy()
        assert np.array_equal(got, base), shape
    assert np.array_equal(spk.spmm(S, tB).cpu().numpy(), base)


def test_default_shapes_by_row_length(spk):
    """The library's default SpMM shape depends on K, the dtype and, for
    16-bit rows of 8 vectors, on whether rows average fewer than 12 nonzeros;
    every default runs and matches the oracle (and the register path bit for
    bit) on a short-row and a long-row pattern."""
    M, N = 600, 500
    g = np.random.default_rng(77)
    short = synth.csr_from_coo(np.repeat(np.arange(M), 4), g.integers(0, N, 4 * M), M, N)
    long_ = synth.csr_from_coo(np.repeat(np.arange(M), 20), g.integers(0, N, 20 * M), M, N)
    want = {  # (pattern, dtype code, K) -> default SpMM shape
        ("short", 1, 64): (8, 1, 4), ("long", 1, 64): (16, 1, 8),
        ("short", 1, 128): (8, 2, 4), ("long", 1, 128): (8, 2, 4),
        ("short", 0, 128): (16, 2, 8), ("long", 0, 64): (16, 1, 8),
    }
    for (name, code, K), shape in want.items():
        rp, ci = short if name == "short" else long_
        vals = g.uniform(-1, 1, ci.size).astype(np.float32)
        S = spk.CSR(rp, ci, (M, N), torch.from_numpy(vals), device=DEV)
        t = S.tune_default(1, code, K)
        assert (t["group_lanes"], t["vecs_per_lane"], t["unroll"]) == shape, (name, code, K, t)
        Bf = g.standard_normal((N, K)).astype(np.float32)
        tB = torch.from_numpy(Bf).to(DEV)
        if code == 1:
            tB = spk.cast(tB, torch.bfloat16)
            Bq = tB.view(torch.int16).cpu().numpy().view(np.uint16)
            fmt = "bf16"
        else:
            Bq, fmt = Bf, None
        got = spk.spmm(S, tB).cpu().numpy()
        assert comp_err(got, oracle.spmm(rp, ci, Bq, vals, fmt_b=fmt),
                        oracle.spmm(rp, ci, Bq, vals, fmt_b=fmt, absmode=True)) <= TOL, (name, code, K)
        assert np.array_equal(got, spk.spmm(S, tB, tune={"variant": 3}).cpu().numpy()), (name, code, K)
