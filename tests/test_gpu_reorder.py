"""Row relabelling for locality (spk_reorder_rows, spk_permute_pattern,
spk_permute_rows / _values): the orders bit-exact against the oracle's
stable sorts and its reverse Cuthill-McKee, the relabelled pattern against a
direct construction, and SDDMM (Eq. 1) / SpMM (Eq. 2) computed on the
relabelled pattern and mapped back, against the oracle on the original
problem; SpMM is bitwise equal to the unrelabelled call when no row is split
(each row then sums its entries in the same order)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import TOL, comp_err, edge_pattern

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def spk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2404_19638_gb300 as m
    return m


def _banded_shuffled(n, w, seed):
    """A band of half-width w whose rows are relabelled at random: the
    locality a relabelling can recover."""
    g = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        lo, hi = max(0, i - w), min(n, i + w + 1)
        c = np.unique(g.integers(lo, hi, w + 1))
        rows.append(np.full(c.size, i)); cols.append(c)
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    lab = g.permutation(n)
    return synth.csr_from_coo(lab[rows], lab[cols], n, n)


PATTERNS = {
    "edges": lambda: edge_pattern(900, 900, seed=41, long_row=700),
    "band": lambda: _banded_shuffled(1500, 6, seed=42),
    "rect": lambda: edge_pattern(700, 1300, seed=43),
}


@pytest.mark.parametrize("name", list(PATTERNS))
@pytest.mark.parametrize("order", ["degree", "leading", "rcm"])
def test_orders_match_oracle(spk, name, order):
    rp, ci = PATTERNS[name]()
    M = rp.size - 1
    N = 1300 if name == "rect" else M
    if order == "rcm" and M != N:
        S = spk.CSR(rp, ci, (M, N), device=DEV)
        with pytest.raises(spk.SpkError):
            spk.Reordering(S, "rcm")
        return
    S = spk.CSR(rp, ci, (M, N), device=DEV)
    R = spk.Reordering(S, order)
    perm = R.perm.cpu().numpy()
    exp = oracle.rcm(rp, ci) if order == "rcm" else oracle.row_order(rp, ci, N, order)
    assert np.array_equal(perm, exp)
    # the relabelled pattern, written out directly
    deg = np.diff(rp)
    rp2 = np.concatenate([[0], np.cumsum(deg[perm])]).astype(np.int32)
    emap = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in perm]).astype(np.int32)
    assert np.array_equal(R.S.rowptr.cpu().numpy(), rp2)
    assert np.array_equal(R.emap.cpu().numpy(), emap)
    assert np.array_equal(R.S.colidx.cpu().numpy(), ci[emap])


@pytest.mark.parametrize("order", ["degree", "leading", "rcm"])
@pytest.mark.parametrize("K,dtype", [(64, torch.float32), (32, torch.float32), (64, torch.bfloat16)])
def test_kernels_through_relabelling(spk, order, K, dtype):
    rp, ci = _banded_shuffled(3000, 9, seed=44) if order != "degree" else edge_pattern(2500, 2500, 45, 3000)
    n = rp.size - 1
    g = np.random.default_rng(K)
    vals = g.uniform(-1, 1, ci.size).astype(np.float32)
    A = g.standard_normal((n, K)).astype(np.float32)
    B = g.standard_normal((n, K)).astype(np.float32)
    S = spk.CSR(rp, ci, (n, n), torch.from_numpy(vals), device=DEV, chunk_work=64)
    R = spk.Reordering(S, order, chunk_work=64)
    tA, tB = torch.from_numpy(A).to(DEV).to(dtype), torch.from_numpy(B).to(DEV).to(dtype)
    out = R.scatter_values(spk.sddmm(R.S, R.gather_rows(tA), tB))
    C = R.scatter_rows(spk.spmm(R.S, tB))
    if dtype == torch.float32:
        Ao, Bo, kw = A, B, {}
    else:
        Ao = tA.view(torch.int16).cpu().numpy().view(np.uint16)
        Bo = tB.view(torch.int16).cpu().numpy().view(np.uint16)
        kw = {"fmt_a": "bf16", "fmt_b": "bf16"}
    ref = oracle.sddmm(rp, ci, Ao, Bo, vals, **kw)
    den = oracle.sddmm(rp, ci, Ao, Bo, vals, absmode=True, **kw)
    assert comp_err(out.cpu().numpy(), ref, den) <= TOL
    kb = {"fmt_b": kw["fmt_b"]} if kw else {}
    assert comp_err(C.cpu().numpy(), oracle.spmm(rp, ci, Bo, vals, **kb),
                    oracle.spmm(rp, ci, Bo, vals, absmode=True, **kb)) <= TOL


def test_spmm_bitwise_without_split_rows(spk):
    rp, ci = _banded_shuffled(2000, 8, seed=46)
    n = rp.size - 1
    g = np.random.default_rng(7)
    vals = torch.from_numpy(g.uniform(-1, 1, ci.size).astype(np.float32)).to(DEV)
    B = torch.from_numpy(g.standard_normal((n, 64)).astype(np.float32)).to(DEV)
    S = spk.CSR(rp, ci, (n, n), vals, device=DEV, chunk_work=512)
    assert S.schedule_info()["npieces"] == 0
    R = spk.Reordering(S, "rcm", chunk_work=512)
    assert R.S.schedule_info()["npieces"] == 0
    assert torch.equal(R.scatter_rows(spk.spmm(R.S, B)), spk.spmm(S, B))


def test_rcm_recovers_the_band(spk):
    """On a shuffled band, reverse Cuthill-McKee brings every entry back within
    a few multiples of the band's half-width of the diagonal."""
    rp, ci = _banded_shuffled(4000, 5, seed=47)
    S = spk.CSR(rp, ci, (4000, 4000), device=DEV)
    R = spk.Reordering(S, "rcm")
    perm = R.perm.cpu().numpy()
    inv = np.empty_like(perm); inv[perm] = np.arange(perm.size)
    rows = np.repeat(np.arange(4000), np.diff(rp))
    assert np.max(np.abs(rows - ci)) > 1000                        # shuffled: entries far from the diagonal
    assert np.max(np.abs(inv[rows] - inv[ci])) <= 4 * 5 + 2        # relabelled: back near it
