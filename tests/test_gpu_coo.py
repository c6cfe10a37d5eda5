"""COO -> CSR on the device (spk_coo_to_csr), bit-exact against the oracle's
two stable counting sorts: the order (row, column) with ties in input order,
the three treatments of repeated coordinates, row pointers, and the values
carried along (summed repeats: FP32 in input order against the oracle's FP64
sum, componentwise).  Edge cases: no entries, empty rows, a single row or
column (no radix pass on that key), sizes spanning many radix tiles and
three passes, and a coordinate outside the matrix."""
import ctypes

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


def _coo(M, N, n, seed, repeat_frac=0.2):
    g = np.random.default_rng(seed)
    rows = g.integers(0, M, n).astype(np.int32)
    cols = g.integers(0, N, n).astype(np.int32)
    k = int(n * repeat_frac)
    if k and n > 2 * k:
        idx = g.integers(0, n - k, k)
        rows[n - k:] = rows[idx]
        cols[n - k:] = cols[idx]                  # exact repeats, later in input order
    vals = g.uniform(-1, 1, n).astype(np.float32)
    return rows, cols, vals


CASES = [(1000, 800, 20000, 1), (1, 500, 3000, 2), (700, 1, 2500, 3), (1, 1, 40, 4), (5000, 3000, 0, 5),
         (3000, 4000, 50, 6), ((1 << 20) + 3, 70000, 300000, 7)]


@pytest.mark.parametrize("M,N,n,seed", CASES)
@pytest.mark.parametrize("dedup", ["keep", "first", "sum"])
def test_coo_to_csr_matches_oracle(spk, M, N, n, seed, dedup):
    rows, cols, vals = _coo(M, N, n, seed)
    mode = {"keep": 0, "first": 1, "sum": 2}[dedup]
    rp, ci, v = spk.coo_to_csr(rows, cols, (M, N), vals, dedup=dedup)
    erp, eci, ev = oracle.coo_to_csr(rows, cols, M, N, vals.astype(np.float64), mode)
    assert np.array_equal(rp.cpu().numpy(), erp)
    assert np.array_equal(ci.cpu().numpy(), eci)
    got = v.cpu().numpy()
    if mode == 2:
        # magnitudes of each output's terms: the oracle's summed |values|
        _, _, den = oracle.coo_to_csr(rows, cols, M, N, np.abs(vals.astype(np.float64)), 2)
        assert comp_err(got, ev, den) <= TOL
    else:
        assert np.array_equal(got.astype(np.float64), ev)
    if mode == 1:
        srp, sci = synth.csr_from_coo(rows, cols, M, N)
        assert np.array_equal(rp.cpu().numpy(), srp) and np.array_equal(ci.cpu().numpy(), sci)
    # no values asked for: the same pattern
    rp2, ci2, v2 = spk.coo_to_csr(rows, cols, (M, N), None, dedup=dedup)
    assert v2 is None and torch.equal(rp2, rp) and torch.equal(ci2, ci)


def test_coo_pattern_runs_the_kernels(spk):
    """A CSR built from shuffled coordinates computes what the sorted pattern does."""
    P = synth.tiny(seed=3, M=900, N=700, deg=9, K=16)
    rows = np.repeat(np.arange(P.M), np.diff(P.rowptr)).astype(np.int32)
    perm = np.random.default_rng(5).permutation(rows.size)
    S = spk.CSR.from_coo(rows[perm], P.colidx[perm], (P.M, P.N), P.vals[perm], dedup="first", chunk_work=64)
    assert torch.equal(S.rowptr.cpu(), torch.from_numpy(P.rowptr)) and torch.equal(S.colidx.cpu(),
                                                                                     torch.from_numpy(P.colidx))
    assert np.array_equal(S.vals.cpu().numpy(), P.vals)
    A, B = torch.from_numpy(P.A).to(DEV), torch.from_numpy(P.B).to(DEV)
    out = spk.sddmm(S, A, B).cpu().numpy()
    assert comp_err(out, oracle.sddmm(P.rowptr, P.colidx, P.A, P.B, P.vals),
                    oracle.sddmm(P.rowptr, P.colidx, P.A, P.B, P.vals, absmode=True)) <= TOL


def test_coo_rejects_out_of_range_coordinates(spk):
    from paper_2404_19638_gb300.binding import SpkError
    rows = np.array([0, 3, 1, 2], np.int32)
    cols = np.array([1, 0, 5, 2], np.int32)              # column 5 of a 4-column matrix
    with pytest.raises(SpkError) as ex:
        spk.coo_to_csr(rows, cols, (4, 4))
    assert ex.value.code == "SPK_ERR_INDEX" and "entry 2" in str(ex.value)
    with pytest.raises(SpkError):
        spk.coo_to_csr(np.array([-1], np.int32), np.array([0], np.int32), (4, 4))
    # the library is still usable afterwards
    rp, ci, _ = spk.coo_to_csr(rows[:2], cols[:2], (4, 4))
    assert rp.cpu().tolist() == [0, 1, 1, 1, 2] and ci.cpu().tolist() == [1, 0]
