"""The seeded generators: shapes, exact degrees, determinism, CSR invariants."""
import numpy as np

import synth


def check_csr(rp, ci, M, N):
    assert rp.dtype == np.int32 and ci.dtype == np.int32
    assert rp.size == M + 1 and rp[0] == 0 and rp[-1] == ci.size
    assert np.all(np.diff(rp.astype(np.int64)) >= 0)
    if ci.size:
        assert ci.min() >= 0 and ci.max() < N
    rows = np.repeat(np.arange(M), np.diff(rp))
    key = rows.astype(np.int64) * N + ci
    assert np.all(np.diff(key) > 0)        # sorted, no duplicates


def test_er_exact_degree():
    rp, ci = synth.er_exact_degree(300, 50, 16, seed=0)
    check_csr(rp, ci, 300, 50)
    assert np.all(np.diff(rp) == 16)
    rp2, ci2 = synth.er_exact_degree(300, 50, 16, seed=0)
    assert np.array_equal(ci, ci2)
    rp3, ci3 = synth.er_exact_degree(300, 50, 16, seed=1)
    assert not np.array_equal(ci, ci3)


def test_rmat_power_law_and_deterministic():
    rp, ci = synth.rmat(12, 8, seed=0)
    check_csr(rp, ci, 4096, 4096)
    deg = np.diff(rp)
    assert ci.size <= 8 * 4096 and ci.size > 4 * 4096
    assert deg[0] == deg.max()              # no permutation: row 0 is the heaviest
    assert (deg == 0).sum() > 0
    rp2, ci2 = synth.rmat(12, 8, seed=0)
    assert np.array_equal(ci, ci2)


def test_rmat_non_power_of_two():
    rp, ci = synth.rmat(0, 16, seed=3, n=1500)
    check_csr(rp, ci, 1500, 1500)


def test_chung_lu_exact_nnz():
    rp, ci = synth.chung_lu(2000, 500, 20000, 1.1, 1, 200, seed=0)
    check_csr(rp, ci, 2000, 500)
    assert ci.size == 20000


def test_tiny_workload_shape():
    P = synth.tiny()
    assert (P.M, P.N, P.K, P.nnz) == (4096, 4096, 32, 65536)
    assert P.A.shape == (4096, 32) and P.B.shape == (4096, 32)
    assert P.vals.min() >= -1 and P.vals.max() <= 1


def test_batch_workload_small():
    ps = synth.batch(seed=0, count=6, n_lo=100, n_hi=400)
    assert len(ps) == 6
    for p in ps:
        check_csr(p.rowptr, p.colidx, p.M, p.N)
        assert p.K in (16, 32, 64)
    assert ps[0].meta["kind"] == "er" and ps[-1].meta["kind"] == "rmat"


def test_rmat20_pattern_matches_the_recorded_figures():
    """The recorded rmat20 pattern (nnz after deduplication, empty rows, the
    heaviest row) that the measurements and their GFLOP/s use."""
    rp, ci = synth.rmat(20, 16, seed=0)
    check_csr(rp, ci, 1 << 20, 1 << 20)
    deg = np.diff(rp.astype(np.int64))
    assert ci.size == 16_086_730
    assert int(deg.max()) == 39_513
    assert round(float(np.mean(deg == 0)), 2) == 0.48
