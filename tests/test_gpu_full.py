"""Full-size configurations, in the launch configuration the benchmark times
(library defaults), checked on sampled rows the oracle computes one by one and
through properties that hold at any size (adjoint identity, determinism)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import TOL, TOL_BF16_X, comp_err

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def spk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2404_19638_gb300 as m
    return m


def _rows_entries(rowptr, rows):
    return np.concatenate([np.arange(rowptr[r], rowptr[r + 1]) for r in rows]).astype(np.int64)


def _sample_cols(colidx, N, count, seed):
    g = np.random.default_rng(seed)
    cdeg = np.bincount(colidx, minlength=N)
    return np.unique(np.concatenate([np.argsort(cdeg)[-6:], [0, N - 1], g.integers(0, N, count)])).astype(np.int64)


def test_tiny_exact_config_all_entries(spk):
    """The plain-method configuration exactly: Erdos-Renyi 4096 x 4096 with 16
    distinct uniform columns per row (65,536 nonzeros), K = 32, values and
    factors uniform [-1, 1] FP32, seed 0; SDDMM (Eq. 1), SpMM (Eq. 2) and
    S^T A in the default launch configuration, every output element against
    the oracle, componentwise at the FP32 tolerance."""
    P = synth.tiny(seed=0)
    assert (P.M, P.N, P.K, P.colidx.size) == (4096, 4096, 32, 65536)
    S = spk.CSR(P.rowptr, P.colidx, (P.M, P.N), torch.from_numpy(P.vals), device=DEV)
    A, B = torch.from_numpy(P.A).to(DEV), torch.from_numpy(P.B).to(DEV)
    out = spk.sddmm(S, A, B).cpu().numpy()
    C = spk.spmm(S, B).cpu().numpy()
    X = spk.spmm_t(S, A).cpu().numpy()
    assert comp_err(out, oracle.sddmm(P.rowptr, P.colidx, P.A, P.B, P.vals),
                    oracle.sddmm(P.rowptr, P.colidx, P.A, P.B, P.vals, absmode=True)) <= TOL
    assert comp_err(C, oracle.spmm(P.rowptr, P.colidx, P.B, P.vals),
                    oracle.spmm(P.rowptr, P.colidx, P.B, P.vals, absmode=True)) <= TOL
    assert comp_err(X, oracle.spmm_t(P.rowptr, P.colidx, P.N, P.A, P.vals),
                    oracle.spmm_t(P.rowptr, P.colidx, P.N, P.A, P.vals, absmode=True)) <= TOL


def test_rmat20_fp32(spk):
    P = synth.rmat_problem(20, 16, 64, seed=0)
    S = spk.CSR(P.rowptr, P.colidx, (P.M, P.N), torch.from_numpy(P.vals), device=DEV)
    A, B = torch.from_numpy(P.A).to(DEV), torch.from_numpy(P.B).to(DEV)
    out = spk.sddmm(S, A, B)
    C = spk.spmm(S, B)
    X = spk.spmm_t(S, A)
    rows = synth.sample_rows(P.rowptr, 1500, seed=1)
    ent = _rows_entries(P.rowptr, rows)
    ref = oracle.sddmm(P.rowptr, P.colidx, P.A, P.B, P.vals, rows=rows)[ent]
    den = oracle.sddmm(P.rowptr, P.colidx, P.A, P.B, P.vals, rows=rows, absmode=True)[ent]
    assert comp_err(out.cpu().numpy()[ent], ref, den) <= TOL
    assert comp_err(C.cpu().numpy()[rows], oracle.spmm(P.rowptr, P.colidx, P.B, P.vals, rows=rows),
                    oracle.spmm(P.rowptr, P.colidx, P.B, P.vals, rows=rows, absmode=True)) <= TOL
    cols = _sample_cols(P.colidx, P.N, 800, seed=2)
    assert comp_err(X.cpu().numpy()[cols], oracle.spmm_t(P.rowptr, P.colidx, P.N, P.A, P.vals, cols=cols),
                    oracle.spmm_t(P.rowptr, P.colidx, P.N, P.A, P.vals, cols=cols, absmode=True)) <= TOL
    # size-independent properties: determinism and the adjoint identity
    assert torch.equal(spk.sddmm(S, A, B), out) and torch.equal(spk.spmm(S, B), C)
    s1 = out.double().sum().item()
    s2 = (A.double() * C.double()).sum().item()
    s3 = (B.double() * X.double()).sum().item()
    scale = (out.double().abs().sum().item() + 1.0)
    assert abs(s1 - s2) <= 1e-6 * scale and abs(s1 - s3) <= 1e-6 * scale


def test_rec_bf16_and_e4m3(spk):
    P = synth.rec(seed=0)
    S = spk.CSR(P.rowptr, P.colidx, (P.M, P.N), torch.from_numpy(P.vals), device=DEV)
    A32, B32 = torch.from_numpy(P.A).to(DEV), torch.from_numpy(P.B).to(DEV)
    rows = synth.sample_rows(P.rowptr, 1200, seed=3)
    ent = _rows_entries(P.rowptr, rows)
    need_b = np.unique(P.colidx[ent])
    # BF16: the GPU cast is the RNE encoding (bit-exact on the rows used)
    Ah, Bh = spk.cast(A32, torch.bfloat16), spk.cast(B32, torch.bfloat16)
    qa = Ah[torch.from_numpy(rows).to(DEV)].view(torch.int16).cpu().numpy().view(np.uint16)
    assert np.array_equal(qa, oracle.encode(P.A[rows], "bf16"))
    qA = np.zeros((P.M, P.K), np.uint16); qA[rows] = qa
    qB = oracle.encode(P.B, "bf16")
    assert np.array_equal(Bh[torch.from_numpy(need_b).to(DEV)].view(torch.int16).cpu().numpy().view(np.uint16),
                          qB[need_b])
    out = spk.sddmm(S, Ah, Bh).cpu().numpy()[ent]
    C = spk.spmm(S, Bh).cpu().numpy()[rows]
    ref_q = oracle.sddmm(P.rowptr, P.colidx, qA, qB, P.vals, rows=rows, fmt_a="bf16", fmt_b="bf16")[ent]
    den_q = oracle.sddmm(P.rowptr, P.colidx, qA, qB, P.vals, rows=rows, fmt_a="bf16", fmt_b="bf16", absmode=True)[ent]
    assert comp_err(out, ref_q, den_q) <= TOL
    ref_x = oracle.sddmm(P.rowptr, P.colidx, P.A, P.B, P.vals, rows=rows)[ent]
    den_x = oracle.sddmm(P.rowptr, P.colidx, P.A, P.B, P.vals, rows=rows, absmode=True)[ent]
    assert comp_err(out, ref_x, den_x) <= TOL_BF16_X
    assert comp_err(C, oracle.spmm(P.rowptr, P.colidx, qB, P.vals, rows=rows, fmt_b="bf16"),
                    oracle.spmm(P.rowptr, P.colidx, qB, P.vals, rows=rows, fmt_b="bf16", absmode=True)) <= TOL
    assert comp_err(C, oracle.spmm(P.rowptr, P.colidx, P.B, P.vals, rows=rows),
                    oracle.spmm(P.rowptr, P.colidx, P.B, P.vals, rows=rows, absmode=True)) <= TOL_BF16_X
    del Ah, Bh
    # E4M3 with per-row scales: quantisation bit-exact on the rows used
    Qa, Sa = spk.quantize_e4m3_rows(A32)
    Qb, Sb = spk.quantize_e4m3_rows(B32)
    oa, osa = oracle.quantize_e4m3_rows(P.A[rows])
    ob, osb = oracle.quantize_e4m3_rows(P.B)
    tr = torch.from_numpy(rows).to(DEV)
    assert np.array_equal(Qa[tr].view(torch.uint8).cpu().numpy(), oa) and np.array_equal(Sa[tr].cpu().numpy(), osa)
    assert np.array_equal(Qb.view(torch.uint8).cpu().numpy(), ob) and np.array_equal(Sb.cpu().numpy(), osb)
    qA8 = np.zeros((P.M, P.K), np.uint8); qA8[rows] = oa
    sA8 = np.ones(P.M, np.float32); sA8[rows] = osa
    out8 = spk.sddmm(S, Qa, Qb, a_scale=Sa, b_scale=Sb).cpu().numpy()[ent]
    ref8 = oracle.sddmm(P.rowptr, P.colidx, qA8, ob, P.vals, rows=rows, a_scale=sA8, b_scale=osb)[ent]
    den8 = oracle.sddmm(P.rowptr, P.colidx, qA8, ob, P.vals, rows=rows, a_scale=sA8, b_scale=osb, absmode=True)[ent]
    assert comp_err(out8, ref8, den8) <= TOL
    assert comp_err(out8, ref_x, den_x) <= 0.13
    C8 = spk.spmm(S, Qb, b_scale=Sb).cpu().numpy()[rows]
    assert comp_err(C8, oracle.spmm(P.rowptr, P.colidx, ob, P.vals, rows=rows, b_scale=osb),
                    oracle.spmm(P.rowptr, P.colidx, ob, P.vals, rows=rows, b_scale=osb, absmode=True)) <= TOL


def test_gnn_forward_backward(spk):
    P = synth.gnn(seed=0)
    S = spk.CSR(P.rowptr, P.colidx, (P.M, P.N), device=DEV)
    H = spk.cast(torch.from_numpy(P.A).to(DEV), torch.bfloat16).requires_grad_()
    qH = oracle.encode(P.A, "bf16")
    g = np.random.default_rng(4)
    dY = g.standard_normal((P.M, P.K)).astype(np.float32)
    Y = spk.autograd.gnn_layer(S, H)
    Y.backward(torch.from_numpy(dY).to(DEV))
    rows = synth.sample_rows(P.rowptr, 400, seed=5)
    rp, ci = P.rowptr, P.colidx
    Hd = oracle.dequantize(qH, "bf16")
    # forward: e = SDDMM(S, H, H) (all entries, needed for S_e^T), Y = SpMM(S_e, H)
    e_full = oracle.sddmm(rp, ci, qH, qH, fmt_a="bf16", fmt_b="bf16")
    Yref = oracle.spmm(rp, ci, qH, e_full, rows=rows, fmt_b="bf16")
    Yabs = oracle.spmm(rp, ci, np.abs(Hd), np.abs(e_full), rows=rows)
    assert comp_err(Y.detach().cpu().numpy()[rows], Yref, Yabs) <= TOL
    # backward: dH = (S.dE) H + (S.dE)^T H + S_e^T dY with dE_e = <dY_i, h_j>
    dE = oracle.sddmm(rp, ci, dY, qH, fmt_b="bf16")
    dEa = oracle.sddmm(rp, ci, np.abs(dY), np.abs(Hd))
    g1 = oracle.spmm(rp, ci, qH, None, dE, rows=rows, fmt_b="bf16")
    g2 = oracle.spmm_t(rp, ci, P.N, qH, None, dE, cols=rows, fmt_y="bf16")
    g3 = oracle.spmm_t(rp, ci, P.N, dY, e_full, cols=rows)
    a1 = oracle.spmm(rp, ci, np.abs(Hd), None, dEa, rows=rows)
    a2 = oracle.spmm_t(rp, ci, P.N, np.abs(Hd), None, dEa, cols=rows)
    a3 = oracle.spmm_t(rp, ci, P.N, np.abs(dY), np.abs(e_full), cols=rows)
    got = H.grad.float().cpu().numpy()[rows]
    assert comp_err(got, g1 + g2 + g3, a1 + a2 + a3) <= 2.0 ** -8 + TOL     # dH is stored in BF16


def test_batch_256_graph_vs_per_matrix(spk):
    probs = synth.batch(seed=0)
    assert len(probs) == 256
    items, keep = [], []
    for k, p in enumerate(probs):
        dt = torch.float32 if k % 4 < 2 else torch.bfloat16
        S = spk.CSR(p.rowptr, p.colidx, (p.M, p.N), torch.from_numpy(p.vals), device=DEV)
        A = torch.from_numpy(p.A).to(DEV).to(dt)
        B = torch.from_numpy(p.B).to(DEV).to(dt)
        if k % 2 == 0:
            out = torch.empty(p.nnz, device=DEV)
            items.append(spk.Item(spk.OP_SDDMM, S, B, out, A=A))
        else:
            out = torch.empty((p.M, p.K), device=DEV)
            items.append(spk.Item(spk.OP_SPMM, S, B, out))
        keep.append((S, A, B, out, k % 2, p, dt))
    batch = spk.Batch(items)
    batch.capture()
    for it in items:
        it.out.fill_(float("nan"))
    batch.replay()
    torch.cuda.synchronize()
    for S, A, B, out, op, p, dt in keep:
        nvec = p.K // (4 if dt == torch.float32 else 8)
        shape = (4, 1, 4) if nvec <= 4 else ((8, 1, 4) if nvec <= 8 else (16, 1, 4))
        tune = {"variant": 2, "group_lanes": shape[0], "vecs_per_lane": shape[1], "unroll": shape[2]}
        want = spk.sddmm(S, A, B, tune=tune) if op == 0 else spk.spmm(S, B, tune=tune)
        assert torch.equal(out, want), (p.name, op)
    for idx in (0, 1, 130, 131, 254, 255):
        S, A, B, out, op, p, dt = keep[idx]
        rows = synth.sample_rows(p.rowptr, 100, seed=idx)
        Aq, Bq = A.float().cpu().numpy(), B.float().cpu().numpy()
        if op == 0:
            ent = _rows_entries(p.rowptr, rows)
            assert comp_err(out.cpu().numpy()[ent], oracle.sddmm(p.rowptr, p.colidx, Aq, Bq, p.vals, rows=rows)[ent],
                            oracle.sddmm(p.rowptr, p.colidx, Aq, Bq, p.vals, rows=rows, absmode=True)[ent]) <= TOL
        else:
            assert comp_err(out.cpu().numpy()[rows], oracle.spmm(p.rowptr, p.colidx, Bq, p.vals, rows=rows),
                            oracle.spmm(p.rowptr, p.colidx, Bq, p.vals, rows=rows, absmode=True)) <= TOL


def test_autotuner_choice_is_correct(spk, tmp_path):
    from paper_2404_19638_gb300.autotune import Autotuner
    P = synth.rmat_problem(14, 16, 64, seed=0, name="rmat14")
    S = spk.CSR(P.rowptr, P.colidx, (P.M, P.N), torch.from_numpy(P.vals), device=DEV)
    A, B = torch.from_numpy(P.A).to(DEV), torch.from_numpy(P.B).to(DEV)
    tuner = Autotuner(cache_path=str(tmp_path / "cache.json"), chunk_works=(256, 512), reps=2)
    best = tuner.tune(S, "sddmm", A, B)
    best2 = Autotuner(cache_path=str(tmp_path / "cache.json")).tune(S, "sddmm", A, B)
    assert best2 == best                                     # served from the cache file
    out = spk.sddmm(S, A, B, tune=best["tune"]).cpu().numpy()
    rows = synth.sample_rows(P.rowptr, 300, seed=1)
    ent = _rows_entries(P.rowptr, rows)
    assert comp_err(out[ent], oracle.sddmm(P.rowptr, P.colidx, P.A, P.B, P.vals, rows=rows)[ent],
                    oracle.sddmm(P.rowptr, P.colidx, P.A, P.B, P.vals, rows=rows, absmode=True)[ent]) <= TOL
    bs = tuner.tune(S, "spmm", None, B)
    C = spk.spmm(S, B, tune=bs["tune"]).cpu().numpy()
    assert comp_err(C[rows], oracle.spmm(P.rowptr, P.colidx, P.B, P.vals, rows=rows),
                    oracle.spmm(P.rowptr, P.colidx, P.B, P.vals, rows=rows, absmode=True)) <= TOL
