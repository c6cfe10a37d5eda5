"""Differentiation (autograd Functions vs the oracle's closed-form gradients)
and the batched persistent launch (vs one launch per matrix, and graph replay)."""
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


def _dense_case(M, N, K, seed):
    rp, ci = edge_pattern(M, N, seed, long_row=1500)
    g = np.random.default_rng(seed)
    vals = g.uniform(-1, 1, ci.size).astype(np.float32)
    A = g.standard_normal((M, K)).astype(np.float32)
    B = g.standard_normal((N, K)).astype(np.float32)
    return rp, ci, vals, A, B


def test_sddmm_backward_vs_oracle(spk):
    M, N, K = 400, 300, 32
    rp, ci, vals, A, B = _dense_case(M, N, K, 1)
    S = spk.CSR(rp, ci, (M, N), device=DEV, chunk_work=128)
    tv = torch.from_numpy(vals).to(DEV).requires_grad_()
    tA = torch.from_numpy(A).to(DEV).requires_grad_()
    tB = torch.from_numpy(B).to(DEV).requires_grad_()
    G = np.random.default_rng(2).standard_normal(ci.size).astype(np.float32)
    out = spk.autograd.sddmm(S, tA, tB, tv)
    out.backward(torch.from_numpy(G).to(DEV))
    dA, dB, ds = oracle.sddmm_grads(rp, ci, A, B, vals, G)
    dAa, dBa, dsa = oracle.sddmm_grads(rp, ci, np.abs(A), np.abs(B), np.abs(vals), np.abs(G))
    assert comp_err(tA.grad.cpu().numpy(), dA, dAa) <= TOL
    assert comp_err(tB.grad.cpu().numpy(), dB, dBa) <= TOL
    assert comp_err(tv.grad.cpu().numpy(), ds, dsa) <= TOL


def test_spmm_backward_vs_oracle(spk):
    M, N, K = 400, 300, 32
    rp, ci, vals, A, B = _dense_case(M, N, K, 3)
    S = spk.CSR(rp, ci, (M, N), device=DEV, chunk_work=128)
    tv = torch.from_numpy(vals).to(DEV).requires_grad_()
    tB = torch.from_numpy(B).to(DEV).requires_grad_()
    dY = np.random.default_rng(4).standard_normal((M, K)).astype(np.float32)
    C = spk.autograd.spmm(S, tB, tv)
    C.backward(torch.from_numpy(dY).to(DEV))
    dB, ds = oracle.spmm_grads(rp, ci, B, vals, dY)
    dBa, dsa = oracle.spmm_grads(rp, ci, np.abs(B), np.abs(vals), np.abs(dY))
    assert comp_err(tB.grad.cpu().numpy(), dB, dBa) <= TOL
    assert comp_err(tv.grad.cpu().numpy(), ds, dsa) <= TOL


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_gnn_layer_scale12(spk, dt):
    """The differentiation workload at its finite-difference size (R-MAT scale
    12, K = 8): GPU backward vs the oracle's FD-checked closed form."""
    P = synth.small_rmat(scale=12, edge_factor=8, K=8, seed=0)
    S = spk.CSR(P.rowptr, P.colidx, (P.M, P.N), device=DEV, chunk_work=256)
    H32 = torch.from_numpy(P.A).to(DEV)
    H = (H32 if dt == torch.float32 else spk.cast(H32, dt)).requires_grad_()
    Hq = P.A if dt == torch.float32 else oracle.encode(P.A, "bf16")
    fmt = None if dt == torch.float32 else "bf16"
    dY = np.random.default_rng(5).standard_normal((P.M, 8)).astype(np.float32)
    Y = spk.autograd.gnn_layer(S, H)
    Y.backward(torch.from_numpy(dY).to(DEV))
    _, Yref = oracle.gnn_forward(P.rowptr, P.colidx, Hq, fmt=fmt)
    Hd = oracle.dequantize(Hq, fmt) if fmt else P.A.astype(np.float64)
    _, Yabs = oracle.gnn_forward(P.rowptr, P.colidx, np.abs(Hd))
    assert comp_err(Y.detach().cpu().numpy(), Yref, Yabs) <= TOL
    g = oracle.gnn_grad(P.rowptr, P.colidx, Hq, dY, fmt=fmt)
    gabs = oracle.gnn_grad(P.rowptr, P.colidx, np.abs(Hd), np.abs(dY))
    got = H.grad.float().cpu().numpy()
    tol = TOL if dt == torch.float32 else 2.0 ** -8 + TOL     # one BF16 rounding of dH
    assert comp_err(got, g, gabs) <= tol
    # composing the two differentiable primitives gives the same gradient
    H2 = H.detach().clone().requires_grad_()
    e = spk.autograd.sddmm(S, H2, H2)
    Y2 = spk.autograd.spmm(S, H2, e)
    Y2.backward(torch.from_numpy(dY).to(DEV))
    assert comp_err(H2.grad.float().cpu().numpy(), g, gabs) <= (TOL if dt == torch.float32 else 3 * 2.0 ** -8)


def _batch_problems(count, seed, n_hi=3000):
    return synth.batch(seed=seed, count=count, n_lo=100, n_hi=n_hi)


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_batch_equals_per_matrix_launches(spk, dt):
    probs = _batch_problems(12, seed=3)
    items, ref = [], []
    keep = []
    for k, p in enumerate(probs):
        S = spk.CSR(p.rowptr, p.colidx, (p.M, p.N), torch.from_numpy(p.vals), device=DEV, chunk_work=128)
        A = torch.from_numpy(p.A).to(DEV).to(dt)
        B = torch.from_numpy(p.B).to(DEV).to(dt)
        op = k % 2
        K = p.K
        if op == 0:
            out = torch.full((p.nnz,), float("nan"), device=DEV)
            items.append(spk.Item(spk.OP_SDDMM, S, B, out, A=A))
        else:
            out = torch.full((p.M, K), float("nan"), device=DEV)
            items.append(spk.Item(spk.OP_SPMM, S, B, out))
        keep.append((S, A, B, out, op, p))
    batch = spk.Batch(items)
    batch.run()
    torch.cuda.synchronize()
    for S, A, B, out, op, p in keep:
        vecn = 4 if dt == torch.float32 else 8
        nvec = p.K // vecn
        shape = (4, 1, 4) if nvec <= 4 else ((8, 1, 4) if nvec <= 8 else (16, 1, 4))
        tune = {"variant": 2, "group_lanes": shape[0], "vecs_per_lane": shape[1], "unroll": shape[2]}
        if op == 0:
            want = spk.sddmm(S, A, B, tune=tune)
        else:
            want = spk.spmm(S, B, tune=tune)
        assert torch.equal(out, want), (op, p.name, p.K)
        # and against the oracle
        Aq = A.float().cpu().numpy(); Bq = B.float().cpu().numpy()
        if op == 0:
            assert comp_err(out.cpu().numpy(), oracle.sddmm(p.rowptr, p.colidx, Aq, Bq, p.vals),
                            oracle.sddmm(p.rowptr, p.colidx, Aq, Bq, p.vals, absmode=True)) <= TOL
        else:
            assert comp_err(out.cpu().numpy(), oracle.spmm(p.rowptr, p.colidx, Bq, p.vals),
                            oracle.spmm(p.rowptr, p.colidx, Bq, p.vals, absmode=True)) <= TOL


def test_batch_graph_replay(spk):
    probs = _batch_problems(8, seed=9)
    items, outs = [], []
    keep = []
    for k, p in enumerate(probs):
        S = spk.CSR(p.rowptr, p.colidx, (p.M, p.N), torch.from_numpy(p.vals), device=DEV, chunk_work=64)
        A = torch.from_numpy(p.A).to(DEV); B = torch.from_numpy(p.B).to(DEV)
        out = torch.zeros((p.M, p.K), device=DEV)
        items.append(spk.Item(spk.OP_SPMM, S, B, out))
        keep.append((S, A, B))
        outs.append(out)
    batch = spk.Batch(items)
    batch.capture()
    for o in outs:
        o.fill_(float("nan"))
    batch.replay()
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    for o in outs:
        o.fill_(float("nan"))
    batch.replay(); batch.replay()
    torch.cuda.synchronize()
    for a, b in zip(first, outs):
        assert torch.equal(a, b)
    for (S, A, B), o, p in zip(keep, outs, probs):
        ref = oracle.spmm(p.rowptr, p.colidx, p.B, p.vals)
        assert comp_err(o.cpu().numpy(), ref, oracle.spmm(p.rowptr, p.colidx, p.B, p.vals, absmode=True)) <= TOL


def test_batch_autotune_keeps_results(spk):
    probs = _batch_problems(10, seed=21)
    items, keep = [], []
    for k, p in enumerate(probs):
        S = spk.CSR(p.rowptr, p.colidx, (p.M, p.N), torch.from_numpy(p.vals), device=DEV, chunk_work=512)
        B = torch.from_numpy(p.B).to(DEV)
        out = torch.full((p.M, p.K), float("nan"), device=DEV)
        items.append(spk.Item(spk.OP_SPMM, S, B, out))
        keep.append((S, B, out, p))
    batch = spk.Batch(items)
    res = batch.autotune((64, 256), reps=2)
    assert res["chunk_work"] in (64, 256) and set(res["ms"]) == {64, 256}
    for S, B, out, p in keep:
        assert S.schedule_info()["chunk_work"] == res["chunk_work"]
        out.fill_(float("nan"))
    batch.run()
    torch.cuda.synchronize()
    for S, B, out, p in keep:
        ref = oracle.spmm(p.rowptr, p.colidx, p.B, p.vals)
        assert comp_err(out.cpu().numpy(), ref, oracle.spmm(p.rowptr, p.colidx, p.B, p.vals, absmode=True)) <= TOL


def _batch_items(spk, probs, dt, W=128):
    items, keep = [], []
    for p in probs:
        S = spk.CSR(p.rowptr, p.colidx, (p.M, p.N), torch.from_numpy(p.vals), device=DEV, chunk_work=W)
        A = torch.from_numpy(p.A).to(DEV).to(dt)
        B = torch.from_numpy(p.B).to(DEV).to(dt)
        out = torch.full((p.nnz,), float("nan"), device=DEV)
        C = torch.full((p.M, p.K), float("nan"), device=DEV)
        items.append(spk.Item(spk.OP_SDDMM, S, B, out, A=A))
        items.append(spk.Item(spk.OP_SPMM, S, B, C))
        keep.append((S, A, B, out, C, p))
    return items, keep


def _check_batch_outputs(keep, dt):
    for S, A, B, out, C, p in keep:
        Aq = A.float().cpu().numpy(); Bq = B.float().cpu().numpy()
        assert comp_err(out.cpu().numpy(), oracle.sddmm(p.rowptr, p.colidx, Aq, Bq, p.vals),
                        oracle.sddmm(p.rowptr, p.colidx, Aq, Bq, p.vals, absmode=True)) <= TOL, p.name
        assert comp_err(C.cpu().numpy(), oracle.spmm(p.rowptr, p.colidx, Bq, p.vals),
                        oracle.spmm(p.rowptr, p.colidx, Bq, p.vals, absmode=True)) <= TOL, p.name


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_batch_every_shape_and_register_budget(spk, dt):
    """Every batched shape of each op (spk_batch_shapes) that fits K, under both
    kernel builds (80 and 96 registers): results against the oracle, and bit
    for bit equal to a standalone launch of the same shape and schedule where
    that shape is compiled standalone."""
    from paper_2404_19638_gb300.binding import batch_shapes, compiled_shapes
    probs = _batch_problems(8, seed=31)
    items, keep = _batch_items(spk, probs, dt)
    batch = spk.Batch(items)
    vecn = 4 if dt == torch.float32 else 8
    standalone = set(compiled_shapes())
    for op in (0, 1):
        for shape in batch_shapes(op):
            G, NV, U = shape
            for k, it in enumerate(items):
                nvec = it.B.size(1) // vecn
                fit = it.op == op and G * NV >= nvec
                batch.set_item_tune(k, {"group_lanes": G, "vecs_per_lane": NV, "unroll": U} if fit else None)
            batch._create()
            for regs in (80, 96):
                batch.set_registers(regs)
                for _, _, _, out, C, _ in keep:
                    out.fill_(float("nan")); C.fill_(float("nan"))
                batch.run()
                torch.cuda.synchronize()
                _check_batch_outputs(keep, dt)
                if shape not in standalone:
                    continue
                tune = {"variant": 2, "group_lanes": G, "vecs_per_lane": NV, "unroll": U}
                for S, A, B, out, C, p in keep:
                    if G * NV < p.K // vecn:
                        continue
                    if op == 0:
                        assert torch.equal(out, spk.sddmm(S, A, B, tune=tune)), (shape, p.name)
                    else:
                        assert torch.equal(C, spk.spmm(S, B, tune=tune)), (shape, p.name)
            batch.set_registers(0)


def test_batch_per_item_autotune(spk):
    """Per-item tuning (chunk size per group of patterns, shape per class,
    register budget): every choice is a valid one and the tuned launch still
    matches the oracle, also after graph capture."""
    from paper_2404_19638_gb300.binding import batch_shapes
    probs = _batch_problems(10, seed=41, n_hi=6000)
    items, keep = _batch_items(spk, probs, torch.float32, W=512)
    batch = spk.Batch(items)
    res = batch.autotune((128, 512), reps=1, per_item=True, min_gain=0.0)
    assert res["chunk_work"] in (128, 512) and res["registers"] in ("default", 80, 96)
    assert res["trials"] > 0 and res["ms_final"] <= min(res["ms"].values())
    for name, shape in res["shapes"].items():
        op = 0 if name.startswith("sddmm") else 1
        assert shape is None or tuple(shape) in batch_shapes(op)
    for S, *_ in keep:
        assert S.schedule_info()["chunk_work"] in (64, 128, 256, 512, 1024)
    batch.capture()
    for _, _, _, out, C, _ in keep:
        out.fill_(float("nan")); C.fill_(float("nan"))
    batch.replay()
    torch.cuda.synchronize()
    _check_batch_outputs(keep, torch.float32)
