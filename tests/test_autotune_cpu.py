"""Host logic of the autotuner: pattern signatures and candidate shapes."""
import re
from pathlib import Path

import numpy as np
import torch

import synth
from paper_2404_19638_gb300.autotune import candidate_shapes, pattern_signature
from paper_2404_19638_gb300.binding import compiled_shapes

ROOT = Path(__file__).resolve().parents[1]


def test_candidates_are_compiled_shapes():
    """The library reports the shape table its kernels were compiled from."""
    src = (ROOT / "paper_2404_19638_gb300" / "csrc" / "common.cuh").read_text()
    block = src[src.index("#define SPK_SHAPES"):src.index("constexpr int kNumShapes")]
    compiled = [tuple(int(v) for v in m) for m in re.findall(r"X\(\d+,\s*(\d+),\s*(\d+),\s*(\d+)\)", block)]
    assert compiled_shapes() == compiled


def test_candidates_cover_the_row():
    for dt, vec in ((torch.float32, 4), (torch.bfloat16, 8), (torch.float8_e4m3fn, 16)):
        for K in (vec, 2 * vec, 4 * vec, 16 * vec, 32 * vec, 64 * vec):
            nvec = K // vec
            cands = candidate_shapes(K, dt)
            assert cands
            for G, NV, U in cands:
                assert (G, NV, U) in compiled_shapes()
                assert G * NV >= min(nvec, 128) or (G, NV, U) == (32, 4, 4)


def test_signature_separates_patterns():
    rp1, ci1 = synth.er_exact_degree(1000, 1000, 8, seed=0)
    rp2, ci2 = synth.er_exact_degree(1000, 1000, 8, seed=1)
    rp3, ci3 = synth.rmat(10, 8, seed=0)
    s1 = pattern_signature(rp1, 1000, 1000)
    assert s1 == pattern_signature(rp2, 1000, 1000)          # same shape and degree histogram
    assert s1 != pattern_signature(rp3, 1024, 1024)
    assert s1 != pattern_signature(rp1, 1000, 1001)
    empty = np.zeros(5, np.int32)
    assert pattern_signature(empty, 4, 4) != pattern_signature(np.arange(5, dtype=np.int32), 4, 4)


def test_cache_round_trip_and_lookup(tmp_path):
    """Entries persist through the JSON cache and are found again by the key of
    a pattern with the same signature (host-only stand-in for a CSR)."""
    import types
    from paper_2404_19638_gb300.autotune import Autotuner
    rp, _ = synth.er_exact_degree(500, 400, 6, seed=2)
    S = types.SimpleNamespace(rowptr=torch.from_numpy(rp), M=500, N=400)
    path = tmp_path / "tune.json"
    t1 = Autotuner(cache_path=str(path))
    assert t1.lookup(S, "spmm", torch.float32, 64) is None
    key = t1.key(S, "spmm", torch.float32, 64)
    t1._cache[key] = {"group_lanes": 16, "vecs_per_lane": 1, "unroll": 8, "chunk_work": 512}
    t1._save()
    t2 = Autotuner(cache_path=str(path))
    assert t2.lookup(S, "spmm", torch.float32, 64) == t1._cache[key]
    assert t2.lookup(S, "spmm", torch.bfloat16, 64) is None          # dtype is part of the key
    assert t2.lookup(S, "sddmm", torch.float32, 64) is None          # so is the operation
