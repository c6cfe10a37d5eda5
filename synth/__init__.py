"""Seeded synthetic inputs for the local SDDMM / SpMM path.

This module only draws random patterns and values.  It holds none of the
method's arithmetic (no products, no sums over nonzeros), so that the CPU
oracle and the CUDA path can both be fed from it while sharing no code.

Every generator takes an integer ``seed`` and derives one independent numpy
PCG64 stream per array from ``(seed, stream_id)``, so that e.g. the values of
a matrix do not change when its pattern generator changes.

Patterns are returned as CSR with int32 ``rowptr`` (M+1) and ``colidx`` (nnz),
columns sorted ascending and unique within a row.

Workload recipes (the synthetic stand-ins for the paper's SuiteSparse graphs
of Sec. 7.1, Table 1, which are not available here):

* ``tiny``   4096 x 4096, exactly 16 distinct uniform columns per row,
             values U[-1,1]; A, B 4096 x 32 U[-1,1].
* ``rmat20`` R-MAT scale 20, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05),
             2^20 * 16 sampled edges, duplicates removed; values U[-1,1];
             A, B 2^20 x 64 N(0,1).
* ``rec``    2,000,000 x 500,000 Chung-Lu bipartite graph with Zipf(1.1)
             weights clipped to [1, 20000], exactly 50,000,000 distinct
             pairs; values uniform on {1..5}; A 2M x 128, B 500K x 128 N(0,1)
             (the low-precision copies are made by the path under test).
* ``gnn``    R-MAT scale 22, edge factor 8, values 1; H 2^22 x 64 N(0, 0.1).
* ``batch``  256 matrices, n log-uniform in [1e3, 2e5]; the first 128
             Erdos-Renyi with an exact degree d ~ U{4..32}, the other 128
             R-MAT edge factor 16 at scale ceil(log2 n) with out-of-range
             endpoints rejected; K ~ U{16,32,64}.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)

# Stream ids: one independent random stream per array of a workload.
_PATTERN, _VALS, _A, _B, _G, _SAMPLE, _META = 0, 1, 2, 3, 4, 5, 6


def rng(seed: int, stream: int, sub: int = 0) -> np.random.Generator:
    """Independent PCG64 stream for (seed, stream, sub)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream), int(sub)])))


# ----------------------------------------------------------------------------
# CSR assembly from sorted unique (row, col) keys
# ----------------------------------------------------------------------------

def _dedup_sorted(keys: np.ndarray) -> np.ndarray:
    keys = np.sort(keys)
    if keys.size == 0:
        return keys
    keep = np.empty(keys.size, dtype=bool)
    keep[0] = True
    np.not_equal(keys[1:], keys[:-1], out=keep[1:])
    return keys[keep]


def csr_from_keys(keys: np.ndarray, M: int, N: int):
    """keys = row * N + col, sorted and unique -> (rowptr int32, colidx int32)."""
    rows = keys // N
    cols = (keys - rows * N).astype(np.int32)
    counts = np.bincount(rows, minlength=M)
    rowptr = np.zeros(M + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 indices")
    return rowptr.astype(np.int32), cols


def csr_from_coo(rows, cols, M: int, N: int):
    """Arbitrary (row, col) lists -> sorted, de-duplicated CSR."""
    keys = np.asarray(rows, dtype=np.int64) * N + np.asarray(cols, dtype=np.int64)
    return csr_from_keys(_dedup_sorted(keys), M, N)


# ----------------------------------------------------------------------------
# Pattern generators
# ----------------------------------------------------------------------------

def er_exact_degree(M: int, N: int, deg: int, seed: int, sub: int = 0):
    """Each row gets exactly ``deg`` distinct columns drawn uniformly from [0, N)."""
    if deg > N:
        raise ValueError("degree exceeds number of columns")
    g = rng(seed, _PATTERN, sub)
    if deg == 0 or M == 0:
        return np.zeros(M + 1, np.int32), np.zeros(0, np.int32)
    cols = g.integers(0, N, size=(M, deg), dtype=np.int64)
    while True:
        cols.sort(axis=1)
        dup = np.zeros_like(cols, dtype=bool)
        dup[:, 1:] = cols[:, 1:] == cols[:, :-1]
        ndup = int(dup.sum())
        if ndup == 0:
            break
        cols[dup] = g.integers(0, N, size=ndup, dtype=np.int64)
    rowptr = (np.arange(M + 1, dtype=np.int64) * deg).astype(np.int32)
    return rowptr, cols.reshape(-1).astype(np.int32)


def rmat_edges(scale: int, n_edges: int, g: np.random.Generator, abcd=RMAT_ABCD):
    """Draw ``n_edges`` R-MAT edges at 2^scale vertices (no permutation, no noise).

    At each of the ``scale`` levels one uniform number picks a quadrant with
    probabilities a (top-left), b (top-right), c (bottom-left), d (bottom-right).
    """
    a, b, c, _ = abcd
    t_ab, t_abc = np.float32(a + b), np.float32(a + b + c)
    t_a = np.float32(a)
    r = np.zeros(n_edges, dtype=np.int64)
    col = np.zeros(n_edges, dtype=np.int64)
    for lvl in range(scale):
        u = g.random(n_edges, dtype=np.float32)
        bit = np.int64(1) << np.int64(scale - 1 - lvl)
        down = u >= t_ab
        right = ((u >= t_a) & (u < t_ab)) | (u >= t_abc)
        r[down] |= bit
        col[right] |= bit
    return r, col


def rmat(scale: int, edge_factor: int, seed: int, n: int | None = None, abcd=RMAT_ABCD, sub: int = 0):
    """R-MAT pattern, duplicates removed.  With ``n`` (not a power of two) the
    graph is drawn at scale ceil(log2 n) and edges with an endpoint >= n are
    rejected until edge_factor * n edges have been kept."""
    g = rng(seed, _PATTERN, sub)
    if n is None:
        n = 1 << scale
        r, c = rmat_edges(scale, edge_factor * n, g, abcd)
    else:
        scale = max(1, math.ceil(math.log2(n)))
        want = edge_factor * n
        rs, cs, have = [], [], 0
        while have < want:
            draw = int((want - have) * 1.3) + 1024
            r, c = rmat_edges(scale, draw, g, abcd)
            ok = (r < n) & (c < n)
            r, c = r[ok], c[ok]
            take = min(want - have, r.size)
            rs.append(r[:take]); cs.append(c[:take]); have += take
        r, c = np.concatenate(rs), np.concatenate(cs)
    return csr_from_coo(r, c, n, n)


def zipf_weights(count: int, alpha: float, lo: int, hi: int, g: np.random.Generator):
    return np.clip(g.zipf(alpha, size=count), lo, hi).astype(np.float64)


def chung_lu(M: int, N: int, nnz: int, alpha: float, dmin: int, dmax: int, seed: int, sub: int = 0):
    """Bipartite Chung-Lu pattern with exactly ``nnz`` distinct (row, col) pairs.

    Row and column weights are Zipf(alpha) draws clipped to [dmin, dmax]; pairs
    are sampled with probability proportional to w_row * w_col until at least
    ``nnz`` distinct pairs exist, and then exactly ``nnz`` of the distinct pairs
    are kept by a seeded uniform choice.
    """
    g = rng(seed, _PATTERN, sub)
    wr = zipf_weights(M, alpha, dmin, dmax, g)
    wc = zipf_weights(N, alpha, dmin, dmax, g)
    cr = np.cumsum(wr); cr /= cr[-1]
    cc = np.cumsum(wc); cc /= cc[-1]
    keys = np.zeros(0, dtype=np.int64)
    while keys.size < nnz:
        draw = int((nnz - keys.size) * 1.15) + 4096
        r = np.minimum(np.searchsorted(cr, g.random(draw), side="right"), M - 1)
        c = np.minimum(np.searchsorted(cc, g.random(draw), side="right"), N - 1)
        keys = _dedup_sorted(np.concatenate([keys, r.astype(np.int64) * N + c]))
    if keys.size > nnz:
        pick = np.sort(g.choice(keys.size, size=nnz, replace=False))
        keys = keys[pick]
    return csr_from_keys(keys, M, N)


# ----------------------------------------------------------------------------
# Dense values
# ----------------------------------------------------------------------------

def uniform(shape, lo, hi, seed: int, stream: int, sub: int = 0, dtype=np.float32):
    return rng(seed, stream, sub).uniform(lo, hi, size=shape).astype(dtype)


def normal(shape, std, seed: int, stream: int, sub: int = 0, dtype=np.float32):
    return (rng(seed, stream, sub).standard_normal(size=shape) * std).astype(dtype)


def uniform_int(shape, lo, hi, seed: int, stream: int, sub: int = 0, dtype=np.float32):
    """Integers uniform on {lo..hi} (inclusive), stored as ``dtype``."""
    return rng(seed, stream, sub).integers(lo, hi + 1, size=shape).astype(dtype)


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    """One sparse matrix S (CSR) with its dense factors (A: M x K, B: N x K)."""
    name: str
    M: int
    N: int
    K: int
    rowptr: np.ndarray
    colidx: np.ndarray
    vals: np.ndarray | None
    A: np.ndarray | None
    B: np.ndarray | None
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.colidx.size)

    def degree_stats(self) -> dict:
        deg = np.diff(self.rowptr.astype(np.int64))
        return {"nnz": self.nnz, "max_deg": int(deg.max(initial=0)),
                "mean_deg": float(deg.mean()) if deg.size else 0.0,
                "empty_rows": int((deg == 0).sum())}


def tiny(seed: int = 0, M: int = 4096, N: int = 4096, deg: int = 16, K: int = 32) -> Problem:
    rp, ci = er_exact_degree(M, N, deg, seed)
    return Problem("tiny", M, N, K, rp, ci,
                   uniform(ci.size, -1.0, 1.0, seed, _VALS),
                   uniform((M, K), -1.0, 1.0, seed, _A),
                   uniform((N, K), -1.0, 1.0, seed, _B))


def dense_blocks(M: int, N: int, blocks: int, density: float, background_deg: int, seed: int,
                 block_shape=(128, 64), aligned: bool = True, sub: int = 0):
    """A sparse background of exactly ``background_deg`` distinct uniform
    columns per row, plus ``blocks`` rectangles of ``block_shape`` whose cells
    are each present with probability ``density`` (at positions that are
    multiples of the block shape when ``aligned``, anywhere otherwise).
    Duplicates are removed.  Returns (rowptr, colidx)."""
    g = rng(seed, _PATTERN, sub)
    rp, ci = er_exact_degree(M, N, background_deg, seed, sub) if background_deg else (np.zeros(M + 1, np.int32),
                                                                                       np.zeros(0, np.int32))
    rows = [np.repeat(np.arange(M), np.diff(rp))]
    cols = [ci.astype(np.int64)]
    bh, bw = block_shape
    for _ in range(blocks):
        if aligned:
            r0 = int(g.integers(0, max(1, M // bh))) * bh
            c0 = int(g.integers(0, max(1, N // bw))) * bw
        else:
            r0 = int(g.integers(0, max(1, M - bh)))
            c0 = int(g.integers(0, max(1, N - bw)))
        cell = g.random((min(bh, M - r0), min(bw, N - c0))) < density
        rr, cc = np.nonzero(cell)
        rows.append(rr + r0)
        cols.append(cc + c0)
    return csr_from_coo(np.concatenate(rows), np.concatenate(cols), M, N)


def rmat_problem(scale: int = 20, edge_factor: int = 16, K: int = 64, seed: int = 0,
                 name: str = "rmat20") -> Problem:
    rp, ci = rmat(scale, edge_factor, seed)
    n = 1 << scale
    return Problem(name, n, n, K, rp, ci,
                   uniform(ci.size, -1.0, 1.0, seed, _VALS),
                   normal((n, K), 1.0, seed, _A),
                   normal((n, K), 1.0, seed, _B),
                   {"scale": scale, "edge_factor": edge_factor, "samples": edge_factor << scale})


def rec(seed: int = 0, M: int = 2_000_000, N: int = 500_000, nnz: int = 50_000_000, K: int = 128) -> Problem:
    rp, ci = chung_lu(M, N, nnz, 1.1, 1, 20000, seed)
    return Problem("rec", M, N, K, rp, ci,
                   uniform_int(ci.size, 1, 5, seed, _VALS),
                   normal((M, K), 1.0, seed, _A),
                   normal((N, K), 1.0, seed, _B))


def gnn(seed: int = 0, scale: int = 22, edge_factor: int = 8, K: int = 64) -> Problem:
    """GNN-layer-shaped input: S is the (unit-valued) R-MAT adjacency, A = B = H."""
    rp, ci = rmat(scale, edge_factor, seed)
    n = 1 << scale
    H = normal((n, K), 0.1, seed, _A)
    return Problem("gnn", n, n, K, rp, ci, None, H, H,
                   {"scale": scale, "edge_factor": edge_factor, "samples": edge_factor << scale})


def batch(seed: int = 0, count: int = 256, n_lo: int = 1000, n_hi: int = 200_000,
          K_choices=(16, 32, 64)) -> list[Problem]:
    """The batching workload: ``count`` independent matrices of uneven size."""
    g = rng(seed, _META)
    ns = np.exp(g.uniform(math.log(n_lo), math.log(n_hi), size=count)).astype(np.int64)
    Ks = g.choice(np.asarray(K_choices), size=count)
    degs = g.integers(4, 33, size=count)
    out = []
    for m in range(count):
        n, K = int(ns[m]), int(Ks[m])
        mseed = seed + m
        if m < count // 2:
            rp, ci = er_exact_degree(n, n, int(degs[m]), mseed)
            kind = {"kind": "er", "deg": int(degs[m])}
        else:
            rp, ci = rmat(0, 16, mseed, n=n)
            kind = {"kind": "rmat", "edge_factor": 16}
        out.append(Problem(f"batch{m}", n, n, K, rp, ci,
                           uniform(ci.size, -1.0, 1.0, mseed, _VALS),
                           uniform((n, K), -1.0, 1.0, mseed, _A),
                           uniform((n, K), -1.0, 1.0, mseed, _B), kind))
    return out


def sample_rows(rowptr: np.ndarray, count: int, seed: int, heavy: int = 8) -> np.ndarray:
    """Rows for sampled checks at full size: the ``heavy`` longest rows, the
    first and last rows, and ``count`` uniform rows (sorted, unique)."""
    M = rowptr.size - 1
    g = rng(seed, _SAMPLE)
    deg = np.diff(rowptr.astype(np.int64))
    pick = [np.argsort(deg)[-heavy:], np.array([0, M - 1]), g.integers(0, M, size=count)]
    return np.unique(np.concatenate(pick)).astype(np.int64)


def small_rmat(scale: int = 12, edge_factor: int = 8, K: int = 8, seed: int = 0, std: float = 0.1) -> Problem:
    """Scaled-down GNN copy for finite-difference checks."""
    rp, ci = rmat(scale, edge_factor, seed)
    n = 1 << scale
    H = normal((n, K), std, seed, _A)
    return Problem(f"rmat{scale}", n, n, K, rp, ci, None, H, H)
