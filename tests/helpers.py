"""Shared test utilities: componentwise error metric and small edge-case patterns.

Error metric (floating point parity): for every output, the absolute
difference divided by the sum of the magnitudes of the terms that form it
(|s_e| sum_k |a_ik b_jk| for SDDMM, sum_e |s_e| |b_jk| for SpMM), i.e. the
error relative to the condition of the sum.  Outputs whose denominator is 0
must match exactly.  FP32 accumulation of n terms is bounded by about
n * 2^-24 in this metric; the tests use 1e-5.
"""
from __future__ import annotations

import numpy as np

import synth

TOL = 1e-5          # FP32-accumulation tolerance against the FP64 oracle on the same inputs
TOL_BF16_X = 2e-2   # BF16 / F16 inputs against the oracle on the original FP32 inputs


def comp_err(got, ref, den) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.asarray(den, dtype=np.float64)
    zero = den == 0
    if np.any(zero) and not np.array_equal(got[zero], ref[zero]):
        return float("inf")
    d = np.abs(got - ref)
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(zero, 0.0, d / np.where(zero, 1.0, den))
    return float(r.max(initial=0.0))


def edge_pattern(M: int, N: int, seed: int, long_row: int = 0, empty_every: int = 5, deg_max: int = 12):
    """Random pattern with empty rows (incl. the first and last), a run of
    empty rows, and optionally one row with ``long_row`` nonzeros."""
    g = np.random.default_rng(seed)
    deg = g.integers(0, deg_max + 1, M)
    deg[::empty_every] = 0
    deg[0] = 0
    deg[M - 1] = 0
    if M > 20:
        deg[10:17] = 0
    rows = np.repeat(np.arange(M), deg)
    cols = g.integers(0, N, rows.size)
    if long_row:
        r = M // 3
        rows = np.concatenate([rows, np.full(long_row, r)])
        cols = np.concatenate([cols, g.integers(0, N, long_row)])
    return synth.csr_from_coo(rows, cols, M, N)


def row_of(rowptr):
    return np.repeat(np.arange(rowptr.size - 1), np.diff(rowptr.astype(np.int64)))
