// Pipelined spans for the 16-byte vector path: each lane group keeps D batches
// of gathered rows in flight in shared memory.
//
// Per group (G lanes), shared memory holds
//   * two index tiles of T = 4G nonzeros (column, COO row, value), filled with
//     ordinary loads when the issue cursor enters a new tile,
//   * a ring of D slots, each holding the U gathered B rows of one batch
//     (lane gl's 16-byte vectors of every row), written by cp.async,
//   * (SDDMM) a ring of D A-row slices, copied when a batch starts a new row.
// The issue cursor runs D-1 batches ahead of the compute cursor.  Every lane
// reads back only the vectors it copied itself, so the only synchronisation
// on gathered data is the lane's own cp.async.wait_group: no waits on other
// lanes, warps or blocks.  Registers no longer bound the bytes in flight:
// the gathers of D-1 batches per group are outstanding while one is reduced.
#pragma once
#include "tiles.cuh"

namespace spk {

constexpr int PIPE_D = 4;   // batches in flight per group (ring slots)

// 32-bit words of shared memory one group uses (host and device).
__host__ __device__ constexpr int pipe_words(int G, int NV, int U, int a_vec16)
{
    // tiles + B ring + A ring (a_vec16 = 16-byte vectors per lane of one A slice)
    return 2 * 3 * 4 * G + PIPE_D * U * NV * G * 4 + PIPE_D * a_vec16 * G * 4;
}

// Fill index tile `buf` with entries [tb, tb + 4G) (column, row, value) using
// ordinary loads; entries past n are left unset.
template <int G>
__device__ __forceinline__ void load_tile(int* tiles, int buf, int64_t tb, int64_t n, int gl, const int32_t* colidx,
                                          const int32_t* rowidx, const float* vals)
{
    constexpr int T = 4 * G;
    int* col = tiles + buf * T;
    int* row = tiles + 2 * T + buf * T;
    int* val = tiles + 4 * T + buf * T;
    const int64_t e = tb + 4 * gl;
    if (e + 4 <= n) {
        *reinterpret_cast<int4*>(col + 4 * gl) = __ldg(reinterpret_cast<const int4*>(colidx + e));
        if (rowidx) *reinterpret_cast<int4*>(row + 4 * gl) = __ldg(reinterpret_cast<const int4*>(rowidx + e));
        if (vals) *reinterpret_cast<int4*>(val + 4 * gl) = __ldg(reinterpret_cast<const int4*>(vals + e));
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (e + k < n) {
                col[4 * gl + k] = __ldg(colidx + e + k);
                if (rowidx) row[4 * gl + k] = __ldg(rowidx + e + k);
                if (vals) val[4 * gl + k] = __float_as_int(__ldg(vals + e + k));
            }
        }
    }
}

// ----------------------------------------------------------------------------
// SDDMM
// ----------------------------------------------------------------------------
template <int DTA, int DTB, int G, int NV, int U, bool KNOWN_ROW>
__device__ __forceinline__ void sddmm_span_pipe(const SddmmArgs& a, const Group<G>& g, int* sm, int64_t r0,
                                                int64_t e0, int64_t e1)
{
    constexpr int VECN = vec_elems(DTB);
    constexpr int T = 4 * G;
    constexpr int D = PIPE_D;
    constexpr int AV = VECN * dt_bytes(DTA) / 16;        // 16-byte vectors per A slice vector
    static_assert(D * U <= T, "the issue cursor may run at most one tile ahead");
    if (e0 >= e1) return;
    int* tiles = sm;
    uint4* bring = reinterpret_cast<uint4*>(sm + 2 * 3 * T);
    uint4* aring = bring + D * U * NV * G;
    const int nvec = a.K / VECN;

    const int64_t pb0 = e0 & ~int64_t(U - 1);
    const int nb = (int)((e1 - pb0 + U - 1) / U);
    const int32_t* rsrc = KNOWN_ROW ? nullptr : a.rowidx;
    int issue_tile = -1;
    int last_issued_row = -1;

    auto issue = [&](int s) {
        const int pos = s * U;
        const int tid = pos / T, buf = tid & 1, off = pos % T;
        if (tid != issue_tile) {
            __syncwarp(g.mask);
            load_tile<G>(tiles, buf, pb0 + (int64_t)tid * T, a.nnz, g.gl, a.colidx, rsrc, nullptr);
            __syncwarp(g.mask);
            issue_tile = tid;
        }
        const int* col = tiles + buf * T;
        const int* row = tiles + 2 * T + buf * T;
        const int slot = s % D;
        int first_row = -1, last_row = -1;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = pb0 + pos + u;
            if (e < e0 || e >= e1) continue;
            const int j = col[off + u];
            const int r = KNOWN_ROW ? (int)r0 : row[off + u];
            if (first_row < 0) first_row = r;
            last_row = r;
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                const int v = t * G + g.gl;
                if (v < nvec)
                    cp_async16(bring + ((slot * U + u) * NV + t) * G + g.gl,
                               reinterpret_cast<const char*>(a.B) + ((int64_t)j * a.ldb + (int64_t)v * VECN) * dt_bytes(DTB), 16);
            }
        }
        if (first_row >= 0 && first_row != last_issued_row) {
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                const int v = t * G + g.gl;
                if (v < nvec) {
#pragma unroll
                    for (int h = 0; h < AV; ++h)
                        cp_async16(aring + ((slot * NV + t) * AV + h) * G + g.gl,
                                   reinterpret_cast<const char*>(a.A) +
                                       ((int64_t)first_row * a.lda + (int64_t)v * VECN) * dt_bytes(DTA) + 16 * h, 16);
                }
            }
        }
        if (last_row >= 0) last_issued_row = last_row;
    };

#pragma unroll 1
    for (int s = 0; s < D - 1; ++s) {
        if (s < nb) issue(s);
        cp_async_commit();
    }

    float av[NV][VECN];
    int a_row = -1;
#pragma unroll 1
    for (int c = 0; c < nb; ++c) {
        if (c + D - 1 < nb) issue(c + D - 1);
        cp_async_commit();
        cp_async_wait<D - 1>();

        const int pos = c * U;
        const int buf = (pos / T) & 1, off = pos % T;
        const int* row = tiles + 2 * T + buf * T;
        const int slot = c % D;
        const int64_t eb = pb0 + pos;
        float sv = 0.f;
        const int64_t ew = eb + g.gl;
        const bool writer = (g.gl < U) && (ew >= e0) && (ew < e1);
        if (writer) {
            sv = a.vals ? __ldg(a.vals + ew) : 1.f;
            if (a.vals2) sv *= __ldg(a.vals2 + ew);
        }
        float p[U];
        bool first = true;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            p[u] = 0.f;
            const int64_t e = eb + u;
            if (e < e0 || e >= e1) continue;
            const int r = KNOWN_ROW ? (int)r0 : row[off + u];
            if (r != a_row) {
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    const int v = t * G + g.gl;
                    if (v >= nvec) {
#pragma unroll
                        for (int q = 0; q < VECN; ++q) av[t][q] = 0.f;
                    } else if (first) {
                        // the batch starts a new row: its A slice arrived with the batch
                        Raw<DTA, VECN> ra;
#pragma unroll
                        for (int h = 0; h < AV; ++h) {
                            const uint4 w = aring[((slot * NV + t) * AV + h) * G + g.gl];
                            ra.w[4 * h] = w.x; ra.w[4 * h + 1] = w.y; ra.w[4 * h + 2] = w.z; ra.w[4 * h + 3] = w.w;
                        }
                        unpack_all<DTA, VECN>(ra, av[t]);
                    } else {
                        // a row change inside the batch (short rows): direct load
                        load_elems<DTA, VECN>(a.A, (int64_t)r * a.lda + (int64_t)v * VECN, av[t]);
                    }
                }
                a_row = r;
            }
            first = false;
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                if (t * G + g.gl >= nvec) continue;
                const uint4 w = bring[((slot * U + u) * NV + t) * G + g.gl];
                Raw<DTB, VECN> rb;
                rb.w[0] = w.x; rb.w[1] = w.y; rb.w[2] = w.z; rb.w[3] = w.w;
                float bf[VECN];
                unpack_all<DTB, VECN>(rb, bf);
#pragma unroll
                for (int q = 0; q < VECN; ++q) p[u] = fmaf(av[t][q], bf[q], p[u]);
            }
            if constexpr (DTA == DT_E4M3) {
                const int j = tiles[buf * T + off + u];
                p[u] *= __ldg(a.a_scale + r) * __ldg(a.b_scale + j);
            }
        }
#pragma unroll
        for (int d = U / 2; d >= 1; d >>= 1) {
            const bool upper = (g.gl & d) != 0;
#pragma unroll
            for (int i = 0; i < d; ++i) {
                const float send = upper ? p[i] : p[i + d];
                const float keep = upper ? p[i + d] : p[i];
                p[i] = keep + __shfl_xor_sync(g.mask, send, d, G);
            }
        }
#pragma unroll
        for (int d = U; d < G; d <<= 1) p[0] += __shfl_xor_sync(g.mask, p[0], d, G);
        if (writer) __stcs(a.out + ew, sv * p[0]);
    }
    cp_async_wait<0>();
    __syncwarp(g.mask);
}


// ----------------------------------------------------------------------------
// SpMM (flush / piece helpers from spmm_impl.cuh)
// ----------------------------------------------------------------------------
template <int VECN, int G, int NV>
__device__ __forceinline__ void write_row(const SpmmArgs& a, const Group<G>& g, int kb, int nvec, int64_t row,
                                          const float (&acc)[NV][VECN]);
template <int VECN, int G, int NV>
__device__ __forceinline__ void zero_row(const SpmmArgs& a, const Group<G>& g, int kb, int nvec, int64_t row);
template <int VECN, int G, int NV>
__device__ __forceinline__ void finish_piece(const SpmmArgs& a, const Group<G>& g, int kb, int nkb, int nvec,
                                             int slot, int s0, int64_t row, const float (&acc)[NV][VECN]);

template <int DTB, int G, int NV, int U, bool KNOWN_ROW>
__device__ __forceinline__ void spmm_span_pipe(const SpmmArgs& a, const Group<G>& g, int* sm, int kb, int nkb,
                                               int64_t r0, int64_t e0, int64_t r1, int64_t e1, const int4 meta,
                                               int head_s0)
{
    constexpr int VECN = vec_elems(DTB);
    constexpr int T = 4 * G;
    constexpr int D = PIPE_D;
    static_assert(D * U <= T, "the issue cursor may run at most one tile ahead");
    int* tiles = sm;
    uint4* bring = reinterpret_cast<uint4*>(sm + 2 * 3 * T);
    const int nvec = a.K / VECN;
    const int vbase = kb * G * NV;

    float acc[NV][VECN];
#pragma unroll
    for (int t = 0; t < NV; ++t)
#pragma unroll
        for (int q = 0; q < VECN; ++q) acc[t][q] = 0.f;
    int64_t cur = r0;
    auto flush = [&](int64_t row) {
        if (!KNOWN_ROW && row == r0 && meta.x >= 0)
            finish_piece<VECN, G, NV>(a, g, kb, nkb, nvec, meta.x, head_s0, row, acc);
        else if (!KNOWN_ROW && row == r1 && meta.y >= 0)
            finish_piece<VECN, G, NV>(a, g, kb, nkb, nvec, meta.y, meta.y, row, acc);
        else
            write_row<VECN, G, NV>(a, g, kb, nvec, row, acc);
    };

    if (e0 < e1) {
        const int64_t pb0 = e0 & ~int64_t(U - 1);
        const int nb = (int)((e1 - pb0 + U - 1) / U);
        const int32_t* rsrc = KNOWN_ROW ? nullptr : a.rowidx;
        const float* vsrc = a.vals_staged ? a.vals : nullptr;
        int issue_tile = -1;

        auto issue = [&](int s) {
            const int pos = s * U;
            const int tid = pos / T, buf = tid & 1, off = pos % T;
            if (tid != issue_tile) {
                __syncwarp(g.mask);
                load_tile<G>(tiles, buf, pb0 + (int64_t)tid * T, a.nnz, g.gl, a.colidx, rsrc, vsrc);
                __syncwarp(g.mask);
                issue_tile = tid;
            }
            const int* col = tiles + buf * T;
            const int slot = s % D;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = pb0 + pos + u;
                if (e < e0 || e >= e1) continue;
                const int j = col[off + u];
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    const int v = vbase + t * G + g.gl;
                    if (v < nvec)
                        cp_async16(bring + ((slot * U + u) * NV + t) * G + g.gl,
                                   reinterpret_cast<const char*>(a.B) + ((int64_t)j * a.ldb + (int64_t)v * VECN) * dt_bytes(DTB), 16);
                }
            }
        };

#pragma unroll 1
        for (int s = 0; s < D - 1; ++s) {
            if (s < nb) issue(s);
            cp_async_commit();
        }
#pragma unroll 1
        for (int c = 0; c < nb; ++c) {
            if (c + D - 1 < nb) issue(c + D - 1);
            cp_async_commit();
            cp_async_wait<D - 1>();

            const int pos = c * U;
            const int buf = (pos / T) & 1, off = pos % T;
            const int* col = tiles + buf * T;
            const int* row = tiles + 2 * T + buf * T;
            const float* val = reinterpret_cast<const float*>(tiles + 4 * T + buf * T);
            const int slot = c % D;
            const int64_t eb = pb0 + pos;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = eb + u;
                if (e < e0 || e >= e1) continue;
                float sv;
                if (a.vals_staged) {
                    sv = val[off + u];
                } else {
                    const int64_t vi = a.vperm ? (int64_t)__ldg(a.vperm + e) : e;
                    sv = a.vals ? __ldg(a.vals + vi) : 1.f;
                    if (a.vals2) sv *= __ldg(a.vals2 + vi);
                }
                if constexpr (DTB == DT_E4M3) sv *= __ldg(a.b_scale + col[off + u]);
                if constexpr (!KNOWN_ROW) {
                    const int r = row[off + u];
                    if (r != cur) {
                        flush(cur);
                        for (int64_t rr = cur + 1; rr < r; ++rr) zero_row<VECN, G, NV>(a, g, kb, nvec, rr);
                        cur = r;
#pragma unroll
                        for (int t = 0; t < NV; ++t)
#pragma unroll
                            for (int q = 0; q < VECN; ++q) acc[t][q] = 0.f;
                    }
                }
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    if (vbase + t * G + g.gl >= nvec) continue;
                    const uint4 w = bring[((slot * U + u) * NV + t) * G + g.gl];
                    Raw<DTB, VECN> rb;
                    rb.w[0] = w.x; rb.w[1] = w.y; rb.w[2] = w.z; rb.w[3] = w.w;
                    float bf[VECN];
                    unpack_all<DTB, VECN>(rb, bf);
#pragma unroll
                    for (int q = 0; q < VECN; ++q) acc[t][q] = fmaf(sv, bf[q], acc[t][q]);
                }
            }
        }
        cp_async_wait<0>();
        __syncwarp(g.mask);
    }
    flush(cur);
    for (int64_t rr = cur + 1; rr <= meta.z; ++rr) zero_row<VECN, G, NV>(a, g, kb, nvec, rr);
}

}  // namespace spk
