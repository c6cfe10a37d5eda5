// Lean spans for the 16-byte vector path: few instructions per nonzero.
//
// Per nonzero the essential work is one gathered row (K * elt bytes, 0.5
// warp-wide 128-bit loads per nonzero at 256 bytes) and K FMAs (K/32 warp
// instructions).  Everything else is overhead to amortise:
//   * index streams are read as 128-bit loads that every lane of a group
//     issues for the same address (one request per group), 4 nonzeros each;
//   * offsets are 32-bit products widened once (row * row-bytes);
//   * a batch whose nonzeros are all valid and all in the current row takes a
//     branch-free path; only span edges and row changes take the general one;
//   * with 8 lanes per row (16-byte vectors, 128-byte lines) a warp-wide load
//     covers four rows at full line efficiency and the per-batch bookkeeping
//     is shared by four nonzeros.
#pragma once
#include "tiles.cuh"

namespace spk {

template <int G>
__device__ __forceinline__ unsigned group_mask(int lane)
{
    return (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
}

// Four consecutive int32 (or float) entries at a 16-byte aligned position.
__device__ __forceinline__ int4 ld4(const int32_t* p) { return __ldg(reinterpret_cast<const int4*>(p)); }

// ----------------------------------------------------------------------------
// SDDMM: a warp walks a span of nonzeros in warp batches of (32/G)*U; group k
// of the warp takes nonzeros [wb + kU, wb + kU + U).  Outputs are per nonzero,
// so the groups never combine results.
// ----------------------------------------------------------------------------
template <int DTA, int DTB, int G, int NV, int U, bool KNOWN_ROW>
__device__ __forceinline__ void sddmm_warp_span(const SddmmArgs& a, int lane, int r0, int e0, int e1)
{
    constexpr int VECN = vec_elems(DTB);
    constexpr int GPW = 32 / G;
    constexpr int WB = GPW * U;
    static_assert(U % 4 == 0 && U <= G, "index batches are read four at a time; U lanes store results");
    const int grp = lane / G, gl = lane % G;
    const unsigned gmask = group_mask<G>(lane);
    const int nvec = a.K / VECN;
    const char* __restrict__ Bb = reinterpret_cast<const char*>(a.B);
    const char* __restrict__ Ab = reinterpret_cast<const char*>(a.A);
    const unsigned ldb_bytes = (unsigned)a.ldb * dt_bytes(DTB);
    const unsigned lda_bytes = (unsigned)a.lda * dt_bytes(DTA);
    bool vin[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) vin[t] = (t * G + gl) < nvec;
    const bool all_vin = (nvec >= G * NV);                     // no lane has a vector past K
    const unsigned lane_off = (unsigned)gl * 16u;              // byte offset of the lane's first vector

    float av[NV][VECN];
    int cur = -1;
    // Indices of the next batch are loaded while the current batch's rows are
    // being gathered, so a batch costs one memory round trip, not two.
    int nj[U], nrow[U];
    bool nfull = false;
    auto load_idx = [&](int eg) {
        nfull = (eg >= e0) && (eg + U <= e1);
        if (nfull) {
#pragma unroll
            for (int u = 0; u < U; u += 4) {
                const int4 c = ld4(a.colidx + eg + u);
                nj[u] = c.x; nj[u + 1] = c.y; nj[u + 2] = c.z; nj[u + 3] = c.w;
                if constexpr (!KNOWN_ROW) {
                    const int4 r = ld4(a.rowidx + eg + u);
                    nrow[u] = r.x; nrow[u + 1] = r.y; nrow[u + 2] = r.z; nrow[u + 3] = r.w;
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = eg + u;
                const bool ok = (e >= e0) && (e < e1);
                nj[u] = ok ? __ldg(a.colidx + e) : -1;
                if constexpr (!KNOWN_ROW) nrow[u] = ok ? __ldg(a.rowidx + e) : -1;
            }
        }
        if constexpr (KNOWN_ROW) {
#pragma unroll
            for (int u = 0; u < U; ++u) nrow[u] = r0;
        }
    };
    const int wb0 = e0 & ~3;
    if (wb0 + grp * U < e1) load_idx(wb0 + grp * U);
    for (int wb = wb0; wb < e1; wb += WB) {
        const int eg = wb + grp * U;
        if (eg >= e1) continue;
        const bool full = nfull;
        int j[U], row[U];
#pragma unroll
        for (int u = 0; u < U; ++u) { j[u] = nj[u]; row[u] = nrow[u]; }
        // the lane that stores nonzero eg + gl fetches its scale early
        const int ew = eg + gl;
        const bool writer = (gl < U) && (ew >= e0) && (ew < e1);
        float sv = 0.f;
        if (writer) {
            sv = a.vals ? __ldg(a.vals + ew) : 1.f;
            if (a.vals2) sv *= __ldg(a.vals2 + ew);
        }
        if (eg + WB < e1) load_idx(eg + WB);
        float p[U];
        if (full && all_vin && row[0] == cur && row[U - 1] == cur) {
            // Common case: U valid nonzeros of the current row, every lane's
            // vectors inside K: unconditional loads, one address per row.
            uint4 bw[U][NV];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint4* brow = reinterpret_cast<const uint4*>(Bb + (size_t)(unsigned)j[u] * ldb_bytes + lane_off);
#pragma unroll
                for (int t = 0; t < NV; ++t) bw[u][t] = __ldg(brow + t * G);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                p[u] = 0.f;
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    Raw<DTB, VECN> rb;
                    rb.w[0] = bw[u][t].x; rb.w[1] = bw[u][t].y; rb.w[2] = bw[u][t].z; rb.w[3] = bw[u][t].w;
                    float bf[VECN];
                    unpack_all<DTB, VECN>(rb, bf);
#pragma unroll
                    for (int q = 0; q < VECN; ++q) p[u] = fmaf(av[t][q], bf[q], p[u]);
                }
            }
        } else {
            Raw<DTB, VECN> bw[U][NV];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const char* brow = Bb + (size_t)(unsigned)j[u] * ldb_bytes;
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    if ((full || j[u] >= 0) && vin[t])
                        load_raw<DTB, VECN>(brow, (int64_t)(t * G + gl) * VECN, bw[u][t]);
                    else
                        zero_raw(bw[u][t]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                p[u] = 0.f;
                if (!full && j[u] < 0) continue;
                if (row[u] != cur) {
                    cur = row[u];
                    const char* arow = Ab + (size_t)(unsigned)cur * lda_bytes;
#pragma unroll
                    for (int t = 0; t < NV; ++t) {
                        if (vin[t]) load_elems<DTA, VECN>(arow, (int64_t)(t * G + gl) * VECN, av[t]);
                        else
#pragma unroll
                            for (int q = 0; q < VECN; ++q) av[t][q] = 0.f;
                    }
                }
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    float bf[VECN];
                    unpack_all<DTB, VECN>(bw[u][t], bf);
#pragma unroll
                    for (int q = 0; q < VECN; ++q) p[u] = fmaf(av[t][q], bf[q], p[u]);
                }
            }
        }
        if constexpr (DTA == DT_E4M3) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (full || j[u] >= 0) p[u] *= __ldg(a.a_scale + row[u]) * __ldg(a.b_scale + j[u]);
        }
        // Reduce-scatter over the low log2(U) lane bits, then butterflies over
        // the remaining G/U lane subsets: nonzero eg + (gl % U) ends in lane gl.
#pragma unroll
        for (int d = U / 2; d >= 1; d >>= 1) {
            const bool upper = (gl & d) != 0;
#pragma unroll
            for (int i = 0; i < d; ++i) {
                const float send = upper ? p[i] : p[i + d];
                const float keep = upper ? p[i + d] : p[i];
                p[i] = keep + __shfl_xor_sync(gmask, send, d, G);
            }
        }
#pragma unroll
        for (int d = U; d < G; d <<= 1) p[0] += __shfl_xor_sync(gmask, p[0], d, G);
        if (writer) __stcs(a.out + ew, sv * p[0]);
    }
}

// ----------------------------------------------------------------------------
// SpMM: a group walks its own span (chunk) U nonzeros at a time, accumulating
// K-slices of the current output row in registers.
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
__device__ __forceinline__ void spmm_group_span(const SpmmArgs& a, const Group<G>& g, int kb, int nkb, int r0,
                                                int e0, int r1, int e1, const int4 meta, int head_s0)
{
    constexpr int VECN = vec_elems(DTB);
    static_assert(U % 4 == 0, "index batches are read four at a time");
    const int gl = g.gl;
    const int nvec = a.K / VECN;
    const int vbase = kb * G * NV;
    const char* __restrict__ Bb = reinterpret_cast<const char*>(a.B);
    const unsigned ldb_bytes = (unsigned)a.ldb * dt_bytes(DTB);
    bool vin[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) vin[t] = (vbase + t * G + gl) < nvec;
    const bool all_vin = (nvec >= vbase + G * NV);            // no lane has a vector past this K block
    const unsigned lane_off = (unsigned)(vbase + gl) * 16u;   // byte offset of the lane's first vector
    const bool vec_vals = a.vals_staged != 0;            // vals alone, 16-byte aligned

    float acc[NV][VECN];
#pragma unroll
    for (int t = 0; t < NV; ++t)
#pragma unroll
        for (int q = 0; q < VECN; ++q) acc[t][q] = 0.f;
    int cur = r0;
    auto flush = [&](int row) {
        if (!KNOWN_ROW && row == r0 && meta.x >= 0)
            finish_piece<VECN, G, NV>(a, g, kb, nkb, nvec, meta.x, head_s0, row, acc);
        else if (!KNOWN_ROW && row == r1 && meta.y >= 0)
            finish_piece<VECN, G, NV>(a, g, kb, nkb, nvec, meta.y, meta.y, row, acc);
        else
            write_row<VECN, G, NV>(a, g, kb, nvec, row, acc);
    };

    // Indices and values of the next batch are loaded while the current
    // batch's rows are being gathered (one memory round trip per batch).
    int nj[U], nrow[U];
    float ns[U];
    bool nfull = false;
    auto load_idx = [&](int eb) {
        nfull = (eb >= e0) && (eb + U <= e1);
        if (nfull) {
#pragma unroll
            for (int u = 0; u < U; u += 4) {
                const int4 c = ld4(a.colidx + eb + u);
                nj[u] = c.x; nj[u + 1] = c.y; nj[u + 2] = c.z; nj[u + 3] = c.w;
                if constexpr (!KNOWN_ROW) {
                    const int4 r = ld4(a.rowidx + eb + u);
                    nrow[u] = r.x; nrow[u + 1] = r.y; nrow[u + 2] = r.z; nrow[u + 3] = r.w;
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = eb + u;
                const bool ok = (e >= e0) && (e < e1);
                nj[u] = ok ? __ldg(a.colidx + e) : -1;
                if constexpr (!KNOWN_ROW) nrow[u] = ok ? __ldg(a.rowidx + e) : -1;
            }
        }
        if constexpr (KNOWN_ROW) {
#pragma unroll
            for (int u = 0; u < U; ++u) nrow[u] = r0;
        }
        if (nfull && vec_vals) {
#pragma unroll
            for (int u = 0; u < U; u += 4) {
                const float4 v4 = __ldg(reinterpret_cast<const float4*>(a.vals + eb + u));
                ns[u] = v4.x; ns[u + 1] = v4.y; ns[u + 2] = v4.z; ns[u + 3] = v4.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float sv = 0.f;
                if (nfull || nj[u] >= 0) {
                    const int e = eb + u;
                    const int vi = a.vperm ? __ldg(a.vperm + e) : e;
                    sv = a.vals ? __ldg(a.vals + vi) : 1.f;
                    if (a.vals2) sv *= __ldg(a.vals2 + vi);
                }
                ns[u] = sv;
            }
        }
    };
    // An empty span (e0 == e1) still rounds down to a batch start below e1:
    // it must not enter the loop, whose indices come from load_idx.
    if (e0 < e1) load_idx(e0 & ~3);
    for (int eb = e0 & ~3; e0 < e1 && eb < e1; eb += U) {
        const bool full = nfull;
        int j[U], row[U];
        float s[U];
#pragma unroll
        for (int u = 0; u < U; ++u) { j[u] = nj[u]; row[u] = nrow[u]; s[u] = ns[u]; }
        if constexpr (DTB == DT_E4M3) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (full || j[u] >= 0) s[u] *= __ldg(a.b_scale + j[u]);
        }
        if (eb + U < e1) load_idx(eb + U);
        if (full && all_vin && (KNOWN_ROW || row[U - 1] == cur)) {
            // Common case: U valid nonzeros of the current row, every lane's
            // vectors inside this K block: unconditional loads.
            uint4 bw[U][NV];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint4* brow = reinterpret_cast<const uint4*>(Bb + (size_t)(unsigned)j[u] * ldb_bytes + lane_off);
#pragma unroll
                for (int t = 0; t < NV; ++t) bw[u][t] = __ldg(brow + t * G);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    Raw<DTB, VECN> rb;
                    rb.w[0] = bw[u][t].x; rb.w[1] = bw[u][t].y; rb.w[2] = bw[u][t].z; rb.w[3] = bw[u][t].w;
                    float bf[VECN];
                    unpack_all<DTB, VECN>(rb, bf);
#pragma unroll
                    for (int q = 0; q < VECN; ++q) acc[t][q] = fmaf(s[u], bf[q], acc[t][q]);
                }
        } else {
            Raw<DTB, VECN> bw[U][NV];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const char* brow = Bb + (size_t)(unsigned)j[u] * ldb_bytes;
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    if ((full || j[u] >= 0) && vin[t])
                        load_raw<DTB, VECN>(brow, (int64_t)(vbase + t * G + gl) * VECN, bw[u][t]);
                    else
                        zero_raw(bw[u][t]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!full && j[u] < 0) continue;
                if constexpr (!KNOWN_ROW) {
                    if (row[u] != cur) {
                        flush(cur);
                        for (int rr = cur + 1; rr < row[u]; ++rr) zero_row<VECN, G, NV>(a, g, kb, nvec, rr);
                        cur = row[u];
#pragma unroll
                        for (int t = 0; t < NV; ++t)
#pragma unroll
                            for (int q = 0; q < VECN; ++q) acc[t][q] = 0.f;
                    }
                }
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    float bf[VECN];
                    unpack_all<DTB, VECN>(bw[u][t], bf);
#pragma unroll
                    for (int q = 0; q < VECN; ++q) acc[t][q] = fmaf(s[u], bf[q], acc[t][q]);
                }
            }
        }
    }
    flush(cur);
    for (int rr = cur + 1; rr <= meta.z; ++rr) zero_row<VECN, G, NV>(a, g, kb, nvec, rr);
}

}  // namespace spk
