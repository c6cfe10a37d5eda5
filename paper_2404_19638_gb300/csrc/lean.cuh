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
//
// Registers bound the gathers in flight (resident warps x U rows), so the hot
// path keeps only the U gathered vectors, the A slice and U partial sums live.
// A batch that is full, inside K and in the current row takes the fast path;
// anything else (span edges, row changes) goes nonzero by nonzero.
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
    const bool all_vin = (nvec >= G * NV);
    const char* __restrict__ Bb = reinterpret_cast<const char*>(a.B) + gl * 16;   // lane's first vector
    const char* __restrict__ Ab = reinterpret_cast<const char*>(a.A);
    const unsigned ldb_bytes = (unsigned)a.ldb * dt_bytes(DTB);
    const unsigned lda_bytes = (unsigned)a.lda * dt_bytes(DTA);

    float av[NV][VECN];
    int cur = -1;
    auto load_a = [&](int r) {
        const char* arow = Ab + (size_t)(unsigned)r * lda_bytes;
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            if (t * G + gl < nvec) load_elems<DTA, VECN>(arow, (int64_t)(t * G + gl) * VECN, av[t]);
            else
#pragma unroll
                for (int q = 0; q < VECN; ++q) av[t][q] = 0.f;
        }
    };
    bool vin[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) vin[t] = all_vin || (t * G + gl < nvec);
    for (int wb = e0 & ~3; wb < e1; wb += WB) {
        const int eg = wb + grp * U;
        if (eg >= e1) continue;
        // One batch body for every case; invalid slots, row changes and K tails
        // are predicates, so the lock-stepped groups of a warp never run two
        // different code paths one after the other.
        const bool full = (eg >= e0) && (eg + U <= e1);
        int j[U], row[U];
        bool ok[U];
        if (full) {
#pragma unroll
            for (int u = 0; u < U; u += 4) {
                const int4 c = ld4(a.colidx + eg + u);
                j[u] = c.x; j[u + 1] = c.y; j[u + 2] = c.z; j[u + 3] = c.w;
                if constexpr (!KNOWN_ROW) {
                    const int4 r = ld4(a.rowidx + eg + u);
                    row[u] = r.x; row[u + 1] = r.y; row[u + 2] = r.z; row[u + 3] = r.w;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) ok[u] = true;
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = eg + u;
                ok[u] = (e >= e0) && (e < e1);
                j[u] = ok[u] ? __ldg(a.colidx + e) : 0;
                if constexpr (!KNOWN_ROW) row[u] = ok[u] ? __ldg(a.rowidx + e) : cur;
            }
        }
        if constexpr (KNOWN_ROW) {
#pragma unroll
            for (int u = 0; u < U; ++u) row[u] = r0;
        }
        uint4 bw[U][NV];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint4* brow = reinterpret_cast<const uint4*>(Bb + (size_t)(unsigned)j[u] * ldb_bytes);
#pragma unroll
            for (int t = 0; t < NV; ++t)
                if (ok[u] && vin[t]) bw[u][t] = __ldg(brow + t * G);
        }
        float sv = 1.f;
        const int ew = eg + gl;
        const bool writer = (gl < U) && (ew >= e0) && (ew < e1);
        if (writer) {
            if (a.vals) sv = __ldg(a.vals + ew);
            if (a.vals2) sv *= __ldg(a.vals2 + ew);
        }
        float p[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            p[u] = 0.f;
            if (!ok[u]) continue;
            if (row[u] != cur) { cur = row[u]; load_a(cur); }
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                if (!vin[t]) continue;
                Raw<DTB, VECN> rb;
                rb.w[0] = bw[u][t].x; rb.w[1] = bw[u][t].y; rb.w[2] = bw[u][t].z; rb.w[3] = bw[u][t].w;
                float bf[VECN];
                unpack_all<DTB, VECN>(rb, bf);
                dot_pairs<VECN>(acc, av[t], bf);
            }
            p[u] = acc.x + acc.y;
            if constexpr (DTA == DT_E4M3) p[u] *= __ldg(a.a_scale + cur) * __ldg(a.b_scale + j[u]);
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
    const bool all_vin = (nvec >= vbase + G * NV);
    const char* __restrict__ Bb = reinterpret_cast<const char*>(a.B) + (vbase + gl) * 16;   // lane's first vector
    const unsigned ldb_bytes = (unsigned)a.ldb * dt_bytes(DTB);
    // vals alone and 16-byte aligned (every head's array too)
    const bool vec_vals = a.vals_staged != 0 && (a.heads == 1 || (a.hstride & 3) == 0);
    // several heads (NV = 1): the lane's columns belong to head (vector / vectors per head),
    // whose value array starts hstride elements after the previous head's
    const float* __restrict__ hvals = a.vals;
    if (a.heads > 1 && a.vals) hvals += (int64_t)min((vbase + gl) / (nvec / a.heads), a.heads - 1) * a.hstride;

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
    auto value = [&](int e) {
        const int vi = a.vperm ? __ldg(a.vperm + e) : e;
        float sv = hvals ? __ldg(hvals + vi) : 1.f;
        if (a.vals2) sv *= __ldg(a.vals2 + vi);
        return sv;
    };

    bool vin[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) vin[t] = all_vin || (vbase + t * G + gl < nvec);
    // An empty span (e0 == e1) still rounds down to a batch start below e1:
    // it must not enter the loop.
    for (int eb = e0 & ~3; e0 < e1 && eb < e1; eb += U) {
        // One batch body for every case (see sddmm_warp_span).
        const bool full = (eb >= e0) && (eb + U <= e1);
        int j[U], row[U];
        bool ok[U];
        float s[U];
        if (full) {
#pragma unroll
            for (int u = 0; u < U; u += 4) {
                const int4 c = ld4(a.colidx + eb + u);
                j[u] = c.x; j[u + 1] = c.y; j[u + 2] = c.z; j[u + 3] = c.w;
                if constexpr (!KNOWN_ROW) {
                    const int4 r = ld4(a.rowidx + eb + u);
                    row[u] = r.x; row[u + 1] = r.y; row[u + 2] = r.z; row[u + 3] = r.w;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) ok[u] = true;
            if (vec_vals) {
#pragma unroll
                for (int u = 0; u < U; u += 4) {
                    const float4 v4 = __ldg(reinterpret_cast<const float4*>(hvals + eb + u));
                    s[u] = v4.x; s[u + 1] = v4.y; s[u + 2] = v4.z; s[u + 3] = v4.w;
                }
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) s[u] = value(eb + u);
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = eb + u;
                ok[u] = (e >= e0) && (e < e1);
                j[u] = ok[u] ? __ldg(a.colidx + e) : 0;
                if constexpr (!KNOWN_ROW) row[u] = ok[u] ? __ldg(a.rowidx + e) : cur;
                s[u] = ok[u] ? value(e) : 0.f;
            }
        }
        if constexpr (KNOWN_ROW) {
#pragma unroll
            for (int u = 0; u < U; ++u) row[u] = r0;
        }
        uint4 bw[U][NV];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint4* brow = reinterpret_cast<const uint4*>(Bb + (size_t)(unsigned)j[u] * ldb_bytes);
#pragma unroll
            for (int t = 0; t < NV; ++t)
                if (ok[u] && vin[t]) bw[u][t] = __ldg(brow + t * G);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!ok[u]) continue;
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
            float sv = s[u];
            if constexpr (DTB == DT_E4M3) sv *= __ldg(a.b_scale + j[u]);
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                if (!vin[t]) continue;
                Raw<DTB, VECN> rb;
                rb.w[0] = bw[u][t].x; rb.w[1] = bw[u][t].y; rb.w[2] = bw[u][t].z; rb.w[3] = bw[u][t].w;
                float bf[VECN];
                unpack_all<DTB, VECN>(rb, bf);
                axpy_pairs<VECN>(acc[t], sv, bf);
            }
        }
    }
    flush(cur);
    for (int rr = cur + 1; rr <= meta.z; ++rr) zero_row<VECN, G, NV>(a, g, kb, nvec, rr);
}

}  // namespace spk
