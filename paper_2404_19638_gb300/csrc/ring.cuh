// Ring spans for the 16-byte vector path: gathered rows travel through a
// per-warp shared-memory ring filled by cp.async, so the bytes in flight are
// bounded by shared memory instead of registers, and the index streams are
// read one tile ahead so that no gather waits on an index load.
//
// Per warp (and for each of its lane groups of G lanes, U nonzeros a batch):
//   * index tiles of RING_T = 128 nonzeros: lane l holds entries 4l..4l+3 of
//     the column (and COO row) stream as one int4 each; the tile after the
//     current one is already in registers, and a group fetches the indices of
//     its batch from the owning lane with shuffles;
//   * a ring of D batch slots.  For every nonzero of a batch, lane gl of
//     the group copies its 16-byte vectors (t*G + gl, t < NV) of the gathered
//     row into the slot and later reads back exactly those vectors, so the
//     only wait on gathered data is the lane's own cp.async.wait_group;
//   * (SDDMM) one A-row slot per group and batch: the first row that starts
//     inside the batch is copied with it; a second new row inside the same
//     batch (rare: three rows meeting within U nonzeros) is read directly;
//   * per-slot metadata (rows, values) written by the group's lanes and read
//     after a __syncwarp.
// The issue cursor runs D - 1 batches ahead of the compute cursor (D = 2 or 4
// slots per warp).
#pragma once
#include "lean.cuh"

namespace spk {

constexpr int RING_T = 128;    // nonzeros per index tile (one int4 per lane)

__device__ __forceinline__ void cpa16(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cpa4(void* smem, const void* gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}

// Shared memory of one SDDMM warp with D batch slots, in bytes (host and
// device): B slots, A slots, then rows / values / second values / batch
// metadata per slot, rounded up to 128 bytes so that every warp's slots stay
// 16-byte aligned.
__host__ __device__ constexpr int sddmm_ring_bytes(int G, int NV, int U, int D)
{
    return (D * (U * NV * 512 + NV * 512 + 3 * (32 / G) * U * 4 + (32 / G) * 4) + 127) / 128 * 128;
}

// Ring kernels run 2-warp CTAs (fine occupancy steps when shared memory is
// the limit); this many fit an SM's 227 KB of shared memory, at most 16.
constexpr int RING_THREADS = 64;
__host__ __device__ constexpr int ring_min_ctas(int bytes_per_warp)
{
    return (232448 / (2 * bytes_per_warp)) > 16 ? 16
                                                 : ((232448 / (2 * bytes_per_warp)) < 1 ? 1 : (232448 / (2 * bytes_per_warp)));
}

// Tile t of a span based at tb0 (16-byte aligned): lane's four entries of
// the column and row streams; entries at or past e1 read as 0.
__device__ __forceinline__ void ring_tile(const int32_t* __restrict__ col, const int32_t* __restrict__ row, int tb0,
                                          int t, int e1, int lane, int4& c, int4& r)
{
    const int e = tb0 + t * RING_T + 4 * lane;
    if (e + 4 <= e1) {
        c = ld4(col + e);
        r = ld4(row + e);
    } else {
        c = make_int4(0, 0, 0, 0);
        r = make_int4(0, 0, 0, 0);
        if (e < e1) { c.x = __ldg(col + e); r.x = __ldg(row + e); }
        if (e + 1 < e1) { c.y = __ldg(col + e + 1); r.y = __ldg(row + e + 1); }
        if (e + 2 < e1) { c.z = __ldg(col + e + 2); r.z = __ldg(row + e + 2); }
    }
}

// Entries u = 0..U-1 of a group's batch from the tile registers of lane src0 + u/4.
template <int U>
__device__ __forceinline__ void ring_fetch(const int4& t, int src0, int (&v)[U])
{
#pragma unroll
    for (int c = 0; c < U / 4; ++c) {
        v[4 * c + 0] = __shfl_sync(0xffffffffu, t.x, src0 + c);
        v[4 * c + 1] = __shfl_sync(0xffffffffu, t.y, src0 + c);
        v[4 * c + 2] = __shfl_sync(0xffffffffu, t.z, src0 + c);
        v[4 * c + 3] = __shfl_sync(0xffffffffu, t.w, src0 + c);
    }
}

// ----------------------------------------------------------------------------
// A slice of one lane (one 16-byte vector of the row of A).  FP32 keeps the
// widened floats; BF16 / F16 keep the packed halves and multiply them with the
// packed halves of B by mixed-precision FMAs (16-bit inputs, FP32 accumulate:
// the product is exact and rounded once into the accumulator, the same result
// as an fmaf on the widened values), so neither operand is unpacked.  Both
// forms accumulate even elements in acc.x and odd ones in acc.y.
// ----------------------------------------------------------------------------
template <int DT>
struct ASlice {
    float f[4];
    __device__ __forceinline__ void set(const uint4 v)
    {
        f[0] = __uint_as_float(v.x); f[1] = __uint_as_float(v.y); f[2] = __uint_as_float(v.z); f[3] = __uint_as_float(v.w);
    }
    __device__ __forceinline__ void zero() { f[0] = f[1] = f[2] = f[3] = 0.f; }
    __device__ __forceinline__ void dot(float2& acc, const uint4 b) const
    {
        acc = __ffma2_rn(make_float2(f[0], f[1]), make_float2(__uint_as_float(b.x), __uint_as_float(b.y)), acc);
        acc = __ffma2_rn(make_float2(f[2], f[3]), make_float2(__uint_as_float(b.z), __uint_as_float(b.w)), acc);
    }
};

template <int DT>
__device__ __forceinline__ void fma_halves(float2& acc, uint32_t a, uint32_t b)
{
    if constexpr (DT == DT_BF16)
        asm("{\n .reg .b16 al, ah, bl, bh;\n mov.b32 {al, ah}, %2;\n mov.b32 {bl, bh}, %3;\n"
            " fma.rn.f32.bf16 %0, al, bl, %0;\n fma.rn.f32.bf16 %1, ah, bh, %1;\n}"
            : "+f"(acc.x), "+f"(acc.y) : "r"(a), "r"(b));
    else
        asm("{\n .reg .b16 al, ah, bl, bh;\n mov.b32 {al, ah}, %2;\n mov.b32 {bl, bh}, %3;\n"
            " fma.rn.f32.f16 %0, al, bl, %0;\n fma.rn.f32.f16 %1, ah, bh, %1;\n}"
            : "+f"(acc.x), "+f"(acc.y) : "r"(a), "r"(b));
}

template <int DT>
struct ASlice16 {
    uint4 w;
    __device__ __forceinline__ void set(const uint4 v) { w = v; }
    __device__ __forceinline__ void zero() { w = make_uint4(0u, 0u, 0u, 0u); }
    __device__ __forceinline__ void dot(float2& acc, const uint4 b) const
    {
        fma_halves<DT>(acc, w.x, b.x);
        fma_halves<DT>(acc, w.y, b.y);
        fma_halves<DT>(acc, w.z, b.z);
        fma_halves<DT>(acc, w.w, b.w);
    }
};
template <> struct ASlice<DT_BF16> : ASlice16<DT_BF16> {};
template <> struct ASlice<DT_F16> : ASlice16<DT_F16> {};

// ----------------------------------------------------------------------------
// SDDMM (Eq. 1) over the span [e0, e1) of one warp; DT is the dtype of both
// dense operands (F32, BF16 or F16).  ALLV: every lane's NV vectors lie
// inside K (no per-vector predicates).
//
// Rows are non-decreasing along a span, so a batch lies in one row exactly
// when its first and last nonzeros do.  Such a full batch takes the fast
// path: no per-nonzero checks, and if its row is not the row of the group's
// previous batch, that row's A slice arrives through the ring with the batch.
// Any other batch (span edge, or a row starting inside the batch) takes the
// general path: the first new row's A slice arrives through the ring, a
// second new row inside the same batch is read directly.
// ----------------------------------------------------------------------------
// NH > 0: several heads, each a block of NH consecutive 16-byte vectors of a
// row (so lane gl's vector t belongs to head (t * G + gl) / NH), one output
// array of nnz values per head (out + head * nnz); NH = 0: one dot per nonzero.
template <int DT, int G, int NV, int U, int D, bool ALLV, int NH = 0>
__device__ __forceinline__ void sddmm_ring_span(const SddmmArgs& a, int lane, unsigned char* wsm, int e0, int e1)
{
    static_assert(NH == 0 || (G % NH == 0 && (U * NV) % NH == 0), "heads must tile the lanes and the batch");
    constexpr int VECN = vec_elems(DT);
    constexpr int GPW = 32 / G;
    constexpr int WB = GPW * U;
    constexpr int BPT = RING_T / WB;
    static_assert(U % 4 == 0 && U <= G && RING_T % WB == 0, "batch shape must tile the index tile");
    if (e0 >= e1) return;
    uint4* ringB = reinterpret_cast<uint4*>(wsm);
    uint4* ringA = ringB + D * U * NV * 32;
    int* mrow = reinterpret_cast<int*>(ringA + D * NV * 32);   // [D][WB]
    float* mval = reinterpret_cast<float*>(mrow + D * WB);      // [D][WB]
    float* mval2 = mval + D * WB;                                // [D][WB]
    int* mmeta = reinterpret_cast<int*>(mval2 + D * WB);         // [D][GPW]

    const int grp = lane / G, gl = lane % G;
    const unsigned gmask = group_mask<G>(lane);
    const int nvec = a.K / VECN;
    bool vin[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) vin[t] = ALLV || (t * G + gl) < nvec;
    const char* __restrict__ Bb = reinterpret_cast<const char*>(a.B) + gl * 16;
    const char* __restrict__ Ab = reinterpret_cast<const char*>(a.A) + gl * 16;
    const unsigned ldb_bytes = (unsigned)a.ldb * dt_bytes(DT);
    const unsigned lda_bytes = (unsigned)a.lda * dt_bytes(DT);
    const float* __restrict__ vals = a.vals;
    const float* __restrict__ vals2 = a.vals2;
    const int tb0 = e0 & ~3;
    const int nb = (e1 - tb0 + WB - 1) / WB;
    const int slot_l = grp * U + gl;                 // writer lane's metadata slot (gl < U)

    int4 tc, tr, nc, nr;
    ring_tile(a.colidx, a.rowidx, tb0, 0, e1, lane, tc, tr);
    ring_tile(a.colidx, a.rowidx, tb0, 1, e1, lane, nc, nr);
    int itile = 0;
    int ilast = -1;                       // row of this group's last scheduled nonzero

    auto issue = [&](int b) {
        if (b < nb) {
            const int t = b / BPT;
            if (t != itile) {
                tc = nc; tr = nr;
                ring_tile(a.colidx, a.rowidx, tb0, t + 1, e1, lane, nc, nr);
                itile = t;
            }
            const int src0 = ((b % BPT) * WB + grp * U) >> 2;
            int j[U], row[U];
            ring_fetch<U>(tc, src0, j);
            ring_fetch<U>(tr, src0, row);
            const int d = b % D;
            const int eg = tb0 + b * WB + grp * U;
            uint4* sB = ringB + d * U * NV * 32 + lane;
            // one decision for the whole warp: a batch that could take the
            // fast path is also right on the general one, and lock-stepped
            // groups running the two paths one after the other cost both
            const bool fast = __all_sync(0xffffffffu, (eg >= e0) && (eg + U <= e1) && (row[0] == row[U - 1]));
            if (fast) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const char* brow = Bb + (size_t)(unsigned)j[u] * ldb_bytes;
#pragma unroll
                    for (int t2 = 0; t2 < NV; ++t2)
                        if (vin[t2]) cpa16(sB + (u * NV + t2) * 32, brow + t2 * G * 16);
                }
                const bool fresh = row[0] != ilast;          // the batch starts a new row
                if (fresh) {
                    const char* arow = Ab + (size_t)(unsigned)row[0] * lda_bytes;
#pragma unroll
                    for (int t2 = 0; t2 < NV; ++t2)
                        if (vin[t2]) cpa16(ringA + (d * NV + t2) * 32 + lane, arow + t2 * G * 16);
                }
                ilast = row[0];
                if (gl < U) {
                    if (vals) cpa4(mval + d * WB + slot_l, vals + eg + gl);
                    if (vals2) cpa4(mval2 + d * WB + slot_l, vals2 + eg + gl);
                }
                if (gl == 0) mmeta[d * GPW + grp] = fresh ? 3 : 1;
            } else {
                int m = 0, prev = ilast, myrow = row[0];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (gl == u) myrow = row[u];
                    const int e = eg + u;
                    if (e < e0 || e >= e1) continue;
                    const char* brow = Bb + (size_t)(unsigned)j[u] * ldb_bytes;
#pragma unroll
                    for (int t2 = 0; t2 < NV; ++t2)
                        if (vin[t2]) cpa16(sB + (u * NV + t2) * 32, brow + t2 * G * 16);
                    m |= (row[u] != prev ? 1 : 0) << u;
                    prev = row[u];
                }
                ilast = prev;
                if (m) {
                    const int ua = __ffs(m) - 1;
                    int ra = row[0];
#pragma unroll
                    for (int u = 1; u < U; ++u)
                        if (u == ua) ra = row[u];
                    const char* arow = Ab + (size_t)(unsigned)ra * lda_bytes;
#pragma unroll
                    for (int t2 = 0; t2 < NV; ++t2)
                        if (vin[t2]) cpa16(ringA + (d * NV + t2) * 32 + lane, arow + t2 * G * 16);
                }
                if (gl < U) {
                    mrow[d * WB + slot_l] = myrow;
                    const int e = eg + gl;
                    if (e >= e0 && e < e1) {
                        if (vals) cpa4(mval + d * WB + slot_l, vals + e);
                        if (vals2) cpa4(mval2 + d * WB + slot_l, vals2 + e);
                    }
                }
                if (gl == 0) mmeta[d * GPW + grp] = m << 1;
            }
        }
        cp_async_commit();
    };

    __syncwarp();
#pragma unroll
    for (int b = 0; b < D - 1; ++b) issue(b);
    ASlice<DT> av[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) av[t].zero();
    for (int b = 0; b < nb; ++b) {
        __syncwarp();
        issue(b + D - 1);
        cp_async_wait<D - 1>();
        __syncwarp();
        const int d = b % D;
        const int eg = tb0 + b * WB + grp * U;
        const int meta = mmeta[d * GPW + grp];
        const uint4* sB = ringB + d * U * NV * 32 + lane;
        constexpr int V = NH ? U * NV : U;               // partial dots this lane reduces
        float p[V];
        if (meta & 1) {                                  // issued on the fast path (a warp-wide decision)
            if (meta & 2) {                              // new row from nonzero 0 on: its A slice is in the ring
#pragma unroll
                for (int t = 0; t < NV; ++t)
                    if (vin[t]) av[t].set(ringA[(d * NV + t) * 32 + lane]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if constexpr (NH == 0) {
                    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int t = 0; t < NV; ++t)
                        if (vin[t]) av[t].dot(acc, sB[(u * NV + t) * 32]);
                    p[u] = acc.x + acc.y;
                } else {
#pragma unroll
                    for (int t = 0; t < NV; ++t) {
                        float2 acc = make_float2(0.f, 0.f);
                        if (vin[t]) av[t].dot(acc, sB[(u * NV + t) * 32]);
                        p[u * NV + t] = acc.x + acc.y;
                    }
                }
            }
        } else {
            const int m = meta >> 1;
            const int ua = m ? __ffs(m) - 1 : U;
#pragma unroll
            for (int k = 0; k < V; ++k) p[k] = 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = eg + u;
                if (e < e0 || e >= e1) continue;
                if ((m >> u) & 1) {
                    if (u == ua) {
#pragma unroll
                        for (int t = 0; t < NV; ++t)
                            if (vin[t]) av[t].set(ringA[(d * NV + t) * 32 + lane]);
                    } else {
                        const int r = mrow[d * WB + grp * U + u];
                        const uint4* arow = reinterpret_cast<const uint4*>(
                            reinterpret_cast<const char*>(a.A) + (size_t)(unsigned)r * lda_bytes) + gl;
#pragma unroll
                        for (int t = 0; t < NV; ++t)
                            if (vin[t]) av[t].set(__ldg(arow + t * G));
                    }
                }
                if constexpr (NH == 0) {
                    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int t = 0; t < NV; ++t)
                        if (vin[t]) av[t].dot(acc, sB[(u * NV + t) * 32]);
                    p[u] = acc.x + acc.y;
                } else {
#pragma unroll
                    for (int t = 0; t < NV; ++t) {
                        float2 acc = make_float2(0.f, 0.f);
                        if (vin[t]) av[t].dot(acc, sB[(u * NV + t) * 32]);
                        p[u * NV + t] = acc.x + acc.y;
                    }
                }
            }
        }
        if constexpr (NH > 0) {
            // Recursive halving over the NH lanes of a head block: after
            // log2(NH) levels lane gl holds C = V / NH finished dots, those of
            // values C * (gl % NH) + i, value k = u * NV + t being nonzero eg + u
            // against vector t of its row, which belongs to head
            // (t * G + gl) / NH = t * (G / NH) + gl / NH.
            constexpr int C = V / NH;
#pragma unroll
            for (int dd = NH / 2, half = V / 2; dd >= 1; dd >>= 1, half >>= 1) {
                const bool upper = (gl & dd) != 0;
#pragma unroll
                for (int i = 0; i < half; ++i) {
                    const float send = upper ? p[i] : p[i + half];
                    const float keep = upper ? p[i + half] : p[i];
                    p[i] = keep + __shfl_xor_sync(gmask, send, dd, G);
                }
            }
            const int kb0 = C * (gl % NH);
#pragma unroll
            for (int i = 0; i < C; ++i) {
                const int k = kb0 + i, u = k / NV, t = k % NV;
                const int ew = eg + u;
                if (ew < e0 || ew >= e1) continue;
                float sv = vals ? mval[d * WB + grp * U + u] : 1.f;
                if (vals2) sv *= mval2[d * WB + grp * U + u];
                const int head = t * (G / NH) + gl / NH;
                __stcs(a.out + (int64_t)head * a.nnz + ew, sv * p[i]);
            }
            continue;
        }
        // Reduce-scatter over the low log2(U) lane bits, then butterflies over
        // the remaining G/U lane subsets: nonzero eg + (gl % U) ends in lane gl.
#pragma unroll
        for (int dd = U / 2; dd >= 1; dd >>= 1) {
            const bool upper = (gl & dd) != 0;
#pragma unroll
            for (int i = 0; i < dd; ++i) {
                const float send = upper ? p[i] : p[i + dd];
                const float keep = upper ? p[i + dd] : p[i];
                p[i] = keep + __shfl_xor_sync(gmask, send, dd, G);
            }
        }
#pragma unroll
        for (int dd = U; dd < G; dd <<= 1) p[0] += __shfl_xor_sync(gmask, p[0], dd, G);
        const int ew = eg + gl;
        if (gl < U && ew >= e0 && ew < e1) {
            float sv = vals ? mval[d * WB + slot_l] : 1.f;
            if (vals2) sv *= mval2[d * WB + slot_l];
            __stcs(a.out + ew, sv * p[0]);
        }
    }
    cp_async_wait<0>();
}

// ----------------------------------------------------------------------------
// SpMM (Eq. 2): a lane group walks its own span (chunk) of the balanced
// schedule, accumulating K-slices of the current output row in registers, as
// in the register path; gathered rows arrive through the warp's ring (two
// slots).  Each group streams its own index tiles of 4G entries: the columns
// one tile ahead in registers (they address the gathers), the COO rows and
// values by cp.async into a double-buffered tile in shared memory (they are
// only read by the compute).  A full batch that stays in the current row
// takes the fast path (no per-nonzero checks); span edges and row changes go
// nonzero by nonzero, flushing finished rows.  Values must be absent or
// 16-byte aligned without a second factor or a slot permutation (other calls
// take the register path).
// ----------------------------------------------------------------------------
// VB: bytes of one lane vector, 16, or 8 for 16-bit operands spread over
// twice the lanes (a group of G lanes then covers G * NV * VB bytes of a row).
// Per warp: two batch slots of gathered rows, the staged COO rows (two tiles
// of 128 entries) and the staged values (two tiles per head).
__host__ __device__ constexpr int spmm_ring_bytes(int NV, int U, int VB = 16, int heads = 1)
{
    return 2 * U * NV * 32 * VB + 2 * 128 * 4 + heads * 2 * 128 * 4;
}

__device__ __forceinline__ void cpa8(void* smem, const void* gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}

template <int VB>
struct LaneVec { using type = uint4; };
template <>
struct LaneVec<8> { using type = uint2; };

template <int DT, int VECN>
__device__ __forceinline__ void unpack_vec(const uint4 v, float (&f)[VECN])
{
    Raw<DT, VECN> r;
    r.w[0] = v.x; r.w[1] = v.y; r.w[2] = v.z; r.w[3] = v.w;
    unpack_all<DT, VECN>(r, f);
}
template <int DT, int VECN>
__device__ __forceinline__ void unpack_vec(const uint2 v, float (&f)[VECN])
{
    Raw<DT, VECN> r;
    r.w[0] = v.x; r.w[1] = v.y;
    unpack_all<DT, VECN>(r, f);
}

template <int DT, int G, int NV, int U, bool ALLV, int VB = 16>
__device__ __forceinline__ void spmm_ring_span(const SpmmArgs& a, const Group<G>& g, uint4* wring16, int kb, int nkb,
                                               int r0, int e0, int r1, int e1, const int4 meta, int head_s0)
{
    static_assert(VB == 16 || (VB == 8 && DT != DT_F32 && DT != DT_E4M3), "8-byte lane vectors are for 16-bit operands");
    using Vec = typename LaneVec<VB>::type;
    constexpr int VECN = VB / dt_bytes(DT);
    Vec* wring = reinterpret_cast<Vec*>(wring16);
    constexpr int TG = 4 * G;                       // entries per group tile (one int4 per lane)
    static_assert(U % 4 == 0 && TG % U == 0 && TG / U >= 2, "batches must tile the group tile");
    const int gl = g.gl;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G;
    const int nvec = a.K / VECN;
    const int vbase = kb * G * NV;
    bool vin[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) vin[t] = ALLV || (vbase + t * G + gl < nvec);
    const char* __restrict__ Bb = reinterpret_cast<const char*>(a.B) + (vbase + gl) * VB;
    const unsigned ldb_bytes = (unsigned)a.ldb * dt_bytes(DT);
    const float* __restrict__ vals = a.vals;
    // tile buffers after the B slots: rows[2][128] then vals[2][128] per warp;
    // group grp owns entries [grp * 4G, (grp + 1) * 4G) of each 128-entry buffer
    int* trow = reinterpret_cast<int*>(wring + 2 * U * NV * 32) + grp * TG;
    float* tval = reinterpret_cast<float*>(reinterpret_cast<int*>(wring + 2 * U * NV * 32) + 2 * 128) + grp * TG;
    // several heads (NV = 1): head h's values in the h-th pair of value tiles;
    // this lane reads the tiles of the head its columns belong to
    float* tval_l = tval;
    if (a.heads > 1) tval_l += min((vbase + gl) / (nvec / a.heads), a.heads - 1) * 256;

    float acc[NV][VECN];
#pragma unroll
    for (int t = 0; t < NV; ++t)
#pragma unroll
        for (int q = 0; q < VECN; ++q) acc[t][q] = 0.f;
    int cur = r0;
    auto flush = [&](int row) {
        if (row == r0 && meta.x >= 0)
            finish_piece<VECN, G, NV>(a, g, kb, nkb, nvec, meta.x, head_s0, row, acc);
        else if (row == r1 && meta.y >= 0)
            finish_piece<VECN, G, NV>(a, g, kb, nkb, nvec, meta.y, meta.y, row, acc);
        else
            write_row<VECN, G, NV>(a, g, kb, nvec, row, acc);
    };

    if (e0 < e1) {
        const int tb0 = e0 & ~3;
        const int nb = (e1 - tb0 + U - 1) / U;
        auto cols = [&](int t) -> int4 {
            const int e = tb0 + t * TG + 4 * gl;
            if (e + 4 <= e1) return ld4(a.colidx + e);
            int4 c = make_int4(0, 0, 0, 0);
            if (e < e1) c.x = __ldg(a.colidx + e);
            if (e + 1 < e1) c.y = __ldg(a.colidx + e + 1);
            if (e + 2 < e1) c.z = __ldg(a.colidx + e + 2);
            return c;
        };
        auto stage_tile = [&](int t) {             // rows and values of tile t into buffer t & 1
            const int e = tb0 + t * TG + 4 * gl;
            const int n = e1 - e;
            if (n <= 0) return;
            const int bytes = n >= 4 ? 16 : 4 * n;
            const int o = (t & 1) * 128 + 4 * gl;
            cp_async16(trow + o, a.rowidx + e, bytes);
            if (vals) {
                if (a.heads == 1) {
                    cp_async16(tval + o, vals + e, bytes);
                } else {
                    for (int h = 0; h < a.heads; ++h) {
                        const float* hv = vals + (int64_t)h * a.hstride + e;
                        if ((a.hstride & 3) == 0) {
                            cp_async16(tval + h * 256 + o, hv, bytes);
                        } else {                    // a head array off 16-byte alignment: four 4-byte copies
                            const int n4 = n >= 4 ? 4 : n;
                            for (int q = 0; q < n4; ++q) cpa4(tval + h * 256 + o + q, hv + q);
                        }
                    }
                }
            }
        };
        int4 tc = cols(0), nc = cols(1);
        int itile = 0;
        stage_tile(0);
        auto issue = [&](int b) {
            if (b < nb) {
                const int t = (b * U) / TG;
                if (t != itile) {
                    tc = nc;
                    nc = cols(t + 1);
                    stage_tile(t);
                    itile = t;
                }
                const int src0 = ((b * U) % TG) >> 2;
                int j[U];
#pragma unroll
                for (int c = 0; c < U / 4; ++c) {
                    j[4 * c + 0] = __shfl_sync(g.mask, tc.x, src0 + c, G);
                    j[4 * c + 1] = __shfl_sync(g.mask, tc.y, src0 + c, G);
                    j[4 * c + 2] = __shfl_sync(g.mask, tc.z, src0 + c, G);
                    j[4 * c + 3] = __shfl_sync(g.mask, tc.w, src0 + c, G);
                }
                const int eb = tb0 + b * U;
                Vec* sl = wring + (b & 1) * U * NV * 32 + lane;
                auto copy_row = [&](int u) {
                    const char* brow = Bb + (size_t)(unsigned)j[u] * ldb_bytes;
#pragma unroll
                    for (int t2 = 0; t2 < NV; ++t2)
                        if (vin[t2]) {
                            if constexpr (VB == 16) cpa16(sl + (u * NV + t2) * 32, brow + t2 * G * 16);
                            else cpa8(sl + (u * NV + t2) * 32, brow + t2 * G * 8);
                        }
                };
                if constexpr (DT == DT_F32 && U >= 8) {
                    if (eb >= e0 && eb + U <= e1) {     // whole batch inside the span: no per-entry guard
#pragma unroll
                        for (int u = 0; u < U; ++u) copy_row(u);
                    } else {
#pragma unroll
                        for (int u = 0; u < U; ++u)
                            if (eb + u >= e0 && eb + u < e1) copy_row(u);
                    }
                } else {                                // 16-bit rows, short batches: one guarded loop
                    const bool full = (eb >= e0) && (eb + U <= e1);
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (!full && (eb + u < e0 || eb + u >= e1)) continue;
                        copy_row(u);
                    }
                }
            }
            cp_async_commit();
        };

        issue(0);
        for (int b = 0; b < nb; ++b) {
            __syncwarp(g.mask);
            issue(b + 1);
            cp_async_wait<1>();
            __syncwarp(g.mask);
            const int eb = tb0 + b * U;
            const Vec* sl = wring + (b & 1) * U * NV * 32 + lane;
            const int o = (((b * U) / TG) & 1) * 128 + (b * U) % TG;
            int rc[U];
            float sc[U];
#pragma unroll
            for (int c = 0; c < U / 4; ++c) {
                const int4 r4 = *reinterpret_cast<const int4*>(trow + o + 4 * c);
                rc[4 * c + 0] = r4.x; rc[4 * c + 1] = r4.y; rc[4 * c + 2] = r4.z; rc[4 * c + 3] = r4.w;
                if (vals) {
                    const float4 v4 = *reinterpret_cast<const float4*>(tval_l + o + 4 * c);
                    sc[4 * c + 0] = v4.x; sc[4 * c + 1] = v4.y; sc[4 * c + 2] = v4.z; sc[4 * c + 3] = v4.w;
                } else {
                    sc[4 * c + 0] = sc[4 * c + 1] = sc[4 * c + 2] = sc[4 * c + 3] = 1.f;
                }
            }
            // one fast/general decision for the lane groups running together
            // (each group walks its own span, so they may have parted): a batch
            // that could take the fast path is also right on the general one,
            // and groups running the two paths one after the other cost both
            if (__all_sync(__activemask(), eb >= e0 && eb + U <= e1 && rc[U - 1] == cur)) {
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int t = 0; t < NV; ++t) {
                        if (!vin[t]) continue;
                        float bf[VECN];
                        unpack_vec<DT, VECN>(sl[(u * NV + t) * 32], bf);
                        axpy_pairs<VECN>(acc[t], sc[u], bf);
                    }
            } else if constexpr (DT == DT_F32 && U >= 8) {
                // a row ends inside the batch, or the batch straddles the
                // span's ends: one copy of the row-change code, entries read
                // back from the staged tiles by a runtime index (measured
                // 3 % faster for FP32 rows in batches of 8; 7 % slower for
                // 16-bit rows and 14 % slower for FP32 batches of 4)
                const int u0 = max(e0 - eb, 0), u1 = min(e1 - eb, U);
#pragma unroll 1
                for (int u = u0; u < u1; ++u) {
                    const int r = trow[o + u];
                    if (r != cur) {
                        flush(cur);
                        for (int rr = cur + 1; rr < r; ++rr) zero_row<VECN, G, NV>(a, g, kb, nvec, rr);
                        cur = r;
#pragma unroll
                        for (int t = 0; t < NV; ++t)
#pragma unroll
                            for (int q = 0; q < VECN; ++q) acc[t][q] = 0.f;
                    }
                    const float sv = vals ? tval_l[o + u] : 1.f;
#pragma unroll
                    for (int t = 0; t < NV; ++t) {
                        if (!vin[t]) continue;
                        float bf[VECN];
                        unpack_vec<DT, VECN>(sl[(u * NV + t) * 32], bf);
                        axpy_pairs<VECN>(acc[t], sv, bf);
                    }
                }
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = eb + u;
                    if (e < e0 || e >= e1) continue;
                    if (rc[u] != cur) {
                        flush(cur);
                        for (int rr = cur + 1; rr < rc[u]; ++rr) zero_row<VECN, G, NV>(a, g, kb, nvec, rr);
                        cur = rc[u];
#pragma unroll
                        for (int t = 0; t < NV; ++t)
#pragma unroll
                            for (int q = 0; q < VECN; ++q) acc[t][q] = 0.f;
                    }
#pragma unroll
                    for (int t = 0; t < NV; ++t) {
                        if (!vin[t]) continue;
                        float bf[VECN];
                        unpack_vec<DT, VECN>(sl[(u * NV + t) * 32], bf);
                        axpy_pairs<VECN>(acc[t], sc[u], bf);
                    }
                }
            }
        }
        cp_async_wait<0>();
        __syncwarp(g.mask);
    }
    flush(cur);
    for (int rr = cur + 1; rr <= meta.z; ++rr) zero_row<VECN, G, NV>(a, g, kb, nvec, rr);
}

}  // namespace spk
