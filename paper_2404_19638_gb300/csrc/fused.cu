// FusedMM: SDDMM cascaded into SpMM (Sec. 2 names the cascade; operands as in
// Eq. 1 and Eq. 2), on one gathered dense matrix B:
//   e_h(i,j) = scale * s_ij * <A[i, head h], B[j, head h]>
//   w_h(i,j) = e_h(i,j), or the softmax of e_h(i, .) over row i
//   Y[i, head h] = sum_j w_h(i,j) * B[j, head h]
// Every gathered row of B serves both products: one gather per nonzero and
// head instead of two, and the scores never travel through HBM (they are
// written only if asked for).
//
// Structure: the SpMM ring span (ring.cuh) with one lane group per span of the
// balanced schedule and one head per grid row (blockIdx.y); a group covers a
// whole head, so each score is complete after a butterfly all-reduce across
// the group.  The A slice of the current row arrives through the ring when a
// batch starts a new row.  Row softmax is online: the group keeps the running
// maximum m, the running sum l and the unnormalised row acc, rescaling by
// exp(m_old - m_new) once per batch.  A row split across chunks leaves
// (acc, m, l) of each piece in its carry slot; the last piece to arrive merges
// them in slot order (log-sum-exp) and writes the row, so results do not
// depend on scheduling.
#include "fused.cuh"
#include "ring.cuh"

namespace spk {

#define SPK_FUSED_SHAPES(X) \
    X(0, 4, 1, 4)           \
    X(1, 8, 1, 4)           \
    X(2, 16, 1, 4)          \
    X(3, 32, 1, 8)          \
    X(4, 32, 2, 4)          \
    X(5, 8, 2, 4)           \
    X(6, 4, 2, 4)

constexpr int kFusedShapes = 7;
static const Shape kFusedShapeList[kFusedShapes] = {
#define X(i, G_, NV_, U_) {G_, NV_, U_},
    SPK_FUSED_SHAPES(X)
#undef X
};

int fused_shape_index(int G, int NV, int U)
{
    for (int i = 0; i < kFusedShapes; ++i)
        if (kFusedShapeList[i].G == G && kFusedShapeList[i].NV == NV && kFusedShapeList[i].U == U) return i;
    return -1;
}

// Shared memory of one warp: B slots, the row/value tiles of the SpMM ring,
// and one A slot per batch slot.
__host__ __device__ constexpr int fused_ring_bytes(int NV, int U) { return spmm_ring_bytes(NV, U) + 2 * NV * 512; }

template <int G>
__device__ __forceinline__ float group_allreduce(const Group<G>& g, float x)
{
#pragma unroll
    for (int d = G / 2; d >= 1; d >>= 1) x += __shfl_xor_sync(g.mask, x, d, G);
    return x;
}

// Slot stride of the carry area, in floats: K partial sums and (max, sum)
// per head, rounded up to 4 floats so that every slot is 16-byte aligned.
__device__ __forceinline__ int64_t fused_slot_floats(const FusedArgs& a)
{
    return ((int64_t)a.K + 2 * a.heads + 3) / 4 * 4;
}

template <int VECN, int G, int NV>
__device__ __forceinline__ void fused_write_row(const FusedArgs& a, const Group<G>& g, int kb, int nvh, int64_t row,
                                                const float (&acc)[NV][VECN], float m, float l)
{
    const float inv = (a.softmax && l > 0.f) ? 1.f / l : 1.f;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        const int v = t * G + g.gl;
        if (v >= nvh) continue;
        float o[VECN];
#pragma unroll
        for (int q = 0; q < VECN; ++q) o[q] = (a.softmax && !(l > 0.f)) ? 0.f : acc[t][q] * inv;
        store_elems<DT_F32, VECN>(a.Y, row * a.ldy + (int64_t)kb * a.dh + (int64_t)v * VECN, o);
    }
    if (a.softmax && a.lse && g.gl == 0) a.lse[row * a.heads + kb] = (l > 0.f) ? m + logf(l) : -INFINITY;
}

template <int VECN, int G, int NV>
__device__ __forceinline__ void fused_zero_row(const FusedArgs& a, const Group<G>& g, int kb, int nvh, int64_t row)
{
    float z[NV][VECN];
#pragma unroll
    for (int t = 0; t < NV; ++t)
#pragma unroll
        for (int q = 0; q < VECN; ++q) z[t][q] = 0.f;
    fused_write_row<VECN, G, NV>(a, g, kb, nvh, row, z, -INFINITY, 0.f);
}

// Deposit one piece of a split row; the last piece to arrive (over all
// pieces and heads) merges them in slot order and writes the row.
template <int VECN, int G, int NV>
__device__ __forceinline__ void fused_finish_piece(const FusedArgs& a, const Group<G>& g, int kb, int nvh, int slot,
                                                   int s0, int64_t row, const float (&acc)[NV][VECN], float m,
                                                   float l)
{
    const int64_t sf = fused_slot_floats(a);
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        const int v = t * G + g.gl;
        if (v < nvh) store_elems<DT_F32, VECN>(a.carry, (int64_t)slot * sf + (int64_t)kb * a.dh + (int64_t)v * VECN, acc[t]);
    }
    if (g.gl == 0) {
        a.carry[(int64_t)slot * sf + a.K + 2 * kb] = m;
        a.carry[(int64_t)slot * sf + a.K + 2 * kb + 1] = l;
    }
    __threadfence();
    __syncwarp(g.mask);
    int last = 0;
    if (g.gl == 0) {
        const int np = __ldcg(a.slot_np + s0);
        const int old = atomicAdd(a.cnt + s0, 1);
        last = (old == np * (int)gridDim.y - 1);     // every piece of every grid row (head) has arrived
    }
    last = __shfl_sync(g.mask, last, 0, G);
    if (!last) return;
    __threadfence();
    const int np = __ldcg(a.slot_np + s0);
    for (int h = 0; h < a.heads; ++h) {
        float M = -INFINITY;
        if (a.softmax)
            for (int sl = s0; sl < s0 + np; ++sl) M = fmaxf(M, __ldcg(a.carry + (int64_t)sl * sf + a.K + 2 * h));
        float L = 0.f;
        float sum[NV][VECN];
#pragma unroll
        for (int t = 0; t < NV; ++t)
#pragma unroll
            for (int q = 0; q < VECN; ++q) sum[t][q] = 0.f;
        for (int sl = s0; sl < s0 + np; ++sl) {
            float c = 1.f;
            if (a.softmax) {
                const float mp = __ldcg(a.carry + (int64_t)sl * sf + a.K + 2 * h);
                const float lp = __ldcg(a.carry + (int64_t)sl * sf + a.K + 2 * h + 1);
                c = (lp > 0.f) ? expf(mp - M) : 0.f;
                L += lp * c;
            }
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                const int v = t * G + g.gl;
                if (v >= nvh) continue;
                float x[VECN];
                load_elems_cg<DT_F32, VECN>(a.carry, (int64_t)sl * sf + (int64_t)h * a.dh + (int64_t)v * VECN, x);
#pragma unroll
                for (int q = 0; q < VECN; ++q) sum[t][q] = a.softmax ? fmaf(x[q], c, sum[t][q]) : sum[t][q] + x[q];
            }
        }
        fused_write_row<VECN, G, NV>(a, g, h, nvh, row, sum, M, L);
    }
    __syncwarp(g.mask);
    if (g.gl == 0) atomicExch(a.cnt + s0, 0);   // ready for the next launch
}

template <int DT, int G, int NV, int U, bool ALLV>
__device__ __forceinline__ void fused_span(const FusedArgs& a, const Group<G>& g, uint4* wring, int kb, int r0,
                                           int e0, int r1, int e1, const int4 meta, int head_s0)
{
    constexpr int VECN = vec_elems(DT);
    constexpr int TG = 4 * G;
    static_assert(U % 4 == 0 && TG % U == 0 && TG / U >= 2 && U <= G, "batches must tile the group tile");
    const int gl = g.gl;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G;
    const int nvh = a.dh / VECN;
    bool vin[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) vin[t] = ALLV || (t * G + gl < nvh);
    const int64_t hoff = (int64_t)kb * a.dh * dt_bytes(DT);           // byte offset of the head's slice
    const char* __restrict__ Bb = reinterpret_cast<const char*>(a.B) + hoff + gl * 16;
    const char* __restrict__ Ab = reinterpret_cast<const char*>(a.A) + hoff + gl * 16;
    const unsigned ldb_bytes = (unsigned)a.ldb * dt_bytes(DT);
    const unsigned lda_bytes = (unsigned)a.lda * dt_bytes(DT);
    const float* __restrict__ vals = a.vals;
    int* trow = reinterpret_cast<int*>(wring + 2 * U * NV * 32) + grp * TG;
    float* tval = reinterpret_cast<float*>(reinterpret_cast<int*>(wring + 2 * U * NV * 32) + 2 * 128) + grp * TG;
    uint4* ringA = reinterpret_cast<uint4*>(reinterpret_cast<int*>(wring + 2 * U * NV * 32) + 4 * 128);
    const float scale = a.scale;
    const bool smax = a.softmax != 0;

    float acc[NV][VECN], av[NV][VECN];
#pragma unroll
    for (int t = 0; t < NV; ++t)
#pragma unroll
        for (int q = 0; q < VECN; ++q) { acc[t][q] = 0.f; av[t][q] = 0.f; }
    float m = -INFINITY, l = 0.f;
    int cur = r0;            // output row being accumulated
    int acur = -1;           // row whose A slice is in av
    auto flush = [&](int row) {
        if (row == r0 && meta.x >= 0)
            fused_finish_piece<VECN, G, NV>(a, g, kb, nvh, meta.x, head_s0, row, acc, m, l);
        else if (row == r1 && meta.y >= 0)
            fused_finish_piece<VECN, G, NV>(a, g, kb, nvh, meta.y, meta.y, row, acc, m, l);
        else
            fused_write_row<VECN, G, NV>(a, g, kb, nvh, row, acc, m, l);
    };
    auto reset = [&]() {
#pragma unroll
        for (int t = 0; t < NV; ++t)
#pragma unroll
            for (int q = 0; q < VECN; ++q) acc[t][q] = 0.f;
        m = -INFINITY;
        l = 0.f;
    };
    // one gathered row: partial dot of the lane's slice with the current A slice
    auto partial = [&](const uint4* sl, int u) {
        float2 d2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            if (!vin[t]) continue;
            const uint4 v = sl[(u * NV + t) * 32];
            Raw<DT, VECN> rb;
            rb.w[0] = v.x; rb.w[1] = v.y; rb.w[2] = v.z; rb.w[3] = v.w;
            float bf[VECN];
            unpack_all<DT, VECN>(rb, bf);
            dot_pairs<VECN>(d2, av[t], bf);
        }
        return d2.x + d2.y;
    };
    auto accumulate = [&](const uint4* sl, int u, float w) {
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            if (!vin[t]) continue;
            const uint4 v = sl[(u * NV + t) * 32];
            Raw<DT, VECN> rb;
            rb.w[0] = v.x; rb.w[1] = v.y; rb.w[2] = v.z; rb.w[3] = v.w;
            float bf[VECN];
            unpack_all<DT, VECN>(rb, bf);
            axpy_pairs<VECN>(acc[t], w, bf);
        }
    };
    auto rescale = [&](float c) {
#pragma unroll
        for (int t = 0; t < NV; ++t)
#pragma unroll
            for (int q = 0; q < VECN; ++q) acc[t][q] *= c;
    };

    if (e0 < e1) {
        const int tb0 = e0 & ~3;
        const int nb = (e1 - tb0 + U - 1) / U;
        // columns and COO rows of tile t in registers (they address the gathers
        // and the A slices); rows and values also go to the shared tile for the compute
        auto cols = [&](int t, int4& c, int4& r) {
            const int e = tb0 + t * TG + 4 * gl;
            if (e + 4 <= e1) {
                c = ld4(a.colidx + e);
                r = ld4(a.rowidx + e);
                return;
            }
            c = make_int4(0, 0, 0, 0);
            r = make_int4(0, 0, 0, 0);
            if (e < e1) { c.x = __ldg(a.colidx + e); r.x = __ldg(a.rowidx + e); }
            if (e + 1 < e1) { c.y = __ldg(a.colidx + e + 1); r.y = __ldg(a.rowidx + e + 1); }
            if (e + 2 < e1) { c.z = __ldg(a.colidx + e + 2); r.z = __ldg(a.rowidx + e + 2); }
        };
        auto stage_tile = [&](int t) {
            const int e = tb0 + t * TG + 4 * gl;
            const int n = e1 - e;
            if (n <= 0) return;
            const int bytes = n >= 4 ? 16 : 4 * n;
            const int o = (t & 1) * 128 + 4 * gl;
            cp_async16(trow + o, a.rowidx + e, bytes);
            if (vals) cp_async16(tval + o, vals + e, bytes);
        };
        int4 tc, tr, nc, nr;
        cols(0, tc, tr);
        cols(1, nc, nr);
        int itile = 0;
        int ilast = -1;
        stage_tile(0);
        auto issue = [&](int b) {
            if (b < nb) {
                const int t = (b * U) / TG;
                if (t != itile) {
                    tc = nc; tr = nr;
                    cols(t + 1, nc, nr);
                    stage_tile(t);
                    itile = t;
                }
                const int src0 = ((b * U) % TG) >> 2;
                int j[U], rws[U];
#pragma unroll
                for (int c = 0; c < U / 4; ++c) {
                    j[4 * c + 0] = __shfl_sync(g.mask, tc.x, src0 + c, G);
                    j[4 * c + 1] = __shfl_sync(g.mask, tc.y, src0 + c, G);
                    j[4 * c + 2] = __shfl_sync(g.mask, tc.z, src0 + c, G);
                    j[4 * c + 3] = __shfl_sync(g.mask, tc.w, src0 + c, G);
                    rws[4 * c + 0] = __shfl_sync(g.mask, tr.x, src0 + c, G);
                    rws[4 * c + 1] = __shfl_sync(g.mask, tr.y, src0 + c, G);
                    rws[4 * c + 2] = __shfl_sync(g.mask, tr.z, src0 + c, G);
                    rws[4 * c + 3] = __shfl_sync(g.mask, tr.w, src0 + c, G);
                }
                const int eb = tb0 + b * U;
                uint4* sl = wring + (b & 1) * U * NV * 32 + lane;
                bool copied = false;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (eb + u < e0 || eb + u >= e1) continue;
                    const char* brow = Bb + (size_t)(unsigned)j[u] * ldb_bytes;
#pragma unroll
                    for (int t2 = 0; t2 < NV; ++t2)
                        if (vin[t2]) cpa16(sl + (u * NV + t2) * 32, brow + t2 * G * 16);
                    if (rws[u] != ilast) {
                        if (!copied) {
                            copied = true;
                            const char* arow = Ab + (size_t)(unsigned)rws[u] * lda_bytes;
#pragma unroll
                            for (int t2 = 0; t2 < NV; ++t2)
                                if (vin[t2]) cpa16(ringA + ((b & 1) * NV + t2) * 32 + lane, arow + t2 * G * 16);
                        }
                        ilast = rws[u];
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
            const uint4* sl = wring + (b & 1) * U * NV * 32 + lane;
            const int o = (((b * U) / TG) & 1) * 128 + (b * U) % TG;
            int rc[U];
            float sc[U];
#pragma unroll
            for (int c = 0; c < U / 4; ++c) {
                const int4 r4 = *reinterpret_cast<const int4*>(trow + o + 4 * c);
                rc[4 * c + 0] = r4.x; rc[4 * c + 1] = r4.y; rc[4 * c + 2] = r4.z; rc[4 * c + 3] = r4.w;
                if (vals) {
                    const float4 v4 = *reinterpret_cast<const float4*>(tval + o + 4 * c);
                    sc[4 * c + 0] = v4.x; sc[4 * c + 1] = v4.y; sc[4 * c + 2] = v4.z; sc[4 * c + 3] = v4.w;
                } else {
                    sc[4 * c + 0] = sc[4 * c + 1] = sc[4 * c + 2] = sc[4 * c + 3] = 1.f;
                }
            }
            float ev[U];
            if (eb >= e0 && eb + U <= e1 && rc[U - 1] == cur && cur == acur) {
                // the whole batch continues the current row: U scores, one rescale
#pragma unroll
                for (int u = 0; u < U; ++u) ev[u] = scale * (sc[u] * group_allreduce<G>(g, partial(sl, u)));
                if (smax) {
                    float mb = m;
#pragma unroll
                    for (int u = 0; u < U; ++u) mb = fmaxf(mb, ev[u]);
                    const float c = (m == -INFINITY) ? 0.f : expf(m - mb);
                    rescale(c);
                    l *= c;
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const float w = expf(ev[u] - mb);
                        l += w;
                        accumulate(sl, u, w);
                    }
                    m = mb;
                } else {
#pragma unroll
                    for (int u = 0; u < U; ++u) accumulate(sl, u, ev[u]);
                }
            } else {
                bool first = true;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    ev[u] = 0.f;
                    const int e = eb + u;
                    if (e < e0 || e >= e1) continue;
                    if (rc[u] != cur) {
                        flush(cur);
                        for (int rr = cur + 1; rr < rc[u]; ++rr) fused_zero_row<VECN, G, NV>(a, g, kb, nvh, rr);
                        cur = rc[u];
                        reset();
                    }
                    if (rc[u] != acur) {
                        if (first) {
#pragma unroll
                            for (int t = 0; t < NV; ++t)
                                if (vin[t]) {
                                    const uint4 v = ringA[((b & 1) * NV + t) * 32 + lane];
                                    Raw<DT, VECN> ra;
                                    ra.w[0] = v.x; ra.w[1] = v.y; ra.w[2] = v.z; ra.w[3] = v.w;
                                    unpack_all<DT, VECN>(ra, av[t]);
                                }
                        } else {
                            const char* arow = reinterpret_cast<const char*>(a.A) + hoff + (size_t)(unsigned)rc[u] * lda_bytes;
#pragma unroll
                            for (int t = 0; t < NV; ++t)
                                if (vin[t]) load_elems<DT, VECN>(arow, (int64_t)(t * G + gl) * VECN, av[t]);
                        }
                        first = false;
                        acur = rc[u];
                    }
                    ev[u] = scale * (sc[u] * group_allreduce<G>(g, partial(sl, u)));
                    if (smax) {
                        const float mb = fmaxf(m, ev[u]);
                        const float c = (m == -INFINITY) ? 0.f : expf(m - mb);
                        rescale(c);
                        const float w = expf(ev[u] - mb);
                        l = l * c + w;
                        accumulate(sl, u, w);
                        m = mb;
                    } else {
                        accumulate(sl, u, ev[u]);
                    }
                }
            }
            if (a.scores) {
                float mine = ev[0];
#pragma unroll
                for (int u = 1; u < U; ++u)
                    if (gl == u) mine = ev[u];
                const int e = eb + gl;
                if (gl < U && e >= e0 && e < e1) __stcs(a.scores + (int64_t)kb * a.nnz + e, mine);
            }
        }
        cp_async_wait<0>();
        __syncwarp(g.mask);
    }
    flush(cur);
    for (int rr = cur + 1; rr <= meta.z; ++rr) fused_zero_row<VECN, G, NV>(a, g, kb, nvh, rr);
}

// CTAs per SM the register budget is cut for: as many as shared memory
// allows, at most 8 (128 registers); 16-bit rows of two vectors a lane keep
// twice the widened elements and get 6 (168 registers) so that they do not spill.
template <int DT, int NV, int U>
constexpr int fused_min_ctas()
{
    return (DT != DT_F32 && NV > 1) ? 6
                                    : (ring_min_ctas(fused_ring_bytes(NV, U)) < 8 ? ring_min_ctas(fused_ring_bytes(NV, U)) : 8);
}

template <int DT, int G, int NV, int U>
__global__ void __launch_bounds__(RING_THREADS, fused_min_ctas<DT, NV, U>()) k_fused(const FusedArgs a)
{
    extern __shared__ __align__(16) unsigned char ring_smem[];
    const Group<G> g;
    uint4* wring = reinterpret_cast<uint4*>(ring_smem) + (threadIdx.x >> 5) * (fused_ring_bytes(NV, U) / 16);
    const int kb = blockIdx.y;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const bool allv = a.dh / vec_elems(DT) >= G * NV;
    for (int64_t c = gid; c < a.nchunks; c += ngroups) {
        const int2 b0 = a.bnd[c], b1 = a.bnd[c + 1];
        const int4 m = a.meta[c];
        if (b1.y == b0.y && m.z < b0.x) continue;          // nothing in this chunk
        const int hs0 = (m.x >= 0) ? __ldg(a.head_s0 + c) : -1;
        if (allv) fused_span<DT, G, NV, U, true>(a, g, wring, kb, b0.x, b0.y, b1.x, b1.y, m, hs0);
        else fused_span<DT, G, NV, U, false>(a, g, wring, kb, b0.x, b0.y, b1.x, b1.y, m, hs0);
    }
}

// ----------------------------------------------------------------------------
// All heads in one group: G = K / VECN lanes, lane gl holds vector gl of every
// row, the heads are consecutive blocks of NH = G / heads lanes.  A gathered
// row serves every head; each head's scores come from a reduction over its
// NH lanes, after which every lane of the head holds the same scores and the
// same softmax state (m, l).  The split-row carry slot holds the K partial
// sums and (m, l) per head; one arrival per piece.
// ----------------------------------------------------------------------------
template <int G, int U>
__device__ __forceinline__ void head_allreduce(const Group<G>& g, int NH, float (&p)[U])
{
    if (NH >= U) {
        // reduce-scatter over the low log2(U) lane bits, butterflies over the
        // rest of the head, then every lane fetches the U sums of its head
#pragma unroll
        for (int dd = U / 2; dd >= 1; dd >>= 1) {
            const bool upper = (g.gl & dd) != 0;
#pragma unroll
            for (int i = 0; i < dd; ++i) {
                const float send = upper ? p[i] : p[i + dd];
                const float keep = upper ? p[i + dd] : p[i];
                p[i] = keep + __shfl_xor_sync(g.mask, send, dd, G);
            }
        }
        for (int dd = U; dd < NH; dd <<= 1) p[0] += __shfl_xor_sync(g.mask, p[0], dd, G);
        const int base = g.gl & ~(NH - 1);
        const float mine = p[0];
#pragma unroll
        for (int u = 0; u < U; ++u) p[u] = __shfl_sync(g.mask, mine, base + u, G);
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u)
            for (int dd = NH / 2; dd >= 1; dd >>= 1) p[u] += __shfl_xor_sync(g.mask, p[u], dd, G);
    }
}

template <int G>
__device__ __forceinline__ float head_allreduce1(const Group<G>& g, int NH, float x)
{
    for (int dd = NH / 2; dd >= 1; dd >>= 1) x += __shfl_xor_sync(g.mask, x, dd, G);
    return x;
}

template <int VECN, int G>
__device__ __forceinline__ void mh_write_row(const FusedArgs& a, const Group<G>& g, int hl, bool hlead, int64_t row,
                                             const float (&acc)[VECN], float m, float l)
{
    const bool empty = a.softmax && !(l > 0.f);
    const float inv = (a.softmax && l > 0.f) ? 1.f / l : 1.f;
    float o[VECN];
#pragma unroll
    for (int q = 0; q < VECN; ++q) o[q] = empty ? 0.f : acc[q] * inv;
    store_elems<DT_F32, VECN>(a.Y, row * a.ldy + (int64_t)g.gl * VECN, o);
    if (a.softmax && a.lse && hlead) a.lse[row * a.heads + hl] = (l > 0.f) ? m + logf(l) : -INFINITY;
}

template <int VECN, int G>
__device__ __forceinline__ void mh_finish_piece(const FusedArgs& a, const Group<G>& g, int hl, bool hlead, int slot,
                                                int s0, int64_t row, const float (&acc)[VECN], float m, float l)
{
    const int64_t sf = fused_slot_floats(a);
    store_elems<DT_F32, VECN>(a.carry, (int64_t)slot * sf + (int64_t)g.gl * VECN, acc);
    if (hlead) {
        a.carry[(int64_t)slot * sf + a.K + 2 * hl] = m;
        a.carry[(int64_t)slot * sf + a.K + 2 * hl + 1] = l;
    }
    __threadfence();
    __syncwarp(g.mask);
    int last = 0;
    if (g.gl == 0) {
        const int np = __ldcg(a.slot_np + s0);
        const int old = atomicAdd(a.cnt + s0, 1);
        last = (old == np - 1);
    }
    last = __shfl_sync(g.mask, last, 0, G);
    if (!last) return;
    __threadfence();
    const int np = __ldcg(a.slot_np + s0);
    float M = -INFINITY;
    if (a.softmax)
        for (int sl = s0; sl < s0 + np; ++sl) M = fmaxf(M, __ldcg(a.carry + (int64_t)sl * sf + a.K + 2 * hl));
    float L = 0.f, sum[VECN];
#pragma unroll
    for (int q = 0; q < VECN; ++q) sum[q] = 0.f;
    for (int sl = s0; sl < s0 + np; ++sl) {
        float c = 1.f;
        if (a.softmax) {
            const float mp = __ldcg(a.carry + (int64_t)sl * sf + a.K + 2 * hl);
            const float lp = __ldcg(a.carry + (int64_t)sl * sf + a.K + 2 * hl + 1);
            c = (lp > 0.f) ? expf(mp - M) : 0.f;
            L += lp * c;
        }
        float x[VECN];
        load_elems_cg<DT_F32, VECN>(a.carry, (int64_t)sl * sf + (int64_t)g.gl * VECN, x);
#pragma unroll
        for (int q = 0; q < VECN; ++q) sum[q] = a.softmax ? fmaf(x[q], c, sum[q]) : sum[q] + x[q];
    }
    mh_write_row<VECN, G>(a, g, hl, hlead, row, sum, M, L);
    __syncwarp(g.mask);
    if (g.gl == 0) atomicExch(a.cnt + s0, 0);
}

template <int DT, int G, int U, int NV>
__device__ __forceinline__ void fused_span_mh(const FusedArgs& a, const Group<G>& g, uint4* wring, int r0, int e0,
                                              int r1, int e1, const int4 meta, int head_s0)
{
    constexpr int VECN = vec_elems(DT);
    constexpr int W = NV * VECN;                    // elements a lane holds: NV adjacent 16-byte vectors
    constexpr int TG = 4 * G;
    static_assert(U % 4 == 0 && TG % U == 0 && TG / U >= 2 && U <= G, "batches must tile the group tile");
    const int gl = g.gl;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G;
    const int NH = G / a.heads;                     // lanes per head
    const int hl = gl / NH;                         // this lane's head
    const bool hlead = (gl % NH) == 0;
    const char* __restrict__ Bb = reinterpret_cast<const char*>(a.B) + gl * 16 * NV;
    const char* __restrict__ Ab = reinterpret_cast<const char*>(a.A) + gl * 16 * NV;
    const unsigned ldb_bytes = (unsigned)a.ldb * dt_bytes(DT);
    const unsigned lda_bytes = (unsigned)a.lda * dt_bytes(DT);
    const float* __restrict__ vals = a.vals;
    int* trow = reinterpret_cast<int*>(wring + 2 * U * NV * 32) + grp * TG;
    float* tval = reinterpret_cast<float*>(reinterpret_cast<int*>(wring + 2 * U * NV * 32) + 2 * 128) + grp * TG;
    uint4* ringA = reinterpret_cast<uint4*>(reinterpret_cast<int*>(wring + 2 * U * NV * 32) + 4 * 128);
    const float scale = a.scale;
    const bool smax = a.softmax != 0;

    float acc[W], av[W];
#pragma unroll
    for (int q = 0; q < W; ++q) { acc[q] = 0.f; av[q] = 0.f; }
    float m = -INFINITY, l = 0.f;
    int cur = r0, acur = -1;
    auto flush = [&](int row) {
        if (row == r0 && meta.x >= 0) mh_finish_piece<W, G>(a, g, hl, hlead, meta.x, head_s0, row, acc, m, l);
        else if (row == r1 && meta.y >= 0) mh_finish_piece<W, G>(a, g, hl, hlead, meta.y, meta.y, row, acc, m, l);
        else mh_write_row<W, G>(a, g, hl, hlead, row, acc, m, l);
    };
    auto zero_out = [&](int row) {
        float z[W];
#pragma unroll
        for (int q = 0; q < W; ++q) z[q] = 0.f;
        mh_write_row<W, G>(a, g, hl, hlead, row, z, -INFINITY, 0.f);
    };
    // the lane's NV vectors, 32 slots apart in the ring, widened to FP32
    auto unpack_v = [&](const uint4* v, float (&f)[W]) {
        Raw<DT, W> r;
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const uint4 x = v[t * 32];
            r.w[4 * t] = x.x; r.w[4 * t + 1] = x.y; r.w[4 * t + 2] = x.z; r.w[4 * t + 3] = x.w;
        }
        unpack_all<DT, W>(r, f);
    };
    auto dot = [&](const float (&bf)[W]) {
        float2 d2 = make_float2(0.f, 0.f);
        dot_pairs<W>(d2, av, bf);
        return d2.x + d2.y;
    };

    if (e0 < e1) {
        const int tb0 = e0 & ~3;
        const int nb = (e1 - tb0 + U - 1) / U;
        auto cols = [&](int t, int4& c, int4& r) {
            const int e = tb0 + t * TG + 4 * gl;
            if (e + 4 <= e1) {
                c = ld4(a.colidx + e);
                r = ld4(a.rowidx + e);
                return;
            }
            c = make_int4(0, 0, 0, 0);
            r = make_int4(0, 0, 0, 0);
            if (e < e1) { c.x = __ldg(a.colidx + e); r.x = __ldg(a.rowidx + e); }
            if (e + 1 < e1) { c.y = __ldg(a.colidx + e + 1); r.y = __ldg(a.rowidx + e + 1); }
            if (e + 2 < e1) { c.z = __ldg(a.colidx + e + 2); r.z = __ldg(a.rowidx + e + 2); }
        };
        auto stage_tile = [&](int t) {
            const int e = tb0 + t * TG + 4 * gl;
            const int n = e1 - e;
            if (n <= 0) return;
            const int bytes = n >= 4 ? 16 : 4 * n;
            const int o = (t & 1) * 128 + 4 * gl;
            cp_async16(trow + o, a.rowidx + e, bytes);
            if (vals) cp_async16(tval + o, vals + e, bytes);
        };
        int4 tc, tr, nc, nr;
        cols(0, tc, tr);
        cols(1, nc, nr);
        int itile = 0, ilast = -1;
        stage_tile(0);
        auto issue = [&](int b) {
            if (b < nb) {
                const int t = (b * U) / TG;
                if (t != itile) {
                    tc = nc; tr = nr;
                    cols(t + 1, nc, nr);
                    stage_tile(t);
                    itile = t;
                }
                const int src0 = ((b * U) % TG) >> 2;
                int j[U], rws[U];
#pragma unroll
                for (int c = 0; c < U / 4; ++c) {
                    j[4 * c + 0] = __shfl_sync(g.mask, tc.x, src0 + c, G);
                    j[4 * c + 1] = __shfl_sync(g.mask, tc.y, src0 + c, G);
                    j[4 * c + 2] = __shfl_sync(g.mask, tc.z, src0 + c, G);
                    j[4 * c + 3] = __shfl_sync(g.mask, tc.w, src0 + c, G);
                    rws[4 * c + 0] = __shfl_sync(g.mask, tr.x, src0 + c, G);
                    rws[4 * c + 1] = __shfl_sync(g.mask, tr.y, src0 + c, G);
                    rws[4 * c + 2] = __shfl_sync(g.mask, tr.z, src0 + c, G);
                    rws[4 * c + 3] = __shfl_sync(g.mask, tr.w, src0 + c, G);
                }
                const int eb = tb0 + b * U;
                uint4* sl = wring + (b & 1) * U * NV * 32 + lane;
                bool copied = false;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (eb + u < e0 || eb + u >= e1) continue;
#pragma unroll
                    for (int t = 0; t < NV; ++t)
                        cpa16(sl + (u * NV + t) * 32, Bb + (size_t)(unsigned)j[u] * ldb_bytes + t * 16);
                    if (rws[u] != ilast) {
                        if (!copied) {
                            copied = true;
#pragma unroll
                            for (int t = 0; t < NV; ++t)
                                cpa16(ringA + ((b & 1) * NV + t) * 32 + lane,
                                      Ab + (size_t)(unsigned)rws[u] * lda_bytes + t * 16);
                        }
                        ilast = rws[u];
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
            const uint4* sl = wring + (b & 1) * U * NV * 32 + lane;
            const int o = (((b * U) / TG) & 1) * 128 + (b * U) % TG;
            int rc[U];
            float sc[U];
#pragma unroll
            for (int c = 0; c < U / 4; ++c) {
                const int4 r4 = *reinterpret_cast<const int4*>(trow + o + 4 * c);
                rc[4 * c + 0] = r4.x; rc[4 * c + 1] = r4.y; rc[4 * c + 2] = r4.z; rc[4 * c + 3] = r4.w;
                if (vals) {
                    const float4 v4 = *reinterpret_cast<const float4*>(tval + o + 4 * c);
                    sc[4 * c + 0] = v4.x; sc[4 * c + 1] = v4.y; sc[4 * c + 2] = v4.z; sc[4 * c + 3] = v4.w;
                } else {
                    sc[4 * c + 0] = sc[4 * c + 1] = sc[4 * c + 2] = sc[4 * c + 3] = 1.f;
                }
            }
            float ev[U];
            if (eb >= e0 && eb + U <= e1 && rc[U - 1] == cur && cur == acur) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    float bf[W];
                    unpack_v(sl + u * NV * 32, bf);
                    ev[u] = dot(bf);
                }
                head_allreduce<G, U>(g, NH, ev);
#pragma unroll
                for (int u = 0; u < U; ++u) ev[u] = scale * (sc[u] * ev[u]);
                if (smax) {
                    float mb = m;
#pragma unroll
                    for (int u = 0; u < U; ++u) mb = fmaxf(mb, ev[u]);
                    const float c = (m == -INFINITY) ? 0.f : expf(m - mb);
#pragma unroll
                    for (int q = 0; q < W; ++q) acc[q] *= c;
                    l *= c;
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const float w = expf(ev[u] - mb);
                        l += w;
                        float bf[W];
                        unpack_v(sl + u * NV * 32, bf);     // re-read: keeps U rows out of registers
                        axpy_pairs<W>(acc, w, bf);
                    }
                    m = mb;
                } else {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        float bf[W];
                        unpack_v(sl + u * NV * 32, bf);
                        axpy_pairs<W>(acc, ev[u], bf);
                    }
                }
            } else {
                // span edge or row change: all U dots first (the A slice switches
                // where a new row starts), one reduction for the batch, then the
                // rows are closed and accumulated in order
                bool first = true;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    ev[u] = 0.f;
                    const int e = eb + u;
                    if (e < e0 || e >= e1) continue;
                    float bfu[W];
                    unpack_v(sl + u * NV * 32, bfu);
                    if (rc[u] != acur) {
                        if (first) unpack_v(ringA + (b & 1) * NV * 32 + lane, av);
                        else load_elems<DT, W>(reinterpret_cast<const char*>(a.A) + (size_t)(unsigned)rc[u] * lda_bytes,
                                               (int64_t)gl * W, av);
                        first = false;
                        acur = rc[u];
                    }
                    ev[u] = dot(bfu);
                }
                head_allreduce<G, U>(g, NH, ev);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = eb + u;
                    if (e < e0 || e >= e1) { ev[u] = 0.f; continue; }
                    ev[u] = scale * (sc[u] * ev[u]);
                    if (rc[u] != cur) {
                        flush(cur);
                        for (int rr = cur + 1; rr < rc[u]; ++rr) zero_out(rr);
                        cur = rc[u];
#pragma unroll
                        for (int q = 0; q < W; ++q) acc[q] = 0.f;
                        m = -INFINITY;
                        l = 0.f;
                    }
                    float bf[W];
                    unpack_v(sl + u * NV * 32, bf);
                    if (smax) {
                        const float mb = fmaxf(m, ev[u]);
                        const float c = (m == -INFINITY) ? 0.f : expf(m - mb);
#pragma unroll
                        for (int q = 0; q < W; ++q) acc[q] *= c;
                        const float w = expf(ev[u] - mb);
                        l = l * c + w;
                        axpy_pairs<W>(acc, w, bf);
                        m = mb;
                    } else {
                        axpy_pairs<W>(acc, ev[u], bf);
                    }
                }
            }
            if (a.scores && hlead) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = eb + u;
                    if (e >= e0 && e < e1) __stcs(a.scores + (int64_t)hl * a.nnz + e, ev[u]);
                }
            }
        }
        cp_async_wait<0>();
        __syncwarp(g.mask);
    }
    flush(cur);
    for (int rr = cur + 1; rr <= meta.z; ++rr) zero_out(rr);
}

__host__ __device__ constexpr int fused_mh_ring_bytes(int U, int NV) { return fused_ring_bytes(NV, U); }

template <int DT, int G, int U, int NV>
__global__ void __launch_bounds__(RING_THREADS, (DT == DT_F32 && NV == 1) ? 8 : 6) k_fused_mh(const FusedArgs a)
{
    extern __shared__ __align__(16) unsigned char ring_smem[];
    const Group<G> g;
    uint4* wring = reinterpret_cast<uint4*>(ring_smem) + (threadIdx.x >> 5) * (fused_mh_ring_bytes(U, NV) / 16);
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    for (int64_t c = gid; c < a.nchunks; c += ngroups) {
        const int2 b0 = a.bnd[c], b1 = a.bnd[c + 1];
        const int4 m = a.meta[c];
        if (b1.y == b0.y && m.z < b0.x) continue;
        const int hs0 = (m.x >= 0) ? __ldg(a.head_s0 + c) : -1;
        fused_span_mh<DT, G, U, NV>(a, g, wring, b0.x, b0.y, b1.x, b1.y, m, hs0);
    }
}

template <int DT>
static cudaError_t launch_fused_mh_t(int G, int NV, const FusedArgs& a, cudaStream_t s)
{
    const void* fn = nullptr;
    // 4 nonzeros a batch (8 measured slower: more registers, fewer warps)
    if (NV == 1) {
        switch (G) {
        case 4: fn = (const void*)&k_fused_mh<DT, 4, 4, 1>; break;
        case 8: fn = (const void*)&k_fused_mh<DT, 8, 4, 1>; break;
        case 16: fn = (const void*)&k_fused_mh<DT, 16, 4, 1>; break;
        case 32: fn = (const void*)&k_fused_mh<DT, 32, 4, 1>; break;
        }
    } else if (NV == 2) {
        switch (G) {
        case 4: fn = (const void*)&k_fused_mh<DT, 4, 4, 2>; break;
        case 8: fn = (const void*)&k_fused_mh<DT, 8, 4, 2>; break;
        case 16: fn = (const void*)&k_fused_mh<DT, 16, 4, 2>; break;
        }
    }
    if (!fn) return cudaErrorInvalidValue;
    constexpr int U = 4;
    if (a.nchunks <= 0) return cudaSuccess;
    const int64_t groups_per_cta = RING_THREADS / G;
    int64_t blocks = (a.nchunks + groups_per_cta - 1) / groups_per_cta;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    const size_t smem = (size_t)(RING_THREADS / 32) * fused_mh_ring_bytes(U, NV);
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3((unsigned)blocks, 1), dim3(RING_THREADS), args, smem, s);
}

cudaError_t launch_fused_mh_nv(int dt, int G, int NV, const FusedArgs& a, cudaStream_t s)
{
    switch (dt) {
    case DT_F32: return launch_fused_mh_t<DT_F32>(G, NV, a, s);
    case DT_BF16: return launch_fused_mh_t<DT_BF16>(G, NV, a, s);
    case DT_F16: return launch_fused_mh_t<DT_F16>(G, NV, a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fused_mh(int dt, int G, const FusedArgs& a, cudaStream_t s)
{
    return launch_fused_mh_nv(dt, G, 1, a, s);
}

template <int DT>
static cudaError_t launch_fused_t(const Launch& L, const FusedArgs& a, cudaStream_t s)
{
    const void* fn = nullptr;
    switch (L.shape) {
#define X(i, G_, NV_, U_) case i: fn = (const void*)&k_fused<DT, G_, NV_, U_>; break;
        SPK_FUSED_SHAPES(X)
#undef X
    }
    if (!fn) return cudaErrorInvalidValue;
    const Shape sh = kFusedShapeList[L.shape];
    if (a.nchunks <= 0) return cudaSuccess;
    const int64_t groups_per_cta = RING_THREADS / sh.G;
    int64_t blocks = (a.nchunks + groups_per_cta - 1) / groups_per_cta;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    if (a.heads > 65535) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(RING_THREADS / 32) * fused_ring_bytes(sh.NV, sh.U);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3((unsigned)blocks, (unsigned)a.heads), dim3(RING_THREADS), args, smem, s);
}

// ----------------------------------------------------------------------------
// Elementwise steps of the FusedMM backward, per head h (grid row) and stored
// entry e of row i (COO row from the schedule):
//   weights:    w = e_h, or exp(e_h - lse[i, h]) with softmax
//   score grad: c = scale * s_e * dw, or scale * s_e * w * (dw - rowdot[i, h])
// Each thread takes kElemIlp entries a block-width apart (coalesced, several
// loads in flight); the grid's x extent is a multiple of the SM count.
// ----------------------------------------------------------------------------
constexpr int kElemThreads = 256;
constexpr int kElemIlp = 4;

static unsigned elem_blocks(int64_t nnz)
{
    const int64_t per = (int64_t)kElemThreads * kElemIlp;
    int64_t b = (nnz + per - 1) / per;
    const int64_t cap = 152 * 8;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

__global__ void __launch_bounds__(kElemThreads) k_fused_weights(const int32_t* __restrict__ rowidx, int64_t nnz,
                                                                int32_t heads, const float* __restrict__ scores,
                                                                const float* __restrict__ lse, float* __restrict__ w)
{
    const int h = blockIdx.y;
    const float* sc = scores + (int64_t)h * nnz;
    float* wo = w + (int64_t)h * nnz;
    const int64_t stride = (int64_t)gridDim.x * kElemThreads * kElemIlp;
    for (int64_t base = (int64_t)blockIdx.x * kElemThreads * kElemIlp + threadIdx.x; base < nnz; base += stride) {
        float x[kElemIlp];
        int r[kElemIlp];
#pragma unroll
        for (int u = 0; u < kElemIlp; ++u) {
            const int64_t e = base + (int64_t)u * kElemThreads;
            x[u] = e < nnz ? __ldg(sc + e) : 0.f;
            r[u] = e < nnz ? __ldg(rowidx + e) : 0;
        }
#pragma unroll
        for (int u = 0; u < kElemIlp; ++u) {
            const int64_t e = base + (int64_t)u * kElemThreads;
            if (e < nnz) wo[e] = expf(x[u] - __ldg(lse + (int64_t)r[u] * heads + h));
        }
    }
}

template <bool SOFTMAX>
__global__ void __launch_bounds__(kElemThreads) k_fused_score_grad(const int32_t* __restrict__ rowidx, int64_t nnz,
                                                                   int32_t heads, float scale,
                                                                   const float* __restrict__ vals,
                                                                   const float* __restrict__ w,
                                                                   const float* __restrict__ dw,
                                                                   const float* __restrict__ rowdot,
                                                                   float* __restrict__ c)
{
    const int h = blockIdx.y;
    const int64_t off = (int64_t)h * nnz;
    const int64_t stride = (int64_t)gridDim.x * kElemThreads * kElemIlp;
    for (int64_t base = (int64_t)blockIdx.x * kElemThreads * kElemIlp + threadIdx.x; base < nnz; base += stride) {
        float g[kElemIlp], ww[kElemIlp], s[kElemIlp];
        int r[kElemIlp];
#pragma unroll
        for (int u = 0; u < kElemIlp; ++u) {
            const int64_t e = base + (int64_t)u * kElemThreads;
            const bool in = e < nnz;
            g[u] = in ? __ldg(dw + off + e) : 0.f;
            s[u] = (in && vals) ? __ldg(vals + e) : 1.f;
            if constexpr (SOFTMAX) {
                ww[u] = in ? __ldg(w + off + e) : 0.f;
                r[u] = in ? __ldg(rowidx + e) : 0;
            }
        }
#pragma unroll
        for (int u = 0; u < kElemIlp; ++u) {
            const int64_t e = base + (int64_t)u * kElemThreads;
            if (e >= nnz) continue;
            float v = g[u];
            if constexpr (SOFTMAX) v = ww[u] * (v - __ldg(rowdot + (int64_t)r[u] * heads + h));
            c[off + e] = (scale * s[u]) * v;
        }
    }
}

// rowdot[i, h] = <dY[i, head h], Y[i, head h]>: with Y[i, h] = sum_j w_ij B[j, h]
// this equals sum_j w_ij <dY_i, B_j> = sum_j w_ij dw_ij, the softmax
// backward's row term, read from two dense rows instead of a sparse row
// (balanced whatever the degree).  One thread per (row, head); 16-byte loads
// when the head's columns and both row strides allow them.
template <bool V4>
__global__ void __launch_bounds__(kElemThreads) k_fused_rowdot(int64_t M, int32_t Kh, int32_t heads,
                                                               const float* __restrict__ dY, int64_t lddy,
                                                               const float* __restrict__ Y, int64_t ldy,
                                                               float* __restrict__ rowdot)
{
    const int64_t n = M * heads;
    for (int64_t q = (int64_t)blockIdx.x * kElemThreads + threadIdx.x; q < n; q += (int64_t)gridDim.x * kElemThreads) {
        const int64_t i = q / heads;
        const int h = (int)(q - i * heads);
        const float* g = dY + i * lddy + (int64_t)h * Kh;
        const float* y = Y + i * ldy + (int64_t)h * Kh;
        float a0 = 0.f, a1 = 0.f;
        if constexpr (V4) {
            for (int c = 0; c < Kh; c += 4) {
                const float4 gv = __ldg(reinterpret_cast<const float4*>(g + c));
                const float4 yv = __ldg(reinterpret_cast<const float4*>(y + c));
                a0 = fmaf(gv.x, yv.x, a0); a1 = fmaf(gv.y, yv.y, a1);
                a0 = fmaf(gv.z, yv.z, a0); a1 = fmaf(gv.w, yv.w, a1);
            }
        } else {
            for (int c = 0; c < Kh; ++c) a0 = fmaf(__ldg(g + c), __ldg(y + c), a0);
        }
        rowdot[q] = a0 + a1;
    }
}

cudaError_t launch_fused_rowdot(int64_t M, int K, int heads, const float* dY, int64_t lddy, const float* Y,
                                int64_t ldy, float* rowdot, cudaStream_t s)
{
    const int64_t n = M * heads;
    if (n <= 0) return cudaSuccess;
    const int Kh = K / heads;
    int64_t blocks = (n + kElemThreads - 1) / kElemThreads;
    if (blocks > 152 * 8) blocks = 152 * 8;
    const bool v4 = Kh % 4 == 0 && (reinterpret_cast<uintptr_t>(dY) & 15u) == 0 &&
                    (reinterpret_cast<uintptr_t>(Y) & 15u) == 0 && (M <= 1 || (lddy % 4 == 0 && ldy % 4 == 0));
    if (v4) k_fused_rowdot<true><<<(unsigned)blocks, kElemThreads, 0, s>>>(M, Kh, heads, dY, lddy, Y, ldy, rowdot);
    else k_fused_rowdot<false><<<(unsigned)blocks, kElemThreads, 0, s>>>(M, Kh, heads, dY, lddy, Y, ldy, rowdot);
    return cudaGetLastError();
}

cudaError_t launch_fused_weights(const int32_t* rowidx, int64_t nnz, int heads, int softmax, const float* scores,
                                 const float* lse, float* w, cudaStream_t s)
{
    if (nnz <= 0 || heads <= 0) return cudaSuccess;
    if (!softmax)
        return cudaMemcpyAsync(w, scores, (size_t)nnz * heads * sizeof(float), cudaMemcpyDeviceToDevice, s);
    k_fused_weights<<<dim3(elem_blocks(nnz), (unsigned)heads), kElemThreads, 0, s>>>(rowidx, nnz, heads, scores,
                                                                                     lse, w);
    return cudaGetLastError();
}

cudaError_t launch_fused_score_grad(const int32_t* rowidx, int64_t nnz, int heads, int softmax, float scale,
                                    const float* vals, const float* w, const float* dw, const float* rowdot,
                                    float* c, cudaStream_t s)
{
    if (nnz <= 0 || heads <= 0) return cudaSuccess;
    const dim3 grid(elem_blocks(nnz), (unsigned)heads);
    if (softmax)
        k_fused_score_grad<true><<<grid, kElemThreads, 0, s>>>(rowidx, nnz, heads, scale, vals, w, dw, rowdot, c);
    else
        k_fused_score_grad<false><<<grid, kElemThreads, 0, s>>>(rowidx, nnz, heads, scale, vals, w, dw, rowdot, c);
    return cudaGetLastError();
}

cudaError_t launch_fused(int dt, const Launch& L, const FusedArgs& a, cudaStream_t s)
{
    switch (dt) {
    case DT_F32: return launch_fused_t<DT_F32>(L, a, s);
    case DT_BF16: return launch_fused_t<DT_BF16>(L, a, s);
    case DT_F16: return launch_fused_t<DT_F16>(L, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace spk
