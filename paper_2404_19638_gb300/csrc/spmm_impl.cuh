// SpMM kernel template: C[i,:] = sum_{e=(i,j)} s_e * B[j,:]  (Sec. 3.2, Eq. 2;
// the fine-grain task is one vector scaling).  Also serves S^T Y through a
// transposed pattern whose values are gathered through a permutation.
//
// A lane group of G lanes owns K-slices of one output row at a time and walks
// a span of consecutive nonzeros U at a time: the indices (and values) arrive
// through shared memory one tile ahead (cp.async, see tiles.cuh); U*NV 16-byte
// gathers of B rows are in flight per lane; FP32 FMAs into registers.
// When the COO row changes, the finished row is stored; rows without
// nonzeros between two stored rows are written as zeros.
//
// Balanced schedule: a chunk is a range of the merged (row ends, nonzeros)
// sequence.  Rows longer than the chunk work are cut into pieces; a piece's
// partial row goes to its carry slot, and the group that delivers the last
// piece of a row (an integer arrival counter; no float atomics, no waiting)
// adds the pieces in chunk order and writes the row.  The sum order is fixed
// by the schedule, so results are bitwise reproducible.
#pragma once
#include "ring.cuh"

namespace spk {

template <int VECN>
__device__ __forceinline__ void write_vec(const SpmmArgs& a, int64_t idx, const float* v)
{
    float o[VECN];
#pragma unroll
    for (int q = 0; q < VECN; ++q) o[q] = v[q];
    switch (a.dtc) {
    case DT_BF16:
        if (a.accumulate) {
            float old[VECN];
            load_elems_cg<DT_BF16, VECN>(a.C, idx, old);
#pragma unroll
            for (int q = 0; q < VECN; ++q) o[q] += old[q];
        }
        store_elems<DT_BF16, VECN>(a.C, idx, o);
        break;
    case DT_F16:
        if (a.accumulate) {
            float old[VECN];
            load_elems_cg<DT_F16, VECN>(a.C, idx, old);
#pragma unroll
            for (int q = 0; q < VECN; ++q) o[q] += old[q];
        }
        store_elems<DT_F16, VECN>(a.C, idx, o);
        break;
    default:
        if (a.accumulate) {
            float old[VECN];
            load_elems_cg<DT_F32, VECN>(a.C, idx, old);
#pragma unroll
            for (int q = 0; q < VECN; ++q) o[q] += old[q];
        }
        store_elems<DT_F32, VECN>(a.C, idx, o);
    }
}

template <int VECN, int G, int NV>
__device__ __forceinline__ void write_row(const SpmmArgs& a, const Group<G>& g, int kb, int nvec, int64_t row,
                                          const float (&acc)[NV][VECN])
{
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        const int v = kb * G * NV + t * G + g.gl;
        if (v < nvec) write_vec<VECN>(a, row * a.ldc + (int64_t)v * VECN, acc[t]);
    }
}

template <int VECN, int G, int NV>
__device__ __forceinline__ void zero_row(const SpmmArgs& a, const Group<G>& g, int kb, int nvec, int64_t row)
{
    if (a.accumulate) return;
    float z[VECN];
#pragma unroll
    for (int q = 0; q < VECN; ++q) z[q] = 0.f;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        const int v = kb * G * NV + t * G + g.gl;
        if (v < nvec) write_vec<VECN>(a, row * a.ldc + (int64_t)v * VECN, z);
    }
}

// Deposit one piece of a split row and, if it is the last to arrive, finish the row.
template <int VECN, int G, int NV>
__device__ __forceinline__ void finish_piece(const SpmmArgs& a, const Group<G>& g, int kb, int nkb, int nvec,
                                             int slot, int s0, int64_t row, const float (&acc)[NV][VECN])
{
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        const int v = kb * G * NV + t * G + g.gl;
        if (v < nvec) store_elems<DT_F32, VECN>(a.carry, (int64_t)slot * a.K + (int64_t)v * VECN, acc[t]);
    }
    __threadfence();
    __syncwarp(g.mask);
    int last = 0;
    if (g.gl == 0) {
        const int np = __ldcg(a.slot_np + s0);
        const int old = atomicAdd(a.cnt + s0, 1);
        last = (old == np * nkb - 1);
    }
    last = __shfl_sync(g.mask, last, 0, G);
    if (!last) return;
    __threadfence();
    const int np = __ldcg(a.slot_np + s0);
    for (int kb2 = 0; kb2 < nkb; ++kb2) {
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const int v = kb2 * G * NV + t * G + g.gl;
            if (v >= nvec) continue;
            float sum[VECN];
#pragma unroll
            for (int q = 0; q < VECN; ++q) sum[q] = 0.f;
            for (int sl = s0; sl < s0 + np; ++sl) {
                float x[VECN];
                load_elems_cg<DT_F32, VECN>(a.carry, (int64_t)sl * a.K + (int64_t)v * VECN, x);
#pragma unroll
                for (int q = 0; q < VECN; ++q) sum[q] += x[q];
            }
            write_vec<VECN>(a, row * a.ldc + (int64_t)v * VECN, sum);
        }
    }
    __syncwarp(g.mask);
    if (g.gl == 0) atomicExch(a.cnt + s0, 0);   // ready for the next launch
}

template <int DTB, int VECN, int G, int NV, int U, bool KNOWN_ROW>
__device__ __forceinline__ void spmm_span(const SpmmArgs& a, const Group<G>& g, int* tiles, int kb, int nkb,
                                          int64_t r0, int64_t e0, int64_t r1, int64_t e1,
                                          const int4 meta, int head_s0)
{
    constexpr int T = TileCfg<G>::T;
    static_assert(T % U == 0, "tile must hold whole batches");
    const int nvec = a.K / VECN;
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

    const int64_t tb0 = e0 & ~int64_t(3);
    const int32_t* rsrc = KNOWN_ROW ? nullptr : a.rowidx;
    const float* vsrc = a.vals_staged ? a.vals : nullptr;
    if (e0 < e1) {
        fill_tile<G>(tiles, 0, tb0, a.nnz, g.gl, a.colidx, rsrc, vsrc);
        cp_async_commit();
    }
    int t = 0;
    for (int64_t tb = tb0; tb < e1; tb += T, ++t) {
        const int buf = t & 1;
        if (tb + T < e1) fill_tile<G>(tiles, buf ^ 1, tb + T, a.nnz, g.gl, a.colidx, rsrc, vsrc);
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp(g.mask);
        const int* colt = tiles + buf * T;
        const int* rowt = tiles + 2 * T + buf * T;
        const float* valt = reinterpret_cast<const float*>(tiles + 4 * T + buf * T);
        for (int b = 0; b < T; b += U) {
            const int64_t eb = tb + b;
            if (eb >= e1) break;
            int j[U], row[U];
            float s[U];
            bool ok[U];
#pragma unroll
            for (int u = 0; u < U; u += 4) {
                const int4 c4 = *reinterpret_cast<const int4*>(colt + b + u);
                j[u] = c4.x; j[u + 1] = c4.y; j[u + 2] = c4.z; j[u + 3] = c4.w;
                if constexpr (KNOWN_ROW) {
                    row[u] = row[u + 1] = row[u + 2] = row[u + 3] = (int)r0;
                } else {
                    const int4 r4 = *reinterpret_cast<const int4*>(rowt + b + u);
                    row[u] = r4.x; row[u + 1] = r4.y; row[u + 2] = r4.z; row[u + 3] = r4.w;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) ok[u] = (eb + u >= e0) && (eb + u < e1);
            if (a.vals_staged) {
#pragma unroll
                for (int u = 0; u < U; u += 4) {
                    const float4 v4 = *reinterpret_cast<const float4*>(valt + b + u);
                    s[u] = v4.x; s[u + 1] = v4.y; s[u + 2] = v4.z; s[u + 3] = v4.w;
                }
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    float sv = 1.f;
                    if (ok[u]) {
                        const int64_t e = eb + u;
                        const int64_t vi = a.vperm ? (int64_t)__ldg(a.vperm + e) : e;
                        if (a.vals) sv = __ldg(a.vals + vi);
                        if (a.vals2) sv *= __ldg(a.vals2 + vi);
                    }
                    s[u] = sv;
                }
            }
            if constexpr (DTB == DT_E4M3) {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (ok[u]) s[u] *= __ldg(a.b_scale + j[u]);
            }
            Raw<DTB, VECN> bw[U][NV];
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int t2 = 0; t2 < NV; ++t2) {
                    const int v = kb * G * NV + t2 * G + g.gl;
                    if (ok[u] && v < nvec) load_raw<DTB, VECN>(a.B, (int64_t)j[u] * a.ldb + (int64_t)v * VECN, bw[u][t2]);
                    else zero_raw(bw[u][t2]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!ok[u]) continue;
                if constexpr (!KNOWN_ROW) {
                    if (row[u] != cur) {
                        flush(cur);
                        for (int64_t rr = cur + 1; rr < row[u]; ++rr) zero_row<VECN, G, NV>(a, g, kb, nvec, rr);
                        cur = row[u];
#pragma unroll
                        for (int t2 = 0; t2 < NV; ++t2)
#pragma unroll
                            for (int q = 0; q < VECN; ++q) acc[t2][q] = 0.f;
                    }
                }
#pragma unroll
                for (int t2 = 0; t2 < NV; ++t2) {
                    float bf[VECN];
                    unpack_all<DTB, VECN>(bw[u][t2], bf);
                    axpy_pairs<VECN>(acc[t2], s[u], bf);
                }
            }
        }
        __syncwarp(g.mask);
    }
    cp_async_wait<0>();
    flush(cur);
    for (int64_t rr = cur + 1; rr <= meta.z; ++rr) zero_row<VECN, G, NV>(a, g, kb, nvec, rr);
}

// One group per span (a chunk of the balanced schedule, or a row).  The
// vector path runs the lean span without shared memory; the element path
// streams index tiles through shared memory.
template <int DTB, int VECN, int G, int NV, int U>
__global__ void __launch_bounds__(256, VECN > 1 ? (U * NV <= 4 ? 4 : (U * NV <= 8 ? 3 : 2)) : min_ctas(U * NV * Raw<DTB, VECN>::NW))
    k_spmm(const SpmmArgs a)
{
    extern __shared__ int smem[];
    const Group<G> g;
    const int kb = blockIdx.y, nkb = gridDim.y;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    int* sm = smem + (threadIdx.x / G) * tile_words(G);
    if (a.bnd) {
        for (int64_t c = gid; c < a.nchunks; c += ngroups) {
            const int2 b0 = a.bnd[c], b1 = a.bnd[c + 1];
            const int4 m = a.meta[c];
            if (b1.y == b0.y && m.z < b0.x) continue;          // nothing in this chunk
            const int hs0 = (m.x >= 0) ? __ldg(a.head_s0 + c) : -1;
            if constexpr (VECN > 1)
                spmm_group_span<DTB, G, NV, U, false>(a, g, kb, nkb, b0.x, b0.y, b1.x, b1.y, m, hs0);
            else
                spmm_span<DTB, VECN, G, NV, U, false>(a, g, sm, kb, nkb, b0.x, b0.y, b1.x, b1.y, m, hs0);
        }
    } else {
        for (int64_t r = gid; r < a.M; r += ngroups) {
            const int e0 = __ldg(a.rowptr + r), e1 = __ldg(a.rowptr + r + 1);
            const int4 m = make_int4(-1, -1, (int)r, 0);
            if constexpr (VECN > 1)
                spmm_group_span<DTB, G, NV, U, true>(a, g, kb, nkb, (int)r, e0, (int)r, e1, m, -1);
            else
                spmm_span<DTB, VECN, G, NV, U, true>(a, g, sm, kb, nkb, r, e0, r, e1, m, -1);
        }
    }
}

// Ring path: one group per span of the balanced schedule, gathered rows
// staged in the warp's shared-memory ring (ring.cuh).
template <int DT, int G, int NV, int U, int VB>
__global__ void __launch_bounds__(RING_THREADS, ring_min_ctas(spmm_ring_bytes(NV, U, VB))) k_spmm_ring(const SpmmArgs a)
{
    extern __shared__ __align__(16) unsigned char ring_smem[];
    const Group<G> g;
    uint4* wring = reinterpret_cast<uint4*>(ring_smem) + (threadIdx.x >> 5) * (spmm_ring_bytes(NV, U, VB, a.heads) / 16);
    const int kb = blockIdx.y, nkb = gridDim.y;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const bool allv = a.K / (VB / dt_bytes(DT)) >= (kb + 1) * G * NV;
    for (int64_t c = gid; c < a.nchunks; c += ngroups) {
        const int2 b0 = a.bnd[c], b1 = a.bnd[c + 1];
        const int4 m = a.meta[c];
        if (b1.y == b0.y && m.z < b0.x) continue;          // nothing in this chunk
        const int hs0 = (m.x >= 0) ? __ldg(a.head_s0 + c) : -1;
        if (allv) spmm_ring_span<DT, G, NV, U, true, VB>(a, g, wring, kb, nkb, b0.x, b0.y, b1.x, b1.y, m, hs0);
        else spmm_ring_span<DT, G, NV, U, false, VB>(a, g, wring, kb, nkb, b0.x, b0.y, b1.x, b1.y, m, hs0);
    }
}

template <int DT, int VB>
inline const void* spmm_ring_kernel_for(int shape)
{
    switch (shape) {
#define X(i, G_, NV_, U_) case i: return (const void*)&k_spmm_ring<DT, G_, NV_, U_, VB>;
        SPK_SHAPES(X)
#undef X
    }
    return nullptr;
}

template <int DTB, int VECN>
inline const void* spmm_kernel_for(int shape)
{
    switch (shape) {
#define X(i, G_, NV_, U_) case i: return (const void*)&k_spmm<DTB, VECN, G_, NV_, U_>;
        SPK_SHAPES(X)
#undef X
    }
    return nullptr;
}

template <int DTB>
cudaError_t launch_spmm_t(const Launch& L, const SpmmArgs& a, cudaStream_t s)
{
    const void* fn = L.vec ? spmm_kernel_for<DTB, vec_elems(DTB)>(L.shape) : spmm_kernel_for<DTB, 1>(L.shape);
    if (!fn) return cudaErrorInvalidValue;
    const Shape sh = shape_at(L.shape);
    const int vecn = L.vec ? vec_elems(DTB) : 1;
    const int nvec = a.K / vecn;
    const int nkb = (nvec + sh.G * sh.NV - 1) / (sh.G * sh.NV);
    const int64_t items = a.bnd ? a.nchunks : a.M;
    if (items <= 0) return cudaSuccess;
    if constexpr (DTB != DT_E4M3) {
        const bool ring_ok = L.vec && L.ring && a.bnd && !a.vperm && !a.vals2 && (!a.vals || a.vals_staged) &&
                             (a.heads == 1 || shape_at(L.shape).NV == 1);
        if (ring_ok) {
            // 16-bit operands whose 16-byte vectors would leave half the group's
            // lanes idle are spread over all of them as 8-byte vectors
            constexpr bool can_half = (DTB == DT_BF16 || DTB == DT_F16);
            const bool half = can_half && 2 * nvec <= sh.G * sh.NV && a.K % 4 == 0;
            const int vb = half ? 8 : 16;
            const void* rf = half ? spmm_ring_kernel_for<DTB, (can_half ? 8 : 16)>(L.shape)
                                  : spmm_ring_kernel_for<DTB, 16>(L.shape);
            if (!rf) return cudaErrorInvalidValue;
            const int nkb2 = half ? (a.K / 4 + sh.G * sh.NV - 1) / (sh.G * sh.NV) : nkb;

            const int64_t groups_per_cta = RING_THREADS / sh.G;
            int64_t blocks = (items + groups_per_cta - 1) / groups_per_cta;
            if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
            if (nkb2 > 65535) return cudaErrorInvalidValue;
            const size_t smem = (size_t)(RING_THREADS / 32) * spmm_ring_bytes(sh.NV, sh.U, vb, a.heads);
            if (smem > 48 * 1024) {
                cudaError_t e = cudaFuncSetAttribute(rf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
            }
            void* args[] = {(void*)&a};
            return cudaLaunchKernel(rf, dim3((unsigned)blocks, (unsigned)nkb2), dim3(RING_THREADS), args, smem, s);
        }
    }
    const int64_t groups_per_cta = L.threads / sh.G;
    int64_t blocks = (items + groups_per_cta - 1) / groups_per_cta;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    if (nkb > 65535) return cudaErrorInvalidValue;
    const size_t smem = L.vec ? 0 : (size_t)groups_per_cta * tile_words(sh.G) * sizeof(int);
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3((unsigned)blocks, (unsigned)nkb), dim3(L.threads), args, smem, s);
}

}  // namespace spk
