// SpMM kernel template: C[i,:] = sum_{e=(i,j)} s_e * B[j,:]  (Sec. 3.2, Eq. 2;
// the fine-grain task is one vector scaling).  Also serves S^T Y through a
// transposed pattern whose values are gathered through a permutation.
//
// A lane group of G lanes owns K-slices of one output row at a time and walks
// a span of consecutive nonzeros U at a time: U broadcast index loads, U*NV
// 16-byte gathers of B rows in flight per lane, FP32 FMAs into registers.
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
#include "common.cuh"

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
__device__ __forceinline__ void spmm_span(const SpmmArgs& a, const Group<G>& g, int kb, int nkb,
                                          int64_t r0, int64_t e0, int64_t r1, int64_t e1,
                                          const int4 meta, int head_s0)
{
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

    for (int64_t eb = e0 & ~int64_t(U - 1); eb < e1; eb += U) {
        int j[U], row[U];
        float s[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = eb + u;
            ok[u] = (e >= e0) && (e < e1);
            j[u] = ok[u] ? __ldg(a.colidx + e) : 0;
            if constexpr (KNOWN_ROW) row[u] = (int)r0;
            else row[u] = ok[u] ? __ldg(a.rowidx + e) : 0;
            const int64_t vi = a.vperm ? (ok[u] ? (int64_t)__ldg(a.vperm + e) : 0) : e;
            float sv = 0.f;
            if (ok[u]) {
                sv = a.vals ? __ldg(a.vals + vi) : 1.f;
                if (a.vals2) sv *= __ldg(a.vals2 + vi);
                if constexpr (DTB == DT_E4M3) sv *= __ldg(a.b_scale + j[u]);
            }
            s[u] = sv;
        }
        float bv[U][NV][VECN];
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                const int v = kb * G * NV + t * G + g.gl;
                if (ok[u] && v < nvec) {
                    load_elems<DTB, VECN>(a.B, (int64_t)j[u] * a.ldb + (int64_t)v * VECN, bv[u][t]);
                } else {
#pragma unroll
                    for (int q = 0; q < VECN; ++q) bv[u][t][q] = 0.f;
                }
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
                    for (int t = 0; t < NV; ++t)
#pragma unroll
                        for (int q = 0; q < VECN; ++q) acc[t][q] = 0.f;
                }
            }
#pragma unroll
            for (int t = 0; t < NV; ++t)
#pragma unroll
                for (int q = 0; q < VECN; ++q) acc[t][q] = fmaf(s[u], bv[u][t][q], acc[t][q]);
        }
    }
    flush(cur);
    for (int64_t rr = cur + 1; rr <= meta.z; ++rr) zero_row<VECN, G, NV>(a, g, kb, nvec, rr);
}

template <int DTB, int VECN, int G, int NV, int U>
__global__ void __launch_bounds__(256) k_spmm(const SpmmArgs a)
{
    const Group<G> g;
    const int kb = blockIdx.y, nkb = gridDim.y;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (a.bnd) {
        for (int64_t c = gid; c < a.nchunks; c += ngroups) {
            const int2 b0 = a.bnd[c], b1 = a.bnd[c + 1];
            const int4 m = a.meta[c];
            if (b1.y == b0.y && m.z < b0.x) continue;          // nothing in this chunk
            const int hs0 = (m.x >= 0) ? __ldg(a.head_s0 + c) : -1;
            spmm_span<DTB, VECN, G, NV, U, false>(a, g, kb, nkb, b0.x, b0.y, b1.x, b1.y, m, hs0);
        }
    } else {
        for (int64_t r = gid; r < a.M; r += ngroups) {
            const int64_t e0 = __ldg(a.rowptr + r), e1 = __ldg(a.rowptr + r + 1);
            spmm_span<DTB, VECN, G, NV, U, true>(a, g, kb, nkb, r, e0, r, e1,
                                                 make_int4(-1, -1, (int)r, 0), -1);
        }
    }
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
    const int64_t groups_per_cta = L.threads / sh.G;
    int64_t blocks = (items + groups_per_cta - 1) / groups_per_cta;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    if (nkb > 65535) return cudaErrorInvalidValue;
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3((unsigned)blocks, (unsigned)nkb), dim3(L.threads), args, 0, s);
}

}  // namespace spk
