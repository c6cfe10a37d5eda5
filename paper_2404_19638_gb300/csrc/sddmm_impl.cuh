// SDDMM kernel template: out_e = s_e * <A[i,:], B[j,:]> for every stored
// e = (i, j) (Sec. 3.2, Eq. 1; the fine-grain task of Sec. 3.2 is one scaled
// inner product).
//
// A lane group of G lanes walks a span of consecutive nonzeros U at a time:
//   1. the U column indices (and COO rows) are read as broadcast loads,
//   2. the U gathered rows of B and the A rows they meet are issued together
//      (an A row is loaded only where the row changes inside the batch), so a
//      batch keeps U*NV 16-byte loads in flight per lane,
//   3. each lane forms U partial dot products over its slice of K,
//   4. a reduce-scatter across the group (U-1 shuffles plus log2(G/U)
//      butterflies, instead of U*log2(G)) leaves the full sum for nonzero u in
//      lane u, which scales it by s_e and stores it (coalesced).
// Spans are whole rows (row-split) or chunks of the balanced schedule, whose
// long rows are cut into pieces; SDDMM outputs are per nonzero, so pieces
// need no combining.
#pragma once
#include "common.cuh"

namespace spk {

template <int DTA, int DTB, int VECN, int G, int NV, int U, bool KNOWN_ROW>
__device__ __forceinline__ void sddmm_span(const SddmmArgs& a, const Group<G>& g, int64_t r0,
                                           int64_t e0, int64_t e1)
{
    const int nvec = a.K / VECN;               // vectors per dense row
    constexpr int PER_BLK = G * NV;
    const int nkb = (nvec + PER_BLK - 1) / PER_BLK;
    float arow[NV][VECN];          // used when the span is one known row
    bool have_arow = false;

    for (int64_t eb = e0 & ~int64_t(U - 1); eb < e1; eb += U) {
        int j[U], row[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = eb + u;
            ok[u] = (e >= e0) && (e < e1);
            j[u] = ok[u] ? __ldg(a.colidx + e) : 0;
            if constexpr (KNOWN_ROW) row[u] = (int)r0;
            else row[u] = ok[u] ? __ldg(a.rowidx + e) : -1;
        }
        float p[U];
#pragma unroll
        for (int u = 0; u < U; ++u) p[u] = 0.f;

        for (int kb = 0; kb < nkb; ++kb) {
            float bv[U][NV][VECN];
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    const int v = kb * PER_BLK + t * G + g.gl;
                    if (ok[u] && v < nvec) {
                        load_elems<DTB, VECN>(a.B, (int64_t)j[u] * a.ldb + (int64_t)v * VECN, bv[u][t]);
                    } else {
#pragma unroll
                        for (int q = 0; q < VECN; ++q) bv[u][t][q] = 0.f;
                    }
                }
            }
            if constexpr (KNOWN_ROW) {
                // One row for the whole span: its A slice is loaded once.
                if (nkb > 1 || !have_arow) {
#pragma unroll
                    for (int t = 0; t < NV; ++t) {
                        const int v = kb * PER_BLK + t * G + g.gl;
                        if (v < nvec) load_elems<DTA, VECN>(a.A, r0 * a.lda + (int64_t)v * VECN, arow[t]);
                        else
#pragma unroll
                            for (int q = 0; q < VECN; ++q) arow[t][q] = 0.f;
                    }
                    have_arow = true;
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int t = 0; t < NV; ++t)
#pragma unroll
                        for (int q = 0; q < VECN; ++q) p[u] = fmaf(arow[t][q], bv[u][t][q], p[u]);
            } else {
                // A rows: loaded where the row changes inside the batch, issued
                // together with the B gathers.
                float av[U][NV][VECN];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool fresh = (u == 0) || (row[u] != row[u > 0 ? u - 1 : 0]) || !ok[u > 0 ? u - 1 : 0];
#pragma unroll
                    for (int t = 0; t < NV; ++t) {
                        const int v = kb * PER_BLK + t * G + g.gl;
                        if (fresh) {
                            if (ok[u] && v < nvec) {
                                load_elems<DTA, VECN>(a.A, (int64_t)row[u] * a.lda + (int64_t)v * VECN, av[u][t]);
                            } else {
#pragma unroll
                                for (int q = 0; q < VECN; ++q) av[u][t][q] = 0.f;
                            }
                        } else {
#pragma unroll
                            for (int q = 0; q < VECN; ++q) av[u][t][q] = av[u > 0 ? u - 1 : 0][t][q];
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int t = 0; t < NV; ++t)
#pragma unroll
                        for (int q = 0; q < VECN; ++q) p[u] = fmaf(av[u][t][q], bv[u][t][q], p[u]);
            }
        }

        if constexpr (DTA == DT_E4M3) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (ok[u]) p[u] *= __ldg(a.a_scale + row[u]) * __ldg(a.b_scale + j[u]);
        }

        // Reduce-scatter over the low log2(U) lane bits: after the stage with
        // distance d, lanes with bit d set keep the upper half of the list.
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
        // Combine the G/U lane subsets that each hold a partial of nonzero gl % U.
#pragma unroll
        for (int d = U; d < G; d <<= 1) p[0] += __shfl_xor_sync(g.mask, p[0], d, G);

        if (g.gl < U) {
            const int64_t e = eb + g.gl;
            if (e >= e0 && e < e1) {
                float s = a.vals ? __ldg(a.vals + e) : 1.f;
                if (a.vals2) s *= __ldg(a.vals2 + e);
                __stcs(a.out + e, s * p[0]);
            }
        }
    }
}

template <int DTA, int DTB, int VECN, int G, int NV, int U>
__global__ void __launch_bounds__(256) k_sddmm(const SddmmArgs a)
{
    const Group<G> g;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (a.bnd) {
        for (int64_t c = gid; c < a.nchunks; c += ngroups) {
            const int2 b0 = a.bnd[c], b1 = a.bnd[c + 1];
            sddmm_span<DTA, DTB, VECN, G, NV, U, false>(a, g, b0.x, b0.y, b1.y);
        }
    } else {
        for (int64_t r = gid; r < a.M; r += ngroups) {
            const int64_t e0 = __ldg(a.rowptr + r), e1 = __ldg(a.rowptr + r + 1);
            sddmm_span<DTA, DTB, VECN, G, NV, U, true>(a, g, r, e0, e1);
        }
    }
}

// Kernel for (dtypes, vector mode, shape index).
template <int DTA, int DTB, int VECN>
inline const void* sddmm_kernel_for(int shape)
{
    switch (shape) {
#define X(i, G_, NV_, U_) case i: return (const void*)&k_sddmm<DTA, DTB, VECN, G_, NV_, U_>;
        SPK_SHAPES(X)
#undef X
    }
    return nullptr;
}

template <int DTA, int DTB>
cudaError_t launch_sddmm_t(const Launch& L, const SddmmArgs& a, cudaStream_t s)
{
    const void* fn = L.vec ? sddmm_kernel_for<DTA, DTB, vec_elems(DTB)>(L.shape)
                           : sddmm_kernel_for<DTA, DTB, 1>(L.shape);
    if (!fn) return cudaErrorInvalidValue;
    const Shape sh = shape_at(L.shape);
    const int64_t items = a.bnd ? a.nchunks : a.M;
    if (items <= 0) return cudaSuccess;
    const int64_t groups_per_cta = L.threads / sh.G;
    int64_t blocks = (items + groups_per_cta - 1) / groups_per_cta;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(L.threads), args, 0, s);
}

}  // namespace spk
