// SDDMM kernel template: out_e = s_e * <A[i,:], B[j,:]> for every stored
// e = (i, j) (Sec. 3.2, Eq. 1; the fine-grain task of Sec. 3.2 is one scaled
// inner product).
//
// A lane group of G lanes walks a span of consecutive nonzeros U at a time:
//   1. the column indices and COO rows of the span arrive through shared
//      memory one tile ahead (cp.async, see tiles.cuh), so gathers never wait
//      on index loads,
//   2. the U gathered rows of B are issued together (U*NV 16-byte loads in
//      flight per lane); the A slice of the current row stays in registers and
//      is reloaded only where the row changes,
//   3. each lane forms U partial dot products over its slice of K,
//   4. a reduce-scatter across the group (U-1 shuffles plus log2(G/U)
//      butterflies, instead of U*log2(G)) leaves the full sum for nonzero u in
//      lane u, which scales it by s_e and stores it (coalesced).
// Spans are whole rows (row-split) or chunks of the balanced schedule, whose
// long rows are cut into pieces; SDDMM outputs are per nonzero, so pieces
// need no combining.
#pragma once
#include "ring.cuh"

namespace spk {

template <int DTA, int DTB, int VECN, int G, int NV, int U, bool KNOWN_ROW>
__device__ __forceinline__ void sddmm_span(const SddmmArgs& a, const Group<G>& g, int* tiles, int64_t r0,
                                           int64_t e0, int64_t e1)
{
    constexpr int T = TileCfg<G>::T;
    static_assert(T % U == 0, "tile must hold whole batches");
    const int nvec = a.K / VECN;               // vectors per dense row
    constexpr int PER_BLK = G * NV;
    const int nkb = (nvec + PER_BLK - 1) / PER_BLK;
    float av[NV][VECN];                        // A slice of row `ra` (single K block only)
    int ra = -1;
    if (e0 >= e1) return;

    const int64_t tb0 = e0 & ~int64_t(3);
    const int32_t* rsrc = KNOWN_ROW ? nullptr : a.rowidx;
    fill_tile<G>(tiles, 0, tb0, a.nnz, g.gl, a.colidx, rsrc, nullptr);
    cp_async_commit();
    int t = 0;
    for (int64_t tb = tb0; tb < e1; tb += T, ++t) {
        const int buf = t & 1;
        if (tb + T < e1) fill_tile<G>(tiles, buf ^ 1, tb + T, a.nnz, g.gl, a.colidx, rsrc, nullptr);
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp(g.mask);
        const int* colt = tiles + buf * T;
        const int* rowt = tiles + 2 * T + buf * T;
        for (int b = 0; b < T; b += U) {
            const int64_t eb = tb + b;
            if (eb >= e1) break;
            int j[U], row[U];
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
            // the lane that will store nonzero gl fetches its value now
            float sv = 0.f;
            const int64_t ew = eb + g.gl;
            const bool writer = (g.gl < U) && (ew >= e0) && (ew < e1);
            if (writer) {
                sv = a.vals ? __ldg(a.vals + ew) : 1.f;
                if (a.vals2) sv *= __ldg(a.vals2 + ew);
            }

            float p[U];
#pragma unroll
            for (int u = 0; u < U; ++u) p[u] = 0.f;
            for (int kb = 0; kb < nkb; ++kb) {
                Raw<DTB, VECN> bw[U][NV];
#pragma unroll
                for (int u = 0; u < U; ++u) {
#pragma unroll
                    for (int t2 = 0; t2 < NV; ++t2) {
                        const int v = kb * PER_BLK + t2 * G + g.gl;
                        if (ok[u] && v < nvec) load_raw<DTB, VECN>(a.B, (int64_t)j[u] * a.ldb + (int64_t)v * VECN, bw[u][t2]);
                        else zero_raw(bw[u][t2]);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (!ok[u]) continue;
                    if (nkb > 1 || row[u] != ra) {
                        // row change (rare inside a batch): reload the A slice
#pragma unroll
                        for (int t2 = 0; t2 < NV; ++t2) {
                            const int v = kb * PER_BLK + t2 * G + g.gl;
                            if (v < nvec) load_elems<DTA, VECN>(a.A, (int64_t)row[u] * a.lda + (int64_t)v * VECN, av[t2]);
                            else
#pragma unroll
                                for (int q = 0; q < VECN; ++q) av[t2][q] = 0.f;
                        }
                        ra = (nkb == 1) ? row[u] : -1;
                    }
#pragma unroll
                    for (int t2 = 0; t2 < NV; ++t2) {
                        float bf[VECN];
                        unpack_all<DTB, VECN>(bw[u][t2], bf);
#pragma unroll
                        for (int q = 0; q < VECN; ++q) p[u] = fmaf(av[t2][q], bf[q], p[u]);
                    }
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

            if (writer) __stcs(a.out + ew, sv * p[0]);
        }
        __syncwarp(g.mask);
    }
    cp_async_wait<0>();
}

// Element path (operands not 16-byte aligned / K not a multiple of a vector):
// one group per span, index tiles in shared memory.
template <int DTA, int DTB, int VECN, int G, int NV, int U>
__global__ void __launch_bounds__(256, min_ctas(U * NV * Raw<DTB, VECN>::NW)) k_sddmm(const SddmmArgs a)
{
    extern __shared__ int smem[];
    int* sm = smem + (threadIdx.x / G) * tile_words(G);
    const Group<G> g;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (a.bnd) {
        for (int64_t c = gid; c < a.nchunks; c += ngroups) {
            const int2 b0 = a.bnd[c], b1 = a.bnd[c + 1];
            sddmm_span<DTA, DTB, VECN, G, NV, U, false>(a, g, sm, b0.x, b0.y, b1.y);
        }
    } else {
        for (int64_t r = gid; r < a.M; r += ngroups) {
            const int64_t e0 = __ldg(a.rowptr + r), e1 = __ldg(a.rowptr + r + 1);
            sddmm_span<DTA, DTB, VECN, G, NV, U, true>(a, g, sm, r, e0, e1);
        }
    }
}

// Vector path: one warp per span (a chunk of the balanced schedule, or a row).
template <int DTA, int DTB, int G, int NV, int U>
__global__ void __launch_bounds__(256, U * NV <= 4 ? 4 : (U * NV <= 8 ? 3 : 2)) k_sddmm_lean(const SddmmArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (a.bnd) {
        for (int64_t c = wid; c < a.nchunks; c += nwarps) {
            const int2 b0 = a.bnd[c], b1 = a.bnd[c + 1];
            sddmm_warp_span<DTA, DTB, G, NV, U, false>(a, lane, b0.x, b0.y, b1.y);
        }
    } else {
        for (int64_t r = wid; r < a.M; r += nwarps) {
            const int e0 = __ldg(a.rowptr + r), e1 = __ldg(a.rowptr + r + 1);
            sddmm_warp_span<DTA, DTB, G, NV, U, true>(a, lane, (int)r, e0, e1);
        }
    }
}

// Ring path: one warp per span of the balanced schedule, gathered rows staged
// in the warp's shared-memory ring of D batch slots (ring.cuh).
template <int DT, int G, int NV, int U, int D>
__global__ void __launch_bounds__(RING_THREADS, ring_min_ctas(sddmm_ring_bytes(G, NV, U, D)))
    k_sddmm_ring(const SddmmArgs a)
{
    extern __shared__ __align__(16) unsigned char ring_smem[];
    const int lane = threadIdx.x & 31;
    unsigned char* wsm = ring_smem + (threadIdx.x >> 5) * sddmm_ring_bytes(G, NV, U, D);
    const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const bool allv = a.K / vec_elems(DT) >= G * NV;
    for (int64_t c = wid; c < a.nchunks; c += nwarps) {
        const int2 b0 = a.bnd[c], b1 = a.bnd[c + 1];
        if (allv) sddmm_ring_span<DT, G, NV, U, D, true>(a, lane, wsm, b0.y, b1.y);
        else sddmm_ring_span<DT, G, NV, U, D, false>(a, lane, wsm, b0.y, b1.y);
    }
}

template <int DT, int D>
inline const void* sddmm_ring_kernel_for(int shape)
{
    switch (shape) {
#define X(i, G_, NV_, U_) case i: return (const void*)&k_sddmm_ring<DT, G_, NV_, U_, D>;
        SPK_SHAPES(X)
#undef X
    }
    return nullptr;
}

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
inline const void* sddmm_lean_kernel_for(int shape)
{
    switch (shape) {
#define X(i, G_, NV_, U_) case i: return (const void*)&k_sddmm_lean<DTA, DTB, G_, NV_, U_>;
        SPK_SHAPES(X)
#undef X
    }
    return nullptr;
}

template <int DTA, int DTB>
cudaError_t launch_sddmm_t(const Launch& L, const SddmmArgs& a, cudaStream_t s)
{
    const Shape sh = shape_at(L.shape);
    const int64_t items = a.bnd ? a.nchunks : a.M;
    if (items <= 0) return cudaSuccess;
    const bool lean = L.vec && (a.K / vec_elems(DTB)) <= sh.G * sh.NV;
    if constexpr (DTA == DTB && DTB != DT_E4M3) {
        if (lean && L.ring && a.bnd) {
            const void* rf = L.stages == 4 ? sddmm_ring_kernel_for<DTB, 4>(L.shape)
                                           : sddmm_ring_kernel_for<DTB, 2>(L.shape);
            if (!rf) return cudaErrorInvalidValue;
            const int warps = RING_THREADS / 32;
            int64_t blocks = (items + warps - 1) / warps;
            if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
            const size_t smem = (size_t)warps * sddmm_ring_bytes(sh.G, sh.NV, sh.U, L.stages == 4 ? 4 : 2);
            if (smem > 48 * 1024) {
                cudaError_t e = cudaFuncSetAttribute(rf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
            }
            void* args[] = {(void*)&a};
            return cudaLaunchKernel(rf, dim3((unsigned)blocks), dim3(RING_THREADS), args, smem, s);
        }
    }
    const void* fn = lean ? sddmm_lean_kernel_for<DTA, DTB>(L.shape)
                          : (L.vec ? sddmm_kernel_for<DTA, DTB, vec_elems(DTB)>(L.shape)
                                   : sddmm_kernel_for<DTA, DTB, 1>(L.shape));
    if (!fn) return cudaErrorInvalidValue;
    const int64_t per_cta = lean ? L.threads / 32 : L.threads / sh.G;     // spans per CTA
    int64_t blocks = (items + per_cta - 1) / per_cta;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    const size_t smem = lean ? 0 : (size_t)(L.threads / sh.G) * tile_words(sh.G) * sizeof(int);
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(L.threads), args, smem, s);
}

}  // namespace spk
