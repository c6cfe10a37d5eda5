// Multi-head SDDMM: per head h (equal slices of K), out[h * nnz + e] =
// s_e * <A[i, head h], B[j, head h]> for every stored e = (i, j) (Eq. 1 on
// each slice), one pass over the pattern for all heads.  The ring span of
// the single-head SDDMM with per-head reductions (ring.cuh, NH > 0).
#include "heads.cuh"
#include "sddmm_impl.cuh"

namespace spk {

template <int DT, int G, int NV, int U, int NH>
__global__ void __launch_bounds__(RING_THREADS, ring_min_ctas(sddmm_ring_bytes(G, NV, U, 2)))
    k_sddmm_ring_mh(const SddmmArgs a)
{
    extern __shared__ __align__(16) unsigned char ring_smem[];
    const int lane = threadIdx.x & 31;
    unsigned char* wsm = ring_smem + (threadIdx.x >> 5) * sddmm_ring_bytes(G, NV, U, 2);
    const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    for (int64_t c = wid; c < a.nchunks; c += nwarps) {
        const int2 b0 = a.bnd[c], b1 = a.bnd[c + 1];
        sddmm_ring_span<DT, G, NV, U, 2, true, NH>(a, lane, wsm, b0.y, b1.y);   // rows are whole lane blocks
    }
}

// (dtype, G, NV, U, NH) compiled: the default SDDMM shapes of K = 32, 64 and
// 128 (FP32) and K = 64, 128 (BF16), every head width that tiles them.
#define SPK_SDDMM_MH(X)                                                                              \
    X(DT_F32, 8, 2, 4, 1) X(DT_F32, 8, 2, 4, 2) X(DT_F32, 8, 2, 4, 4) X(DT_F32, 8, 2, 4, 8)          \
    X(DT_F32, 4, 2, 4, 1) X(DT_F32, 4, 2, 4, 2) X(DT_F32, 4, 2, 4, 4)                                \
    X(DT_F32, 8, 4, 4, 1) X(DT_F32, 8, 4, 4, 2) X(DT_F32, 8, 4, 4, 4) X(DT_F32, 8, 4, 4, 8)          \
    X(DT_BF16, 4, 2, 4, 1) X(DT_BF16, 4, 2, 4, 2) X(DT_BF16, 4, 2, 4, 4)                             \
    X(DT_BF16, 8, 2, 4, 1) X(DT_BF16, 8, 2, 4, 2) X(DT_BF16, 8, 2, 4, 4) X(DT_BF16, 8, 2, 4, 8)

static const void* sddmm_mh_fn(int dt, int G, int NV, int U, int NH)
{
#define X(DT_, G_, NV_, U_, NH_)                                                     \
    if (dt == DT_ && G == G_ && NV == NV_ && U == U_ && NH == NH_)                   \
        return (const void*)&k_sddmm_ring_mh<DT_, G_, NV_, U_, NH_>;
    SPK_SDDMM_MH(X)
#undef X
    return nullptr;
}

bool sddmm_mh_supported(int dt, int G, int NV, int U, int NH) { return sddmm_mh_fn(dt, G, NV, U, NH) != nullptr; }

cudaError_t launch_sddmm_mh(int dt, int G, int NV, int U, int NH, const SddmmArgs& a, cudaStream_t s)
{
    const void* fn = sddmm_mh_fn(dt, G, NV, U, NH);
    if (!fn) return cudaErrorInvalidValue;
    if (a.nchunks <= 0) return cudaSuccess;
    const int warps = RING_THREADS / 32;
    int64_t blocks = (a.nchunks + warps - 1) / warps;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    const size_t smem = (size_t)warps * sddmm_ring_bytes(G, NV, U, 2);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(RING_THREADS), args, smem, s);
}

}  // namespace spk
