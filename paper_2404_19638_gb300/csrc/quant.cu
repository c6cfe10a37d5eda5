// Precision kernels for the low-precision factor formats: round-to-nearest-even
// casts of FP32 to BF16 / F16, and per-row E4M3 quantisation (scale = row amax
// / 448, the largest finite E4M3 magnitude; saturating conversion).
#include "common.cuh"

namespace spk {

template <int DT>
__global__ void k_cast(const float* __restrict__ x, int64_t n, void* __restrict__ out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned short* o = reinterpret_cast<unsigned short*>(out);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float v = __ldcs(x + i);
        o[i] = (DT == DT_BF16) ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : __half_as_ushort(__float2half_rn(v));
    }
}

cudaError_t launch_cast(const float* x, int64_t n, int dt, void* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (dt == DT_BF16) k_cast<DT_BF16><<<(unsigned)blocks, 256, 0, s>>>(x, n, out);
    else k_cast<DT_F16><<<(unsigned)blocks, 256, 0, s>>>(x, n, out);
    return cudaGetLastError();
}

// One warp per row: amax by a warp max-reduction, then code = E4M3(x / scale)
// with an IEEE binary32 division.
__global__ void k_quant_e4m3(const float* __restrict__ X, int64_t M, int64_t K, int64_t ldx, uint8_t* __restrict__ Q,
                             int64_t ldq, float* __restrict__ scales)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < M; r += nwarps) {
        const float* x = X + r * ldx;
        float amax = 0.f;
        for (int64_t k = lane; k < K; k += 32) amax = fmaxf(amax, fabsf(x[k]));
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, d));
        const float scale = amax > 0.f ? __fdiv_rn(amax, 448.0f) : 1.0f;
        if (lane == 0) scales[r] = scale;
        for (int64_t k = lane; k < K; k += 32)
            Q[r * ldq + k] = (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(x[k], scale), __NV_SATFINITE, __NV_E4M3);
    }
}

cudaError_t launch_quant_e4m3(const float* X, int64_t M, int64_t K, int64_t ldx, uint8_t* Q, int64_t ldq,
                              float* scales, cudaStream_t s)
{
    if (M <= 0) return cudaSuccess;
    int64_t blocks = (M * 32 + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_quant_e4m3<<<(unsigned)blocks, 256, 0, s>>>(X, M, K, ldx, Q, ldq, scales);
    return cudaGetLastError();
}

}  // namespace spk
