// Precision kernels for the low-precision factor formats: round-to-nearest-even
// casts of FP32 to BF16 / F16, and per-row E4M3 quantisation (scale = row amax
// / 448, the largest finite E4M3 magnitude; saturating conversion).
#include "common.cuh"

namespace spk {

// Cast: 8 elements per thread and step (two 16-byte loads, one 16-byte store)
// when both buffers are 16-byte aligned; a scalar loop covers the tail and
// unaligned buffers.  Every element is rounded on its own (RNE), so the
// vector and scalar forms give the same bits.
template <int DT>
__device__ __forceinline__ uint32_t cvt_pair(float a, float b)
{
    if constexpr (DT == DT_BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
}

template <int DT>
__global__ void __launch_bounds__(256) k_cast(const float* __restrict__ x, int64_t n, void* __restrict__ out, int vec)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned short* o = reinterpret_cast<unsigned short*>(out);
    int64_t done = 0;
    if (vec) {
        const int64_t n8 = n >> 3;
        const float4* x4 = reinterpret_cast<const float4*>(x);
        uint4* o4 = reinterpret_cast<uint4*>(out);
        for (int64_t i = t0; i < n8; i += stride) {
            const float4 a = __ldcs(x4 + 2 * i), b = __ldcs(x4 + 2 * i + 1);
            uint4 r;
            r.x = cvt_pair<DT>(a.x, a.y); r.y = cvt_pair<DT>(a.z, a.w);
            r.z = cvt_pair<DT>(b.x, b.y); r.w = cvt_pair<DT>(b.z, b.w);
            __stcs(o4 + i, r);
        }
        done = n8 << 3;
    }
    for (int64_t i = done + t0; i < n; i += stride) {
        const float v = __ldcs(x + i);
        o[i] = (DT == DT_BF16) ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : __half_as_ushort(__float2half_rn(v));
    }
}

cudaError_t launch_cast(const float* x, int64_t n, int dt, void* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
    int64_t blocks = ((vec ? n / 8 : n) + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (dt == DT_BF16) k_cast<DT_BF16><<<(unsigned)blocks, 256, 0, s>>>(x, n, out, vec);
    else k_cast<DT_F16><<<(unsigned)blocks, 256, 0, s>>>(x, n, out, vec);
    return cudaGetLastError();
}

// Per-row E4M3 quantisation.  L lanes share a row (32 / L rows per warp); a
// lane owns 4-element pieces k = 4 * (lane + L * c): amax by a max-reduction
// over the L lanes, scale = amax / 448 (1 for an all-zero row), then each
// code = E4M3(x / scale) with an IEEE binary32 division and saturation.
// VEC: 16-byte aligned rows (ldx % 4 == 0) and 4-byte aligned codes
// (ldq % 4 == 0, K % 4 == 0); else one element at a time.
template <int L, bool VEC>
__global__ void __launch_bounds__(256) k_quant_e4m3(const float* __restrict__ X, int64_t M, int64_t K, int64_t ldx,
                                                  uint8_t* __restrict__ Q, int64_t ldq, float* __restrict__ scales)
{
    constexpr int RPW = 32 / L;
    const int lane = threadIdx.x & 31, sl = lane % L;
    const unsigned mask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (lane & ~(L - 1)));
    const int64_t nrg = ((int64_t)gridDim.x * blockDim.x >> 5) * RPW;
    for (int64_t r = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW + lane / L; r - lane / L < M;
         r += nrg) {
        const bool live = r < M;
        const float* x = X + (live ? r : 0) * ldx;
        float amax = 0.f;
        if (live) {
            if (VEC) {
                for (int64_t k = 4 * sl; k < K; k += 4 * L) {
                    const float4 v = __ldg(reinterpret_cast<const float4*>(x + k));
                    amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
                }
            } else {
                for (int64_t k = sl; k < K; k += L) amax = fmaxf(amax, fabsf(__ldg(x + k)));
            }
        }
#pragma unroll
        for (int d = L / 2; d >= 1; d >>= 1) amax = fmaxf(amax, __shfl_xor_sync(mask, amax, d, L));
        if (!live) continue;
        const float scale = amax > 0.f ? __fdiv_rn(amax, 448.0f) : 1.0f;
        if (sl == 0) scales[r] = scale;
        if (VEC) {
            for (int64_t k = 4 * sl; k < K; k += 4 * L) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(x + k));
                uint32_t w = 0;
                w |= (uint32_t)(uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(v.x, scale), __NV_SATFINITE, __NV_E4M3);
                w |= (uint32_t)(uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(v.y, scale), __NV_SATFINITE, __NV_E4M3) << 8;
                w |= (uint32_t)(uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(v.z, scale), __NV_SATFINITE, __NV_E4M3) << 16;
                w |= (uint32_t)(uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(v.w, scale), __NV_SATFINITE, __NV_E4M3) << 24;
                *reinterpret_cast<uint32_t*>(Q + r * ldq + k) = w;
            }
        } else {
            for (int64_t k = sl; k < K; k += L)
                Q[r * ldq + k] = (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(__ldg(x + k), scale), __NV_SATFINITE, __NV_E4M3);
        }
    }
}

template <int L, bool VEC>
static cudaError_t quant_launch(const float* X, int64_t M, int64_t K, int64_t ldx, uint8_t* Q, int64_t ldq,
                                float* scales, cudaStream_t s)
{
    const int64_t warps = (M + (32 / L) - 1) / (32 / L);
    int64_t blocks = (warps * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_quant_e4m3<L, VEC><<<(unsigned)blocks, 256, 0, s>>>(X, M, K, ldx, Q, ldq, scales);
    return cudaGetLastError();
}

cudaError_t launch_quant_e4m3(const float* X, int64_t M, int64_t K, int64_t ldx, uint8_t* Q, int64_t ldq,
                              float* scales, cudaStream_t s)
{
    if (M <= 0) return cudaSuccess;
    const bool vec = (reinterpret_cast<uintptr_t>(X) & 15u) == 0 && ldx % 4 == 0 && K % 4 == 0 &&
                     (reinterpret_cast<uintptr_t>(Q) & 3u) == 0 && ldq % 4 == 0;
    if (!vec) return quant_launch<32, false>(X, M, K, ldx, Q, ldq, scales, s);
    if (K <= 16) return quant_launch<4, true>(X, M, K, ldx, Q, ldq, scales, s);
    if (K <= 32) return quant_launch<8, true>(X, M, K, ldx, Q, ldq, scales, s);
    if (K <= 64) return quant_launch<16, true>(X, M, K, ldx, Q, ldq, scales, s);
    return quant_launch<32, true>(X, M, K, ldx, Q, ldq, scales, s);
}

}  // namespace spk
