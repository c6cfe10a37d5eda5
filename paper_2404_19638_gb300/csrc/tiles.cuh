// Index tiles: a lane group streams the index arrays of its span (column,
// COO row, value per nonzero) through shared memory with cp.async, one tile
// ahead of the compute, so that the gathers of B rows never wait on index
// loads.  A tile holds 4*G nonzeros (one 16-byte copy per lane per array);
// two tiles per group are double-buffered.
#pragma once
#include "common.cuh"

namespace spk {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Shared-memory words per group: 2 buffers x T entries x (col, row, val).
template <int G>
struct TileCfg {
    static constexpr int T = 4 * G;
    static constexpr int WORDS = 2 * 3 * T;
};

// Host-side size of one group's tiles, in 32-bit words.
__host__ __device__ constexpr int tile_words(int G) { return 2 * 3 * 4 * G; }

template <int G>
__device__ __forceinline__ int* group_tiles(int* smem)
{
    return smem + (threadIdx.x / G) * TileCfg<G>::WORDS;
}

// Copy entries [tb, tb + T) of up to three int32/float arrays into buffer
// `buf`; entries at or past `n` are not read (zero-filled or left unset).
template <int G>
__device__ __forceinline__ void fill_tile(int* tiles, int buf, int64_t tb, int64_t n, int gl, const int32_t* colidx,
                                          const int32_t* rowidx, const float* vals)
{
    constexpr int T = TileCfg<G>::T;
    int* col = tiles + buf * T;
    int* row = tiles + 2 * T + buf * T;
    float* val = reinterpret_cast<float*>(tiles + 4 * T + buf * T);
#pragma unroll
    for (int q = gl; q < T / 4; q += G) {
        const int64_t e = tb + 4 * q;
        const int64_t rem = n - e;
        if (rem <= 0) continue;
        const int bytes = rem >= 4 ? 16 : (int)rem * 4;
        cp_async16(col + 4 * q, colidx + e, bytes);
        if (rowidx) cp_async16(row + 4 * q, rowidx + e, bytes);
        if (vals) cp_async16(val + 4 * q, vals + e, bytes);
    }
}

}  // namespace spk
