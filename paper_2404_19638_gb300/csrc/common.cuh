// Internal declarations shared by the CUDA translation units of libspk.
//
// Data layout in HBM (all caller-owned):
//   S      CSR, int32 rowptr[M+1], colidx[nnz]; values FP32 per call
//   A, B   row-major, leading dimension in elements, one "row" = one dense
//          vector a_i / b_j of Sec. 3.1
//   out    SDDMM: FP32 per nonzero, in colidx order; SpMM: C row-major
// A lane group of G lanes owns one dense row at a time; lane gl holds the
// 16-byte vectors v = gl + G*t (t < NV) of each K block, so one warp-wide
// 128-bit load covers whole 128-byte lines of the gathered rows.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>
#include <stddef.h>

#include "spk.h"

namespace spk {

enum : int { DT_F32 = 0, DT_BF16 = 1, DT_F16 = 2, DT_E4M3 = 3 };

__host__ __device__ constexpr int dt_bytes(int dt) { return dt == DT_F32 ? 4 : (dt == DT_E4M3 ? 1 : 2); }
// Elements in one 16-byte vector of the gathered operand.
__host__ __device__ constexpr int vec_elems(int dt) { return 16 / dt_bytes(dt); }

// ----------------------------------------------------------------------------
// Element loads: N consecutive elements of type DT at element index idx,
// widened to float.  The address must be aligned to min(16, N * bytes).
// Gathered rows are read through the read-only path (ld.global.nc).
// ----------------------------------------------------------------------------
template <int DT>
__device__ __forceinline__ float unpack_one(const uint32_t* w, int k)
{
    if constexpr (DT == DT_F32) {
        return __uint_as_float(w[k]);
    } else if constexpr (DT == DT_BF16) {
        uint32_t x = w[k >> 1];
        return __uint_as_float((k & 1) ? (x & 0xffff0000u) : (x << 16));
    } else if constexpr (DT == DT_F16) {
        uint32_t x = w[k >> 1];
        unsigned short h = (unsigned short)((k & 1) ? (x >> 16) : (x & 0xffffu));
        return __half2float(__ushort_as_half(h));
    } else {
        uint32_t x = w[k >> 2];
        __nv_fp8_storage_t q = (__nv_fp8_storage_t)((x >> (8 * (k & 3))) & 0xffu);
        __half_raw hr = __nv_cvt_fp8_to_halfraw(q, __NV_E4M3);
        return __half2float(__half(hr));
    }
}

template <int DT, int N>
__device__ __forceinline__ void load_elems(const void* base, int64_t idx, float* out)
{
    constexpr int TB = N * dt_bytes(DT);
    constexpr int NW = (TB + 3) / 4;
    uint32_t w[NW];
    const char* p = reinterpret_cast<const char*>(base) + idx * dt_bytes(DT);
    if constexpr (TB >= 16) {
#pragma unroll
        for (int q = 0; q < TB / 16; ++q) {
            uint4 v = __ldg(reinterpret_cast<const uint4*>(p) + q);
            w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
        }
    } else if constexpr (TB == 8) {
        uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
        w[0] = v.x; w[1] = v.y;
    } else if constexpr (TB == 4) {
        w[0] = __ldg(reinterpret_cast<const unsigned int*>(p));
    } else if constexpr (TB == 2) {
        w[0] = __ldg(reinterpret_cast<const unsigned short*>(p));
    } else {
        w[0] = __ldg(reinterpret_cast<const unsigned char*>(p));
    }
    if constexpr (DT == DT_E4M3 && N >= 2) {
#pragma unroll
        for (int k = 0; k < N; k += 2) {
            uint32_t x = w[k >> 2];
            __nv_fp8x2_storage_t q2 = (__nv_fp8x2_storage_t)((x >> (8 * (k & 3))) & 0xffffu);
            __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(q2, __NV_E4M3);
            float2 f = __half22float2(__half2(hr));
            out[k] = f.x; out[k + 1] = f.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) out[k] = unpack_one<DT>(w, k);
    }
}

// Dot-product accumulation in element pairs: acc.x collects the even
// elements, acc.y the odd ones, one packed FMA (two IEEE fused multiply-adds,
// round to nearest) per pair; the caller adds acc.x + acc.y once per dot.
template <int N>
__device__ __forceinline__ void dot_pairs(float2& acc, const float* a, const float* b)
{
    static_assert(N % 2 == 0, "pairs");
#pragma unroll
    for (int q = 0; q < N; q += 2) acc = __ffma2_rn(make_float2(a[q], a[q + 1]), make_float2(b[q], b[q + 1]), acc);
}

// acc[q] += s * b[q] for N elements (pairs through the packed FMA; the result
// of every element is the same as one fmaf).
template <int N>
__device__ __forceinline__ void axpy_pairs(float* acc, float s, const float* b)
{
    if constexpr (N % 2 == 0) {
#pragma unroll
        for (int q = 0; q < N; q += 2) {
            const float2 r = __ffma2_rn(make_float2(s, s), make_float2(b[q], b[q + 1]), make_float2(acc[q], acc[q + 1]));
            acc[q] = r.x;
            acc[q + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) acc[q] = fmaf(s, b[q], acc[q]);
    }
}

// Raw (still packed) elements: gathered rows stay packed in registers while
// their loads are in flight and are widened at the FMA, so a 16-byte vector
// costs 4 registers whatever the dtype.
template <int DT, int N>
struct Raw {
    static constexpr int TB = N * dt_bytes(DT);
    static constexpr int NW = (TB + 3) / 4;
    uint32_t w[NW];
};

template <int DT, int N>
__device__ __forceinline__ void load_raw(const void* base, int64_t idx, Raw<DT, N>& r)
{
    constexpr int TB = Raw<DT, N>::TB;
    const char* p = reinterpret_cast<const char*>(base) + idx * dt_bytes(DT);
    if constexpr (TB >= 16) {
#pragma unroll
        for (int q = 0; q < TB / 16; ++q) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(p) + q);
            r.w[4 * q] = v.x; r.w[4 * q + 1] = v.y; r.w[4 * q + 2] = v.z; r.w[4 * q + 3] = v.w;
        }
    } else if constexpr (TB == 8) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
        r.w[0] = v.x; r.w[1] = v.y;
    } else if constexpr (TB == 4) {
        r.w[0] = __ldg(reinterpret_cast<const unsigned int*>(p));
    } else if constexpr (TB == 2) {
        r.w[0] = __ldg(reinterpret_cast<const unsigned short*>(p));
    } else {
        r.w[0] = __ldg(reinterpret_cast<const unsigned char*>(p));
    }
}

template <int DT, int N>
__device__ __forceinline__ void zero_raw(Raw<DT, N>& r)
{
#pragma unroll
    for (int k = 0; k < Raw<DT, N>::NW; ++k) r.w[k] = 0u;
}

// Widen all N elements of a raw vector.
template <int DT, int N>
__device__ __forceinline__ void unpack_all(const Raw<DT, N>& r, float* out)
{
    if constexpr (DT == DT_E4M3 && N >= 2) {
#pragma unroll
        for (int k = 0; k < N; k += 2) {
            const uint32_t x = r.w[k >> 2];
            const __nv_fp8x2_storage_t q2 = (__nv_fp8x2_storage_t)((x >> (8 * (k & 3))) & 0xffffu);
            const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(q2, __NV_E4M3);
            const float2 f = __half22float2(__half2(hr));
            out[k] = f.x; out[k + 1] = f.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) out[k] = unpack_one<DT>(r.w, k);
    }
}

// Plain (coherent, L1-bypassing) load of C for accumulate and of the carry rows.
template <int DT, int N>
__device__ __forceinline__ void load_elems_cg(const void* base, int64_t idx, float* out)
{
    constexpr int TB = N * dt_bytes(DT);
    constexpr int NW = (TB + 3) / 4;
    uint32_t w[NW];
    const char* p = reinterpret_cast<const char*>(base) + idx * dt_bytes(DT);
    if constexpr (TB >= 16) {
#pragma unroll
        for (int q = 0; q < TB / 16; ++q) {
            uint4 v = __ldcg(reinterpret_cast<const uint4*>(p) + q);
            w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
        }
    } else if constexpr (TB == 8) {
        uint2 v = __ldcg(reinterpret_cast<const uint2*>(p));
        w[0] = v.x; w[1] = v.y;
    } else if constexpr (TB == 4) {
        w[0] = __ldcg(reinterpret_cast<const unsigned int*>(p));
    } else {
        w[0] = __ldcg(reinterpret_cast<const unsigned short*>(p));
    }
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] = unpack_one<DT>(w, k);
}

// Store N floats as DT (F32, BF16 or F16; round-to-nearest-even), streaming
// (evict-first) so that output rows do not displace gathered rows in L2.
template <int DT, int N>
__device__ __forceinline__ void store_elems(void* base, int64_t idx, const float* v)
{
    constexpr int TB = N * dt_bytes(DT);
    constexpr int NW = (TB + 3) / 4;
    uint32_t w[NW];
    if constexpr (DT == DT_F32) {
#pragma unroll
        for (int k = 0; k < N; ++k) w[k] = __float_as_uint(v[k]);
    } else if constexpr (N == 1) {
        unsigned short h = (DT == DT_BF16) ? __bfloat16_as_ushort(__float2bfloat16_rn(v[0]))
                                           : __half_as_ushort(__float2half_rn(v[0]));
        w[0] = h;
    } else {
#pragma unroll
        for (int k = 0; k < N; k += 2) {
            uint32_t lo, hi;
            if constexpr (DT == DT_BF16) {
                lo = __bfloat16_as_ushort(__float2bfloat16_rn(v[k]));
                hi = __bfloat16_as_ushort(__float2bfloat16_rn(v[k + 1]));
            } else {
                lo = __half_as_ushort(__float2half_rn(v[k]));
                hi = __half_as_ushort(__float2half_rn(v[k + 1]));
            }
            w[k >> 1] = lo | (hi << 16);
        }
    }
    char* p = reinterpret_cast<char*>(base) + idx * dt_bytes(DT);
    if constexpr (TB >= 16) {
#pragma unroll
        for (int q = 0; q < TB / 16; ++q)
            __stcs(reinterpret_cast<uint4*>(p) + q, make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]));
    } else if constexpr (TB == 8) {
        __stcs(reinterpret_cast<uint2*>(p), make_uint2(w[0], w[1]));
    } else if constexpr (TB == 4) {
        __stcs(reinterpret_cast<unsigned int*>(p), w[0]);
    } else {
        *reinterpret_cast<unsigned short*>(p) = (unsigned short)w[0];
    }
}

// Resident 256-thread CTAs per SM a kernel is compiled for, from the
// registers of gathered rows each lane keeps in flight (U x NV raw vectors).
__host__ __device__ constexpr int min_ctas(int inflight_regs)
{
    return inflight_regs <= 16 ? 3 : (inflight_regs <= 32 ? 2 : 1);
}

// Lane group of G lanes inside a warp.
template <int G>
struct Group {
    int gl;          // lane within the group
    unsigned mask;   // members, for *_sync intrinsics
    __device__ __forceinline__ Group()
    {
        const int lane = threadIdx.x & 31;
        gl = lane & (G - 1);
        mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    }
};

// ----------------------------------------------------------------------------
// Kernel arguments
// ----------------------------------------------------------------------------
struct SddmmArgs {
    int64_t M, N, nnz;
    int32_t K;
    const int32_t* rowptr;
    const int32_t* colidx;
    const int32_t* rowidx;    // COO row of every nonzero (balanced schedule only)
    const float* vals;        // NULL = ones
    const float* vals2;       // NULL = ones
    const void* A; int64_t lda; const float* a_scale;
    const void* B; int64_t ldb; const float* b_scale;
    float* out;
    const int2* bnd;          // chunk boundaries (row, nonzero); NULL = row-split
    int64_t nchunks;
};

struct SpmmArgs {
    int64_t M, N, nnz;
    int32_t K;
    int32_t vals_staged;      // vals is 16-byte aligned and used alone: stream it with the indices
    int32_t heads = 1;        // value arrays, one per equal slice of K (1: one array for all columns)
    int64_t hstride = 0;      // elements from one head's value array to the next
    const int32_t* rowptr;
    const int32_t* colidx;
    const int32_t* rowidx;
    const int32_t* vperm;     // values index through this permutation (S^T), or NULL
    const float* vals;
    const float* vals2;
    const void* B; int64_t ldb; const float* b_scale;
    void* C; int64_t ldc; int32_t dtc; int32_t accumulate;
    const int2* bnd;          // NULL = row-split
    const int4* meta;         // {head slot, tail slot, last row, unused} per chunk
    const int32_t* head_s0;   // first slot of the split row a chunk's head piece belongs to
    const int32_t* slot_np;   // pieces of the split row starting at a slot
    int32_t* cnt;             // arrival counters per split row (self-resetting)
    float* carry;             // partial rows, K floats per slot
    int64_t nchunks;
};

// FusedMM: SDDMM cascaded into SpMM on one dense matrix B, per head of
// heads equal slices of K (dh = K / heads): scores e = scale * s * <a_i, b_j>
// over the head's slice, weights w = e or the row softmax of e, and
// Y[i, head] = sum_j w_ij * B[j, head].
struct FusedArgs {
    int64_t M, N, nnz;
    int32_t K, heads, dh;
    int32_t softmax;
    float scale;
    const int32_t* rowptr;
    const int32_t* colidx;
    const int32_t* rowidx;
    const float* vals;        // NULL = ones; 16-byte aligned
    const void* A; int64_t lda;
    const void* B; int64_t ldb;
    float* Y; int64_t ldy;
    float* scores;            // heads x nnz (head-major), or NULL
    float* lse;               // M x heads: max + log(sum) of each softmax row, or NULL
    const int2* bnd;
    const int4* meta;
    const int32_t* head_s0;
    const int32_t* slot_np;
    int32_t* cnt;
    float* carry;             // split-row pieces: K partial sums + (max, sum) per head, per slot
    int64_t nchunks;
};

// Kernel shape: lanes per group, 16-byte vectors per lane, nonzeros in flight.
struct Shape { int G, NV, U; };

// Shapes compiled into the library, indexed by position.
#define SPK_SHAPES(X) \
    X(0, 4, 1, 4)     \
    X(1, 8, 1, 8)     \
    X(2, 16, 1, 8)    \
    X(3, 32, 1, 8)    \
    X(4, 8, 2, 8)     \
    X(5, 16, 2, 8)    \
    X(6, 32, 2, 4)    \
    X(7, 4, 2, 4)     \
    X(8, 32, 4, 4)    \
    X(9, 16, 1, 4)    \
    X(10, 8, 2, 4)    \
    X(11, 8, 1, 4)    \
    X(12, 8, 4, 4)

constexpr int kNumShapes = 13;
int shape_index(int G, int NV, int U);   // -1 if not compiled
Shape shape_at(int i);

struct Launch {
    int shape;         // index into SPK_SHAPES
    bool vec;          // 16-byte vector mode (else one element per lane slot)
    int threads;
    bool chunks;       // balanced schedule
    bool ring;         // stage gathered rows in a shared-memory ring where the path has one
    int stages;        // batch slots of the ring (2 or 4)
};

// Launchers (one per dtype family; defined in the sddmm_*.cu / spmm_*.cu files).
cudaError_t launch_sddmm(int dta, int dtb, const Launch& L, const SddmmArgs& a, cudaStream_t s);
cudaError_t launch_spmm(int dtb, const Launch& L, const SpmmArgs& a, cudaStream_t s);

cudaError_t launch_sddmm_f32(int dta, const Launch& L, const SddmmArgs& a, cudaStream_t s);
cudaError_t launch_sddmm_bf16(int dta, const Launch& L, const SddmmArgs& a, cudaStream_t s);
cudaError_t launch_sddmm_f16(int dta, const Launch& L, const SddmmArgs& a, cudaStream_t s);
cudaError_t launch_sddmm_e4m3(int dta, const Launch& L, const SddmmArgs& a, cudaStream_t s);
cudaError_t launch_spmm_f32(const Launch& L, const SpmmArgs& a, cudaStream_t s);
cudaError_t launch_spmm_bf16(const Launch& L, const SpmmArgs& a, cudaStream_t s);
cudaError_t launch_spmm_f16(const Launch& L, const SpmmArgs& a, cudaStream_t s);
cudaError_t launch_spmm_e4m3(const Launch& L, const SpmmArgs& a, cudaStream_t s);

// ----------------------------------------------------------------------------
// Schedule / plan helpers (schedule.cu, transpose.cu)
// ----------------------------------------------------------------------------
struct SchedLayout {
    int64_t nchunks;
    size_t rowidx, bnd, meta, head_s0, slot_np, cnt, pieces, scan_tmp, total;
};
SchedLayout sched_layout(int64_t M, int64_t nnz, int32_t W);
size_t scan_temp_bytes(int64_t n);
cudaError_t scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, void* tmp, cudaStream_t s);
cudaError_t build_schedule(const int32_t* rowptr, int64_t M, int64_t nnz, int32_t W, char* storage,
                           const SchedLayout& L, int64_t* npieces_out, cudaStream_t s);
cudaError_t launch_validate(const int32_t* rowptr, const int32_t* colidx, int64_t M, int64_t N, int64_t nnz,
                            int32_t* report, cudaStream_t s);

struct TplanLayout {
    size_t colptr, rowidx, perm, sched, total;          // storage
    size_t keys0, keys1, vals0, vals1, hist, scan_tmp, temp_total;  // temp
    int64_t nblocks;
    int passes;
    SchedLayout sl;
};
TplanLayout tplan_layout(int64_t M, int64_t N, int64_t nnz, int32_t W);
cudaError_t launch_fused(int dt, const Launch& L, const FusedArgs& a, cudaStream_t s);
cudaError_t launch_fused_mh(int dt, int G, const FusedArgs& a, cudaStream_t s);
cudaError_t launch_fused_weights(const int32_t* rowidx, int64_t nnz, int heads, int softmax, const float* scores,
                                 const float* lse, float* w, cudaStream_t s);
cudaError_t launch_fused_rowdot(int64_t M, int K, int heads, const float* dY, int64_t lddy, const float* Y,
                                int64_t ldy, float* rowdot, cudaStream_t s);
cudaError_t launch_fused_score_grad(const int32_t* rowidx, int64_t nnz, int heads, int softmax, float scale,
                                    const float* vals, const float* w, const float* dw, const float* rowdot,
                                    float* c, cudaStream_t s);
int fused_shape_index(int G, int NV, int U);   // -1 if not compiled
cudaError_t launch_permute_vals(const int32_t* perm, const float* vals, const float* vals2, int64_t nnz, float* out,
                                cudaStream_t s);
cudaError_t build_transpose(const int32_t* rowptr, const int32_t* colidx, int64_t M, int64_t N, int64_t nnz,
                            char* storage, char* temp, const TplanLayout& L, cudaStream_t s);
// Stable LSD radix sort of n int32 keys (8 bits per pass, `passes` passes over
// the low bits) carrying int32 values (NULL = the identity 0..n-1); the result
// lands in k0/v0 or k1/v1 (pointers returned; keys/vals themselves when n = 0
// or passes = 0).  hist: radix_hist_bytes(n); scan_tmp: scan_temp_bytes of the
// histogram's entries (radix_tiles(n) * 256).
int radix_passes(int64_t range);          // passes that cover keys in [0, range)
int64_t radix_tiles(int64_t n);
size_t radix_hist_bytes(int64_t n);
cudaError_t radix_sort_i32(const int32_t* keys, const int32_t* vals, int64_t n, int passes, int32_t* k0, int32_t* k1,
                           int32_t* v0, int32_t* v1, int32_t* hist, void* scan_tmp, const int32_t** keys_out,
                           const int32_t** vals_out, cudaStream_t s);
// Row relabelling (reorder.cu)
size_t reorder_temp_bytes(int64_t M);
cudaError_t row_order(const int32_t* rowptr, const int32_t* colidx, int64_t M, int64_t N, int64_t nnz, int kind,
                      int32_t* perm, char* temp, int* host_status, cudaStream_t s);
cudaError_t permute_pattern(const int32_t* rowptr, const int32_t* colidx, int64_t M, const int32_t* perm,
                            int32_t* rowptr2, int32_t* colidx2, int32_t* emap, char* temp, cudaStream_t s);
cudaError_t permute_rows(const void* X, int64_t ldx_b, int64_t M, int64_t bytes, const int32_t* perm, int scatter,
                         void* Y, int64_t ldy_b, cudaStream_t s);
cudaError_t permute_values(const float* x, const int32_t* map, int64_t n, int scatter, float* y, cudaStream_t s);
// Dense row-panel tiles on the tensor cores (tc.cu)
struct TcArgs {
    int64_t M, N;
    int32_t K;
    const void* A; int64_t lda;      // BF16, M x K
    const void* B; int64_t ldb;      // BF16, N x K
    const int4* tiles;               // {panel, column tile, first entry, entries} per dense tile
    const int32_t* ent_slot;         // slot in S of each dense-tile entry
    const int32_t* ent_ij;           // (row in panel) << 16 | (column in tile)
    const float* vals;               // NULL = ones
    float* out;
    int32_t* status;                 // set to 1 if a tensor-core wait ran out
    int32_t unarmed = 0;             // 1: issue no MMA and no commit, so the wait runs out (tests only)
};
size_t tc_sddmm_smem(int K);
cudaError_t launch_tc_sddmm(const TcArgs& a, int64_t ntiles, cudaStream_t s);
struct TcLayout {
    size_t tiles, ent_slot, ent_ij, rowptr, colidx, emap, status, sched, total;     // storage
    size_t rows, key, k0, k1, v0, v1, key2, order, kp, start, runid, runbeg, dense, entries, tileix, entoff, isdense,
        cnt, hist, scan, temp_total;
    int64_t max_tiles;
    SchedLayout sl;
};
TcLayout tc_layout(int64_t M, int64_t N, int64_t nnz, int32_t threshold, int32_t W);
cudaError_t tc_plan_build(const int32_t* rowptr, const int32_t* colidx, int64_t M, int64_t N, int64_t nnz,
                          int32_t threshold, char* storage, char* temp, const TcLayout& L, int64_t* ntiles,
                          int64_t* dense_nnz, cudaStream_t s);
cudaError_t launch_scatter_scale(const int32_t* map, const float* vals, const float* x, int64_t n, float* out,
                                 cudaStream_t s);
// COO -> CSR (coo.cu)
size_t coo_temp_bytes(int64_t M, int64_t N, int64_t nnz);
cudaError_t coo_to_csr(int64_t M, int64_t N, int64_t nnz, const int32_t* rows, const int32_t* cols, const float* vals,
                       int dedup, int32_t* rowptr, int32_t* colidx, float* vals_out, int64_t* nnz_out,
                       int32_t* first_bad, char* temp, cudaStream_t s);

cudaError_t launch_cast(const float* x, int64_t n, int dt, void* out, cudaStream_t s);
cudaError_t launch_quant_e4m3(const float* X, int64_t M, int64_t K, int64_t ldx, uint8_t* Q, int64_t ldq,
                              float* scales, cudaStream_t s);

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace spk

// Host-side handle types (opaque in the C header).
struct spk_csr_s {
    int64_t M, N, nnz;
    const int32_t* rowptr;
    const int32_t* colidx;
    const int32_t* vperm;     // set for the transposed pattern of a plan
    // balanced schedule (in caller storage)
    bool has_sched;
    int32_t W;
    int64_t nchunks, npieces;
    const int32_t* rowidx;
    const int2* bnd;
    const int4* meta;
    const int32_t* head_s0;
    const int32_t* slot_np;
    int32_t* cnt;
};

struct spk_tcplan_s {
    spk_csr_s Rest;           // entries outside dense tiles (with their schedule); rowptr/colidx in storage
    const int4* tiles;
    const int32_t* ent_slot;
    const int32_t* ent_ij;
    const int32_t* emap;      // slot in S of each remainder entry
    int32_t* status;
    int64_t M, N, nnz, ntiles, dense_nnz;
    int32_t threshold;
};

struct spk_tplan_s {
    spk_csr_s St;             // pattern of S^T (rowptr = colptr, colidx = rowidx), vperm = perm
    const int32_t* colptr;
    const int32_t* rowidx;
    const int32_t* perm;
    int64_t M, N;             // of S
};
