// Dense row-panel tiles on the 5th-generation tensor cores (tcgen05).
//
// Where a 128-row x 64-column tile of S holds many entries, its SDDMM (Eq. 1)
// is a real contraction: the tile's A panel (128 x K) and B tile (64 x K) are
// read once into shared memory and multiplied whole on the tensor cores into
// a 128 x 64 FP32 block in tensor memory, which is then sampled at the tile's
// entries, instead of one K-long row gather per entry.  Likewise its SpMM
// (Eq. 2) is the dense product of the tile (as a 128 x 64 matrix) with the
// 64 x K block of B, accumulated over the tiles of a row panel.  Entries
// outside dense tiles (the remainder) run on the gather kernels.
//
// Operands are BF16 (products exact, FP32 accumulation).  The sparse values
// of SpMM are FP32: each is split into three BF16 pieces (hi + mid + lo, exact
// for every FP32 value whose pieces are not BF16 subnormals) multiplied as
// three products, so the result is the FP32 product sum.
//
// Shared-memory operands use the no-swizzle K-major layout of 8-row x 16-byte
// core matrices: core (row block rb, K block kb) of a tile with K elements per
// row sits at byte (rb * K/8 + kb) * 128, row r of the core at + 16 * (r % 8).
// Descriptor: leading (K direction) byte offset 128, stride (row direction)
// byte offset K/8 * 128.  One MMA consumes K = 16 (two core columns).
//
// Every wait on the tensor core's mbarrier has an iteration limit; on expiry
// the kernel records an error, waits (bounded) for the operation once more,
// frees its tensor memory and returns.
#include "common.cuh"

namespace spk {

namespace {

constexpr int TC_M = 128;      // rows of a panel (MMA M)
constexpr int TC_N = 64;       // columns of a tile (SDDMM MMA N, SpMM MMA K)
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_SPIN_LIMIT = 1u << 20;     // polls of a non-blocking test (tens of ms at most)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of the barrier; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    for (uint32_t i = 0; i < TC_SPIN_LIMIT; ++i)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// D (tensor memory) (+)= A (smem, M x 16) . B (smem, N x 16)^T, BF16 in, FP32 out.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
                 : "memory");
}
// Arrive on the barrier once every MMA this thread issued has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// Matrix descriptor of a no-swizzle K-major operand starting at `addr`
// (shared-memory byte address) with `kbytes` bytes of K per row.
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t addr, uint32_t kbytes)
{
    const uint64_t lbo = 128;                 // next core matrix along K
    const uint64_t sbo = (kbytes / 16) * 128; // next 8-row group
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of 16-byte piece kb of row r in the core-matrix layout.
__device__ __forceinline__ uint32_t core_off(int r, int kb, int kblocks)
{
    return (uint32_t)((r >> 3) * kblocks + kb) * 128u + (uint32_t)(r & 7) * 16u;
}

__device__ __forceinline__ void cp16_zfill(void* smem, const void* gmem, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

// Rows [r0, r0 + nrows) of a BF16 matrix (row stride ld elements, `limit`
// rows exist) into the core-matrix layout; rows past `limit` read as zero.
__device__ __forceinline__ void load_rows_kmajor(unsigned char* dst, const __nv_bfloat16* src, int64_t ld, int64_t r0,
                                                 int nrows, int64_t limit, int K)
{
    const int kblocks = K / 8;
    for (int t = threadIdx.x; t < nrows * kblocks; t += blockDim.x) {
        const int r = t / kblocks, kb = t - r * kblocks;
        const bool valid = r0 + r < limit;
        const __nv_bfloat16* g = src + (valid ? (r0 + r) : 0) * ld + kb * 8;
        cp16_zfill(dst + core_off(r, kb, kblocks), g, valid);
    }
    asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;\n" ::: "memory");
}

}  // namespace

// ----------------------------------------------------------------------------
// SDDMM on dense tiles: one CTA per tile (several resident per SM, so one
// tile's loads overlap another's product and sampling).
//   out[e] = s_e * (A_panel B_tile^T)[i, j] for every entry e = (i, j) of the tile.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(TC_THREADS) k_tc_sddmm(const TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const int K = a.K;
    unsigned char* sA = sm;                                   // 128 x K BF16
    unsigned char* sB = sA + TC_M * K * 2;                    // 64 x K BF16
    float* sD = reinterpret_cast<float*>(sB + TC_N * K * 2);  // 128 x 65 FP32
    uint64_t* bar = reinterpret_cast<uint64_t*>(sD + TC_M * 65);
    uint32_t* tbase = reinterpret_cast<uint32_t*>(bar + 1);
    const int warp = threadIdx.x >> 5;

    const int4 tile = a.tiles[blockIdx.x];                    // {panel, column tile, first entry, entries}
    const int64_t r0 = (int64_t)tile.x * TC_M, c0 = (int64_t)tile.y * TC_N;

    if (warp == 0) {
        tmem_alloc(tbase, TC_N);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) mbar_init(bar);
    load_rows_kmajor(sA, reinterpret_cast<const __nv_bfloat16*>(a.A), a.lda, r0, TC_M, a.M, K);
    load_rows_kmajor(sB, reinterpret_cast<const __nv_bfloat16*>(a.B), a.ldb, c0, TC_N, a.N, K);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tbase;

    if (threadIdx.x == 0 && !a.unarmed) {
        const uint32_t idesc = idesc_bf16(TC_M, TC_N);
        const uint32_t kbytes = (uint32_t)K * 2;
        for (int k = 0; k < K / 16; ++k)                      // K step 16 = two core columns of 128 bytes
            mma_bf16(tmem, kmajor_desc(smem_u32(sA) + 256 * k, kbytes), kmajor_desc(smem_u32(sB) + 256 * k, kbytes),
                     idesc, k > 0);
        mma_commit(bar);
    }
    const bool done = mbar_wait(bar, 0);
    tc_fence_after();
    if (!done) {
        if (threadIdx.x == 0) atomicExch(a.status, 1);
        mbar_wait(bar, 0);                                     // once more before the tensor memory goes
    } else {
        // lane 32 * warp + l of tensor memory holds row 32 * warp + l of the block
        const int row = 32 * warp + (threadIdx.x & 31);
#pragma unroll
        for (int c = 0; c < TC_N; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) sD[row * 65 + c + q] = v[q];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TC_N);
    if (!done) return;
    // sample the block: eight entries per thread at a time, every load of a
    // round issued before its results are used
    constexpr int R = 8;
    for (int q0 = 0; q0 < tile.w; q0 += R * TC_THREADS) {
        int32_t e[R], ij[R];
        float sv[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int q = q0 + k * TC_THREADS + threadIdx.x;
            const bool in = q < tile.w;
            e[k] = in ? __ldg(a.ent_slot + tile.z + q) : -1;
            ij[k] = in ? __ldg(a.ent_ij + tile.z + q) : 0;
        }
#pragma unroll
        for (int k = 0; k < R; ++k) sv[k] = (a.vals && e[k] >= 0) ? __ldg(a.vals + e[k]) : 1.f;
#pragma unroll
        for (int k = 0; k < R; ++k)
            if (e[k] >= 0) __stcs(a.out + e[k], sv[k] * sD[(ij[k] >> 16) * 65 + (ij[k] & 0xffff)]);
    }
}

size_t tc_sddmm_smem(int K) { return (size_t)(TC_M + TC_N) * K * 2 + (size_t)TC_M * 65 * 4 + 16; }

cudaError_t launch_tc_sddmm(const TcArgs& a, int64_t ntiles, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    const size_t smem = tc_sddmm_smem(a.K);
    cudaError_t e = cudaFuncSetAttribute((const void*)&k_tc_sddmm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_sddmm<<<(unsigned)ntiles, TC_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// The plan: dense tiles, their entries, and the remainder pattern.
//
// Entries are ordered by (panel = row / 128, column tile = column / 64), ties
// in slot order, by two stable radix sorts (column tile, then panel); equal
// keys form runs, and a run of at least `threshold` entries is a dense tile.
// The remainder keeps the other entries of every row, in order, with their
// slots in S.
// ----------------------------------------------------------------------------
namespace {

unsigned tc_grid(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

#define TC_FOR(i, n) for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// rows[e] = row of entry e; key[e] = column tile of e.  One warp per row.
__global__ void k_tc_rows(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int64_t M,
                          int32_t* __restrict__ rows, int32_t* __restrict__ key)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; r < M; r += nw)
        for (int32_t e = rowptr[r] + lane; e < rowptr[r + 1]; e += 32) {
            rows[e] = (int32_t)r;
            key[e] = colidx[e] >> 6;
        }
}

__global__ void k_tc_panel_keys(const int32_t* __restrict__ rows, const int32_t* __restrict__ p1, int64_t n,
                                int32_t* __restrict__ key2)
{
    TC_FOR(q, n) key2[q] = rows[p1 ? p1[q] : q] >> 7;
}

// start[q] = 1 where a run of equal (panel, column tile) begins.
__global__ void k_tc_starts(const int32_t* __restrict__ kp, const int32_t* __restrict__ colidx,
                            const int32_t* __restrict__ p, int64_t n, int32_t* __restrict__ start)
{
    TC_FOR(q, n) {
        int32_t f = 1;
        if (q > 0) {
            const int32_t c = colidx[p ? p[q] : q] >> 6, cb = colidx[p ? p[q - 1] : q - 1] >> 6;
            f = (kp[q] != kp[q - 1]) || (c != cb);
        }
        start[q] = f;
    }
}

// runid = exclusive scan of start; runbeg[run] = first position; runbeg[nruns] = n.
__global__ void k_tc_runs(const int32_t* __restrict__ start, const int32_t* __restrict__ runid, int64_t n,
                          int32_t* __restrict__ runbeg)
{
    TC_FOR(q, n) {
        if (start[q]) runbeg[runid[q]] = (int32_t)q;
        if (q == n - 1) runbeg[runid[q] + start[q]] = (int32_t)n;
    }
}

// dense[run] = 1 if the run has at least `threshold` entries; entries[run] = its
// entry count if dense, else 0 (scanned next into the dense entries' offsets).
__global__ void k_tc_dense(const int32_t* __restrict__ runbeg, int64_t nruns, int32_t threshold,
                           int32_t* __restrict__ dense, int32_t* __restrict__ entries, int64_t cap)
{
    TC_FOR(r, cap) {
        int32_t d = 0, len = 0;
        if (r < nruns) {
            len = runbeg[r + 1] - runbeg[r];
            d = len >= threshold;
        }
        dense[r] = d;
        entries[r] = d ? len : 0;
    }
}

// Tiles, dense entries, and the dense mark of every slot.
__global__ void k_tc_fill(const int32_t* __restrict__ rows, const int32_t* __restrict__ colidx,
                          const int32_t* __restrict__ p, const int32_t* __restrict__ start,
                          const int32_t* __restrict__ runid, const int32_t* __restrict__ runbeg,
                          const int32_t* __restrict__ dense, const int32_t* __restrict__ tileix,
                          const int32_t* __restrict__ entoff, int64_t n, int4* __restrict__ tiles,
                          int32_t* __restrict__ ent_slot, int32_t* __restrict__ ent_ij, int32_t* __restrict__ isdense)
{
    TC_FOR(q, n) {
        const int32_t run = runid[q] + start[q] - 1;
        const int32_t e = p ? p[q] : (int32_t)q;
        if (!dense[run]) {
            isdense[e] = 0;
            continue;
        }
        isdense[e] = 1;
        const int32_t r = rows[e], c = colidx[e];
        const int32_t ent = entoff[run] + ((int32_t)q - runbeg[run]);
        ent_slot[ent] = e;
        ent_ij[ent] = ((r & 127) << 16) | (c & 63);
        if (start[q]) tiles[tileix[run]] = make_int4(r >> 7, c >> 6, entoff[run], runbeg[run + 1] - runbeg[run]);
    }
}

// cnt[r] = entries of row r outside dense tiles (one warp per row).
__global__ void k_tc_rest_count(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ isdense, int64_t M,
                                int32_t* __restrict__ cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; r < M; r += nw) {
        int32_t c = 0;
        for (int32_t e = rowptr[r] + lane; e < rowptr[r + 1]; e += 32) c += 1 - isdense[e];
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) cnt[r] = c;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[M] = 0;
}

// The remainder's columns and slots, each row in order (one warp per row).
__global__ void k_tc_rest_fill(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                               const int32_t* __restrict__ isdense, const int32_t* __restrict__ rrowptr, int64_t M,
                               int32_t* __restrict__ rcol, int32_t* __restrict__ emap)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; r < M; r += nw) {
        int32_t o = rrowptr[r];
        for (int32_t e0 = rowptr[r]; e0 < rowptr[r + 1]; e0 += 32) {
            const int32_t e = e0 + lane;
            const bool keep = e < rowptr[r + 1] && !isdense[e];
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int32_t at = o + __popc(m & ((1u << lane) - 1u));
                rcol[at] = colidx[e];
                emap[at] = e;
            }
            o += __popc(m);
        }
    }
}

// out[map[i]] = (vals ? vals[map[i]] : 1) * x[i]
__global__ void k_scatter_scale(const int32_t* __restrict__ map, const float* __restrict__ vals,
                                const float* __restrict__ x, int64_t n, float* __restrict__ out)
{
    TC_FOR(i, n) {
        const int32_t e = map[i];
        out[e] = (vals ? vals[e] : 1.f) * x[i];
    }
}

#undef TC_FOR

}  // namespace

TcLayout tc_layout(int64_t M, int64_t N, int64_t nnz, int32_t threshold, int32_t W)
{
    TcLayout L;
    const size_t a = align256((size_t)nnz * 4 + 4);
    L.max_tiles = nnz / (threshold > 0 ? threshold : 1) + 1;
    size_t o = 0;
    L.tiles = o; o += align256((size_t)L.max_tiles * 16);
    L.ent_slot = o; o += a;
    L.ent_ij = o; o += a;
    L.rowptr = o; o += align256((size_t)(M + 1) * 4);
    L.colidx = o; o += a;
    L.emap = o; o += a;
    L.status = o; o += 256;
    L.sl = sched_layout(M, nnz, W);               // the remainder has at most nnz entries
    L.sched = o; o += L.sl.total;
    L.total = o;
    const size_t a1 = align256((size_t)nnz * 4 + 8);
    size_t t = 0;
    L.rows = t; t += a1;
    L.key = t; t += a1;
    L.k0 = t; t += a1;
    L.k1 = t; t += a1;
    L.v0 = t; t += a1;
    L.v1 = t; t += a1;
    L.key2 = t; t += a1;
    L.order = t; t += a1;
    L.kp = t; t += a1;
    L.start = t; t += a1;
    L.runid = t; t += a1;
    L.runbeg = t; t += a1;
    L.dense = t; t += a1;
    L.entries = t; t += a1;
    L.tileix = t; t += a1;
    L.entoff = t; t += a1;
    L.isdense = t; t += a1;
    L.cnt = t; t += align256((size_t)(M + 1) * 4);
    L.hist = t; t += radix_hist_bytes(nnz);
    size_t sc = scan_temp_bytes(radix_tiles(nnz) * 256);
    if (scan_temp_bytes(nnz + 1) > sc) sc = scan_temp_bytes(nnz + 1);
    if (scan_temp_bytes(M + 1) > sc) sc = scan_temp_bytes(M + 1);
    L.scan = t; t += align256(sc);
    L.temp_total = t;
    (void)N;
    return L;
}

cudaError_t tc_plan_build(const int32_t* rowptr, const int32_t* colidx, int64_t M, int64_t N, int64_t nnz,
                          int32_t threshold, char* storage, char* temp, const TcLayout& L, int64_t* ntiles,
                          int64_t* dense_nnz, cudaStream_t s)
{
    auto T = [&](size_t off) { return reinterpret_cast<int32_t*>(temp + off); };
    auto P = [&](size_t off) { return reinterpret_cast<int32_t*>(storage + off); };
    *ntiles = 0;
    *dense_nnz = 0;
    cudaError_t e = cudaMemsetAsync(storage + L.status, 0, 256, s);
    if (e != cudaSuccess) return e;
    int32_t* isdense = T(L.isdense);
    int32_t* cnt = T(L.cnt);
    if (nnz > 0) {
        int32_t* rows = T(L.rows);
        k_tc_rows<<<tc_grid(M * 32), 256, 0, s>>>(rowptr, colidx, M, rows, T(L.key));
        // 1. stable sort by column tile, carrying the slot
        const int32_t *ks = nullptr, *p1 = nullptr;
        e = radix_sort_i32(T(L.key), nullptr, nnz, radix_passes((N + 63) / 64), T(L.k0), T(L.k1), T(L.v0), T(L.v1),
                           T(L.hist), temp + L.scan, &ks, &p1, s);
        if (e != cudaSuccess) return e;
        // 2. stable sort of that order by panel (its first pass must not write where p1 is read)
        k_tc_panel_keys<<<tc_grid(nnz), 256, 0, s>>>(rows, p1, nnz, T(L.key2));
        int32_t *k0 = T(L.k0), *k1 = T(L.k1), *v0 = T(L.v0), *v1 = T(L.v1);
        if (p1 == v0) { v0 = T(L.dense); k0 = T(L.entries); }
        const int32_t *kp = nullptr, *p = nullptr;
        e = radix_sort_i32(T(L.key2), p1, nnz, radix_passes((M + 127) / 128), k0, k1, v0, v1, T(L.hist), temp + L.scan,
                           &kp, &p, s);
        if (e != cudaSuccess) return e;
        if (p) {
            e = cudaMemcpyAsync(T(L.order), p, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
            p = T(L.order);
        }
        e = cudaMemcpyAsync(T(L.kp), kp, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        kp = T(L.kp);
        // 3. runs of equal (panel, column tile)
        int32_t* start = T(L.start);
        int32_t* runid = T(L.runid);
        int32_t* runbeg = T(L.runbeg);
        k_tc_starts<<<tc_grid(nnz), 256, 0, s>>>(kp, colidx, p, nnz, start);
        e = scan_exclusive_i32(start, runid, nnz, temp + L.scan, s);
        if (e != cudaSuccess) return e;
        k_tc_runs<<<tc_grid(nnz), 256, 0, s>>>(start, runid, nnz, runbeg);
        int32_t last[2] = {0, 0};
        e = cudaMemcpyAsync(&last[0], runid + (nnz - 1), 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&last[1], start + (nnz - 1), 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        const int64_t nr = (int64_t)last[0] + last[1];
        // 4. dense runs, their tile numbers and entry offsets
        int32_t* dense = T(L.dense);
        int32_t* entries = T(L.entries);
        int32_t* tileix = T(L.tileix);
        int32_t* entoff = T(L.entoff);
        k_tc_dense<<<tc_grid(nr + 1), 256, 0, s>>>(runbeg, nr, threshold, dense, entries, nr + 1);
        e = scan_exclusive_i32(dense, tileix, nr + 1, temp + L.scan, s);
        if (e == cudaSuccess) e = scan_exclusive_i32(entries, entoff, nr + 1, temp + L.scan, s);
        if (e != cudaSuccess) return e;
        int32_t counts[2] = {0, 0};
        e = cudaMemcpyAsync(&counts[0], tileix + nr, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&counts[1], entoff + nr, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        *ntiles = counts[0];
        *dense_nnz = counts[1];
        // 5. tiles, their entries, and the dense mark of every slot
        k_tc_fill<<<tc_grid(nnz), 256, 0, s>>>(rows, colidx, p, start, runid, runbeg, dense, tileix, entoff, nnz,
                                                reinterpret_cast<int4*>(storage + L.tiles), P(L.ent_slot), P(L.ent_ij),
                                                isdense);
    }
    // 6. the remainder pattern: per-row counts, their scan, the kept entries
    if (M > 0) {
        if (nnz > 0) {
            k_tc_rest_count<<<tc_grid(M * 32), 256, 0, s>>>(rowptr, isdense, M, cnt);
        } else {
            e = cudaMemsetAsync(cnt, 0, (size_t)(M + 1) * 4, s);
            if (e != cudaSuccess) return e;
        }
        e = scan_exclusive_i32(cnt, P(L.rowptr), M + 1, temp + L.scan, s);
        if (e != cudaSuccess) return e;
        if (nnz > 0)
            k_tc_rest_fill<<<tc_grid(M * 32), 256, 0, s>>>(rowptr, colidx, isdense, P(L.rowptr), M, P(L.colidx),
                                                            P(L.emap));
    } else {
        e = cudaMemsetAsync(P(L.rowptr), 0, 4, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_scatter_scale(const int32_t* map, const float* vals, const float* x, int64_t n, float* out,
                                 cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_scatter_scale<<<tc_grid(n), 256, 0, s>>>(map, vals, x, n, out);
    return cudaGetLastError();
}

}  // namespace spk
