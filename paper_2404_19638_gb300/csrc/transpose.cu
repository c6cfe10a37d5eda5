// Transpose plan: the CSC of S (= CSR of S^T) and the CSR slot of every CSC
// slot.  SpMM^T, the adjoint of SpMM in the pair of Sec. 3.2, runs as an SpMM
// over this pattern with the values gathered through `perm`; the plan depends
// only on the pattern, so it is built once (Sec. 5.1).
//
// Built by a stable least-significant-digit radix sort of (column, nonzero
// index) pairs, 8 bits per pass: per-tile digit histograms, one exclusive scan
// over the digit-major histogram table, and a scatter that ranks equal digits
// inside a tile in index order (warp match + per-warp digit counts), so that
// rows stay ascending inside every column.
#include "common.cuh"

namespace spk {

constexpr int RX_THREADS = 256;
constexpr int RX_ROUNDS = 16;
constexpr int RX_TILE = RX_THREADS * RX_ROUNDS;
constexpr int RX_DIGITS = 256;
constexpr int RX_WARPS = RX_THREADS / 32;

TplanLayout tplan_layout(int64_t M, int64_t N, int64_t nnz, int32_t W)
{
    TplanLayout L;
    size_t off = 0;
    L.colptr = off; off += align256((size_t)(N + 1) * 4);
    L.rowidx = off; off += align256((size_t)nnz * 4 + 4);
    L.perm = off;   off += align256((size_t)nnz * 4 + 4);
    L.sl = sched_layout(N, nnz, W);
    L.sched = off;  off += L.sl.total;
    L.total = off;

    L.passes = radix_passes(N);
    L.nblocks = radix_tiles(nnz);
    size_t t = 0;
    L.keys0 = t; t += align256((size_t)nnz * 4 + 4);
    L.keys1 = t; t += align256((size_t)nnz * 4 + 4);
    L.vals0 = t; t += align256((size_t)nnz * 4 + 4);
    L.vals1 = t; t += align256((size_t)nnz * 4 + 4);
    L.hist = t;  t += align256((size_t)L.nblocks * RX_DIGITS * 4);
    L.scan_tmp = t; t += align256(scan_temp_bytes(L.nblocks * RX_DIGITS));
    L.temp_total = t;
    return L;
}

// hist[d * nblocks + b] = count of digit d in tile b.
__global__ void __launch_bounds__(RX_THREADS) k_rx_hist(const int32_t* keys, int64_t n, int shift, int64_t nblocks,
                                                       int32_t* hist)
{
    __shared__ int32_t h[RX_DIGITS];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RX_TILE;
    for (int k = 0; k < RX_ROUNDS; ++k) {
        const int64_t i = base + (int64_t)k * RX_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xff], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile.  offs = exclusive scan of hist.  vals_in == NULL
// means the identity (the nonzero index).
__global__ void __launch_bounds__(RX_THREADS) k_rx_scatter(const int32_t* keys_in, const int32_t* vals_in, int64_t n,
                                                          int shift, int64_t nblocks, const int32_t* offs,
                                                          int32_t* keys_out, int32_t* vals_out)
{
    __shared__ int32_t base_d[RX_DIGITS];            // next free slot per digit
    __shared__ int32_t wcnt[RX_WARPS][RX_DIGITS];    // per-warp digit counts, then offsets
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base_d[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    const int64_t tile = (int64_t)blockIdx.x * RX_TILE;
    for (int k = 0; k < RX_ROUNDS; ++k) {
#pragma unroll
        for (int w = 0; w < RX_WARPS; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const int64_t i = tile + (int64_t)k * RX_THREADS + tid;
        const bool valid = i < n;
        const int32_t key = valid ? keys_in[i] : 0;
        const int digit = valid ? ((key >> shift) & 0xff) : RX_DIGITS;   // invalid items form their own class
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {   // thread tid owns digit tid: warp offsets in index order
            int32_t run = base_d[tid];
#pragma unroll
            for (int w = 0; w < RX_WARPS; ++w) {
                const int32_t c = wcnt[w][tid];
                wcnt[w][tid] = run;
                run += c;
            }
            base_d[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const int32_t pos = wcnt[warp][digit] + rank;
            keys_out[pos] = key;
            vals_out[pos] = vals_in ? vals_in[i] : (int32_t)i;
        }
        __syncthreads();
    }
}

__global__ void k_iota(int32_t* out, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int32_t)i;
}

// colptr[j] = number of sorted keys < j.
__global__ void k_colptr(const int32_t* sorted, int64_t nnz, int64_t N, int32_t* colptr)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j > N) return;
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (sorted[mid] < j) lo = mid + 1; else hi = mid;
    }
    colptr[j] = (int32_t)lo;
}

// rowidx[p] = row of CSR slot perm[p] (last r with rowptr[r] <= perm[p]).
__global__ void k_rows_of(const int32_t* rowptr, int64_t M, const int32_t* perm, int64_t nnz, int32_t* rowidx)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    const int32_t e = perm[p];
    int64_t lo = 0, hi = M - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(rowptr + mid) <= e) lo = mid; else hi = mid - 1;
    }
    rowidx[p] = (int32_t)lo;
}

// Values of S^T in CSC slot order: out[p] = vals[perm[p]] * vals2[perm[p]]
// (absent factors are 1), the same single FP32 product the SpMM kernels form.
__global__ void k_permute_vals(const int32_t* __restrict__ perm, const float* __restrict__ vals,
                               const float* __restrict__ vals2, int64_t nnz, float* __restrict__ out)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = __ldg(perm + p);
        float v = vals ? __ldg(vals + e) : 1.f;
        if (vals2) v *= __ldg(vals2 + e);
        out[p] = v;
    }
}

cudaError_t launch_permute_vals(const int32_t* perm, const float* vals, const float* vals2, int64_t nnz, float* out,
                                cudaStream_t s)
{
    if (nnz <= 0) return cudaSuccess;
    int64_t blocks = (nnz + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_permute_vals<<<(unsigned)blocks, 256, 0, s>>>(perm, vals, vals2, nnz, out);
    return cudaGetLastError();
}

int radix_passes(int64_t range)
{
    int bits = 0;
    while (bits < 31 && (int64_t(1) << bits) < range) ++bits;
    return (bits + 7) / 8;
}

int64_t radix_tiles(int64_t n) { return n < 1 ? 1 : (n + RX_TILE - 1) / RX_TILE; }

size_t radix_hist_bytes(int64_t n) { return align256((size_t)radix_tiles(n) * RX_DIGITS * 4); }

cudaError_t radix_sort_i32(const int32_t* keys, const int32_t* vals, int64_t n, int passes, int32_t* k0, int32_t* k1,
                           int32_t* v0, int32_t* v1, int32_t* hist, void* scan_tmp, const int32_t** keys_out,
                           const int32_t** vals_out, cudaStream_t s)
{
    const int64_t nblocks = radix_tiles(n);
    const int32_t* kin = keys;
    const int32_t* vin = vals;
    for (int p = 0; n > 0 && p < passes; ++p) {
        int32_t* kout = (p & 1) ? k1 : k0;
        int32_t* vout = (p & 1) ? v1 : v0;
        k_rx_hist<<<(unsigned)nblocks, RX_THREADS, 0, s>>>(kin, n, 8 * p, nblocks, hist);
        cudaError_t err = scan_exclusive_i32(hist, hist, nblocks * RX_DIGITS, scan_tmp, s);
        if (err != cudaSuccess) return err;
        k_rx_scatter<<<(unsigned)nblocks, RX_THREADS, 0, s>>>(kin, vin, n, 8 * p, nblocks, hist, kout, vout);
        kin = kout; vin = vout;
    }
    *keys_out = kin;
    *vals_out = vin;
    return cudaGetLastError();
}

cudaError_t build_transpose(const int32_t* rowptr, const int32_t* colidx, int64_t M, int64_t N, int64_t nnz,
                            char* storage, char* temp, const TplanLayout& L, cudaStream_t s)
{
    int32_t* colptr = reinterpret_cast<int32_t*>(storage + L.colptr);
    int32_t* rowidx = reinterpret_cast<int32_t*>(storage + L.rowidx);
    int32_t* perm = reinterpret_cast<int32_t*>(storage + L.perm);
    int32_t* k0 = reinterpret_cast<int32_t*>(temp + L.keys0);
    int32_t* k1 = reinterpret_cast<int32_t*>(temp + L.keys1);
    int32_t* v0 = reinterpret_cast<int32_t*>(temp + L.vals0);
    int32_t* v1 = reinterpret_cast<int32_t*>(temp + L.vals1);
    int32_t* hist = reinterpret_cast<int32_t*>(temp + L.hist);
    cudaError_t err;

    const int32_t* sorted_keys = colidx;
    const int32_t* sorted_vals = nullptr;
    if (nnz > 0) {
        err = radix_sort_i32(colidx, nullptr, nnz, L.passes, k0, k1, v0, v1, hist, temp + L.scan_tmp, &sorted_keys,
                             &sorted_vals, s);
        if (err != cudaSuccess) return err;
    }
    // perm: sorted values (identity when no pass ran, i.e. N <= 1)
    if (nnz > 0) {
        if (sorted_vals) {
            err = cudaMemcpyAsync(perm, sorted_vals, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s);
        } else {
            // N <= 1: every key is 0 and the CSR order is already sorted.
            k_iota<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(perm, nnz);
            err = cudaGetLastError();
        }
        if (err != cudaSuccess) return err;
    }
    k_colptr<<<(unsigned)((N + 1 + 255) / 256), 256, 0, s>>>(sorted_keys, nnz, N, colptr);
    if (nnz > 0)
        k_rows_of<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(rowptr, M, perm, nnz, rowidx);
    return cudaGetLastError();
}

}  // namespace spk
