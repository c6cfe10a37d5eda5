// Pattern-only setup kernels: exclusive scan, the balanced (merge-path)
// schedule with its split-row bookkeeping, the COO row view, and the CSR
// validation kernel.  All of it depends only on the sparsity pattern, so it is
// built once and reused while values change (Sec. 5.1).
#include <climits>

#include "common.cuh"

namespace spk {

// ----------------------------------------------------------------------------
// Exclusive scan of int32 (reduce-then-scan, recursive on the block totals).
// ----------------------------------------------------------------------------
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

size_t scan_temp_bytes(int64_t n)
{
    size_t bytes = 0;
    int64_t m = n;
    while (m > SCAN_TILE) {
        m = (m + SCAN_TILE - 1) / SCAN_TILE;
        bytes += align256((size_t)m * sizeof(int32_t));
    }
    return bytes + 256;
}

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t x, int32_t* total)
{
    __shared__ int32_t warp_sums[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int32_t w = (lane < SCAN_THREADS / 32) ? warp_sums[lane] : 0;
        int32_t wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = wi - w;   // exclusive over warps
        if (lane == SCAN_THREADS / 32 - 1) *total = wi;
    }
    __syncthreads();
    const int32_t r = warp_sums[warp] + incl - x;
    __syncthreads();
    return r;
}

// Scans each tile; writes the tile total to sums[blockIdx.x] (if sums != NULL).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const int32_t* in, int32_t* out, int64_t n,
                                                             int32_t* sums)
{
    __shared__ int32_t total;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t t = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        v[q] = (base + q < n) ? in[base + q] : 0;
        t += v[q];
    }
    int32_t run = block_exclusive_scan(t, &total);
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < n) out[base + q] = run;
        run += v[q];
    }
    if (sums && threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_add(int32_t* out, int64_t n, const int32_t* offs)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / SCAN_TILE];
}

cudaError_t scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, void* tmp, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        k_scan_tiles<<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr);
        return cudaGetLastError();
    }
    int32_t* sums = reinterpret_cast<int32_t*>(tmp);
    char* rest = reinterpret_cast<char*>(tmp) + align256((size_t)tiles * sizeof(int32_t));
    k_scan_tiles<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, sums);
    cudaError_t err = scan_exclusive_i32(sums, sums, tiles, rest, s);
    if (err != cudaSuccess) return err;
    k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, sums);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Balanced schedule
// ----------------------------------------------------------------------------
SchedLayout sched_layout(int64_t M, int64_t nnz, int32_t W)
{
    SchedLayout L;
    L.nchunks = (M + nnz + W - 1) / W;
    if (L.nchunks < 1) L.nchunks = 1;
    size_t off = 0;
    L.rowidx = off;   off += align256((size_t)nnz * 4 + 4);
    L.bnd = off;      off += align256((size_t)(L.nchunks + 1) * 8);
    L.meta = off;     off += align256((size_t)L.nchunks * 16);
    L.head_s0 = off;  off += align256((size_t)L.nchunks * 4);
    L.slot_np = off;  off += align256((size_t)L.nchunks * 8 + 4);
    L.cnt = off;      off += align256((size_t)L.nchunks * 8 + 4);
    L.pieces = off;   off += align256((size_t)(L.nchunks + 1) * 4);
    L.scan_tmp = off; off += align256(scan_temp_bytes(L.nchunks + 1));
    L.total = off;
    return L;
}

// Rows finished after d steps of the merge of the row ends rowptr[1..M] with
// the nonzero indices 0..nnz-1, a row end going first when rowptr[r+1] <= e.
// Largest r in [max(0, d - nnz), min(d, M)] with rowptr[r] <= d - r.
__device__ __forceinline__ int64_t merge_path_rows(const int32_t* rowptr, int64_t M, int64_t nnz, int64_t d)
{
    int64_t lo = d - nnz > 0 ? d - nnz : 0;
    int64_t hi = d < M ? d : M;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)__ldg(rowptr + mid) <= d - mid) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Boundary c at merge diagonal min(c*W, M+nnz).  A point (r, rowptr[r+1]) of a
// non-empty row r (its nonzeros done, its end not yet taken) is moved to
// (r+1, rowptr[r+1]);
// a cut inside a row of at most W nonzeros is moved back to the row start.
__global__ void k_sched_bounds(const int32_t* rowptr, int64_t M, int64_t nnz, int32_t W, int64_t nchunks,
                               int2* bnd, int32_t raw)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > nchunks) return;
    int64_t d = c * (int64_t)W;
    if (d > M + nnz) d = M + nnz;
    int64_t r = merge_path_rows(rowptr, M, nnz, d);
    int64_t e = d - r;
    if (!raw) {
        if (r < M && e > rowptr[r] && e >= rowptr[r + 1]) r += 1;
        if (r < M && e > rowptr[r] && (int64_t)rowptr[r + 1] - rowptr[r] <= W) e = rowptr[r];
    }
    bnd[c] = make_int2((int)r, (int)e);
}

__device__ __forceinline__ void chunk_flags(const int2* bnd, const int32_t* rowptr, int64_t M, int64_t c,
                                            int& head, int& tail, int& r_last)
{
    const int2 b0 = bnd[c], b1 = bnd[c + 1];
    head = (b0.x < M && b0.y > rowptr[b0.x]) ? 1 : 0;                 // starts inside a row
    const bool ends_inside = (b1.x < M && b1.y > rowptr[b1.x]);
    tail = (ends_inside && !(b0.x == b1.x && head)) ? 1 : 0;           // first piece of a split row
    r_last = ends_inside ? b1.x : b1.x - 1;
}

__global__ void k_sched_pieces(const int2* bnd, const int32_t* rowptr, int64_t M, int64_t nchunks,
                               int32_t* pieces)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > nchunks) return;
    if (c == nchunks) { pieces[c] = 0; return; }
    int head, tail, r_last;
    chunk_flags(bnd, rowptr, M, c, head, tail, r_last);
    pieces[c] = head + tail;
}

// Slots are numbered chunk by chunk (head piece before tail piece), so the
// pieces of one split row get consecutive slots s0, s0+1, ...
__global__ void k_sched_meta(const int2* bnd, const int32_t* rowptr, int64_t M, int64_t nchunks,
                             const int32_t* base, int4* meta, int32_t* head_s0, int32_t* slot_np, int32_t* cnt)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    int head, tail, r_last;
    chunk_flags(bnd, rowptr, M, c, head, tail, r_last);
    const int hs = head ? base[c] : -1;
    const int ts = tail ? base[c] + head : -1;
    meta[c] = make_int4(hs, ts, r_last, 0);
    if (!tail) return;
    // This chunk holds the first piece of split row r; the following chunks
    // that start inside r hold the rest.
    const int r = bnd[c + 1].x;
    const int rstart = rowptr[r];
    int np = 1;
    for (int64_t c2 = c + 1; c2 < nchunks; ++c2) {
        const int2 b = bnd[c2];
        if (b.x != r || b.y <= rstart) break;
        head_s0[c2] = ts;
        ++np;
    }
    slot_np[ts] = np;
    cnt[ts] = 0;
}

// COO view: rowidx[e] = row of nonzero e (one warp per row).
__global__ void k_coo_rows(const int32_t* rowptr, int64_t M, int32_t* rowidx)
{
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < M; r += nwarps) {
        const int e0 = rowptr[r], e1 = rowptr[r + 1];
        for (int e = e0 + lane; e < e1; e += 32) rowidx[e] = (int)r;
    }
}

cudaError_t build_schedule(const int32_t* rowptr, int64_t M, int64_t nnz, int32_t W, char* storage,
                           const SchedLayout& L, int64_t* npieces_out, cudaStream_t s)
{
    int32_t* rowidx = reinterpret_cast<int32_t*>(storage + L.rowidx);
    int2* bnd = reinterpret_cast<int2*>(storage + L.bnd);
    int4* meta = reinterpret_cast<int4*>(storage + L.meta);
    int32_t* head_s0 = reinterpret_cast<int32_t*>(storage + L.head_s0);
    int32_t* slot_np = reinterpret_cast<int32_t*>(storage + L.slot_np);
    int32_t* cnt = reinterpret_cast<int32_t*>(storage + L.cnt);
    int32_t* pieces = reinterpret_cast<int32_t*>(storage + L.pieces);
    const int64_t nc = L.nchunks;
    const unsigned gb = (unsigned)((nc + 1 + 255) / 256);

    if (M > 0 && nnz > 0) {
        const int64_t warps = M < (1 << 20) ? M : (1 << 20);
        k_coo_rows<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(rowptr, M, rowidx);
    }
    k_sched_bounds<<<gb, 256, 0, s>>>(rowptr, M, nnz, W, nc, bnd, 0);
    k_sched_pieces<<<gb, 256, 0, s>>>(bnd, rowptr, M, nc, pieces);
    cudaError_t err = scan_exclusive_i32(pieces, pieces, nc + 1, storage + L.scan_tmp, s);
    if (err != cudaSuccess) return err;
    k_sched_meta<<<gb, 256, 0, s>>>(bnd, rowptr, M, nc, pieces, meta, head_s0, slot_np, cnt);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    int32_t np = 0;
    err = cudaMemcpyAsync(&np, pieces + nc, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (err != cudaSuccess) return err;
    err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return err;
    *npieces_out = np;
    return cudaSuccess;
}

// Raw merge-path boundaries (no snapping), for tests against a walk of the merge.
cudaError_t launch_merge_path_bounds(const int32_t* rowptr, int64_t M, int64_t nnz, int32_t W, int64_t n,
                                     int2* out, cudaStream_t s)
{
    k_sched_bounds<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(rowptr, M, nnz, W, n, out, 1);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Validation: report = {first error code, first bad index, bad count, unsorted}
// codes: 1 rowptr[0] != 0, 2 rowptr decreases, 3 rowptr[M] != nnz,
//        4 column out of range, 5 rowptr entry outside [0, nnz]
// ----------------------------------------------------------------------------
__global__ void k_validate_init(int32_t* rep)
{
    rep[0] = 0; rep[1] = INT_MAX; rep[2] = 0; rep[3] = 0;
}

__device__ __forceinline__ void report(int32_t* rep, int code, int64_t idx)
{
    atomicCAS(rep, 0, code);
    atomicMin(rep + 1, (int)(idx < INT_MAX ? idx : INT_MAX));
    atomicAdd(rep + 2, 1);
}

__global__ void k_validate(const int32_t* rowptr, const int32_t* colidx, int64_t M, int64_t N, int64_t nnz,
                           int32_t* rep)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > M) return;
    const int64_t a = rowptr[r];
    if (r == 0 && a != 0) report(rep, 1, 0);
    if (a < 0 || a > nnz) { report(rep, 5, r); return; }
    if (r == M) {
        if (a != nnz) report(rep, 3, M);
        return;
    }
    const int64_t b = rowptr[r + 1];
    if (b < a) { report(rep, 2, r); return; }
    if (b > nnz) return;   // reported by thread r+1
    int prev = -1;
    bool unsorted = false;
    for (int64_t e = a; e < b; ++e) {
        const int c = colidx[e];
        if (c < 0 || c >= N) report(rep, 4, e);
        if (c <= prev) unsorted = true;
        prev = c;
    }
    if (unsorted) atomicOr(rep + 3, 1);
}

cudaError_t launch_validate(const int32_t* rowptr, const int32_t* colidx, int64_t M, int64_t N, int64_t nnz,
                            int32_t* rep, cudaStream_t s)
{
    k_validate_init<<<1, 1, 0, s>>>(rep);
    k_validate<<<(unsigned)((M + 1 + 255) / 256), 256, 0, s>>>(rowptr, colidx, M, N, nnz, rep);
    return cudaGetLastError();
}

}  // namespace spk
