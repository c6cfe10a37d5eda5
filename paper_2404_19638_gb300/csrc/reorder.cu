// Row relabelling for locality.  The paper localises indices before its
// Compute phase (Sec. 5.2: each processor renumbers the rows and columns it
// holds and drops the empty ones); on one GPU the counterpart is a relabelling
// of S's rows that brings rows touching the same B rows close together, so
// that a CTA's gathers share L2 lines.  The relabelled pattern keeps the
// original column ids (B is read as it is) and records, for every entry, its
// slot in the original pattern.
//
// Orders (perm[p] = original row placed at position p; ties keep the original
// order): by degree (most entries first), by leading column (smallest column
// first, rows without entries last) — both stable device radix sorts of a
// per-row key — and reverse Cuthill-McKee on the symmetric graph of a square
// pattern (Cuthill & McKee 1969, reversed after George 1971), run on the host.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace spk {

namespace {

unsigned grid_of(int64_t n, int per = 256)
{
    int64_t b = (n + per - 1) / per;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

// key[i] = INT32_MAX - degree (degree order) or the smallest column of the row
// (N for an empty row: leading-column order).
__global__ void k_row_keys(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int64_t M,
                           int64_t N, int kind, int32_t* __restrict__ key)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e0 = rowptr[i], e1 = rowptr[i + 1];
        if (kind == 1) {
            key[i] = INT32_MAX - (e1 - e0);
        } else {
            int32_t m = (int32_t)N;
            for (int32_t e = e0; e < e1; ++e) m = min(m, colidx[e]);
            key[i] = m;
        }
    }
}

// deg2[p] = degree of row perm[p].
__global__ void k_perm_degrees(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ perm, int64_t M,
                               int32_t* __restrict__ deg2)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = perm[p];
        deg2[p] = rowptr[r + 1] - rowptr[r];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) deg2[M] = 0;      // the scan's last input: rowptr2[M] = the sum
}

// One warp per relabelled row: its entries, in their original order, and
// the original slot of each.
__global__ void k_perm_copy(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                            const int32_t* __restrict__ perm, const int32_t* __restrict__ rowptr2, int64_t M,
                            int32_t* __restrict__ colidx2, int32_t* __restrict__ emap)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; p < M; p += nw) {
        const int32_t r = perm[p];
        const int32_t e0 = rowptr[r], n = rowptr[r + 1] - e0, o = rowptr2[p];
        for (int32_t q = lane; q < n; q += 32) {
            colidx2[o + q] = colidx[e0 + q];
            emap[o + q] = e0 + q;
        }
    }
}

// Y[p] = X[perm[p]] (gather) or Y[perm[p]] = X[p] (scatter), rows of `bytes`
// bytes; 16-byte pieces when every row start is 16-byte aligned, else bytes.
template <bool VEC>
__global__ void k_permute_rows(const char* __restrict__ X, int64_t ldx_b, int64_t M, int64_t bytes,
                               const int32_t* __restrict__ perm, int scatter, char* __restrict__ Y, int64_t ldy_b)
{
    const int64_t per = VEC ? bytes / 16 : bytes;
    const int64_t total = M * per;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / per, q = t - p * per;
        const int64_t r = perm[p];
        const int64_t src = scatter ? p : r, dst = scatter ? r : p;
        if (VEC)
            reinterpret_cast<uint4*>(Y + dst * ldy_b)[q] = __ldg(reinterpret_cast<const uint4*>(X + src * ldx_b) + q);
        else
            Y[dst * ldy_b + q] = X[src * ldx_b + q];
    }
}

// y[i] = x[map[i]] (gather) or y[map[i]] = x[i] (scatter).
__global__ void k_permute_values(const float* __restrict__ x, const int32_t* __restrict__ map, int64_t n, int scatter,
                                 float* __restrict__ y)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (scatter) y[map[i]] = x[i];
        else y[i] = x[map[i]];
    }
}

struct ReorderLayout {
    size_t key, k1, v0, v1, hist, scan, total;
};

ReorderLayout reorder_layout(int64_t M)
{
    ReorderLayout L;
    const size_t a = align256((size_t)M * 4 + 4);
    size_t o = 0;
    L.key = o; o += a;
    L.k1 = o; o += a;
    L.v0 = o; o += a;
    L.v1 = o; o += a;
    L.hist = o; o += radix_hist_bytes(M);
    const size_t sc = std::max(scan_temp_bytes(radix_tiles(M) * 256), scan_temp_bytes(M + 1));
    L.scan = o; o += align256(sc);
    L.total = o;
    return L;
}

// Reverse Cuthill-McKee on the host (the order is a one-time plan).
int rcm_host(int64_t M, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci, std::vector<int32_t>& perm)
{
    std::vector<int64_t> deg(M, 0), start(M + 1, 0), fill(M, 0);
    for (int64_t i = 0; i < M; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int64_t j = ci[e];
            if (j < 0 || j >= M) return 2;
            if (j != i) { deg[i]++; deg[j]++; }
        }
    for (int64_t i = 0; i < M; ++i) start[i + 1] = start[i] + deg[i];
    std::vector<int32_t> adj((size_t)start[M]);
    for (int64_t i = 0; i < M; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int64_t j = ci[e];
            if (j == i) continue;
            adj[start[i] + fill[i]++] = (int32_t)j;
            adj[start[j] + fill[j]++] = (int32_t)i;
        }
    auto less = [&](int32_t x, int32_t y) { return deg[x] != deg[y] ? deg[x] < deg[y] : x < y; };
    std::vector<int32_t> byd(M);
    for (int64_t i = 0; i < M; ++i) byd[i] = (int32_t)i;
    std::sort(byd.begin(), byd.end(), less);
    std::vector<char> seen(M, 0);
    std::vector<int32_t> order;
    order.reserve(M);
    int64_t head = 0, next = 0;
    while ((int64_t)order.size() < M) {
        while (seen[byd[next]]) ++next;
        seen[byd[next]] = 1;
        order.push_back(byd[next]);
        while (head < (int64_t)order.size()) {
            const int32_t v = order[head++];
            const size_t first = order.size();
            for (int64_t q = start[v]; q < start[v + 1]; ++q) {
                const int32_t w = adj[q];
                if (!seen[w]) { seen[w] = 1; order.push_back(w); }
            }
            std::sort(order.begin() + first, order.end(), less);
        }
    }
    perm.assign(order.rbegin(), order.rend());
    return 0;
}

}  // namespace

size_t reorder_temp_bytes(int64_t M) { return reorder_layout(M).total; }

cudaError_t row_order(const int32_t* rowptr, const int32_t* colidx, int64_t M, int64_t N, int64_t nnz, int kind,
                      int32_t* perm, char* temp, int* host_status, cudaStream_t s)
{
    *host_status = 0;
    if (M == 0) return cudaSuccess;
    if (kind == 3) {
        std::vector<int32_t> rp(M + 1), ci(nnz), pm;
        cudaError_t e = cudaMemcpyAsync(rp.data(), rowptr, (size_t)(M + 1) * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(ci.data(), colidx, (size_t)nnz * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        *host_status = rcm_host(M, rp, ci, pm);
        if (*host_status) return cudaSuccess;
        e = cudaMemcpyAsync(perm, pm.data(), (size_t)M * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);     // pm is freed on return
        return e;
    }
    const ReorderLayout L = reorder_layout(M);
    auto at = [&](size_t off) { return reinterpret_cast<int32_t*>(temp + off); };
    k_row_keys<<<grid_of(M), 256, 0, s>>>(rowptr, colidx, M, N, kind, at(L.key));
    const int passes = kind == 1 ? 4 : radix_passes(N + 1);
    const int32_t *ks = nullptr, *vs = nullptr;
    // key ping-pong: the pass outputs go to k1, then back over the keys
    cudaError_t e = radix_sort_i32(at(L.key), nullptr, M, passes, at(L.k1), at(L.key), at(L.v0), at(L.v1), at(L.hist),
                                   temp + L.scan, &ks, &vs, s);
    if (e != cudaSuccess) return e;
    (void)ks;
    // vs: the sorted identity, i.e. the order (NULL only if no pass ran, which M >= 1 excludes)
    return cudaMemcpyAsync(perm, vs, (size_t)M * 4, cudaMemcpyDeviceToDevice, s);
}

cudaError_t permute_pattern(const int32_t* rowptr, const int32_t* colidx, int64_t M, const int32_t* perm,
                            int32_t* rowptr2, int32_t* colidx2, int32_t* emap, char* temp, cudaStream_t s)
{
    const ReorderLayout L = reorder_layout(M);
    int32_t* deg2 = reinterpret_cast<int32_t*>(temp + L.key);
    if (M > 0) k_perm_degrees<<<grid_of(M), 256, 0, s>>>(rowptr, perm, M, deg2);   // M == 0: below
    if (M == 0) return cudaMemsetAsync(rowptr2, 0, 4, s);
    cudaError_t e = scan_exclusive_i32(deg2, rowptr2, M + 1, temp + L.scan, s);
    if (e != cudaSuccess) return e;
    if (M > 0) k_perm_copy<<<grid_of(M * 32), 256, 0, s>>>(rowptr, colidx, perm, rowptr2, M, colidx2, emap);
    return cudaGetLastError();
}

cudaError_t permute_rows(const void* X, int64_t ldx_b, int64_t M, int64_t bytes, const int32_t* perm, int scatter,
                         void* Y, int64_t ldy_b, cudaStream_t s)
{
    if (M == 0 || bytes == 0) return cudaSuccess;
    const bool vec = ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15u) == 0 &&
                     ldx_b % 16 == 0 && ldy_b % 16 == 0 && bytes % 16 == 0;
    const int64_t total = vec ? M * (bytes / 16) : M * bytes;
    if (vec)
        k_permute_rows<true><<<grid_of(total), 256, 0, s>>>(reinterpret_cast<const char*>(X), ldx_b, M, bytes, perm,
                                                             scatter, reinterpret_cast<char*>(Y), ldy_b);
    else
        k_permute_rows<false><<<grid_of(total), 256, 0, s>>>(reinterpret_cast<const char*>(X), ldx_b, M, bytes, perm,
                                                              scatter, reinterpret_cast<char*>(Y), ldy_b);
    return cudaGetLastError();
}

cudaError_t permute_values(const float* x, const int32_t* map, int64_t n, int scatter, float* y, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_permute_values<<<grid_of(n), 256, 0, s>>>(x, map, n, scatter, y);
    return cudaGetLastError();
}

}  // namespace spk
