// COO -> CSR on the device.  The paper states S by its nonzeros s_ij, i.e. by
// coordinates (Sec. 3.1); the kernels stream CSR, so a caller holding
// coordinates converts once per pattern (the pattern is fixed while values
// change, Sec. 5.1).
//
// Order: (row, column), ties in input order: a stable LSD radix sort on the
// column carrying the input slot, a gather of each slot's row, and a stable
// radix sort on the row carrying the slot.  Repeated (row, column) entries are
// kept (dedup 0), reduced to the first in input order (1), or to one entry
// holding the FP32 sum of their values in input order (2).  Row pointers come
// from a lower-bound search per row on the output rows.
#include "common.cuh"

namespace spk {

namespace {

struct CooLayout {
    size_t k0, k1, v0, v1, hist, scan, keys2, rs, perm, flag, pos, rout, report, total;
};

CooLayout coo_layout(int64_t M, int64_t N, int64_t nnz)
{
    CooLayout L;
    const size_t a = align256((size_t)nnz * 4 + 4);
    const int64_t nh = radix_tiles(nnz) * 256;
    size_t o = 0;
    L.k0 = o; o += a;
    L.k1 = o; o += a;
    L.v0 = o; o += a;
    L.v1 = o; o += a;
    L.hist = o; o += radix_hist_bytes(nnz);
    const size_t scan = scan_temp_bytes(nh) > scan_temp_bytes(nnz + 1) ? scan_temp_bytes(nh) : scan_temp_bytes(nnz + 1);
    L.scan = o; o += align256(scan);
    L.keys2 = o; o += a;
    L.rs = o; o += a;
    L.perm = o; o += a;
    L.flag = o; o += a;
    L.pos = o; o += a;
    L.rout = o; o += a;
    L.report = o; o += 256;        // {first bad index, output count}
    L.total = o;
    (void)M; (void)N;
    return L;
}

// report[0] = smallest input slot with a coordinate out of range (INT32_MAX if none).
__global__ void k_coo_check(const int32_t* __restrict__ rows, const int32_t* __restrict__ cols, int64_t nnz,
                            int64_t M, int64_t N, int32_t* report)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = rows[e], c = cols[e];
        if (r < 0 || r >= M || c < 0 || c >= N) atomicMin(report, (int32_t)e);
    }
}

// keys2[i] = rows[p1[i]] (p1 NULL: the identity).
__global__ void k_coo_rows_of_slots(const int32_t* __restrict__ rows, const int32_t* __restrict__ p1, int64_t n,
                                    int32_t* __restrict__ keys2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        keys2[i] = rows[p1 ? p1[i] : i];
}

// Sorted columns (and, for dedup, the first-of-run flags).
__global__ void k_coo_gather(const int32_t* __restrict__ rs, const int32_t* __restrict__ cols,
                             const int32_t* __restrict__ p, int64_t n, int32_t* __restrict__ cs,
                             int32_t* __restrict__ flag)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cols[p ? p[i] : i];
        cs[i] = c;
        if (flag) {
            int32_t f = 1;
            if (i > 0) f = (rs[i] != rs[i - 1]) || (c != cols[p ? p[i - 1] : i - 1]);
            flag[i] = f;
        }
    }
}

// Outputs: dedup 0 copies every sorted entry; otherwise the first of each run
// of equal (row, column) writes its slot pos[i], with the first value (1) or
// the run's values summed in input order (2).  report[1] = output count.
__global__ void k_coo_emit(const int32_t* __restrict__ rs, const int32_t* __restrict__ cs,
                           const int32_t* __restrict__ p, const float* __restrict__ vals,
                           const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, int64_t n, int dedup,
                           int32_t* __restrict__ rout, int32_t* __restrict__ colidx, float* __restrict__ vals_out,
                           int32_t* report)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = p ? p[i] : i;
        if (dedup == 0) {
            rout[i] = rs[i];
            colidx[i] = cs[i];
            if (vals_out) vals_out[i] = vals ? vals[slot] : 1.f;
            if (i == n - 1) report[1] = (int32_t)n;
            continue;
        }
        if (!flag[i]) continue;
        const int32_t o = pos[i];
        rout[o] = rs[i];
        colidx[o] = cs[i];
        if (vals_out) {
            float v = vals ? vals[slot] : 1.f;
            if (dedup == 2 && vals)
                for (int64_t q = i + 1; q < n && !flag[q]; ++q) v += vals[p ? p[q] : q];
            vals_out[o] = v;
        }
    }
    if (dedup != 0 && blockIdx.x == 0 && threadIdx.x == 0 && n > 0) report[1] = pos[n - 1] + flag[n - 1];
}

// rowptr[r] = number of output entries with row < r, r = 0..M (the output
// count is read on the device).
__global__ void k_coo_rowptr(const int32_t* __restrict__ rout, const int32_t* __restrict__ report, int64_t M,
                             int32_t* __restrict__ rowptr)
{
    const int64_t n = report[1];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= M; r += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (rout[mid] < r) lo = mid + 1; else hi = mid;
        }
        rowptr[r] = (int32_t)lo;
    }
}

unsigned grid_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

}  // namespace

size_t coo_temp_bytes(int64_t M, int64_t N, int64_t nnz) { return coo_layout(M, N, nnz).total; }

cudaError_t coo_to_csr(int64_t M, int64_t N, int64_t nnz, const int32_t* rows, const int32_t* cols, const float* vals,
                       int dedup, int32_t* rowptr, int32_t* colidx, float* vals_out, int64_t* nnz_out,
                       int32_t* first_bad, char* temp, cudaStream_t s)
{
    const CooLayout L = coo_layout(M, N, nnz);
    auto at = [&](size_t off) { return reinterpret_cast<int32_t*>(temp + off); };
    int32_t* report = at(L.report);
    const int32_t init[2] = {INT32_MAX, 0};
    cudaError_t e = cudaMemcpyAsync(report, init, sizeof init, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if (nnz > 0) {
        k_coo_check<<<grid_for(nnz), 256, 0, s>>>(rows, cols, nnz, M, N, report);
        // 1. stable sort by column, carrying the input slot
        const int32_t *kc = nullptr, *p1 = nullptr;
        e = radix_sort_i32(cols, nullptr, nnz, radix_passes(N), at(L.k0), at(L.k1), at(L.v0), at(L.v1),
                           at(L.hist), temp + L.scan, &kc, &p1, s);
        if (e != cudaSuccess) return e;
        // 2. the row of each slot in that order, then a stable sort by row
        //    (its buffers must not be the ones holding p1)
        k_coo_rows_of_slots<<<grid_for(nnz), 256, 0, s>>>(rows, p1, nnz, at(L.keys2));
        const int32_t *rs = nullptr, *p = nullptr;
        int32_t* k0 = at(L.k0); int32_t* k1 = at(L.k1);
        int32_t* v0 = at(L.v0); int32_t* v1 = at(L.v1);
        if (p1 == v0) { v0 = at(L.flag); k0 = at(L.pos); }          // keep p1 intact while it is read
        else if (p1 == v1) { v1 = at(L.flag); k1 = at(L.pos); }
        e = radix_sort_i32(at(L.keys2), p1, nnz, radix_passes(M), k0, k1, v0, v1, at(L.hist), temp + L.scan, &rs, &p,
                           s);
        if (e != cudaSuccess) return e;
        // copy the final permutation and rows out of the sort buffers that
        // the flags / positions may reuse
        int32_t* p_fix = at(L.perm);
        int32_t* rs_fix = at(L.rs);
        if (p) {
            e = cudaMemcpyAsync(p_fix, p, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
            p = p_fix;
        }
        e = cudaMemcpyAsync(rs_fix, rs, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        rs = rs_fix;
        int32_t* cs = at(L.k0);
        int32_t* flag = dedup ? at(L.flag) : nullptr;
        k_coo_gather<<<grid_for(nnz), 256, 0, s>>>(rs, cols, p, nnz, cs, flag);
        int32_t* pos = at(L.pos);
        if (dedup) {
            e = scan_exclusive_i32(flag, pos, nnz, temp + L.scan, s);
            if (e != cudaSuccess) return e;
        }
        k_coo_emit<<<grid_for(nnz), 256, 0, s>>>(rs, cs, p, vals, flag, pos, nnz, dedup, at(L.rout), colidx,
                                                  vals_out, report);
    }
    k_coo_rowptr<<<grid_for(M + 1), 256, 0, s>>>(at(L.rout), report, M, rowptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int32_t host[2];
    e = cudaMemcpyAsync(host, report, sizeof host, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *first_bad = host[0] == INT32_MAX ? -1 : host[0];
    *nnz_out = host[1];
    return cudaSuccess;
}

}  // namespace spk
