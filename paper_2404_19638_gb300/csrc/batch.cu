// Batched persistent launch: many independent SDDMM / SpMM problems of uneven
// size in ONE kernel, each warp staging its gathers through a shared-memory
// ring (ring.cuh).  Each item is cut into work units (one warp's worth of
// balanced-schedule chunks, times the K blocks of an SpMM); a persistent grid
// of one wave of CTAs pulls units off a device counter.  No warp ever waits on
// another: split SpMM rows are finished by their last-arriving piece (see
// spmm_impl.cuh), and the last warp to leave resets the counters, so the run
// can be captured in a CUDA graph and replayed.
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sddmm_impl.cuh"
#include "spmm_impl.cuh"

namespace spk {

struct BatchDesc {
    int32_t op;      // 0 SDDMM, 1 SpMM
    int32_t cls;     // (dtype, shape) class of the device routine
    int32_t nkb;     // K blocks (SpMM)
    int32_t gpw;     // lane groups per warp = 32 / G
    SddmmArgs sd;
    SpmmArgs sp;
};

// (G, NV, U) shapes available to batched items, per op; class = dtype * 8 +
// position in the op's list.  Each (op, class) routine is a separate
// non-inlined function, so the merged kernel needs no more registers than its
// largest routine.
#define SPK_BATCH_SDDMM_SHAPES(X) \
    X(0, 4, 1, 4)                 \
    X(1, 8, 1, 4)                 \
    X(2, 16, 1, 4)
#define SPK_BATCH_SPMM_SHAPES(X) \
    X(0, 4, 1, 4)                \
    X(1, 8, 1, 4)                \
    X(2, 16, 1, 4)               \
    X(3, 4, 1, 8)                \
    X(4, 8, 1, 8)                \
    X(5, 16, 1, 8)

constexpr int kBatchSddmmShapes = 3;
constexpr int kBatchSpmmShapes = 6;
static const Shape kBatchSddmmList[kBatchSddmmShapes] = {
#define X(i, G_, NV_, U_) {G_, NV_, U_},
    SPK_BATCH_SDDMM_SHAPES(X)
#undef X
};
static const Shape kBatchSpmmList[kBatchSpmmShapes] = {
#define X(i, G_, NV_, U_) {G_, NV_, U_},
    SPK_BATCH_SPMM_SHAPES(X)
#undef X
};

constexpr int kBatchThreads = 128;

// Shared-memory ring of one warp for one (op, shape); a batch gives every warp
// the largest ring among its items' shapes.
static int batch_ring_bytes(int op, const Shape& sh)
{
    const int b = op == 0 ? sddmm_ring_bytes(sh.G, sh.NV, sh.U, 2) : spmm_ring_bytes(sh.NV, sh.U);
    return (b + 127) / 128 * 128;
}

// SDDMM: one chunk per warp (groups take interleaved batches of it), gathered
// rows through the warp's ring (ring.cuh).
template <int DT, int G, int NV, int U>
__device__ __noinline__ void batch_sddmm_unit(const SddmmArgs& a, int64_t unit, unsigned char* wsm)
{
    if (unit >= a.nchunks) return;
    const int2 b0 = a.bnd[unit], b1 = a.bnd[unit + 1];
    if (a.K / vec_elems(DT) >= G * NV) sddmm_ring_span<DT, G, NV, U, 2, true>(a, threadIdx.x & 31, wsm, b0.y, b1.y);
    else sddmm_ring_span<DT, G, NV, U, 2, false>(a, threadIdx.x & 31, wsm, b0.y, b1.y);
}

// SpMM: one chunk per lane group, 32/G consecutive chunks per unit.
template <int DT, int G, int NV, int U>
__device__ __noinline__ void batch_spmm_unit(const SpmmArgs& a, int64_t unit, int nkb, unsigned char* wsm)
{
    const Group<G> g;
    const int kb = (int)(unit % nkb);
    const int64_t c = (unit / nkb) * (32 / G) + ((threadIdx.x & 31) / G);
    if (c >= a.nchunks) return;
    const int2 b0 = a.bnd[c], b1 = a.bnd[c + 1];
    const int4 m = a.meta[c];
    if (b1.y == b0.y && m.z < b0.x) return;
    const int hs0 = (m.x >= 0) ? __ldg(a.head_s0 + c) : -1;
    uint4* wring = reinterpret_cast<uint4*>(wsm);
    if (a.K / vec_elems(DT) >= (kb + 1) * G * NV)
        spmm_ring_span<DT, G, NV, U, true>(a, g, wring, kb, nkb, b0.x, b0.y, b1.x, b1.y, m, hs0);
    else
        spmm_ring_span<DT, G, NV, U, false>(a, g, wring, kb, nkb, b0.x, b0.y, b1.x, b1.y, m, hs0);
}

// MINB: CTAs per SM the register budget is cut for (6: 80 registers; 5: 96
// registers, for batches with 8-nonzero SpMM batches or BF16 operands, whose
// routines would spill at 80).
template <int MINB>
__global__ void __launch_bounds__(kBatchThreads, MINB) k_batch(const BatchDesc* __restrict__ descs, int32_t count,
                                                  const int64_t* __restrict__ unit_begin, int64_t total_units,
                                                  unsigned long long* counter, unsigned int* done, int32_t ring_bytes)
{
    extern __shared__ __align__(16) unsigned char batch_smem[];
    unsigned char* wsm = batch_smem + (threadIdx.x >> 5) * ring_bytes;
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(counter, 1ull);
        u = __shfl_sync(0xffffffffu, u, 0);
        if ((int64_t)u >= total_units) break;
        int lo = 0, hi = count - 1;                  // last item with unit_begin <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(unit_begin + mid) <= (int64_t)u) lo = mid; else hi = mid - 1;
        }
        const BatchDesc& d = descs[lo];
        const int64_t local = (int64_t)u - __ldg(unit_begin + lo);
        const int cls = d.cls;
        if (d.op == 0) {
            switch (cls) {
#define X(i, G_, NV_, U_)                                                           \
    case i: batch_sddmm_unit<DT_F32, G_, NV_, U_>(d.sd, local, wsm); break;         \
    case 8 + i: batch_sddmm_unit<DT_BF16, G_, NV_, U_>(d.sd, local, wsm); break;
                SPK_BATCH_SDDMM_SHAPES(X)
#undef X
            }
        } else {
            switch (cls) {
#define X(i, G_, NV_, U_)                                                           \
    case i: batch_spmm_unit<DT_F32, G_, NV_, U_>(d.sp, local, d.nkb, wsm); break;   \
    case 8 + i: batch_spmm_unit<DT_BF16, G_, NV_, U_>(d.sp, local, d.nkb, wsm); break;
                SPK_BATCH_SPMM_SHAPES(X)
#undef X
            }
        }
        __syncwarp();
    }
    // Leave: the last warp of the grid resets the counters for the next run.
    if (lane == 0) {
        __threadfence();
        const unsigned total_warps = gridDim.x * (blockDim.x / 32);
        const unsigned old = atomicAdd(done, 1u);
        if (old == total_warps - 1) {
            atomicExch(counter, 0ull);
            atomicExch(done, 0u);
        }
    }
}

}  // namespace spk

using namespace spk;

struct spk_batch_s {
    int32_t count;
    int64_t total_units;
    int32_t grid;
    int32_t ring_bytes;              // per warp: the largest ring among the items' shapes
    bool wide;                       // the 96-register kernel build (see plan_batch)
    bool wide_default;               // the build plan_batch chose
    const BatchDesc* d_descs;
    const int64_t* d_unit_begin;
    unsigned long long* d_counter;
    unsigned int* d_done;
};

// The library-wide last-error slot lives in api.cu.
extern "C" void spk_internal_set_error(const char* msg);

static spk_status bfail(spk_status s, const std::string& msg)
{
    spk_internal_set_error(msg.c_str());
    return s;
}

struct BatchPlan {
    std::vector<BatchDesc> descs;
    std::vector<int64_t> unit_begin;
    size_t off_descs, off_units, off_counter, off_done, off_carry, total;
    std::vector<size_t> carry_off;   // per item (SpMM), relative to off_carry
    int ring_bytes = 0;              // per warp
    bool wide = false;               // some item batches 8 nonzeros or has BF16 operands
};

static spk_status plan_batch(const spk_batch_item* items, int32_t count, BatchPlan& P)
{
    if (!items || count <= 0) return bfail(SPK_ERR_ARG, "spk_batch: items is NULL or count <= 0");
    P.descs.assign(count, BatchDesc());
    P.unit_begin.assign((size_t)count + 1, 0);
    P.carry_off.assign(count, 0);
    size_t carry = 0;
    int64_t units = 0;
    for (int32_t m = 0; m < count; ++m) {
        const spk_batch_item& it = items[m];
        const std::string where = "spk_batch item " + std::to_string(m) + ": ";
        if (it.op != 0 && it.op != 1) return bfail(SPK_ERR_ARG, where + "op must be 0 (SDDMM) or 1 (SpMM)");
        if (!it.S) return bfail(SPK_ERR_ARG, where + "S is NULL");
        const spk_csr_s* S = it.S;
        if (S->vperm) return bfail(SPK_ERR_ARG, where + "transposed patterns are not batched");
        if (!S->has_sched) return bfail(SPK_ERR_STATE, where + "pattern needs spk_schedule_build first");
        if (it.dt != SPK_F32 && it.dt != SPK_BF16) return bfail(SPK_ERR_DTYPE, where + "dtype must be F32 or BF16");
        if (it.K < 1) return bfail(SPK_ERR_SHAPE, where + "K must be >= 1");
        const int vecn = vec_elems(it.dt);
        if (it.K % vecn) return bfail(SPK_ERR_UNSUPPORTED, where + "K must be a multiple of 16 bytes of elements");
        if (it.ldb < it.K || (it.ldb * dt_bytes(it.dt)) % 16 || (reinterpret_cast<uintptr_t>(it.B) & 15))
            return bfail(SPK_ERR_SHAPE, where + "B must be 16-byte aligned with ldb >= K");
        // row addresses are formed with 32-bit byte strides
        const int64_t max_ld = (int64_t)0xFFFFFFFFu / dt_bytes(it.dt);
        if (it.ldb > max_ld || (it.op == 0 && it.lda > max_ld))
            return bfail(SPK_ERR_SHAPE, where + "row strides must be below 4 GiB");
        if (S->nnz > 0 && !it.B) return bfail(SPK_ERR_ARG, where + "B is NULL");
        if (!it.out && (it.op == 1 ? S->M > 0 : S->nnz > 0)) return bfail(SPK_ERR_ARG, where + "out is NULL");
        if (it.op == 0) {
            if (it.lda < it.K || (it.lda * dt_bytes(it.dt)) % 16 || (reinterpret_cast<uintptr_t>(it.A) & 15))
                return bfail(SPK_ERR_SHAPE, where + "A must be 16-byte aligned with lda >= K");
            if (S->nnz > 0 && !it.A) return bfail(SPK_ERR_ARG, where + "A is NULL");
        } else {
            if (it.ldc < it.K || (it.ldc * 4) % 16 || (reinterpret_cast<uintptr_t>(it.out) & 15))
                return bfail(SPK_ERR_SHAPE, where + "C must be 16-byte aligned FP32 with ldc >= K");
            for (int32_t q = 0; q < m; ++q)
                if (items[q].op == 1 && items[q].S == it.S)
                    return bfail(SPK_ERR_ARG, where + "two SpMM items share one pattern handle");
        }
        // shape
        const int nvec = it.K / vecn;
        // Batched shapes: one K block of at most 16 vectors of 16 bytes
        // (K <= 64 in FP32, <= 128 in BF16).
        if (nvec > 16) return bfail(SPK_ERR_UNSUPPORTED, where + "batched K is limited to 16 vectors of 16 bytes");
        int G, NV = 1, U = 4;
        if (nvec <= 4) G = 4;
        else if (nvec <= 8) G = 8;
        else G = 16;
        if (it.tune) {
            if (it.tune->group_lanes) G = it.tune->group_lanes;
            if (it.tune->vecs_per_lane) NV = it.tune->vecs_per_lane;
            if (it.tune->unroll) U = it.tune->unroll;
        }
        const Shape* list = it.op == 0 ? kBatchSddmmList : kBatchSpmmList;
        const int nlist = it.op == 0 ? kBatchSddmmShapes : kBatchSpmmShapes;
        int sidx = -1;
        for (int q = 0; q < nlist; ++q)
            if (list[q].G == G && list[q].NV == NV && list[q].U == U) sidx = q;
        if (sidx < 0 || G * NV < nvec)
            return bfail(SPK_ERR_UNSUPPORTED, where + "shape not available in batched mode");
        const int rb = batch_ring_bytes(it.op, list[sidx]);
        if (rb > P.ring_bytes) P.ring_bytes = rb;
        if (list[sidx].U > 4 || it.dt == SPK_BF16) P.wide = true;
        BatchDesc& d = P.descs[m];
        d.op = it.op;
        d.cls = (it.dt == SPK_BF16 ? 8 : 0) + sidx;
        d.gpw = 32 / G;
        d.nkb = 1;
        const int64_t wunits = (S->nchunks + d.gpw - 1) / d.gpw;
        if (it.op == 0) {
            SddmmArgs& a = d.sd;
            a.M = S->M; a.N = S->N; a.nnz = S->nnz; a.K = it.K;
            a.rowptr = S->rowptr; a.colidx = S->colidx; a.rowidx = S->rowidx;
            a.vals = it.vals; a.vals2 = nullptr;
            a.A = it.A; a.lda = it.lda; a.a_scale = nullptr;
            a.B = it.B; a.ldb = it.ldb; a.b_scale = nullptr;
            a.out = reinterpret_cast<float*>(it.out);
            a.bnd = S->bnd; a.nchunks = S->nchunks;
            P.unit_begin[m + 1] = units + (S->nnz > 0 ? S->nchunks : 0);     // one chunk per warp
        } else {
            d.nkb = (nvec + G * NV - 1) / (G * NV);
            SpmmArgs& a = d.sp;
            a.M = S->M; a.N = S->N; a.nnz = S->nnz; a.K = it.K;
            a.rowptr = S->rowptr; a.colidx = S->colidx; a.rowidx = S->rowidx; a.vperm = nullptr;
            a.vals = it.vals; a.vals2 = nullptr;
            a.vals_staged = (it.vals && (reinterpret_cast<uintptr_t>(it.vals) & 15u) == 0) ? 1 : 0;
            a.B = it.B; a.ldb = it.ldb; a.b_scale = nullptr;
            a.C = it.out; a.ldc = it.ldc; a.dtc = SPK_F32; a.accumulate = 0;
            a.bnd = S->bnd; a.meta = S->meta; a.head_s0 = S->head_s0; a.slot_np = S->slot_np; a.cnt = S->cnt;
            a.carry = nullptr;   // set at create time
            a.nchunks = S->nchunks;
            P.carry_off[m] = carry;
            carry += align256((size_t)S->npieces * it.K * 4);
            P.unit_begin[m + 1] = units + (S->M > 0 ? wunits * d.nkb : 0);
        }
        units = P.unit_begin[m + 1];
    }
    size_t off = 0;
    P.off_descs = off;   off += align256(sizeof(BatchDesc) * (size_t)count);
    P.off_units = off;   off += align256(sizeof(int64_t) * ((size_t)count + 1));
    P.off_counter = off; off += 256;
    P.off_done = off;    off += 256;
    P.off_carry = off;   off += carry;
    P.total = off;
    return SPK_OK;
}

// One wave of CTAs of the chosen kernel build on the current device, with
// 4 warps x ring_bytes of shared memory per CTA.
static cudaError_t batch_grid(bool wide, int ring_bytes, int* grid)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = (size_t)(kBatchThreads / 32) * ring_bytes;
    const void* fn = wide ? (const void*)&k_batch<5> : (const void*)&k_batch<6>;
    if (e == cudaSuccess && smem > 48 * 1024)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchThreads, smem);
    *grid = sms * (per_sm > 0 ? per_sm : 1);
    return e;
}

extern "C" spk_status spk_batch_size(const spk_batch_item* items, int32_t count, size_t* bytes)
{
    if (!bytes) return bfail(SPK_ERR_ARG, "spk_batch_size: bytes is NULL");
    BatchPlan P;
    spk_status s = plan_batch(items, count, P);
    if (s != SPK_OK) return s;
    *bytes = P.total;
    return SPK_OK;
}

extern "C" spk_status spk_batch_create(const spk_batch_item* items, int32_t count, void* storage, size_t bytes,
                                       spk_batch* out, void* stream)
{
    if (!out) return bfail(SPK_ERR_ARG, "spk_batch_create: out is NULL");
    *out = nullptr;
    BatchPlan P;
    spk_status s = plan_batch(items, count, P);
    if (s != SPK_OK) return s;
    if (!storage || bytes < P.total) return bfail(SPK_ERR_WORKSPACE, "spk_batch_create: storage too small");
    if (reinterpret_cast<uintptr_t>(storage) & 255u)
        return bfail(SPK_ERR_WORKSPACE, "spk_batch_create: storage must be 256-byte aligned");
    char* st = reinterpret_cast<char*>(storage);
    for (int32_t m = 0; m < count; ++m)
        if (P.descs[m].op == 1) P.descs[m].sp.carry = reinterpret_cast<float*>(st + P.off_carry + P.carry_off[m]);
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(st + P.off_descs, P.descs.data(), sizeof(BatchDesc) * count,
                                    cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st + P.off_units, P.unit_begin.data(), sizeof(int64_t) * (count + 1),
                            cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(st + P.off_counter, 0, 512, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return bfail(SPK_ERR_CUDA, std::string("spk_batch_create: ") + cudaGetErrorString(e));
    int grid = 0;
    e = batch_grid(P.wide, P.ring_bytes, &grid);
    if (e != cudaSuccess) return bfail(SPK_ERR_CUDA, std::string("spk_batch_create: ") + cudaGetErrorString(e));
    spk_batch_s* B = new (std::nothrow) spk_batch_s();
    if (!B) return bfail(SPK_ERR_ARG, "spk_batch_create: out of host memory");
    B->count = count;
    B->total_units = P.unit_begin[count];
    B->grid = grid;
    B->ring_bytes = P.ring_bytes;
    B->wide = P.wide;
    B->wide_default = P.wide;
    B->d_descs = reinterpret_cast<const BatchDesc*>(st + P.off_descs);
    B->d_unit_begin = reinterpret_cast<const int64_t*>(st + P.off_units);
    B->d_counter = reinterpret_cast<unsigned long long*>(st + P.off_counter);
    B->d_done = reinterpret_cast<unsigned int*>(st + P.off_done);
    *out = B;
    return SPK_OK;
}

extern "C" spk_status spk_batch_run(spk_batch B, void* stream)
{
    if (!B) return bfail(SPK_ERR_ARG, "spk_batch_run: handle is NULL");
    if (B->total_units == 0) return SPK_OK;
    const size_t smem = (size_t)(kBatchThreads / 32) * B->ring_bytes;
    if (B->wide)
        k_batch<5><<<B->grid, kBatchThreads, smem, (cudaStream_t)stream>>>(B->d_descs, B->count, B->d_unit_begin,
                                                                          B->total_units, B->d_counter, B->d_done,
                                                                          B->ring_bytes);
    else
        k_batch<6><<<B->grid, kBatchThreads, smem, (cudaStream_t)stream>>>(B->d_descs, B->count, B->d_unit_begin,
                                                                          B->total_units, B->d_counter, B->d_done,
                                                                          B->ring_bytes);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(SPK_ERR_CUDA, std::string("spk_batch_run: ") + cudaGetErrorString(e));
    return SPK_OK;
}

extern "C" int32_t spk_batch_shapes(int32_t op, int32_t* out, int32_t capacity)
{
    if (op != 0 && op != 1) return 0;
    const Shape* list = op == 0 ? kBatchSddmmList : kBatchSpmmList;
    const int n = op == 0 ? kBatchSddmmShapes : kBatchSpmmShapes;
    for (int i = 0; out && i < n && i < capacity; ++i) {
        out[3 * i] = list[i].G;
        out[3 * i + 1] = list[i].NV;
        out[3 * i + 2] = list[i].U;
    }
    return n;
}

extern "C" spk_status spk_batch_set_registers(spk_batch B, int32_t regs)
{
    if (!B) return bfail(SPK_ERR_ARG, "spk_batch_set_registers: handle is NULL");
    if (regs != 0 && regs != 80 && regs != 96)
        return bfail(SPK_ERR_ARG, "spk_batch_set_registers: regs must be 0, 80 or 96");
    const bool wide = regs == 0 ? B->wide_default : regs == 96;
    int grid = 0;
    cudaError_t e = batch_grid(wide, B->ring_bytes, &grid);
    if (e != cudaSuccess) return bfail(SPK_ERR_CUDA, std::string("spk_batch_set_registers: ") + cudaGetErrorString(e));
    B->wide = wide;
    B->grid = grid;
    return SPK_OK;
}

extern "C" spk_status spk_batch_info(spk_batch B, int64_t* work_units, int32_t* ctas)
{
    if (!B) return bfail(SPK_ERR_ARG, "spk_batch_info: handle is NULL");
    if (work_units) *work_units = B->total_units;
    if (ctas) *ctas = B->grid;
    return SPK_OK;
}

extern "C" spk_status spk_batch_destroy(spk_batch B)
{
    delete B;
    return SPK_OK;
}
