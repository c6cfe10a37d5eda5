// Host side of the C ABI declared in include/spk.h: argument checks (all
// before any CUDA call), handles, kernel-shape selection and dispatch.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "common.cuh"
#include "fused.cuh"
#include "heads.cuh"

namespace spk {

cudaError_t launch_merge_path_bounds(const int32_t* rowptr, int64_t M, int64_t nnz, int32_t W, int64_t n,
                                     int2* out, cudaStream_t s);

static const Shape kShapes[kNumShapes] = {
#define X(i, G_, NV_, U_) {G_, NV_, U_},
    SPK_SHAPES(X)
#undef X
};

int shape_index(int G, int NV, int U)
{
    for (int i = 0; i < kNumShapes; ++i)
        if (kShapes[i].G == G && kShapes[i].NV == NV && kShapes[i].U == U) return i;
    return -1;
}

Shape shape_at(int i) { return kShapes[i]; }

cudaError_t launch_sddmm(int dta, int dtb, const Launch& L, const SddmmArgs& a, cudaStream_t s)
{
    switch (dtb) {
    case DT_F32: return launch_sddmm_f32(dta, L, a, s);
    case DT_BF16: return launch_sddmm_bf16(dta, L, a, s);
    case DT_F16: return launch_sddmm_f16(dta, L, a, s);
    case DT_E4M3: return launch_sddmm_e4m3(dta, L, a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_spmm(int dtb, const Launch& L, const SpmmArgs& a, cudaStream_t s)
{
    switch (dtb) {
    case DT_F32: return launch_spmm_f32(L, a, s);
    case DT_BF16: return launch_spmm_bf16(L, a, s);
    case DT_F16: return launch_spmm_f16(L, a, s);
    case DT_E4M3: return launch_spmm_e4m3(L, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace spk

using namespace spk;

// ----------------------------------------------------------------------------
// Errors
// ----------------------------------------------------------------------------
static thread_local std::string g_err;

static spk_status fail(spk_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

static spk_status cuda_fail(cudaError_t e, const char* where)
{
    return fail(SPK_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define REQUIRE(cond, status, ...) \
    do {                           \
        if (!(cond)) return fail(status, __VA_ARGS__); \
    } while (0)

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
// The gather kernels form a row's address as row x (row stride in bytes) with
// the stride held in 32 bits: a row stride must stay below 4 GiB.
static bool stride32(int64_t ld, int dt) { return ld <= (int64_t)0xFFFFFFFFu / dt_bytes(dt); }
static bool valid_dt(int dt) { return dt >= SPK_F32 && dt <= SPK_E4M3; }

extern "C" const char* spk_status_string(spk_status s)
{
    switch (s) {
    case SPK_OK: return "ok";
    case SPK_ERR_ARG: return "invalid argument";
    case SPK_ERR_SHAPE: return "invalid shape";
    case SPK_ERR_INDEX: return "malformed sparse pattern";
    case SPK_ERR_DTYPE: return "unsupported dtype";
    case SPK_ERR_WORKSPACE: return "workspace too small or misaligned";
    case SPK_ERR_CUDA: return "CUDA error";
    case SPK_ERR_TIMEOUT: return "device wait timed out";
    case SPK_ERR_UNSUPPORTED: return "unsupported size";
    case SPK_ERR_STATE: return "handle not ready";
    }
    return "unknown status";
}

extern "C" const char* spk_last_error(void) { return g_err.c_str(); }
// Not in the public header: lets other translation units set the message.
extern "C" void spk_internal_set_error(const char* msg) { g_err = msg ? msg : ""; }
extern "C" int32_t spk_version(void) { return 10000; }

// ----------------------------------------------------------------------------
// Pattern handles
// ----------------------------------------------------------------------------
extern "C" spk_status spk_csr_create(spk_csr* out, int64_t M, int64_t N, int64_t nnz, const int32_t* rowptr,
                                     const int32_t* colidx)
{
    REQUIRE(out, SPK_ERR_ARG, "spk_csr_create: out is NULL");
    *out = nullptr;
    REQUIRE(M >= 0 && N >= 0 && nnz >= 0, SPK_ERR_ARG, "spk_csr_create: negative size (M=%lld N=%lld nnz=%lld)",
            (long long)M, (long long)N, (long long)nnz);
    REQUIRE(M < INT32_MAX && N < INT32_MAX && nnz < INT32_MAX, SPK_ERR_UNSUPPORTED,
            "spk_csr_create: sizes must be below 2^31-1 (int32 indices)");
    REQUIRE(rowptr, SPK_ERR_ARG, "spk_csr_create: rowptr is NULL");
    REQUIRE(colidx || nnz == 0, SPK_ERR_ARG, "spk_csr_create: colidx is NULL");
    REQUIRE(nnz == 0 || N > 0, SPK_ERR_SHAPE, "spk_csr_create: nonzeros in a matrix with no columns");
    REQUIRE(nnz == 0 || aligned16(colidx), SPK_ERR_ARG, "spk_csr_create: colidx must be 16-byte aligned");
    spk_csr_s* S = new (std::nothrow) spk_csr_s();
    REQUIRE(S, SPK_ERR_ARG, "spk_csr_create: out of host memory");
    S->M = M; S->N = N; S->nnz = nnz;
    S->rowptr = rowptr; S->colidx = colidx;
    *out = S;
    return SPK_OK;
}

extern "C" spk_status spk_csr_destroy(spk_csr S)
{
    delete S;
    return SPK_OK;
}

extern "C" spk_status spk_csr_validate(spk_csr S, int32_t* d_report, void* stream)
{
    REQUIRE(S, SPK_ERR_ARG, "spk_csr_validate: S is NULL");
    REQUIRE(d_report, SPK_ERR_ARG, "spk_csr_validate: report is NULL");
    cudaError_t e = launch_validate(S->rowptr, S->colidx, S->M, S->N, S->nnz, d_report, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_csr_validate");
    return SPK_OK;
}

// ----------------------------------------------------------------------------
// Schedule
// ----------------------------------------------------------------------------
static int32_t chunk_work_or_default(int32_t W) { return W == 0 ? 512 : W; }

extern "C" spk_status spk_schedule_size(spk_csr S, int32_t chunk_work, size_t* bytes)
{
    REQUIRE(S && bytes, SPK_ERR_ARG, "spk_schedule_size: NULL argument");
    const int32_t W = chunk_work_or_default(chunk_work);
    REQUIRE(W >= 32 && W <= (1 << 20), SPK_ERR_ARG, "spk_schedule_size: chunk_work %d outside [32, 2^20]", W);
    *bytes = sched_layout(S->M, S->nnz, W).total;
    return SPK_OK;
}

static spk_status attach_schedule(spk_csr_s* S, int32_t W, void* storage, size_t bytes, cudaStream_t s)
{
    const SchedLayout L = sched_layout(S->M, S->nnz, W);
    REQUIRE(storage, SPK_ERR_WORKSPACE, "schedule storage is NULL");
    REQUIRE(bytes >= L.total, SPK_ERR_WORKSPACE, "schedule storage has %zu bytes, needs %zu", bytes, L.total);
    REQUIRE((reinterpret_cast<uintptr_t>(storage) & 255u) == 0, SPK_ERR_WORKSPACE,
            "schedule storage must be 256-byte aligned");
    char* st = reinterpret_cast<char*>(storage);
    int64_t np = 0;
    S->has_sched = false;
    cudaError_t e = build_schedule(S->rowptr, S->M, S->nnz, W, st, L, &np, s);
    if (e != cudaSuccess) return cuda_fail(e, "schedule build");
    S->has_sched = true;
    S->W = W;
    S->nchunks = L.nchunks;
    S->npieces = np;
    S->rowidx = reinterpret_cast<const int32_t*>(st + L.rowidx);
    S->bnd = reinterpret_cast<const int2*>(st + L.bnd);
    S->meta = reinterpret_cast<const int4*>(st + L.meta);
    S->head_s0 = reinterpret_cast<const int32_t*>(st + L.head_s0);
    S->slot_np = reinterpret_cast<const int32_t*>(st + L.slot_np);
    S->cnt = reinterpret_cast<int32_t*>(st + L.cnt);
    return SPK_OK;
}

extern "C" spk_status spk_schedule_build(spk_csr S, int32_t chunk_work, void* storage, size_t bytes, void* stream)
{
    REQUIRE(S, SPK_ERR_ARG, "spk_schedule_build: S is NULL");
    const int32_t W = chunk_work_or_default(chunk_work);
    REQUIRE(W >= 32 && W <= (1 << 20), SPK_ERR_ARG, "spk_schedule_build: chunk_work %d outside [32, 2^20]", W);
    return attach_schedule(S, W, storage, bytes, (cudaStream_t)stream);
}

extern "C" spk_status spk_schedule_info(spk_csr S, int64_t* nchunks, int64_t* npieces, int32_t* chunk_work)
{
    REQUIRE(S, SPK_ERR_ARG, "spk_schedule_info: S is NULL");
    REQUIRE(S->has_sched, SPK_ERR_STATE, "spk_schedule_info: no schedule attached");
    if (nchunks) *nchunks = S->nchunks;
    if (npieces) *npieces = S->npieces;
    if (chunk_work) *chunk_work = S->W;
    return SPK_OK;
}

extern "C" spk_status spk_schedule_bounds(spk_csr S, int32_t* d_out, void* stream)
{
    REQUIRE(S && d_out, SPK_ERR_ARG, "spk_schedule_bounds: NULL argument");
    REQUIRE(S->has_sched, SPK_ERR_STATE, "spk_schedule_bounds: no schedule attached");
    cudaError_t e = cudaMemcpyAsync(d_out, S->bnd, (size_t)(S->nchunks + 1) * 8, cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_schedule_bounds");
    return SPK_OK;
}

// Raw merge-path split points (row, nonzero) at diagonals 0, W, 2W, ... (n+1
// of them): not part of the public header; used by tests to check the search.
extern "C" spk_status spk_merge_path_points(spk_csr S, int32_t W, int64_t n, int32_t* d_out, void* stream)
{
    REQUIRE(S && d_out && W > 0 && n >= 0, SPK_ERR_ARG, "spk_merge_path_points: bad argument");
    cudaError_t e = launch_merge_path_bounds(S->rowptr, S->M, S->nnz, W, n, reinterpret_cast<int2*>(d_out),
                                             (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_merge_path_points");
    return SPK_OK;
}

// ----------------------------------------------------------------------------
// COO -> CSR
// ----------------------------------------------------------------------------
extern "C" spk_status spk_coo_to_csr_size(int64_t M, int64_t N, int64_t nnz, size_t* temp_bytes)
{
    REQUIRE(temp_bytes, SPK_ERR_ARG, "spk_coo_to_csr_size: temp_bytes is NULL");
    REQUIRE(M >= 0 && N >= 0 && nnz >= 0, SPK_ERR_ARG, "spk_coo_to_csr_size: negative size");
    REQUIRE(M < INT32_MAX && N < INT32_MAX && nnz < INT32_MAX, SPK_ERR_UNSUPPORTED,
            "spk_coo_to_csr_size: sizes must be below 2^31-1 (int32 indices)");
    *temp_bytes = coo_temp_bytes(M, N, nnz);
    return SPK_OK;
}

extern "C" spk_status spk_coo_to_csr(int64_t M, int64_t N, int64_t nnz, const int32_t* rows, const int32_t* cols,
                                     const float* vals, int32_t dedup, int32_t* rowptr, int32_t* colidx,
                                     float* vals_out, int64_t* nnz_out, void* temp, size_t temp_bytes, void* stream)
{
    REQUIRE(nnz_out, SPK_ERR_ARG, "spk_coo_to_csr: nnz_out is NULL");
    *nnz_out = 0;
    REQUIRE(M >= 0 && N >= 0 && nnz >= 0, SPK_ERR_ARG, "spk_coo_to_csr: negative size");
    REQUIRE(M < INT32_MAX && N < INT32_MAX && nnz < INT32_MAX, SPK_ERR_UNSUPPORTED,
            "spk_coo_to_csr: sizes must be below 2^31-1 (int32 indices)");
    REQUIRE(dedup >= 0 && dedup <= 2, SPK_ERR_ARG, "spk_coo_to_csr: dedup must be 0, 1 or 2");
    REQUIRE(rowptr, SPK_ERR_ARG, "spk_coo_to_csr: rowptr is NULL");
    REQUIRE(nnz == 0 || (rows && cols && colidx), SPK_ERR_ARG, "spk_coo_to_csr: NULL coordinate array");
    REQUIRE(nnz == 0 || N > 0, SPK_ERR_SHAPE, "spk_coo_to_csr: entries in a matrix with no columns");
    const size_t need = coo_temp_bytes(M, N, nnz);
    REQUIRE(temp && temp_bytes >= need, SPK_ERR_WORKSPACE, "spk_coo_to_csr: temp has %zu bytes, needs %zu",
            temp ? temp_bytes : (size_t)0, need);
    REQUIRE((reinterpret_cast<uintptr_t>(temp) & 255u) == 0, SPK_ERR_WORKSPACE,
            "spk_coo_to_csr: temp must be 256-byte aligned");
    int32_t bad = -1;
    int64_t n = 0;
    cudaError_t e = coo_to_csr(M, N, nnz, rows, cols, vals, dedup, rowptr, colidx, vals_out, &n, &bad,
                               reinterpret_cast<char*>(temp), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_coo_to_csr");
    REQUIRE(bad < 0, SPK_ERR_INDEX, "spk_coo_to_csr: entry %d has a coordinate outside the %lld x %lld matrix", bad,
            (long long)M, (long long)N);
    *nnz_out = n;
    return SPK_OK;
}

// ----------------------------------------------------------------------------
// Row relabelling for locality
// ----------------------------------------------------------------------------
extern "C" spk_status spk_reorder_size(spk_csr S, size_t* temp_bytes)
{
    REQUIRE(S && temp_bytes, SPK_ERR_ARG, "spk_reorder_size: NULL argument");
    *temp_bytes = reorder_temp_bytes(S->M);
    return SPK_OK;
}

extern "C" spk_status spk_reorder_rows(spk_csr S, int32_t order, int32_t* perm, void* temp, size_t temp_bytes,
                                       void* stream)
{
    REQUIRE(S, SPK_ERR_ARG, "spk_reorder_rows: S is NULL");
    REQUIRE(order >= SPK_ORDER_DEGREE && order <= SPK_ORDER_RCM, SPK_ERR_ARG,
            "spk_reorder_rows: order must be SPK_ORDER_DEGREE, SPK_ORDER_LEADING_COLUMN or SPK_ORDER_RCM");
    REQUIRE(order != SPK_ORDER_RCM || S->M == S->N, SPK_ERR_SHAPE,
            "spk_reorder_rows: reverse Cuthill-McKee needs a square pattern (got %lld x %lld)", (long long)S->M,
            (long long)S->N);
    REQUIRE(S->M == 0 || perm, SPK_ERR_ARG, "spk_reorder_rows: perm is NULL");
    const size_t need = reorder_temp_bytes(S->M);
    REQUIRE(order == SPK_ORDER_RCM || (temp && temp_bytes >= need), SPK_ERR_WORKSPACE,
            "spk_reorder_rows: temp has %zu bytes, needs %zu", temp ? temp_bytes : (size_t)0, need);
    REQUIRE(order == SPK_ORDER_RCM || (reinterpret_cast<uintptr_t>(temp) & 255u) == 0, SPK_ERR_WORKSPACE,
            "spk_reorder_rows: temp must be 256-byte aligned");
    int hs = 0;
    cudaError_t e = row_order(S->rowptr, S->colidx, S->M, S->N, S->nnz, order, perm, reinterpret_cast<char*>(temp),
                              &hs, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_reorder_rows");
    REQUIRE(hs == 0, SPK_ERR_INDEX, "spk_reorder_rows: a column index is outside the square pattern");
    return SPK_OK;
}

extern "C" spk_status spk_permute_pattern(spk_csr S, const int32_t* perm, int32_t* rowptr_out, int32_t* colidx_out,
                                          int32_t* emap, void* temp, size_t temp_bytes, void* stream)
{
    REQUIRE(S, SPK_ERR_ARG, "spk_permute_pattern: S is NULL");
    REQUIRE(rowptr_out && (S->M == 0 || perm) && (S->nnz == 0 || (colidx_out && emap)), SPK_ERR_ARG,
            "spk_permute_pattern: NULL array");
    const size_t need = reorder_temp_bytes(S->M);
    REQUIRE(temp && temp_bytes >= need, SPK_ERR_WORKSPACE, "spk_permute_pattern: temp has %zu bytes, needs %zu",
            temp ? temp_bytes : (size_t)0, need);
    REQUIRE((reinterpret_cast<uintptr_t>(temp) & 255u) == 0, SPK_ERR_WORKSPACE,
            "spk_permute_pattern: temp must be 256-byte aligned");
    cudaError_t e = permute_pattern(S->rowptr, S->colidx, S->M, perm, rowptr_out, colidx_out, emap,
                                    reinterpret_cast<char*>(temp), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_permute_pattern");
    return SPK_OK;
}

extern "C" spk_status spk_permute_rows(const void* X, int64_t ldx, spk_dtype dt, int64_t M, int32_t K,
                                       const int32_t* perm, int32_t scatter, void* Y, int64_t ldy, void* stream)
{
    REQUIRE(valid_dt(dt), SPK_ERR_DTYPE, "spk_permute_rows: unknown dtype");
    REQUIRE(M >= 0 && K >= 0 && ldx >= K && ldy >= K, SPK_ERR_SHAPE, "spk_permute_rows: bad shape");
    REQUIRE(scatter == 0 || scatter == 1, SPK_ERR_ARG, "spk_permute_rows: scatter must be 0 or 1");
    REQUIRE(M == 0 || K == 0 || (X && Y && perm), SPK_ERR_ARG, "spk_permute_rows: NULL array");
    REQUIRE(X != Y || M == 0 || K == 0, SPK_ERR_ARG, "spk_permute_rows: X and Y must not be the same buffer");
    const int64_t b = dt_bytes(dt);
    cudaError_t e = permute_rows(X, ldx * b, M, (int64_t)K * b, perm, scatter, Y, ldy * b, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_permute_rows");
    return SPK_OK;
}

extern "C" spk_status spk_permute_values(const float* x, const int32_t* map, int64_t n, int32_t scatter, float* y,
                                         void* stream)
{
    REQUIRE(n >= 0 && (scatter == 0 || scatter == 1), SPK_ERR_ARG, "spk_permute_values: bad argument");
    REQUIRE(n == 0 || (x && map && y && x != y), SPK_ERR_ARG, "spk_permute_values: NULL or aliased array");
    cudaError_t e = permute_values(x, map, n, scatter, y, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_permute_values");
    return SPK_OK;
}

// ----------------------------------------------------------------------------
// Kernel shape selection
// ----------------------------------------------------------------------------
enum { OP_SDDMM = 0, OP_SPMM = 1, OP_SPMM_T = 2 };

// Default lane-group shape for a row of nvec 16-byte vectors, from shape
// sweeps on GB300 with the L2 flushed before each launch (R-MAT scale 20 and
// 22 with K = 64, the K = 128 Chung-Lu pattern of 50M nonzeros):
//   SDDMM: 4 lanes x 2 vectors at 8 vectors a row, 8 lanes x 2 vectors at 16,
//          8 lanes x 4 vectors at 32, 4 nonzeros in flight;
//   SpMM (and S^T Y): one vector a lane on 16 lanes with 8 nonzeros in
//          flight at 16 vectors; 16 lanes x 2 vectors x 8 at 32 (rec FP32
//          1.90 ms against 2.24 for 8 x 4 x 4).  16-bit rows of 8 vectors
//          spread over 16 lanes as 8-byte vectors (8 nonzeros in flight) when
//          rows are long (rmat20, 15 nonzeros a row: 0.412 ms), else 8 lanes
//          of 16-byte vectors with 4 in flight (R-MAT scale 22, 8 a row:
//          0.803 ms against 0.867); 16-bit rows of 16 vectors take 8 lanes x
//          2 vectors x 4 (rec BF16 1.26 ms against 1.58 for 32 lanes of
//          8-byte vectors).
static void default_shape(int op, int nvec, int* G, int* NV, int* U, bool half16 = false, bool short_rows = false)
{
    *U = 4;
    if (op != OP_SDDMM && half16) {
        if (nvec <= 4) { *G = 8; *NV = 1; return; }                 // 8-byte vectors over 8 lanes
        if (nvec <= 8) {
            if (short_rows) { *G = 8; *NV = 1; return; }              // 16-byte vectors
            *G = 16; *NV = 1; *U = 8; return;                        // 8-byte vectors
        }
        if (nvec <= 16) { *G = 8; *NV = 2; return; }                 // 16-byte vectors
    }
    if (nvec <= 4) { *G = 4; *NV = 1; }
    else if (nvec <= 8) { *G = (op == OP_SDDMM) ? 4 : 8; *NV = (op == OP_SDDMM) ? 2 : 1; }
    else if (nvec <= 16) {
        *G = (op == OP_SDDMM) ? 8 : 16;
        *NV = (op == OP_SDDMM) ? 2 : 1;
        *U = (op == OP_SDDMM) ? 4 : 8;
    }
    else if (nvec <= 32) {
        *G = (op == OP_SDDMM) ? 8 : 16;
        *NV = (op == OP_SDDMM) ? 4 : 2;
        *U = (op == OP_SDDMM) ? 4 : 8;
    }
    else if (nvec <= 64) { *G = 32; *NV = 2; }
    else { *G = 32; *NV = 4; }
}

static spk_status resolve(const spk_csr_s* S, int op, int dtb, int K, bool vec, const spk_tune* t, Launch* L)
{
    const int variant = (t && t->variant) ? t->variant : (S->has_sched ? 2 : 1);
    REQUIRE(variant >= 1 && variant <= 3, SPK_ERR_ARG, "tune.variant %d is not 0, 1, 2 or 3", variant);
    REQUIRE(variant == 1 || S->has_sched, SPK_ERR_STATE, "balanced variant needs spk_schedule_build first");
    const int vecn = vec ? vec_elems(dtb) : 1;
    const int nvec = K / vecn;
    int G, NV, U;
    const bool half16 = vec && (variant == 2) && (dtb == SPK_BF16 || dtb == SPK_F16) && K % 4 == 0;
    const bool short_rows = S->M > 0 && S->nnz < 12 * S->M;            // fewer than 12 nonzeros a row
    default_shape(op, nvec, &G, &NV, &U, half16, short_rows);
    if (t && t->group_lanes) G = t->group_lanes;
    if (t && t->vecs_per_lane) NV = t->vecs_per_lane;
    if (t && t->unroll) U = t->unroll;
    const int idx = shape_index(G, NV, U);
    REQUIRE(idx >= 0, SPK_ERR_UNSUPPORTED, "no kernel compiled for group_lanes=%d vecs_per_lane=%d unroll=%d",
            G, NV, U);
    const int threads = (t && t->cta_threads) ? t->cta_threads : 128;
    REQUIRE(threads == 128 || threads == 256, SPK_ERR_ARG, "tune.cta_threads must be 128 or 256");
    L->shape = idx;
    L->vec = vec;
    L->threads = threads;
    L->chunks = (variant >= 2);
    L->ring = (variant == 2);
    const int stages = (t && t->stages) ? t->stages : 2;
    REQUIRE(stages == 2 || stages == 4, SPK_ERR_ARG, "tune.stages must be 2 or 4");
    L->stages = stages;
    return SPK_OK;
}

extern "C" int32_t spk_shapes(int32_t* out, int32_t capacity)
{
    if (out)
        for (int i = 0; i < kNumShapes && i < capacity; ++i) {
            const Shape sh = shape_at(i);
            out[3 * i] = sh.G;
            out[3 * i + 1] = sh.NV;
            out[3 * i + 2] = sh.U;
        }
    return kNumShapes;
}

extern "C" spk_status spk_tune_default(spk_csr S, int32_t op, spk_dtype dt, int32_t K, spk_tune* out)
{
    REQUIRE(S && out, SPK_ERR_ARG, "spk_tune_default: NULL argument");
    REQUIRE(op >= 0 && op <= 2 && valid_dt(dt) && K >= 1, SPK_ERR_ARG, "spk_tune_default: bad op/dtype/K");
    const bool vec = (K % vec_elems(dt)) == 0;
    Launch L;
    const spk_csr_s* P = S;
    spk_status st = resolve(P, op, dt, K, vec, nullptr, &L);
    if (st != SPK_OK) return st;
    const Shape sh = shape_at(L.shape);
    out->variant = L.chunks ? (L.ring ? 2 : 3) : 1;
    out->group_lanes = sh.G;
    out->vecs_per_lane = sh.NV;
    out->unroll = sh.U;
    out->cta_threads = L.threads;
    out->stages = L.stages;
    return SPK_OK;
}

// ----------------------------------------------------------------------------
// SDDMM
// ----------------------------------------------------------------------------
extern "C" spk_status spk_sddmm(spk_csr S, const float* vals, const float* vals2, spk_dtype dta, const void* A,
                                int64_t lda, const float* a_scale, spk_dtype dtb, const void* B, int64_t ldb,
                                const float* b_scale, int32_t K, float* out, const spk_tune* tune, void* stream)
{
    REQUIRE(S, SPK_ERR_ARG, "spk_sddmm: S is NULL");
    REQUIRE(valid_dt(dta) && valid_dt(dtb), SPK_ERR_DTYPE, "spk_sddmm: unknown dtype");
    REQUIRE(dta == dtb || (dta == SPK_F32 && (dtb == SPK_BF16 || dtb == SPK_F16)), SPK_ERR_DTYPE,
            "spk_sddmm: dtype pair (%d, %d) not supported", (int)dta, (int)dtb);
    REQUIRE(K >= 1, SPK_ERR_SHAPE, "spk_sddmm: K must be >= 1 (got %d)", K);
    REQUIRE(lda >= K && ldb >= K, SPK_ERR_SHAPE, "spk_sddmm: leading dimensions must be >= K");
    REQUIRE(stride32(lda, dta) && stride32(ldb, dtb), SPK_ERR_SHAPE, "spk_sddmm: row strides must be below 4 GiB");
    REQUIRE(S->nnz == 0 || (A && B && out), SPK_ERR_ARG, "spk_sddmm: NULL operand");
    REQUIRE(dta != SPK_E4M3 || (a_scale && b_scale), SPK_ERR_ARG, "spk_sddmm: E4M3 needs a_scale and b_scale");
    REQUIRE(!S->vperm, SPK_ERR_ARG, "spk_sddmm: pattern belongs to a transpose plan");
    if (S->nnz == 0) return SPK_OK;
    const int vecn = vec_elems(dtb);
    const bool vec = (K % vecn) == 0 && aligned16(A) && aligned16(B) && (lda * dt_bytes(dta)) % 16 == 0 &&
                     (ldb * dt_bytes(dtb)) % 16 == 0;
    Launch L;
    spk_status st = resolve(S, OP_SDDMM, dtb, K, vec, tune, &L);
    if (st != SPK_OK) return st;
    SddmmArgs a;
    a.M = S->M; a.N = S->N; a.nnz = S->nnz; a.K = K;
    a.rowptr = S->rowptr; a.colidx = S->colidx; a.rowidx = S->rowidx;
    a.vals = vals; a.vals2 = vals2;
    a.A = A; a.lda = lda; a.a_scale = a_scale;
    a.B = B; a.ldb = ldb; a.b_scale = b_scale;
    a.out = out;
    a.bnd = L.chunks ? S->bnd : nullptr;
    a.nchunks = S->nchunks;
    cudaError_t e = launch_sddmm(dta, dtb, L, a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_sddmm launch");
    return SPK_OK;
}

// Several heads (equal slices of K): out[h * nnz + e] = s_e * <A[i, head h], B[j, head h]>.
extern "C" spk_status spk_sddmm_mh(spk_csr S, const float* vals, int32_t heads, spk_dtype dt, const void* A,
                                   int64_t lda, const void* B, int64_t ldb, int32_t K, float* out, void* stream)
{
    REQUIRE(S, SPK_ERR_ARG, "spk_sddmm_mh: S is NULL");
    REQUIRE(dt == SPK_F32 || dt == SPK_BF16, SPK_ERR_DTYPE, "spk_sddmm_mh: dtype must be F32 or BF16");
    REQUIRE(K >= 1 && heads >= 1 && K % heads == 0, SPK_ERR_SHAPE,
            "spk_sddmm_mh: K (%d) must be a positive multiple of heads (%d)", K, heads);
    REQUIRE(lda >= K && ldb >= K, SPK_ERR_SHAPE, "spk_sddmm_mh: leading dimensions must be >= K");
    REQUIRE(stride32(lda, dt) && stride32(ldb, dt), SPK_ERR_SHAPE, "spk_sddmm_mh: row strides must be below 4 GiB");
    REQUIRE(S->nnz == 0 || (A && B && out), SPK_ERR_ARG, "spk_sddmm_mh: NULL operand");
    REQUIRE(!S->vperm, SPK_ERR_ARG, "spk_sddmm_mh: pattern belongs to a transpose plan");
    REQUIRE(S->has_sched, SPK_ERR_STATE, "spk_sddmm_mh: needs spk_schedule_build first");
    const int vecn = vec_elems(dt);
    REQUIRE(aligned16(A) && aligned16(B) && (lda * dt_bytes(dt)) % 16 == 0 && (ldb * dt_bytes(dt)) % 16 == 0 &&
                (!vals || aligned16(vals)),
            SPK_ERR_SHAPE, "spk_sddmm_mh: A, B (and vals) must be 16-byte aligned with 16-byte row strides");
    REQUIRE((K / heads) % vecn == 0, SPK_ERR_UNSUPPORTED,
            "spk_sddmm_mh: a head of %d elements is not a whole number of 16-byte vectors", K / heads);
    const int nv = K / vecn, nh = nv / heads;
    int G, NV, U;
    default_shape(OP_SDDMM, nv, &G, &NV, &U);
    REQUIRE(heads > 1 || nv == G * NV, SPK_ERR_UNSUPPORTED, "spk_sddmm_mh: K = %d has no whole lane block", K);
    REQUIRE(heads == 1 || (nv == G * NV && sddmm_mh_supported(dt, G, NV, U, nh)), SPK_ERR_UNSUPPORTED,
            "spk_sddmm_mh: no kernel for K = %d in %d heads (rows of %d vectors over %d lanes x %d)", K, heads, nv, G,
            NV);
    if (S->nnz == 0) return SPK_OK;
    if (heads == 1)
        return spk_sddmm(S, vals, nullptr, dt, A, lda, nullptr, dt, B, ldb, nullptr, K, out, nullptr, stream);
    SddmmArgs a;
    a.M = S->M; a.N = S->N; a.nnz = S->nnz; a.K = K;
    a.rowptr = S->rowptr; a.colidx = S->colidx; a.rowidx = S->rowidx;
    a.vals = vals; a.vals2 = nullptr;
    a.A = A; a.lda = lda; a.a_scale = nullptr;
    a.B = B; a.ldb = ldb; a.b_scale = nullptr;
    a.out = out;
    a.bnd = S->bnd;
    a.nchunks = S->nchunks;
    cudaError_t e = launch_sddmm_mh(dt, G, NV, U, nh, a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_sddmm_mh launch");
    return SPK_OK;
}

// ----------------------------------------------------------------------------
// SpMM / SpMM^T
// ----------------------------------------------------------------------------
extern "C" spk_status spk_spmm_workspace_size(spk_csr S, int32_t K, size_t* bytes)
{
    REQUIRE(S && bytes && K >= 1, SPK_ERR_ARG, "spk_spmm_workspace_size: bad argument");
    *bytes = S->has_sched ? (size_t)S->npieces * (size_t)K * 4 : 0;
    return SPK_OK;
}

static spk_status spmm_common(const char* name, const spk_csr_s* S, const float* vals, const float* vals2,
                              spk_dtype dtb, const void* B, int64_t ldb, const float* b_scale, int32_t K,
                              spk_dtype dtc, void* C, int64_t ldc, int32_t accumulate, void* ws, size_t ws_bytes,
                              const spk_tune* tune, cudaStream_t stream, bool vals_in_slot_order = false,
                              bool check_only = false, int32_t heads = 1, int64_t hstride = 0)
{
    REQUIRE(valid_dt(dtb), SPK_ERR_DTYPE, "%s: unknown input dtype", name);
    REQUIRE(dtc == SPK_F32 || dtc == SPK_BF16 || dtc == SPK_F16, SPK_ERR_DTYPE,
            "%s: output dtype must be F32, BF16 or F16", name);
    REQUIRE(K >= 1, SPK_ERR_SHAPE, "%s: K must be >= 1 (got %d)", name, K);
    REQUIRE(ldb >= K && ldc >= K, SPK_ERR_SHAPE, "%s: leading dimensions must be >= K", name);
    REQUIRE(stride32(ldb, dtb), SPK_ERR_SHAPE, "%s: the row stride of the dense input must be below 4 GiB", name);
    REQUIRE(accumulate == 0 || accumulate == 1, SPK_ERR_ARG, "%s: accumulate must be 0 or 1", name);
    REQUIRE(S->M == 0 || C, SPK_ERR_ARG, "%s: output is NULL", name);
    REQUIRE(S->nnz == 0 || B, SPK_ERR_ARG, "%s: dense input is NULL", name);
    REQUIRE(dtb != SPK_E4M3 || b_scale, SPK_ERR_ARG, "%s: E4M3 input needs row scales", name);
    if (S->M == 0) return SPK_OK;
    const int vecn = vec_elems(dtb);
    const bool vec = (K % vecn) == 0 && aligned16(B) && aligned16(C) && (ldb * dt_bytes(dtb)) % 16 == 0 &&
                     (ldc * dt_bytes(dtc)) % 16 == 0;
    Launch L;
    spk_status st;
    if (heads > 1) {
        // one head per lane: one 16-byte vector per lane (NV = 1), G lanes per K block
        REQUIRE(vec, SPK_ERR_UNSUPPORTED, "%s: several heads need 16-byte aligned rows and K a multiple of %d", name,
                vecn);
        const int nv = K / vecn;
        REQUIRE(nv % heads == 0, SPK_ERR_UNSUPPORTED, "%s: %d vectors per row do not split into %d heads", name, nv,
                heads);
        const int G = nv <= 4 ? 4 : (nv <= 8 ? 8 : (nv <= 16 ? 16 : 32));
        spk_tune t{};
        t.variant = S->has_sched ? 2 : 1;
        t.group_lanes = G;
        t.vecs_per_lane = 1;
        t.unroll = G == 4 ? 4 : 8;
        st = resolve(S, OP_SPMM, dtb, K, vec, &t, &L);
    } else {
        st = resolve(S, OP_SPMM, dtb, K, vec, tune, &L);
    }
    if (st != SPK_OK) return st;
    if (L.chunks && S->npieces > 0) {
        const size_t need = (size_t)S->npieces * (size_t)K * 4;
        REQUIRE(ws && ws_bytes >= need, SPK_ERR_WORKSPACE, "%s: workspace has %zu bytes, needs %zu", name,
                ws ? ws_bytes : (size_t)0, need);
        REQUIRE(aligned16(ws), SPK_ERR_WORKSPACE, "%s: workspace must be 16-byte aligned", name);
    }
    if (check_only) return SPK_OK;
    SpmmArgs a;
    a.M = S->M; a.N = S->N; a.nnz = S->nnz; a.K = K;
    a.rowptr = S->rowptr; a.colidx = S->colidx; a.rowidx = S->rowidx;
    a.vperm = vals_in_slot_order ? nullptr : S->vperm;
    a.vals = vals; a.vals2 = vals2;
    // staged values: through the index tiles (several heads: one pair of
    // tiles each; a head array off 16-byte alignment is staged 4 bytes at a time)
    a.vals_staged = (vals && !vals2 && !a.vperm && aligned16(vals)) ? 1 : 0;
    a.heads = heads;
    a.hstride = hstride;
    a.B = B; a.ldb = ldb; a.b_scale = b_scale;
    a.C = C; a.ldc = ldc; a.dtc = dtc; a.accumulate = accumulate;
    a.bnd = L.chunks ? S->bnd : nullptr;
    a.meta = S->meta; a.head_s0 = S->head_s0; a.slot_np = S->slot_np; a.cnt = S->cnt;
    a.carry = reinterpret_cast<float*>(ws);
    a.nchunks = S->nchunks;
    cudaError_t e = launch_spmm(dtb, L, a, stream);
    if (e != cudaSuccess) return cuda_fail(e, name);
    return SPK_OK;
}

extern "C" spk_status spk_spmm(spk_csr S, const float* vals, const float* vals2, spk_dtype dtb, const void* B,
                               int64_t ldb, const float* b_scale, int32_t K, spk_dtype dtc, void* C, int64_t ldc,
                               int32_t accumulate, void* workspace, size_t ws_bytes, const spk_tune* tune,
                               void* stream)
{
    REQUIRE(S, SPK_ERR_ARG, "spk_spmm: S is NULL");
    return spmm_common("spk_spmm", S, vals, vals2, dtb, B, ldb, b_scale, K, dtc, C, ldc, accumulate, workspace,
                       ws_bytes, tune, (cudaStream_t)stream);
}

// Several heads (equal slices of K), each with its own value array.
extern "C" spk_status spk_spmm_mh(spk_csr S, const float* vals, int64_t hstride, int32_t heads, spk_dtype dtb,
                                  const void* B, int64_t ldb, int32_t K, float* C, int64_t ldc, int32_t accumulate,
                                  void* workspace, size_t ws_bytes, void* stream)
{
    REQUIRE(S, SPK_ERR_ARG, "spk_spmm_mh: S is NULL");
    REQUIRE(!S->vperm, SPK_ERR_ARG, "spk_spmm_mh: pattern belongs to a transpose plan");
    REQUIRE(heads >= 1 && K >= 1 && K % heads == 0, SPK_ERR_SHAPE, "spk_spmm_mh: K (%d) must be a multiple of heads (%d)",
            K, heads);
    REQUIRE(dtb == SPK_F32 || dtb == SPK_BF16 || dtb == SPK_F16, SPK_ERR_DTYPE, "spk_spmm_mh: B must be F32, BF16 or F16");
    REQUIRE(heads == 1 || !vals || hstride >= S->nnz, SPK_ERR_ARG, "spk_spmm_mh: hstride below nnz");
    return spmm_common("spk_spmm_mh", S, vals, nullptr, dtb, B, ldb, nullptr, K, SPK_F32, C, ldc, accumulate, workspace,
                       ws_bytes, nullptr, (cudaStream_t)stream, false, false, heads, hstride);
}

// ----------------------------------------------------------------------------
// FusedMM (SDDMM cascaded into SpMM), per head, optional row softmax
// ----------------------------------------------------------------------------
extern "C" spk_status spk_fusedmm_workspace_size(spk_csr S, int32_t K, int32_t heads, size_t* bytes)
{
    REQUIRE(S && bytes && K >= 1 && heads >= 1, SPK_ERR_ARG, "spk_fusedmm_workspace_size: bad argument");
    *bytes = S->has_sched ? (size_t)S->npieces * (((size_t)K + 2 * (size_t)heads + 3) / 4 * 4) * 4 : 0;
    return SPK_OK;
}

extern "C" spk_status spk_fusedmm(spk_csr S, const float* vals, float scale, int32_t softmax, spk_dtype dt,
                                  const void* A, int64_t lda, const void* B, int64_t ldb, int32_t K, int32_t heads,
                                  float* Y, int64_t ldy, float* scores, float* lse, void* workspace, size_t ws_bytes,
                                  const spk_tune* tune, void* stream)
{
    REQUIRE(S, SPK_ERR_ARG, "spk_fusedmm: S is NULL");
    REQUIRE(!S->vperm, SPK_ERR_ARG, "spk_fusedmm: pattern belongs to a transpose plan");
    REQUIRE(S->has_sched, SPK_ERR_STATE, "spk_fusedmm: needs spk_schedule_build first");
    REQUIRE(dt == SPK_F32 || dt == SPK_BF16 || dt == SPK_F16, SPK_ERR_DTYPE, "spk_fusedmm: dtype must be F32, BF16 or F16");
    REQUIRE(K >= 1 && heads >= 1 && K % heads == 0, SPK_ERR_SHAPE, "spk_fusedmm: K (%d) must be a multiple of heads (%d)",
            K, heads);
    REQUIRE(softmax == 0 || softmax == 1, SPK_ERR_ARG, "spk_fusedmm: softmax must be 0 or 1");
    const int vecn = vec_elems(dt);
    const int dh = K / heads;
    REQUIRE(dh % vecn == 0, SPK_ERR_UNSUPPORTED, "spk_fusedmm: head width %d is not a multiple of %d elements", dh,
            vecn);
    REQUIRE(lda >= K && ldb >= K && ldy >= K, SPK_ERR_SHAPE, "spk_fusedmm: leading dimensions must be >= K");
    REQUIRE(stride32(lda, dt) && stride32(ldb, dt), SPK_ERR_SHAPE, "spk_fusedmm: row strides must be below 4 GiB");
    REQUIRE(S->nnz == 0 || (A && B), SPK_ERR_ARG, "spk_fusedmm: NULL operand");
    REQUIRE(S->M == 0 || Y, SPK_ERR_ARG, "spk_fusedmm: Y is NULL");
    REQUIRE(aligned16(A) && aligned16(B) && aligned16(Y) && (lda * dt_bytes(dt)) % 16 == 0 &&
                (ldb * dt_bytes(dt)) % 16 == 0 && ldy % 4 == 0,
            SPK_ERR_SHAPE, "spk_fusedmm: A, B, Y must be 16-byte aligned with 16-byte row strides");
    REQUIRE(!vals || aligned16(vals), SPK_ERR_ARG, "spk_fusedmm: vals must be 16-byte aligned");
    const int nvh = dh / vecn;
    const int nv = K / vecn;
    // Kernel choice.  The all-heads kernel (one lane group per row, heads as
    // blocks of G / heads lanes, NV adjacent vectors a lane) when a row is at
    // most 32 vectors and the heads split the lanes evenly; else, or when a
    // shape is asked for, the one-head-per-grid-row kernel.  Measured on
    // rmat20, K = 64, GB300: one head runs best on the one-head kernel (FP32
    // 8 lanes x 2 vectors 0.85 ms, 16-bit 8 lanes 0.86 ms, against 1.16 / 1.24
    // on the all-heads kernel); 16-bit rows with 4 or more heads on the
    // all-heads kernel with 2 vectors a lane (1.21 ms against 1.32).
    // tune.vecs_per_lane alone (no group_lanes, no unroll) asks for the
    // all-heads kernel with that many vectors a lane (1 or 2).
    const bool mh_asked = tune && tune->vecs_per_lane && !tune->group_lanes && !tune->unroll;
    const bool shaped = tune && (tune->group_lanes || tune->unroll || (tune->vecs_per_lane && !mh_asked));
    const bool one_head = heads == 1 && ((dt == SPK_F32 && nvh == 16) || (dt != SPK_F32 && nvh == 8));
    auto mh_fits = [&](int nvl) {
        const int g = nv / nvl;
        return nv % nvl == 0 && (g == 4 || g == 8 || g == 16 || (g == 32 && nvl == 1)) && g % heads == 0;
    };
    int mh_nv = 1;
    if (mh_asked) {
        mh_nv = tune->vecs_per_lane;
        REQUIRE(mh_nv == 1 || mh_nv == 2, SPK_ERR_ARG, "spk_fusedmm: vecs_per_lane must be 1 or 2 for the all-heads kernel");
        REQUIRE(mh_fits(mh_nv), SPK_ERR_UNSUPPORTED,
                "spk_fusedmm: %d vectors a row do not split into %d heads of %d-vector lanes", nv, heads, mh_nv);
    } else if (dt != SPK_F32 && heads >= 4 && mh_fits(2)) {
        mh_nv = 2;
    }
    const bool mh = mh_asked || (!shaped && !one_head && mh_fits(mh_nv));
    int G, NV = 1, U = 4, idx = -1;
    if (!mh) {
        if (nvh <= 4) G = 4;
        else if (nvh <= 8) G = 8;
        else if (nvh <= 16) G = 16;
        else if (nvh <= 32) { G = 32; U = 8; }
        else { G = 32; NV = 2; }
        if (one_head && dt == SPK_F32) { G = 8; NV = 2; }
        if (one_head && dt != SPK_F32) { G = 8; NV = 1; }
        if (tune && tune->group_lanes) G = tune->group_lanes;
        if (tune && tune->vecs_per_lane) NV = tune->vecs_per_lane;
        if (tune && tune->unroll) U = tune->unroll;
        idx = fused_shape_index(G, NV, U);
        REQUIRE(idx >= 0, SPK_ERR_UNSUPPORTED, "spk_fusedmm: no kernel for group_lanes=%d vecs_per_lane=%d unroll=%d",
                G, NV, U);
        REQUIRE(G * NV >= nvh, SPK_ERR_UNSUPPORTED, "spk_fusedmm: a group of %d x %d vectors cannot hold a head of %d",
                G, NV, nvh);
    }
    const size_t need = (size_t)S->npieces * (((size_t)K + 2 * (size_t)heads + 3) / 4 * 4) * 4;
    if (need > 0) {
        REQUIRE(workspace && ws_bytes >= need, SPK_ERR_WORKSPACE, "spk_fusedmm: workspace has %zu bytes, needs %zu",
                workspace ? ws_bytes : (size_t)0, need);
        REQUIRE(aligned16(workspace), SPK_ERR_WORKSPACE, "spk_fusedmm: workspace must be 16-byte aligned");
    }
    if (S->M == 0) return SPK_OK;
    FusedArgs a;
    a.M = S->M; a.N = S->N; a.nnz = S->nnz; a.K = K; a.heads = heads; a.dh = dh;
    a.softmax = softmax; a.scale = scale;
    a.rowptr = S->rowptr; a.colidx = S->colidx; a.rowidx = S->rowidx; a.vals = vals;
    a.A = A; a.lda = lda; a.B = B; a.ldb = ldb; a.Y = Y; a.ldy = ldy; a.scores = scores; a.lse = lse;
    a.bnd = S->bnd; a.meta = S->meta; a.head_s0 = S->head_s0; a.slot_np = S->slot_np; a.cnt = S->cnt;
    a.carry = reinterpret_cast<float*>(workspace);
    a.nchunks = S->nchunks;
    cudaError_t e;
    if (mh) {
        e = launch_fused_mh_nv(dt, nv / mh_nv, mh_nv, a, (cudaStream_t)stream);
    } else {
        Launch L;
        L.shape = idx; L.vec = true; L.threads = 64; L.chunks = true; L.ring = true; L.stages = 2;
        e = launch_fused(dt, L, a, (cudaStream_t)stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "spk_fusedmm");
    return SPK_OK;
}

extern "C" spk_status spk_fused_weights(spk_csr S, int32_t heads, int32_t softmax, const float* scores,
                                        const float* lse, float* w, void* stream)
{
    REQUIRE(S && heads >= 1 && heads <= 65535 && (softmax == 0 || softmax == 1), SPK_ERR_ARG,
            "spk_fused_weights: bad argument");
    REQUIRE(S->has_sched, SPK_ERR_STATE, "spk_fused_weights: needs spk_schedule_build first");
    REQUIRE(S->nnz == 0 || (scores && w && (!softmax || lse)), SPK_ERR_ARG, "spk_fused_weights: NULL array");
    cudaError_t e = launch_fused_weights(S->rowidx, S->nnz, heads, softmax, scores, lse, w, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_fused_weights");
    return SPK_OK;
}

extern "C" spk_status spk_fused_rowdot(int64_t M, int32_t K, int32_t heads, const float* dY, int64_t lddy,
                                       const float* Y, int64_t ldy, float* rowdot, void* stream)
{
    REQUIRE(M >= 0 && K >= 1 && heads >= 1 && K % heads == 0, SPK_ERR_SHAPE,
            "spk_fused_rowdot: need M >= 0 and K a positive multiple of heads");
    REQUIRE(M == 0 || (dY && Y && rowdot), SPK_ERR_ARG, "spk_fused_rowdot: NULL array");
    REQUIRE(M <= 1 || (lddy >= K && ldy >= K), SPK_ERR_SHAPE, "spk_fused_rowdot: row strides below K");
    cudaError_t e = launch_fused_rowdot(M, K, heads, dY, lddy, Y, ldy, rowdot, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_fused_rowdot");
    return SPK_OK;
}

extern "C" spk_status spk_fused_score_grad(spk_csr S, int32_t heads, int32_t softmax, float scale, const float* vals,
                                           const float* w, const float* dw, const float* rowdot, float* c,
                                           void* stream)
{
    REQUIRE(S && heads >= 1 && heads <= 65535 && (softmax == 0 || softmax == 1), SPK_ERR_ARG,
            "spk_fused_score_grad: bad argument");
    REQUIRE(S->has_sched, SPK_ERR_STATE, "spk_fused_score_grad: needs spk_schedule_build first");
    REQUIRE(S->nnz == 0 || (dw && c && (!softmax || (w && rowdot))), SPK_ERR_ARG,
            "spk_fused_score_grad: NULL array");
    cudaError_t e = launch_fused_score_grad(S->rowidx, S->nnz, heads, softmax, scale, vals, w, dw, rowdot, c,
                                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_fused_score_grad");
    return SPK_OK;
}

// ----------------------------------------------------------------------------
// SpMM with library-held scratch
// ----------------------------------------------------------------------------
// Carry slots of spk_spmm_static.  A file-scope device array: every GPU that
// loads the library holds SPK_STATIC_SCRATCH_BYTES of it until the process
// exits.  In host code `g_static_scratch` is only a stand-in for the symbol;
// its device address comes from cudaGetSymbolAddress, taken with the device
// current on the first spk_spmm_static call in each CUDA context of that
// device.  The cache is keyed on the context's unique ID, so after
// cudaDeviceReset (which destroys the primary context; the module, and with
// it the array, is loaded again in the next one) the address is taken anew.
static __device__ __align__(256) float g_static_scratch[SPK_STATIC_SCRATCH_BYTES / sizeof(float)];

static constexpr int kMaxStaticDevices = 64;
static std::mutex g_static_mu;
struct StaticAddr {
    unsigned long long ctx_id;   // unique ID of the context the address belongs to (0 = none yet)
    void* addr;
};
static StaticAddr g_static_addr[kMaxStaticDevices];

// Driver entry points for the current context and its ID, fetched through the
// runtime (the library does not link the driver library itself).
typedef int (*ctx_get_current_fn)(void** ctx);
typedef int (*ctx_get_id_fn)(void* ctx, unsigned long long* id);

static spk_status current_context_id(unsigned long long* id)
{
    static ctx_get_current_fn get_current = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return cuda_fail(e, "spk_spmm_static: driver entry point cuCtxGetCurrent");
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return cuda_fail(e, "spk_spmm_static: driver entry point cuCtxGetId");
        REQUIRE(q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess && f1 && f2, SPK_ERR_CUDA,
                "spk_spmm_static: the driver does not provide cuCtxGetCurrent / cuCtxGetId");
        get_current = reinterpret_cast<ctx_get_current_fn>(f1);
        get_id = reinterpret_cast<ctx_get_id_fn>(f2);
    }
    void* ctx = nullptr;
    int r = get_current(&ctx);
    REQUIRE(r == 0, SPK_ERR_CUDA, "spk_spmm_static: cuCtxGetCurrent failed (%d)", r);
    REQUIRE(ctx, SPK_ERR_STATE, "spk_spmm_static: no CUDA context is current on this thread");
    r = get_id(ctx, id);
    REQUIRE(r == 0, SPK_ERR_CUDA, "spk_spmm_static: cuCtxGetId failed (%d)", r);
    return SPK_OK;
}

static spk_status static_scratch_address(void** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "spk_spmm_static: cudaGetDevice");
    REQUIRE(dev >= 0 && dev < kMaxStaticDevices, SPK_ERR_UNSUPPORTED,
            "spk_spmm_static: device ordinal %d is beyond the %d supported", dev, kMaxStaticDevices);
    // cudaGetSymbolAddress also makes the device's primary context current if
    // no context is yet, so look the symbol up before asking for the context.
    void* p = nullptr;
    std::lock_guard<std::mutex> lock(g_static_mu);
    unsigned long long id = 0;
    const bool cached = g_static_addr[dev].addr != nullptr;
    if (!cached) {
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "spk_spmm_static: cudaGetSymbolAddress");
    }
    spk_status st = current_context_id(&id);
    if (st != SPK_OK) return st;
    if (cached && g_static_addr[dev].ctx_id == id) {
        *out = g_static_addr[dev].addr;
        return SPK_OK;
    }
    if (cached) {                 // another context than the cached address belongs to
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "spk_spmm_static: cudaGetSymbolAddress");
    }
    REQUIRE(p && (reinterpret_cast<uintptr_t>(p) & 255u) == 0, SPK_ERR_CUDA,
            "spk_spmm_static: scratch symbol address is NULL or misaligned");
    g_static_addr[dev].ctx_id = id;
    g_static_addr[dev].addr = p;
    *out = p;
    return SPK_OK;
}

extern "C" spk_status spk_spmm_static(spk_csr S, const float* vals, const float* vals2, spk_dtype dtb,
                                      const void* B, int64_t ldb, const float* b_scale, int32_t K, spk_dtype dtc,
                                      void* C, int64_t ldc, int32_t accumulate, const spk_tune* tune,
                                      void* stream)
{
    REQUIRE(S, SPK_ERR_ARG, "spk_spmm_static: S is NULL");
    REQUIRE(K >= 1, SPK_ERR_SHAPE, "spk_spmm_static: K must be >= 1 (got %d)", K);
    // Only the balanced schedule's split rows use carry slots: a row-split
    // call (tune.variant = 1) needs no scratch whatever K is.
    const int variant = (tune && tune->variant) ? tune->variant : (S->has_sched ? 2 : 1);
    const size_t need = (variant >= 2 && S->has_sched) ? (size_t)S->npieces * (size_t)K * 4 : 0;
    REQUIRE(need <= (size_t)SPK_STATIC_SCRATCH_BYTES, SPK_ERR_WORKSPACE,
            "spk_spmm_static: %lld split-row pieces x K = %d need %zu bytes of scratch, above the %zu bytes "
            "held by the library (use spk_spmm with a caller workspace)",
            (long long)S->npieces, K, need, (size_t)SPK_STATIC_SCRATCH_BYTES);
    // No slot of the scratch has to start at zero: within one call every carry
    // slot is written before it is read, so nothing is cleared.  (The arrival
    // counters of split rows live in the schedule storage and the kernel
    // returns them to zero.)
    void* ws = nullptr;
    spk_status st = static_scratch_address(&ws);
    if (st != SPK_OK) return st;
    return spmm_common("spk_spmm_static", S, vals, vals2, dtb, B, ldb, b_scale, K, dtc, C, ldc, accumulate, ws,
                       (size_t)SPK_STATIC_SCRATCH_BYTES, tune, (cudaStream_t)stream);
}

// ----------------------------------------------------------------------------
// Dense row-panel tiles on the tensor cores
// ----------------------------------------------------------------------------
static int32_t tc_threshold_or_default(int32_t t) { return t == 0 ? 1024 : t; }

extern "C" spk_status spk_tc_plan_size(spk_csr S, int32_t threshold, int32_t chunk_work, size_t* storage_bytes,
                                       size_t* temp_bytes)
{
    REQUIRE(S && storage_bytes && temp_bytes, SPK_ERR_ARG, "spk_tc_plan_size: NULL argument");
    const int32_t th = tc_threshold_or_default(threshold), W = chunk_work_or_default(chunk_work);
    REQUIRE(th >= 1 && th <= 128 * 64, SPK_ERR_ARG, "spk_tc_plan_size: threshold %d outside [1, 8192]", th);
    REQUIRE(W >= 32 && W <= (1 << 20), SPK_ERR_ARG, "spk_tc_plan_size: chunk_work %d outside [32, 2^20]", W);
    const TcLayout L = tc_layout(S->M, S->N, S->nnz, th, W);
    *storage_bytes = L.total;
    *temp_bytes = L.temp_total;
    return SPK_OK;
}

extern "C" spk_status spk_tc_plan_build(spk_csr S, int32_t threshold, int32_t chunk_work, void* storage,
                                        size_t storage_bytes, void* temp, size_t temp_bytes, spk_tcplan* out,
                                        void* stream)
{
    REQUIRE(S && out, SPK_ERR_ARG, "spk_tc_plan_build: NULL argument");
    *out = nullptr;
    REQUIRE(!S->vperm, SPK_ERR_ARG, "spk_tc_plan_build: pattern belongs to a transpose plan");
    const int32_t th = tc_threshold_or_default(threshold), W = chunk_work_or_default(chunk_work);
    REQUIRE(th >= 1 && th <= 128 * 64, SPK_ERR_ARG, "spk_tc_plan_build: threshold %d outside [1, 8192]", th);
    REQUIRE(W >= 32 && W <= (1 << 20), SPK_ERR_ARG, "spk_tc_plan_build: chunk_work %d outside [32, 2^20]", W);
    const TcLayout L = tc_layout(S->M, S->N, S->nnz, th, W);
    REQUIRE(storage && storage_bytes >= L.total, SPK_ERR_WORKSPACE, "spk_tc_plan_build: storage needs %zu bytes",
            L.total);
    REQUIRE(temp && temp_bytes >= L.temp_total, SPK_ERR_WORKSPACE, "spk_tc_plan_build: temp needs %zu bytes",
            L.temp_total);
    REQUIRE((reinterpret_cast<uintptr_t>(storage) & 255u) == 0 && (reinterpret_cast<uintptr_t>(temp) & 255u) == 0,
            SPK_ERR_WORKSPACE, "spk_tc_plan_build: buffers must be 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    char* st = reinterpret_cast<char*>(storage);
    int64_t nt = 0, nd = 0;
    cudaError_t e = tc_plan_build(S->rowptr, S->colidx, S->M, S->N, S->nnz, th, st, reinterpret_cast<char*>(temp), L,
                                  &nt, &nd, s);
    if (e != cudaSuccess) return cuda_fail(e, "spk_tc_plan_build");
    spk_tcplan_s* P = new (std::nothrow) spk_tcplan_s();
    REQUIRE(P, SPK_ERR_ARG, "spk_tc_plan_build: out of host memory");
    P->M = S->M; P->N = S->N; P->nnz = S->nnz; P->ntiles = nt; P->dense_nnz = nd; P->threshold = th;
    P->tiles = reinterpret_cast<const int4*>(st + L.tiles);
    P->ent_slot = reinterpret_cast<const int32_t*>(st + L.ent_slot);
    P->ent_ij = reinterpret_cast<const int32_t*>(st + L.ent_ij);
    P->emap = reinterpret_cast<const int32_t*>(st + L.emap);
    P->status = reinterpret_cast<int32_t*>(st + L.status);
    spk_csr_s& R = P->Rest;
    R = spk_csr_s();
    R.M = S->M; R.N = S->N; R.nnz = S->nnz - nd;
    R.rowptr = reinterpret_cast<const int32_t*>(st + L.rowptr);
    R.colidx = reinterpret_cast<const int32_t*>(st + L.colidx);
    spk_status ss = attach_schedule(&R, W, st + L.sched, L.sl.total, s);
    if (ss != SPK_OK) { delete P; return ss; }
    *out = P;
    return SPK_OK;
}

extern "C" spk_status spk_tc_plan_info(spk_tcplan P, int64_t* tiles, int64_t* dense_nnz, int64_t* rest_nnz)
{
    REQUIRE(P, SPK_ERR_ARG, "spk_tc_plan_info: P is NULL");
    if (tiles) *tiles = P->ntiles;
    if (dense_nnz) *dense_nnz = P->dense_nnz;
    if (rest_nnz) *rest_nnz = P->Rest.nnz;
    return SPK_OK;
}

extern "C" spk_status spk_tc_plan_arrays(spk_tcplan P, const int32_t** tiles, const int32_t** ent_slot,
                                         const int32_t** rest_rowptr, const int32_t** rest_colidx,
                                         const int32_t** rest_emap, int32_t** status)
{
    REQUIRE(P, SPK_ERR_ARG, "spk_tc_plan_arrays: P is NULL");
    if (tiles) *tiles = reinterpret_cast<const int32_t*>(P->tiles);
    if (ent_slot) *ent_slot = P->ent_slot;
    if (rest_rowptr) *rest_rowptr = P->Rest.rowptr;
    if (rest_colidx) *rest_colidx = P->Rest.colidx;
    if (rest_emap) *rest_emap = P->emap;
    if (status) *status = P->status;
    return SPK_OK;
}

extern "C" spk_status spk_tc_plan_destroy(spk_tcplan P)
{
    delete P;
    return SPK_OK;
}

extern "C" spk_status spk_tc_sddmm_workspace_size(spk_tcplan P, size_t* bytes)
{
    REQUIRE(P && bytes, SPK_ERR_ARG, "spk_tc_sddmm_workspace_size: NULL argument");
    *bytes = align256((size_t)P->Rest.nnz * 4);
    return SPK_OK;
}

extern "C" spk_status spk_tc_sddmm(spk_tcplan P, const float* vals, spk_dtype dt, const void* A, int64_t lda,
                                   const void* B, int64_t ldb, int32_t K, float* out, void* workspace,
                                   size_t ws_bytes, const spk_tune* tune, void* stream)
{
    REQUIRE(P, SPK_ERR_ARG, "spk_tc_sddmm: P is NULL");
    REQUIRE(dt == SPK_BF16, SPK_ERR_DTYPE, "spk_tc_sddmm: the tensor-core tiles take BF16 operands");
    REQUIRE(K >= 16 && K <= 256 && K % 16 == 0, SPK_ERR_SHAPE, "spk_tc_sddmm: K must be a multiple of 16 in [16, 256]");
    REQUIRE(lda >= K && ldb >= K, SPK_ERR_SHAPE, "spk_tc_sddmm: leading dimensions must be >= K");
    REQUIRE(P->nnz == 0 || (A && B && out), SPK_ERR_ARG, "spk_tc_sddmm: NULL operand");
    REQUIRE(aligned16(A) && aligned16(B) && (lda * 2) % 16 == 0 && (ldb * 2) % 16 == 0, SPK_ERR_SHAPE,
            "spk_tc_sddmm: A and B must be 16-byte aligned with 16-byte row strides");
    const size_t need = align256((size_t)P->Rest.nnz * 4);
    REQUIRE(P->Rest.nnz == 0 || (workspace && ws_bytes >= need), SPK_ERR_WORKSPACE,
            "spk_tc_sddmm: workspace has %zu bytes, needs %zu", workspace ? ws_bytes : (size_t)0, need);
    REQUIRE(aligned16(workspace), SPK_ERR_WORKSPACE, "spk_tc_sddmm: workspace must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    // the remainder on the gather kernels (unit values), then scaled into place
    if (P->Rest.nnz > 0) {
        float* rest = reinterpret_cast<float*>(workspace);
        spk_status st = spk_sddmm(&P->Rest, nullptr, nullptr, dt, A, lda, nullptr, dt, B, ldb, nullptr, K, rest, tune,
                                  stream);
        if (st != SPK_OK) return st;
        cudaError_t e = launch_scatter_scale(P->emap, vals, rest, P->Rest.nnz, out, s);
        if (e != cudaSuccess) return cuda_fail(e, "spk_tc_sddmm remainder");
    }
    TcArgs a;
    a.M = P->M; a.N = P->N; a.K = K;
    a.A = A; a.lda = lda; a.B = B; a.ldb = ldb;
    a.tiles = P->tiles; a.ent_slot = P->ent_slot; a.ent_ij = P->ent_ij;
    a.vals = vals; a.out = out; a.status = P->status;
    cudaError_t e = launch_tc_sddmm(a, P->ntiles, s);
    if (e != cudaSuccess) return cuda_fail(e, "spk_tc_sddmm tiles");
    return SPK_OK;
}

// Not in the public header: the tile kernel with no MMA issued and nothing
// committed, so that every tile's bounded wait on the tensor core's barrier
// runs out; the kernel then sets the plan's status word, frees its tensor
// memory and returns, leaving `out` untouched.  Tests use it to check that
// path without a fault or a hang.
extern "C" spk_status spk_tc_sddmm_unarmed(spk_tcplan P, const void* A, int64_t lda, const void* B, int64_t ldb,
                                           int32_t K, float* out, void* stream)
{
    REQUIRE(P && A && B && out && K >= 16 && K <= 256 && K % 16 == 0 && lda >= K && ldb >= K, SPK_ERR_ARG,
            "spk_tc_sddmm_unarmed: bad argument");
    REQUIRE(aligned16(A) && aligned16(B) && (lda * 2) % 16 == 0 && (ldb * 2) % 16 == 0, SPK_ERR_SHAPE,
            "spk_tc_sddmm_unarmed: A and B must be 16-byte aligned with 16-byte row strides");
    TcArgs a;
    a.M = P->M; a.N = P->N; a.K = K;
    a.A = A; a.lda = lda; a.B = B; a.ldb = ldb;
    a.tiles = P->tiles; a.ent_slot = P->ent_slot; a.ent_ij = P->ent_ij;
    a.vals = nullptr; a.out = out; a.status = P->status;
    a.unarmed = 1;
    cudaError_t e = launch_tc_sddmm(a, P->ntiles, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_tc_sddmm_unarmed");
    return SPK_OK;
}

// ----------------------------------------------------------------------------
// Transpose plan
// ----------------------------------------------------------------------------
extern "C" spk_status spk_tplan_size(spk_csr S, int32_t chunk_work, size_t* storage_bytes, size_t* temp_bytes)
{
    REQUIRE(S && storage_bytes && temp_bytes, SPK_ERR_ARG, "spk_tplan_size: NULL argument");
    const int32_t W = chunk_work_or_default(chunk_work);
    REQUIRE(W >= 32 && W <= (1 << 20), SPK_ERR_ARG, "spk_tplan_size: chunk_work %d outside [32, 2^20]", W);
    const TplanLayout L = tplan_layout(S->M, S->N, S->nnz, W);
    *storage_bytes = L.total;
    *temp_bytes = L.temp_total;
    return SPK_OK;
}

extern "C" spk_status spk_tplan_build(spk_csr S, int32_t chunk_work, void* storage, size_t storage_bytes,
                                      void* temp, size_t temp_bytes, spk_tplan* out, void* stream)
{
    REQUIRE(S && out, SPK_ERR_ARG, "spk_tplan_build: NULL argument");
    *out = nullptr;
    REQUIRE(!S->vperm, SPK_ERR_ARG, "spk_tplan_build: pattern already belongs to a transpose plan");
    const int32_t W = chunk_work_or_default(chunk_work);
    REQUIRE(W >= 32 && W <= (1 << 20), SPK_ERR_ARG, "spk_tplan_build: chunk_work %d outside [32, 2^20]", W);
    const TplanLayout L = tplan_layout(S->M, S->N, S->nnz, W);
    REQUIRE(storage && storage_bytes >= L.total, SPK_ERR_WORKSPACE, "spk_tplan_build: storage needs %zu bytes",
            L.total);
    REQUIRE(temp && temp_bytes >= L.temp_total, SPK_ERR_WORKSPACE, "spk_tplan_build: temp needs %zu bytes",
            L.temp_total);
    REQUIRE((reinterpret_cast<uintptr_t>(storage) & 255u) == 0 && (reinterpret_cast<uintptr_t>(temp) & 255u) == 0,
            SPK_ERR_WORKSPACE, "spk_tplan_build: buffers must be 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    char* st = reinterpret_cast<char*>(storage);
    cudaError_t e = build_transpose(S->rowptr, S->colidx, S->M, S->N, S->nnz, st, reinterpret_cast<char*>(temp), L, s);
    if (e != cudaSuccess) return cuda_fail(e, "spk_tplan_build");
    spk_tplan_s* P = new (std::nothrow) spk_tplan_s();
    REQUIRE(P, SPK_ERR_ARG, "spk_tplan_build: out of host memory");
    P->M = S->M; P->N = S->N;
    P->colptr = reinterpret_cast<const int32_t*>(st + L.colptr);
    P->rowidx = reinterpret_cast<const int32_t*>(st + L.rowidx);
    P->perm = reinterpret_cast<const int32_t*>(st + L.perm);
    spk_csr_s& T = P->St;
    T = spk_csr_s();
    T.M = S->N; T.N = S->M; T.nnz = S->nnz;
    T.rowptr = P->colptr; T.colidx = P->rowidx; T.vperm = P->perm;
    spk_status ss = attach_schedule(&T, W, st + L.sched, L.sl.total, s);
    if (ss != SPK_OK) { delete P; return ss; }
    *out = P;
    return SPK_OK;
}

extern "C" spk_status spk_tplan_arrays(spk_tplan P, const int32_t** colptr, const int32_t** rowidx,
                                       const int32_t** perm)
{
    REQUIRE(P, SPK_ERR_ARG, "spk_tplan_arrays: P is NULL");
    if (colptr) *colptr = P->colptr;
    if (rowidx) *rowidx = P->rowidx;
    if (perm) *perm = P->perm;
    return SPK_OK;
}

extern "C" spk_status spk_tplan_destroy(spk_tplan P)
{
    delete P;
    return SPK_OK;
}

// Workspace of S^T Y: the values in CSC slot order (nnz floats, 256-byte
// aligned block), then the carry rows of split rows of S^T.
static size_t spmm_t_vals_bytes(const spk_tplan_s* P) { return ((size_t)P->St.nnz * 4 + 255) & ~(size_t)255; }

extern "C" spk_status spk_spmm_t_workspace_size(spk_tplan P, int32_t K, size_t* bytes)
{
    REQUIRE(P && bytes && K >= 1, SPK_ERR_ARG, "spk_spmm_t_workspace_size: bad argument");
    *bytes = spmm_t_vals_bytes(P) + (size_t)P->St.npieces * (size_t)K * 4;
    return SPK_OK;
}

extern "C" spk_status spk_spmm_t(spk_tplan P, const float* vals, const float* vals2, spk_dtype dty, const void* Y,
                                 int64_t ldy, const float* y_scale, int32_t K, spk_dtype dtx, void* X, int64_t ldx,
                                 int32_t accumulate, void* workspace, size_t ws_bytes, const spk_tune* tune,
                                 void* stream)
{
    REQUIRE(P, SPK_ERR_ARG, "spk_spmm_t: P is NULL");
    REQUIRE(K >= 1, SPK_ERR_SHAPE, "spk_spmm_t: K must be >= 1 (got %d)", K);
    const size_t vb = spmm_t_vals_bytes(P);
    const size_t need = vb + (size_t)P->St.npieces * (size_t)K * 4;
    REQUIRE(need == 0 || (workspace && ws_bytes >= need), SPK_ERR_WORKSPACE,
            "spk_spmm_t: workspace has %zu bytes, needs %zu", workspace ? ws_bytes : (size_t)0, need);
    REQUIRE((reinterpret_cast<uintptr_t>(workspace) & 255u) == 0, SPK_ERR_WORKSPACE,
            "spk_spmm_t: workspace must be 256-byte aligned");
    if (!workspace) ws_bytes = 0;
    REQUIRE(valid_dt(dty), SPK_ERR_DTYPE, "spk_spmm_t: unknown input dtype");
    char* w = reinterpret_cast<char*>(workspace);
    // every argument check of the SpMM on S^T runs before the value permutation
    spk_status st = spmm_common("spk_spmm_t", &P->St, (vals || vals2) ? reinterpret_cast<const float*>(w) : nullptr,
                                nullptr, dty, Y, ldy, y_scale, K, dtx, X, ldx, accumulate, w ? w + vb : nullptr,
                                w ? ws_bytes - vb : 0, tune, (cudaStream_t)stream, true, true);
    if (st != SPK_OK) return st;
    const float* vt = nullptr;
    if ((vals || vals2) && P->St.nnz > 0) {
        float* out = reinterpret_cast<float*>(w);
        cudaError_t e = launch_permute_vals(P->perm, vals, vals2, P->St.nnz, out, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "spk_spmm_t value permutation");
        vt = out;
    }
    return spmm_common("spk_spmm_t", &P->St, vt, nullptr, dty, Y, ldy, y_scale, K, dtx, X, ldx, accumulate,
                       w ? w + vb : nullptr, w ? ws_bytes - vb : 0, tune, (cudaStream_t)stream, true);
}

// S^T Y with one value array per head: the arrays go to CSC slot order in the
// workspace (heads x round_up(nnz, 4) floats), then the multi-head SpMM on S^T.
static size_t spmm_t_mh_vals_bytes(const spk_tplan_s* P, int32_t heads)
{
    return (((size_t)P->St.nnz + 3) / 4 * 4 * (size_t)heads * 4 + 255) & ~(size_t)255;
}

extern "C" spk_status spk_spmm_t_mh_workspace_size(spk_tplan P, int32_t K, int32_t heads, size_t* bytes)
{
    REQUIRE(P && bytes && K >= 1 && heads >= 1, SPK_ERR_ARG, "spk_spmm_t_mh_workspace_size: bad argument");
    *bytes = spmm_t_mh_vals_bytes(P, heads) + (size_t)P->St.npieces * (size_t)K * 4;
    return SPK_OK;
}

extern "C" spk_status spk_spmm_t_mh(spk_tplan P, const float* vals, int64_t hstride, int32_t heads, spk_dtype dty,
                                    const void* Y, int64_t ldy, int32_t K, float* X, int64_t ldx, int32_t accumulate,
                                    void* workspace, size_t ws_bytes, void* stream)
{
    REQUIRE(P, SPK_ERR_ARG, "spk_spmm_t_mh: P is NULL");
    REQUIRE(heads >= 1 && K >= 1 && K % heads == 0, SPK_ERR_SHAPE,
            "spk_spmm_t_mh: K (%d) must be a multiple of heads (%d)", K, heads);
    REQUIRE(dty == SPK_F32 || dty == SPK_BF16 || dty == SPK_F16, SPK_ERR_DTYPE, "spk_spmm_t_mh: Y must be F32, BF16 or F16");
    REQUIRE(heads == 1 || !vals || hstride >= P->St.nnz, SPK_ERR_ARG, "spk_spmm_t_mh: hstride below nnz");
    const size_t vb = spmm_t_mh_vals_bytes(P, heads);
    const size_t need = vb + (size_t)P->St.npieces * (size_t)K * 4;
    REQUIRE(workspace && ws_bytes >= need, SPK_ERR_WORKSPACE, "spk_spmm_t_mh: workspace has %zu bytes, needs %zu",
            workspace ? ws_bytes : (size_t)0, need);
    REQUIRE((reinterpret_cast<uintptr_t>(workspace) & 255u) == 0, SPK_ERR_WORKSPACE,
            "spk_spmm_t_mh: workspace must be 256-byte aligned");
    char* w = reinterpret_cast<char*>(workspace);
    const int64_t ws_stride = (P->St.nnz + 3) / 4 * 4;
    const float* vt = vals ? reinterpret_cast<const float*>(w) : nullptr;
    spk_status st = spmm_common("spk_spmm_t_mh", &P->St, vt, nullptr, dty, Y, ldy, nullptr, K, SPK_F32, X, ldx,
                                accumulate, w + vb, ws_bytes - vb, nullptr, (cudaStream_t)stream, true, true, heads,
                                ws_stride);
    if (st != SPK_OK) return st;
    if (vals && P->St.nnz > 0)
        for (int h = 0; h < heads; ++h) {
            cudaError_t e = launch_permute_vals(P->perm, vals + (int64_t)h * hstride, nullptr, P->St.nnz,
                                                reinterpret_cast<float*>(w) + (int64_t)h * ws_stride, (cudaStream_t)stream);
            if (e != cudaSuccess) return cuda_fail(e, "spk_spmm_t_mh value permutation");
        }
    return spmm_common("spk_spmm_t_mh", &P->St, vt, nullptr, dty, Y, ldy, nullptr, K, SPK_F32, X, ldx, accumulate,
                       w + vb, ws_bytes - vb, nullptr, (cudaStream_t)stream, true, false, heads, ws_stride);
}

// ----------------------------------------------------------------------------
// Precision
// ----------------------------------------------------------------------------
extern "C" spk_status spk_cast(const float* x, int64_t n, spk_dtype dt, void* out, void* stream)
{
    REQUIRE(n >= 0, SPK_ERR_ARG, "spk_cast: negative size");
    REQUIRE(dt == SPK_BF16 || dt == SPK_F16, SPK_ERR_DTYPE, "spk_cast: target must be BF16 or F16");
    REQUIRE(n == 0 || (x && out), SPK_ERR_ARG, "spk_cast: NULL buffer");
    cudaError_t e = launch_cast(x, n, dt, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_cast");
    return SPK_OK;
}

extern "C" spk_status spk_quantize_e4m3_rows(const float* X, int64_t M, int64_t K, int64_t ldx, uint8_t* Q,
                                             int64_t ldq, float* scales, void* stream)
{
    REQUIRE(M >= 0 && K >= 1, SPK_ERR_SHAPE, "spk_quantize_e4m3_rows: bad shape");
    REQUIRE(ldx >= K && ldq >= K, SPK_ERR_SHAPE, "spk_quantize_e4m3_rows: leading dimensions must be >= K");
    REQUIRE(M == 0 || (X && Q && scales), SPK_ERR_ARG, "spk_quantize_e4m3_rows: NULL buffer");
    cudaError_t e = launch_quant_e4m3(X, M, K, ldx, Q, ldq, scales, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spk_quantize_e4m3_rows");
    return SPK_OK;
}
