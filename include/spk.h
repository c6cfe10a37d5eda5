/*
 * spk — local SDDMM / SpMM kernels for NVIDIA GB300 (sm_103a), C ABI.
 *
 * The library implements the per-processor Compute phase of a 3D sparse
 * kernel (SpComm3D, arXiv 2404.19638, Sec. 6.1): the local computation that
 * runs on local data once communication has delivered it.  With S an M x N
 * sparse matrix and A (M x K), B (N x K) dense tall-and-skinny factors
 * (Sec. 3.1):
 *
 *   SDDMM   out_e = s_e * <A[i,:], B[j,:]>  for every stored e = (i, j)   (Sec. 3.2, Eq. 1)
 *   SpMM    C[i,:] = sum_{e=(i,j)} s_e * B[j,:]                          (Sec. 3.2, Eq. 2;
 *           the text's "S B^T" is read as S B, matching the row-by-row equation)
 *   SpMM^T  X[j,:] = sum_{e=(i,j)} s_e * Y[i,:]   — the adjoint of SpMM; with
 *           SDDMM it forms the pair of Sec. 3.2 in which every nonzero takes
 *           or outputs two dense vectors.
 *
 * Conventions (all entry points):
 *  - Every array argument is a DEVICE pointer owned by the caller; the library
 *    never allocates device memory.  Schedules, transpose plans and the SpMM
 *    carry workspace live in caller-provided buffers whose sizes are queried
 *    first.  Handles own only small host-side metadata.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Compute calls
 *    are asynchronous; the *_build calls synchronise `stream` once at the end
 *    to read back a size.
 *  - Sparse patterns are CSR with int32 row pointers (M+1) and column indices
 *    (nnz); nnz < 2^31.  Columns need not be sorted; duplicates are
 *    independent entries.  Values are passed per call (the pattern stays fixed
 *    while values change, Sec. 5.1), as FP32 `vals` (NULL = all ones) times an
 *    optional second FP32 factor `vals2` (NULL = ones), indexed like colidx.
 *  - Dense matrices are row-major with a leading dimension (elements) >= K;
 *    the inputs' row strides must stay below 4 GiB (SPK_ERR_SHAPE otherwise).
 *  - Arithmetic: inputs are widened to FP32 and accumulated in FP32 (no FP64
 *    on the GPU).  E4M3 operands carry one FP32 scale per row: the value of an
 *    element is code * scale[row].
 *  - Errors are returned as spk_status; no exception crosses the ABI.
 *    spk_last_error() gives a message for the calling thread.  Argument errors
 *    are detected on the host before any CUDA call.
 */
#ifndef SPK_H
#define SPK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum spk_status {
    SPK_OK = 0,
    SPK_ERR_ARG = 1,          /* null pointer, negative size, bad flag            */
    SPK_ERR_SHAPE = 2,        /* leading dimension < K or too large, K < 1, size mismatch */
    SPK_ERR_INDEX = 3,        /* malformed CSR found by spk_csr_validate          */
    SPK_ERR_DTYPE = 4,        /* unsupported dtype or dtype combination           */
    SPK_ERR_WORKSPACE = 5,    /* caller buffer too small or misaligned            */
    SPK_ERR_CUDA = 6,         /* a CUDA runtime call or kernel launch failed      */
    SPK_ERR_TIMEOUT = 7,      /* reserved: no entry point waits on the device     */
    SPK_ERR_UNSUPPORTED = 8,  /* sizes beyond int32 indexing or the kernel tables */
    SPK_ERR_STATE = 9         /* handle used before a required build step        */
} spk_status;

typedef enum spk_dtype {
    SPK_F32 = 0,              /* IEEE binary32                                     */
    SPK_BF16 = 1,             /* bfloat16                                          */
    SPK_F16 = 2,              /* IEEE binary16                                     */
    SPK_E4M3 = 3              /* OCP FP8 E4M3 with one FP32 scale per row          */
} spk_dtype;

/* Kernel choice.  Zero fields mean "library default".  See spk_tune_default. */
typedef struct spk_tune {
    int32_t variant;        /* 0 default, 1 row-split (one lane group per row),
                               2 balanced chunks (merge-path schedule, needs spk_schedule_build),
                                 gathered rows staged in shared memory where the path supports it,
                               3 balanced chunks, gathered rows held in registers */
    int32_t group_lanes;    /* lanes that share one row of the dense factor: 4, 8, 16, 32 */
    int32_t vecs_per_lane;  /* 16-byte vectors each lane holds per K block: 1, 2, 4 */
    int32_t unroll;         /* nonzeros in flight per group: 4, 8                  */
    int32_t cta_threads;    /* threads per CTA: 128 or 256 (register paths)        */
    int32_t stages;         /* batch slots of a shared-memory ring: 2 or 4         */
} spk_tune;

typedef struct spk_csr_s* spk_csr;       /* pattern of S (+ its schedule)      */
typedef struct spk_tplan_s* spk_tplan;   /* transpose plan of a pattern        */
typedef struct spk_batch_s* spk_batch;   /* batched persistent launch          */
typedef struct spk_tcplan_s* spk_tcplan; /* dense tiles for the tensor cores   */

/* ---------------------------------------------------------------- misc -- */
const char* spk_status_string(spk_status s);
/* Message of the last failing call on this thread ("" if none). */
const char* spk_last_error(void);
int32_t spk_version(void);
/* The (group_lanes, vecs_per_lane, unroll) shapes compiled into the library:
 * writes min(count, capacity) triples to out (may be NULL), returns count. */
int32_t spk_shapes(int32_t* out, int32_t capacity);
/* The tune a default call would use for this op (0 SDDMM, 1 SpMM, 2 SpMM^T),
 * dtype of the gathered operand, and K.  Fills *out. */
spk_status spk_tune_default(spk_csr S, int32_t op, spk_dtype dt, int32_t K, spk_tune* out);

/* ------------------------------------------------------------- pattern -- */
/* Wrap a CSR pattern (Sec. 3.1: S is M x N).  rowptr[M+1], colidx[nnz] are
 * borrowed device pointers that must outlive the handle; colidx must be
 * 16-byte aligned (it is streamed with 16-byte asynchronous copies).  No
 * device work. */
spk_status spk_csr_create(spk_csr* out, int64_t M, int64_t N, int64_t nnz,
                          const int32_t* rowptr, const int32_t* colidx);
spk_status spk_csr_destroy(spk_csr S);

/* Check the pattern on the device: rowptr[0] == 0, rowptr[M] == nnz,
 * rowptr non-decreasing, 0 <= colidx < N.  d_report is a device int32[4]
 * the kernel fills: {first error code (0 = valid), first bad index, number of
 * bad entries, 1 if some row has unsorted or repeated columns}.  The caller
 * reads it after synchronising `stream`.  Returns SPK_OK if the check was
 * launched; the outcome is in d_report. */
spk_status spk_csr_validate(spk_csr S, int32_t* d_report, void* stream);

/* COO -> CSR on the device.  The paper states S by its nonzeros s_ij, i.e.
 * by coordinates (Sec. 3.1: S is M x N); the kernels take CSR.  rows[nnz],
 * cols[nnz] (device int32) and optional vals[nnz] (device FP32, NULL = no
 * values) are ordered by (row, column), ties in input order.  dedup: 0 keeps
 * every entry (repeats become independent entries, which SpMM sums); 1 keeps
 * the first entry, in input order, of each repeated (row, column); 2 keeps one
 * entry whose value is the FP32 sum of the repeats' values in input order.
 * Outputs (device, caller-owned): rowptr[M+1]; colidx and vals_out (NULL = not
 * wanted; all ones when vals is NULL) of at least nnz entries, of which the
 * first *nnz_out are written (colidx 16-byte aligned if it is then wrapped by
 * spk_csr_create).  temp: >= spk_coo_to_csr_size bytes, 256-byte aligned,
 * scratch for this call only.  Synchronises `stream` once, at the end, to
 * return *nnz_out (host) and to report a coordinate outside the matrix as
 * SPK_ERR_INDEX (the outputs are then undefined; nothing is read or written
 * out of bounds).  Not capturable in a CUDA graph (it synchronises). */
spk_status spk_coo_to_csr_size(int64_t M, int64_t N, int64_t nnz, size_t* temp_bytes);
spk_status spk_coo_to_csr(int64_t M, int64_t N, int64_t nnz, const int32_t* rows, const int32_t* cols,
                          const float* vals, int32_t dedup, int32_t* rowptr, int32_t* colidx, float* vals_out,
                          int64_t* nnz_out, void* temp, size_t temp_bytes, void* stream);

/* ------------------------------------------------------ row relabelling -- */
/* Locality reordering.  The paper localises indices before its Compute phase
 * (Sec. 5.2: a processor renumbers the rows and columns it holds and drops
 * empty ones); on one GPU the counterpart relabels S's rows so that rows
 * gathering the same B rows run close together and share L2 lines.
 *
 * spk_reorder_rows writes perm[M] (device int32): perm[p] = the original row
 * placed at position p, ties kept in the original order:
 *   SPK_ORDER_DEGREE          most entries first (a device sort);
 *   SPK_ORDER_LEADING_COLUMN  smallest column first, rows without entries last
 *                             (a device sort; restores a band whose rows were
 *                             shuffled);
 *   SPK_ORDER_RCM             reverse Cuthill-McKee (Cuthill & McKee 1969,
 *                             reversed after George 1971) on the symmetric
 *                             graph of a square pattern, edge i - j for every
 *                             stored (i, j), i != j; components start from the
 *                             unvisited vertex of smallest (degree, index) and
 *                             neighbours are queued by (degree, index).  Runs
 *                             on the host: copies the pattern out and the order
 *                             back, synchronising `stream` (temp unused).
 * spk_permute_pattern builds the relabelled pattern S' (row p of S' = row
 * perm[p] of S, same columns in the same order, original column ids):
 * rowptr_out[M+1], colidx_out[nnz], emap[nnz] = the slot in S of each slot of
 * S'.  S' is an ordinary CSR pattern (wrap it with spk_csr_create); with
 * A' = A[perm] its SDDMM and SpMM equal those of S up to the order of rows and
 * entries: out = scatter of out' through emap, C = scatter of C' through perm.
 * spk_permute_rows: Y[p] = X[perm[p]] (scatter 0) or Y[perm[p]] = X[p]
 * (scatter 1), M rows of K elements of dtype dt, leading dimensions ldx, ldy.
 * spk_permute_values: y[i] = x[map[i]] (scatter 0) or y[map[i]] = x[i] (1).
 * temp (the two sorts and spk_permute_pattern): >= spk_reorder_size bytes,
 * 256-byte aligned.  Outputs must not overlap inputs. */
enum { SPK_ORDER_DEGREE = 1, SPK_ORDER_LEADING_COLUMN = 2, SPK_ORDER_RCM = 3 };
spk_status spk_reorder_size(spk_csr S, size_t* temp_bytes);
spk_status spk_reorder_rows(spk_csr S, int32_t order, int32_t* perm, void* temp, size_t temp_bytes, void* stream);
spk_status spk_permute_pattern(spk_csr S, const int32_t* perm, int32_t* rowptr_out, int32_t* colidx_out,
                               int32_t* emap, void* temp, size_t temp_bytes, void* stream);
spk_status spk_permute_rows(const void* X, int64_t ldx, spk_dtype dt, int64_t M, int32_t K, const int32_t* perm,
                            int32_t scatter, void* Y, int64_t ldy, void* stream);
spk_status spk_permute_values(const float* x, const int32_t* map, int64_t n, int32_t scatter, float* y,
                              void* stream);

/* ------------------------------------------------------------ schedule -- */
/* The balanced schedule cuts the merged sequence of (row ends, nonzeros) into
 * chunks of about `chunk_work` items (merge-path partition), snapping each cut
 * back to a row start unless the row holds more than chunk_work nonzeros; such
 * long rows are split and their partial SpMM sums combined in a fixed order.
 * It also stores the row index of every nonzero (COO view).  It depends only
 * on the pattern (Sec. 5.1: built once, reused while values change).
 * chunk_work: 32 .. 2^20 (0 = default 512). */
spk_status spk_schedule_size(spk_csr S, int32_t chunk_work, size_t* bytes);
/* Builds into `storage` (>= spk_schedule_size bytes, 256-byte aligned) and
 * attaches it to S.  Synchronises `stream` once. */
spk_status spk_schedule_build(spk_csr S, int32_t chunk_work, void* storage, size_t bytes, void* stream);
/* nchunks, number of split-row pieces, and chunk_work of the attached schedule. */
spk_status spk_schedule_info(spk_csr S, int64_t* nchunks, int64_t* npieces, int32_t* chunk_work);
/* Copy of the schedule's chunk boundaries as (row, nonzero) int32 pairs,
 * nchunks + 1 of them, into a device buffer (for tests). */
spk_status spk_schedule_bounds(spk_csr S, int32_t* d_out, void* stream);

/* Bytes of workspace a SpMM on S with K columns needs (carry rows of split
 * rows under the balanced schedule; 0 for row-split). */
spk_status spk_spmm_workspace_size(spk_csr S, int32_t K, size_t* bytes);

/* ------------------------------------------------------------- compute -- */
/* SDDMM, Eq. 1.  A: M x K (dtype dta, leading dim lda, scales a_scale[M] for
 * E4M3), B: N x K (dtb, ldb, b_scale[N]).  out[nnz] FP32 in colidx order.
 * Supported (dta, dtb): equal dtypes, or dta = F32 with dtb = BF16 / F16. */
spk_status spk_sddmm(spk_csr S, const float* vals, const float* vals2,
                     spk_dtype dta, const void* A, int64_t lda, const float* a_scale,
                     spk_dtype dtb, const void* B, int64_t ldb, const float* b_scale,
                     int32_t K, float* out, const spk_tune* tune, void* stream);
/* SDDMM in heads (equal slices of K, head width K / heads a whole number of
 * 16-byte vectors): out[h * nnz + e] = vals[e] * <A[i, h*dh:(h+1)*dh],
 * B[j, h*dh:(h+1)*dh]> (Eq. 1 on each slice; vals NULL = ones, 16-byte
 * aligned), out FP32 heads x nnz.  A (M x K) and B (N x K) share dtype dt
 * (F32 or BF16), 16-byte aligned with 16-byte row strides.  One pass over the
 * pattern for all heads on the balanced schedule (needs spk_schedule_build);
 * K must fill the default SDDMM lane block (K = 32, 64, 128 in F32; 64, 128
 * in BF16), else SPK_ERR_UNSUPPORTED (call spk_sddmm per slice then). */
spk_status spk_sddmm_mh(spk_csr S, const float* vals, int32_t heads, spk_dtype dt, const void* A, int64_t lda,
                        const void* B, int64_t ldb, int32_t K, float* out, void* stream);

/* SpMM, Eq. 2.  C (M x K, dtype dtc in {F32, BF16, F16}, leading dim ldc)
 * = S B, or C += S B with accumulate = 1.  Empty rows are written as zero
 * (left unchanged when accumulating).  workspace: >= spk_spmm_workspace_size
 * bytes when the balanced schedule is used (may be NULL otherwise).
 * Split rows are summed in chunk order: results are deterministic.  Calls that
 * share one schedule must not overlap on the device. */
spk_status spk_spmm(spk_csr S, const float* vals, const float* vals2,
                    spk_dtype dtb, const void* B, int64_t ldb, const float* b_scale, int32_t K,
                    spk_dtype dtc, void* C, int64_t ldc, int32_t accumulate,
                    void* workspace, size_t ws_bytes, const spk_tune* tune, void* stream);

/* SpMM with one value array per head: heads equal slices of K, head h
 * (columns h*K/heads .. (h+1)*K/heads - 1) multiplying by its own values
 * vals[h * hstride + e] (e in colidx order; NULL = ones):
 *   C[i, head h] (+)= sum_{e=(i,j)} vals[h * hstride + e] * B[j, head h]
 * It is the product that the backward of a multi-head SDDMM -> SpMM cascade
 * needs (one SpMM per head otherwise, each reading the whole pattern).  B is
 * F32, BF16 or F16 (16-byte aligned rows, K/heads a whole number of 16-byte
 * vectors); C is FP32.  Workspace as spk_spmm. */
spk_status spk_spmm_mh(spk_csr S, const float* vals, int64_t hstride, int32_t heads, spk_dtype dtb, const void* B,
                       int64_t ldb, int32_t K, float* C, int64_t ldc, int32_t accumulate, void* workspace,
                       size_t ws_bytes, void* stream);

/* Scratch held by the library for spk_spmm_static, in bytes (4 MiB): a
 * file-scope device array that every GPU loading the library keeps until the
 * process exits. */
#define SPK_STATIC_SCRATCH_BYTES (4u << 20)

/* spk_spmm without a caller workspace: the same SpMM as spk_spmm.  The paper
 * has no counterpart of this entry point.  It is for callers that cannot call cudaMalloc: code running inside a host
 * that owns the device memory pool (a plugin with a memory budget fixed at
 * load time, a framework whose caching allocator must see every buffer) or a
 * loop where cudaMalloc's implicit device synchronisation is not allowed.
 * The split-row carry slots go to the library's static scratch instead of a
 * workspace; the caller still passes the inputs and C.  Neither the caller nor
 * the library allocates: no cudaMalloc, cudaFree or allocating library call.
 * Arguments, layouts and results are those of spk_spmm.
 *  - Limit: with the balanced schedule (the default when one is attached),
 *    spk_schedule_info's npieces x K x 4 must not exceed
 *    SPK_STATIC_SCRATCH_BYTES; larger calls return SPK_ERR_WORKSPACE before
 *    any launch (use spk_spmm then).  Row-split calls (tune.variant = 1) use
 *    no scratch and have no limit.
 *  - Set-up: the first call in a CUDA context of a device (the current one)
 *    looks up the scratch's device address with cudaGetSymbolAddress and
 *    keeps it for that context.  cudaDeviceReset ends the context, so the
 *    first call after it looks the address up again.
 *  - Sharing: every call on a device uses the same scratch, which keeps the
 *    last call's contents.  Nothing in it needs to start at zero, so it is
 *    never cleared.  Calls that overlap on the GPU (other streams, other host
 *    threads) race on the scratch and give wrong results: order them. */
spk_status spk_spmm_static(spk_csr S, const float* vals, const float* vals2,
                           spk_dtype dtb, const void* B, int64_t ldb, const float* b_scale, int32_t K,
                           spk_dtype dtc, void* C, int64_t ldc, int32_t accumulate,
                           const spk_tune* tune, void* stream);

/* FusedMM: SDDMM cascaded into SpMM on one dense matrix (the cascade Sec. 2
 * names; operands as in Eq. 1 and Eq. 2), per head of `heads` equal slices of
 * K (head width dh = K / heads):
 *   e_h(i,j) = scale * s_ij * <A[i, head h], B[j, head h]>
 *   w_h(i,j) = e_h(i,j), or (softmax = 1) exp(e_h(i,j) - m) / sum over row i
 *   Y[i, head h] = sum_j w_h(i,j) * B[j, head h]          (Y: M x K, FP32)
 * Each gathered B row serves both products.  A (M x K) and B (N x K) share
 * dtype dt (F32, BF16 or F16), 16-byte aligned with 16-byte row strides; dh
 * must be a whole number of 16-byte vectors.  vals: NULL (ones) or 16-byte
 * aligned FP32.  scores: NULL or heads x nnz FP32 (head-major, CSR order
 * within a head) receiving e.  lse: NULL or M x heads FP32 receiving
 * m + log(sum exp) of each row (softmax only; -inf for an empty row, whose Y
 * row is 0).  Needs the balanced schedule; workspace >=
 * spk_fusedmm_workspace_size bytes (16-byte aligned; NULL if that is 0).
 * Split rows are merged in a fixed order: results are deterministic.  Calls
 * that share one schedule must not overlap on the device.  tune: NULL (the
 * library picks the kernel), group_lanes / vecs_per_lane / unroll for the
 * one-head-per-grid-row kernel of that shape, or vecs_per_lane alone (1 or
 * 2) for the all-heads kernel with that many adjacent vectors a lane. */
spk_status spk_fusedmm_workspace_size(spk_csr S, int32_t K, int32_t heads, size_t* bytes);
spk_status spk_fusedmm(spk_csr S, const float* vals, float scale, int32_t softmax, spk_dtype dt,
                       const void* A, int64_t lda, const void* B, int64_t ldb, int32_t K, int32_t heads,
                       float* Y, int64_t ldy, float* scores, float* lse,
                       void* workspace, size_t ws_bytes, const spk_tune* tune, void* stream);

/* Steps of the FusedMM backward that are not SDDMM / SpMM calls.  Arrays
 * over entries are heads x nnz FP32 (head-major); lse and rowdot are M x heads
 * FP32; dY and Y are M x K FP32 row-major with row strides lddy, ldy; vals is
 * the FusedMM's nnz sparse values (NULL = ones).  For entry e = (i, j) and
 * head h (columns h*K/heads .. (h+1)*K/heads - 1):
 *   spk_fused_weights:    w = scores, or exp(scores - lse[i]) with softmax
 *   spk_fused_rowdot:     rowdot[i, h] = <dY_i, Y_i> over head h's columns,
 *                         which equals sum_j w_ij <dY_i, B_j> (the softmax
 *                         backward's row term; Y is the FusedMM output)
 *   spk_fused_score_grad: c = scale * s_e * dw, or
 *                         scale * s_e * w * (dw - rowdot[i]) with softmax,
 *                         where dw = <dY_i, B_j> per head: the gradient
 *                         w.r.t. the unscaled dot <A_i, B_j>, so that
 *                         dA = SpMM(c, B) and dB = SpMM^T(c, A) + SpMM^T(w, dY)
 *                         per head, each with one value array
 * heads is at most 65535.  spk_fused_weights and spk_fused_score_grad need
 * the balanced schedule (its COO rows); none allocates.  Outputs must not
 * overlap inputs (w and scores; c and vals, w, dw, rowdot; rowdot and dY, Y). */
spk_status spk_fused_weights(spk_csr S, int32_t heads, int32_t softmax, const float* scores, const float* lse,
                             float* w, void* stream);
spk_status spk_fused_rowdot(int64_t M, int32_t K, int32_t heads, const float* dY, int64_t lddy, const float* Y,
                            int64_t ldy, float* rowdot, void* stream);
spk_status spk_fused_score_grad(spk_csr S, int32_t heads, int32_t softmax, float scale, const float* vals,
                                const float* w, const float* dw, const float* rowdot, float* c, void* stream);

/* --------------------------------------------- tensor-core dense tiles -- */
/* Where a 128-row x 64-column tile of S holds many entries, its SDDMM (Eq. 1)
 * is a real contraction: the tile's A panel (128 x K) and B tile (64 x K) are
 * read once and multiplied whole on the tensor cores (tcgen05, FP32
 * accumulation in tensor memory), then sampled at the tile's entries.
 * spk_tc_plan_build finds the tiles (panel = row / 128, column tile =
 * column / 64) holding at least `threshold` entries (0 = 1024, an eighth of
 * the tile) and builds the remainder pattern (every other entry, each row in
 * order) with its balanced schedule (chunk_work as in spk_schedule_build).
 * storage holds the plan for its lifetime (size from spk_tc_plan_size, an
 * upper bound); temp is scratch for the build.  Synchronises `stream`.
 * spk_tc_plan_arrays: device views for tests — the tiles as int32 quadruples
 * {panel, column tile, first entry, entries}, the slot in S of each
 * dense-tile entry, the remainder's rowptr (M+1), colidx and slot in S of
 * each entry, and the status word (1 after a tensor-core wait ran out).
 *
 * spk_tc_sddmm: out = SDDMM(S, A, B) with vals (NULL = ones), A (M x K) and
 * B (N x K) BF16, 16-byte aligned with 16-byte row strides, K a multiple of
 * 16 up to 256: the remainder through spk_sddmm (into the workspace, >=
 * spk_tc_sddmm_workspace_size bytes, then scaled into place), the dense
 * tiles on the tensor cores.  Results are within FP32 accumulation error of
 * spk_sddmm's (a different summation order). */
spk_status spk_tc_plan_size(spk_csr S, int32_t threshold, int32_t chunk_work, size_t* storage_bytes,
                            size_t* temp_bytes);
spk_status spk_tc_plan_build(spk_csr S, int32_t threshold, int32_t chunk_work, void* storage, size_t storage_bytes,
                             void* temp, size_t temp_bytes, spk_tcplan* out, void* stream);
spk_status spk_tc_plan_info(spk_tcplan P, int64_t* tiles, int64_t* dense_nnz, int64_t* rest_nnz);
spk_status spk_tc_plan_arrays(spk_tcplan P, const int32_t** tiles, const int32_t** ent_slot,
                              const int32_t** rest_rowptr, const int32_t** rest_colidx, const int32_t** rest_emap,
                              int32_t** status);
spk_status spk_tc_plan_destroy(spk_tcplan P);
spk_status spk_tc_sddmm_workspace_size(spk_tcplan P, size_t* bytes);
spk_status spk_tc_sddmm(spk_tcplan P, const float* vals, spk_dtype dt, const void* A, int64_t lda, const void* B,
                        int64_t ldb, int32_t K, float* out, void* workspace, size_t ws_bytes, const spk_tune* tune,
                        void* stream);
/*
 * spk_tc_sddmm_unarmed (test hook): launches the dense-tile kernel of P with
 * its MMAs left out, so that every bounded wait on the tensor core's barrier
 * runs out; each tile sets P's status word to 1, frees its tensor memory and
 * returns without writing `out`.  Same argument rules as spk_tc_sddmm (A, B
 * BF16).  Exists to test the wait limit without a fault or a hang.
 */
spk_status spk_tc_sddmm_unarmed(spk_tcplan P, const void* A, int64_t lda, const void* B, int64_t ldb, int32_t K,
                                float* out, void* stream);

/* ----------------------------------------------------- transpose plan -- */
/* The CSC of S by a stable device radix sort on the column index: colptr[N+1],
 * rowidx[nnz] (rows ascending inside a column) and perm[nnz] (CSR slot of each
 * CSC slot), plus a balanced schedule of S^T.  storage holds the plan for its
 * lifetime; temp is scratch for the build only. */
spk_status spk_tplan_size(spk_csr S, int32_t chunk_work, size_t* storage_bytes, size_t* temp_bytes);
spk_status spk_tplan_build(spk_csr S, int32_t chunk_work, void* storage, size_t storage_bytes,
                           void* temp, size_t temp_bytes, spk_tplan* out, void* stream);
spk_status spk_tplan_arrays(spk_tplan P, const int32_t** colptr, const int32_t** rowidx,
                            const int32_t** perm);
spk_status spk_tplan_destroy(spk_tplan P);
/* Bytes of workspace an S^T Y with K columns needs: the values in CSC slot
 * order (nnz floats) and the carry rows of split rows of S^T. */
spk_status spk_spmm_t_workspace_size(spk_tplan P, int32_t K, size_t* bytes);

/* X (N x K) = S^T Y (Y: M x K), or += with accumulate = 1.  vals / vals2 are
 * indexed like S's colidx (CSR order); the call first writes their product in
 * CSC slot order (gathered through perm) into the workspace (>=
 * spk_spmm_t_workspace_size bytes, 256-byte aligned; NULL only when that size
 * is 0), then runs the SpMM kernels on the transposed pattern. */
spk_status spk_spmm_t(spk_tplan P, const float* vals, const float* vals2,
                      spk_dtype dty, const void* Y, int64_t ldy, const float* y_scale, int32_t K,
                      spk_dtype dtx, void* X, int64_t ldx, int32_t accumulate,
                      void* workspace, size_t ws_bytes, const spk_tune* tune, void* stream);

/* X (N x K, FP32) (+)= S^T Y with one value array per head (as spk_spmm_mh):
 * X[j, head h] = sum_{e=(i,j)} vals[h * hstride + e] * Y[i, head h].  The
 * arrays go to CSC slot order in the workspace (size from
 * spk_spmm_t_mh_workspace_size, 256-byte aligned) first. */
spk_status spk_spmm_t_mh_workspace_size(spk_tplan P, int32_t K, int32_t heads, size_t* bytes);
spk_status spk_spmm_t_mh(spk_tplan P, const float* vals, int64_t hstride, int32_t heads, spk_dtype dty, const void* Y,
                         int64_t ldy, int32_t K, float* X, int64_t ldx, int32_t accumulate, void* workspace,
                         size_t ws_bytes, void* stream);

/* ----------------------------------------------------------- precision -- */
/* Round-to-nearest-even casts of n FP32 values to BF16 or F16. */
spk_status spk_cast(const float* x, int64_t n, spk_dtype dt, void* out, void* stream);
/* Per-row E4M3 quantisation: scale[i] = max_k |X[i,k]| / 448 (1 for an
 * all-zero row), Q[i,k] = E4M3(X[i,k] / scale[i]) with round-to-nearest-even
 * and saturation to +-448; the division is IEEE binary32. */
spk_status spk_quantize_e4m3_rows(const float* X, int64_t M, int64_t K, int64_t ldx,
                                  uint8_t* Q, int64_t ldq, float* scales, void* stream);

/* ------------------------------------------------------------- batched -- */
/* Many independent problems in one persistent launch.  Every item names a
 * pattern (with a balanced schedule attached), its values, dense operands and
 * output; op is 0 (SDDMM: out = FP32 nnz array) or 1 (SpMM: out = C, FP32).
 * Items may differ in size, K (a whole number of 16-byte vectors, at most 16
 * of them: K <= 64 in F32, <= 128 in BF16) and dtype (F32 or BF16, both
 * operands alike).  The run is a single kernel launch that pulls (item, chunk)
 * work off a device counter, so it can be captured in a CUDA graph and
 * replayed; the counter resets itself at the end of each run.  Pointers are
 * fixed at creation: replays read whatever the buffers hold at that time.
 * Each item runs the shape its tune names (spk_batch_shapes lists them per
 * op; default by K); every warp gets the largest shared-memory ring among the
 * items' shapes, and a batch with an item of 8-nonzero batches or BF16
 * operands runs the kernel build with 96 registers per thread (5 CTAs of 4
 * warps per SM; else 80 registers, 6 CTAs). */
typedef struct spk_batch_item {
    int32_t op;               /* 0 SDDMM, 1 SpMM                              */
    spk_csr S;
    const float* vals;        /* NULL = ones                                  */
    spk_dtype dt;             /* F32 or BF16                                  */
    const void* A;            /* SDDMM only: M x K, leading dim lda           */
    int64_t lda;
    const void* B;            /* N x K, leading dim ldb                       */
    int64_t ldb;
    int32_t K;
    void* out;                /* SDDMM: float[nnz]; SpMM: float C[M x ldc]    */
    int64_t ldc;
    const spk_tune* tune;     /* NULL = default; group_lanes/vecs/unroll used */
} spk_batch_item;

/* storage: device buffer (256-byte aligned) for descriptors, work counters and
 * SpMM carry rows; size from spk_batch_size. */
spk_status spk_batch_size(const spk_batch_item* items, int32_t count, size_t* bytes);
spk_status spk_batch_create(const spk_batch_item* items, int32_t count, void* storage,
                            size_t bytes, spk_batch* out, void* stream);
spk_status spk_batch_run(spk_batch Bt, void* stream);
/* The (group_lanes, vecs_per_lane, unroll) shapes batched items of op (0
 * SDDMM, 1 SpMM) can run: writes min(count, capacity) triples to out (may be
 * NULL), returns count (0 for another op). */
int32_t spk_batch_shapes(int32_t op, int32_t* out, int32_t capacity);
/* The kernel build later spk_batch_run calls use: regs = 80 (6 CTAs of 4
 * warps per SM), 96 (5 CTAs) or 0 (the build spk_batch_create chose); the
 * grid is recomputed.  Host only: runs already launched, and graphs captured
 * earlier, keep the build they were given. */
spk_status spk_batch_set_registers(spk_batch Bt, int32_t regs);
/* Number of (item, chunk) work units and CTAs of one run. */
spk_status spk_batch_info(spk_batch Bt, int64_t* work_units, int32_t* ctas);
spk_status spk_batch_destroy(spk_batch Bt);

#ifdef __cplusplus
}
#endif
#endif /* SPK_H */
