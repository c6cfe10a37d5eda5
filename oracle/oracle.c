/*
 * Plain FP64 CPU oracle for the local SDDMM / SpMM computation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * include this file: it exists so that tests, the smoke check and the timed
 * CPU baseline can compare the CUDA path against a slow, obviously correct
 * restatement of the paper's definitions.  It shares no code, header or
 * constant with the CUDA sources.
 *
 * Every routine is a direct loop over the definition, accumulating in double:
 *   SDDMM   c_e = s_e * <a_i, b_j> for every stored e = (i, j)      (Sec. 3.2, Eq. 1)
 *   SpMM    a_i = sum_j s_ij * b_j                                   (Sec. 3.2, Eq. 2)
 *   SpMM^T  x_j = sum_i s_ij * y_i  (the adjoint pair of Sec. 3.2: each nonzero
 *           takes / outputs two dense vectors)
 *   FusedMM y_i = sum_j w_ij * b_j with w = the SDDMM scores (Sec. 2: SDDMM
 *           cascaded into SpMM), per head, optionally row-softmax weights
 * plus the bookkeeping the GPU path needs a reference for:
 *   - a stable counting-sort transpose (CSR -> CSC with slot permutation),
 *   - COO -> CSR by two stable counting sorts, with duplicate handling,
 *   - the reverse Cuthill-McKee order of a square pattern (a row relabelling
 *     for locality; not the paper's, the single-GPU stand-in for its
 *     localisation of indices),
 *   - the merge-path split point of the (row ends, nonzeros) merge, by walking,
 *   - number-format encoders / decoders written from the format definitions
 *     (IEEE binary16, bfloat16 = top half of binary32, OCP FP8 E4M3),
 *   - per-row E4M3 quantisation with scale = amax / 448.
 *
 * Build: gcc -O2 -fPIC -shared -std=c11 (no -ffast-math: the float division in
 * the quantiser must stay the IEEE single-precision operation).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

enum { OR_F32 = 0, OR_BF16 = 1, OR_F16 = 2, OR_E4M3 = 3, OR_F64 = 4 };

/* ------------------------------------------------------------------------- */
/* Number formats, from their definitions                                    */
/* ------------------------------------------------------------------------- */

/* bfloat16: the upper 16 bits of an IEEE binary32 pattern. */
double oracle_decode_bf16(uint32_t h)
{
    uint32_t bits = (h & 0xFFFFu) << 16;
    float f;
    memcpy(&f, &bits, sizeof f);
    return (double)f;
}

/* IEEE binary16: 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits. */
double oracle_decode_f16(uint32_t h)
{
    int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0)
        v = ldexp((double)m, -24);                 /* subnormal: m/1024 * 2^-14 */
    else if (e == 31)
        v = m ? NAN : INFINITY;
    else
        v = ldexp(1.0 + m / 1024.0, e - 15);
    return s ? -v : v;
}

/* OCP FP8 E4M3: 1 sign bit, 4 exponent bits (bias 7), 3 mantissa bits, no
 * infinities, S.1111.111 is NaN, largest finite magnitude 448. */
double oracle_decode_e4m3(uint32_t q)
{
    int s = (q >> 7) & 1, e = (q >> 3) & 15, m = q & 7;
    double v;
    if (e == 15 && m == 7)
        v = NAN;
    else if (e == 0)
        v = ldexp((double)m / 8.0, -6);            /* subnormal */
    else
        v = ldexp(1.0 + m / 8.0, e - 7);
    return s ? -v : v;
}

typedef double (*decode_fn)(uint32_t);

/* Round-to-nearest, ties-to-even, by searching the (monotone) magnitudes of
 * the non-negative codes 0..max_code.  `beyond` is the magnitude of the first
 * value past max_code in the unbounded-exponent format (the IEEE overflow
 * threshold), and `overflow_code` what a magnitude rounding there becomes. */
static uint32_t encode_nearest(double x, decode_fn dec, uint32_t max_code, double beyond,
                               uint32_t overflow_code, uint32_t sign_bit, uint32_t nan_code)
{
    if (isnan(x))
        return nan_code;
    uint32_t sign = signbit(x) ? sign_bit : 0;
    double ax = fabs(x);
    /* largest code with magnitude <= ax */
    uint32_t lo = 0, hi = max_code;
    if (ax >= dec(max_code)) {
        lo = max_code;
    } else {
        while (lo < hi) {                          /* invariant: dec(lo) <= ax */
            uint32_t mid = lo + (hi - lo + 1) / 2;
            if (dec(mid) <= ax) lo = mid; else hi = mid - 1;
        }
    }
    double vlo = dec(lo);
    if (vlo == ax)
        return sign | lo;
    double vhi = (lo == max_code) ? beyond : dec(lo + 1);
    double dlo = ax - vlo, dhi = vhi - ax;
    uint32_t pick;
    if (dlo < dhi) pick = lo;
    else if (dhi < dlo) pick = lo + 1;
    else pick = (lo & 1) ? lo + 1 : lo;            /* tie: even code */
    if (pick > max_code)
        pick = overflow_code;
    return sign | pick;
}

uint32_t oracle_encode_bf16(float x)
{
    /* beyond the largest finite bf16 (0x7F7F) the next step is 2^128 -> inf */
    return encode_nearest((double)x, oracle_decode_bf16, 0x7F7Fu, ldexp(1.0, 128),
                          0x7F80u, 0x8000u, 0x7FC0u | (signbit(x) ? 0x8000u : 0));
}

uint32_t oracle_encode_f16(float x)
{
    return encode_nearest((double)x, oracle_decode_f16, 0x7BFFu, 65536.0,
                          0x7C00u, 0x8000u, 0x7E00u | (signbit(x) ? 0x8000u : 0));
}

/* Saturating E4M3: magnitudes past 448 clamp to 448 instead of overflowing. */
uint32_t oracle_encode_e4m3(float x)
{
    return encode_nearest((double)x, oracle_decode_e4m3, 0x7Eu, 480.0,
                          0x7Eu, 0x80u, 0x7Fu | (signbit(x) ? 0x80u : 0));
}

void oracle_encode_array(int dtype, int64_t n, const float* x, void* out)
{
    for (int64_t i = 0; i < n; ++i) {
        if (dtype == OR_BF16) ((uint16_t*)out)[i] = (uint16_t)oracle_encode_bf16(x[i]);
        else if (dtype == OR_F16) ((uint16_t*)out)[i] = (uint16_t)oracle_encode_f16(x[i]);
        else if (dtype == OR_E4M3) ((uint8_t*)out)[i] = (uint8_t)oracle_encode_e4m3(x[i]);
    }
}

/* Per-row E4M3 quantisation: scale_i = amax_i / 448 (1 for an all-zero row),
 * code = E4M3_satfinite_RNE(x / scale_i), the division in binary32. */
void oracle_quantize_e4m3_rows(int64_t M, int64_t K, const float* x, int64_t ldx,
                               uint8_t* codes, int64_t ldq, float* scales)
{
    for (int64_t i = 0; i < M; ++i) {
        float amax = 0.0f;
        for (int64_t k = 0; k < K; ++k) {
            float a = fabsf(x[i * ldx + k]);
            if (a > amax) amax = a;
        }
        float scale = (amax > 0.0f) ? amax / 448.0f : 1.0f;
        scales[i] = scale;
        for (int64_t k = 0; k < K; ++k) {
            float q = x[i * ldx + k] / scale;
            codes[i * ldq + k] = (uint8_t)oracle_encode_e4m3(q);
        }
    }
}

/* One dense element, dequantised to double: value(code) * row_scale. */
static double elem(int dtype, const void* p, int64_t idx, const float* scale, int64_t row)
{
    double v;
    switch (dtype) {
    case OR_F32:  v = (double)((const float*)p)[idx]; break;
    case OR_BF16: v = oracle_decode_bf16(((const uint16_t*)p)[idx]); break;
    case OR_F16:  v = oracle_decode_f16(((const uint16_t*)p)[idx]); break;
    case OR_E4M3: v = oracle_decode_e4m3(((const uint8_t*)p)[idx]); break;
    case OR_F64:  v = ((const double*)p)[idx]; break;
    default:      v = NAN;
    }
    if (scale) v *= (double)scale[row];
    return v;
}

static double sval(const double* vals, const double* vals2, int64_t e)
{
    double s = vals ? vals[e] : 1.0;
    if (vals2) s *= vals2[e];
    return s;
}

/* ------------------------------------------------------------------------- */
/* SDDMM (Eq. 1): out[e] = s_e * sum_k A[i,k] * B[j,k]                        */
/* With abs_mode, every term is replaced by its magnitude (the condition     */
/* denominator |s_e| * sum_k |a_ik b_jk| used by the componentwise error).   */
/* Only rows listed in `rows` (all rows if rows == NULL) are written.        */
/* ------------------------------------------------------------------------- */
int oracle_sddmm(int64_t M, int64_t N, int64_t K,
                 const int32_t* rowptr, const int32_t* colidx,
                 const double* vals, const double* vals2, int abs_mode,
                 int dta, const void* A, int64_t lda, const float* a_scale,
                 int dtb, const void* B, int64_t ldb, const float* b_scale,
                 int64_t nrows, const int64_t* rows, double* out)
{
    int64_t count = rows ? nrows : M;
    for (int64_t q = 0; q < count; ++q) {
        int64_t i = rows ? rows[q] : q;
        if (i < 0 || i >= M) return 1;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            int64_t j = colidx[e];
            if (j < 0 || j >= N) return 2;
            double acc = 0.0;
            for (int64_t k = 0; k < K; ++k) {
                double t = elem(dta, A, i * lda + k, a_scale, i) * elem(dtb, B, j * ldb + k, b_scale, j);
                acc += abs_mode ? fabs(t) : t;
            }
            double s = sval(vals, vals2, e);
            out[e] = abs_mode ? fabs(s) * acc : s * acc;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* SpMM (Eq. 2): C[q,:] = sum_{e in row i} s_e * B[j_e,:] for i = rows[q].    */
/* ------------------------------------------------------------------------- */
int oracle_spmm(int64_t M, int64_t N, int64_t K,
                const int32_t* rowptr, const int32_t* colidx,
                const double* vals, const double* vals2, int abs_mode,
                int dtb, const void* B, int64_t ldb, const float* b_scale,
                int64_t nrows, const int64_t* rows, double* C)
{
    int64_t count = rows ? nrows : M;
    for (int64_t q = 0; q < count; ++q) {
        int64_t i = rows ? rows[q] : q;
        if (i < 0 || i >= M) return 1;
        double* c = C + q * K;
        for (int64_t k = 0; k < K; ++k) c[k] = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            int64_t j = colidx[e];
            if (j < 0 || j >= N) return 2;
            double s = sval(vals, vals2, e);
            for (int64_t k = 0; k < K; ++k) {
                double t = s * elem(dtb, B, j * ldb + k, b_scale, j);
                c[k] += abs_mode ? fabs(t) : t;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* FusedMM: the SDDMM -> SpMM cascade (Sec. 2) on the operands of Eq. 1 and   */
/* Eq. 2, per head h of H equal slices of K (width D = K / H):                */
/*   e_h(i,j) = scale * s_ij * sum_{k in head h} A[i,k] * B[j,k]              */
/*   w_h(i,j) = e_h(i,j), or with row_softmax                                 */
/*            = exp(e_h(i,j) - m) / sum_{j' in row i} exp(e_h(i,j') - m),     */
/*              m = max_{j' in row i} e_h(i,j')                               */
/*   Y[q, head h] = sum_{j in row i} w_h(i,j) * B[j, head h],   i = rows[q]   */
/* abs_mode: the condition denominator of Y: |w| |B| summed, where a plain    */
/* weight is replaced by |scale s_ij| sum_k |A[i,k] B[j,k]| (softmax weights  */
/* are already positive).  scores[h * nnz + e] = e_h of entry e and           */
/* lse[q * H + h] = m + log(sum) (-inf for an empty row) when requested.      */
/* ------------------------------------------------------------------------- */
static void head_score(int dta, const void* A, int64_t lda, int dtb, const void* B, int64_t ldb, int64_t i,
                       int64_t j, int64_t k0, int64_t D, double sv, double scale, double* score, double* score_abs)
{
    double dot = 0.0, dabs = 0.0;
    for (int64_t k = k0; k < k0 + D; ++k) {
        double t = elem(dta, A, i * lda + k, NULL, i) * elem(dtb, B, j * ldb + k, NULL, j);
        dot += t;
        dabs += fabs(t);
    }
    *score = scale * sv * dot;
    *score_abs = fabs(scale * sv) * dabs;
}

int oracle_fusedmm(int64_t M, int64_t N, int64_t K, int64_t H,
                   const int32_t* rowptr, const int32_t* colidx, const double* vals,
                   double scale, int row_softmax, int abs_mode,
                   int dta, const void* A, int64_t lda, int dtb, const void* B, int64_t ldb,
                   int64_t nrows, const int64_t* rows, double* Y, double* scores, double* lse)
{
    if (H < 1 || K % H != 0) return 3;
    int64_t D = K / H, nnz = rowptr[M];
    int64_t count = rows ? nrows : M;
    for (int64_t q = 0; q < count; ++q) {
        int64_t i = rows ? rows[q] : q;
        if (i < 0 || i >= M) return 1;
        double* y = Y + q * K;
        for (int64_t k = 0; k < K; ++k) y[k] = 0.0;
        for (int64_t h = 0; h < H; ++h) {
            int64_t k0 = h * D;
            double m = -INFINITY, l = 0.0, sc, sa;
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                int64_t j = colidx[e];
                if (j < 0 || j >= N) return 2;
                head_score(dta, A, lda, dtb, B, ldb, i, j, k0, D, vals ? vals[e] : 1.0, scale, &sc, &sa);
                if (scores) scores[h * nnz + e] = sc;
                if (sc > m) m = sc;
            }
            if (row_softmax)
                for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                    head_score(dta, A, lda, dtb, B, ldb, i, colidx[e], k0, D, vals ? vals[e] : 1.0, scale, &sc, &sa);
                    l += exp(sc - m);
                }
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                int64_t j = colidx[e];
                head_score(dta, A, lda, dtb, B, ldb, i, j, k0, D, vals ? vals[e] : 1.0, scale, &sc, &sa);
                double w = row_softmax ? exp(sc - m) / l : sc;
                double wa = row_softmax ? w : sa;
                for (int64_t k = k0; k < k0 + D; ++k) {
                    double b = elem(dtb, B, j * ldb + k, NULL, j);
                    y[k] += abs_mode ? wa * fabs(b) : w * b;
                }
            }
            if (lse) lse[q * H + h] = (rowptr[i + 1] > rowptr[i]) ? m + log(l) : -INFINITY;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* SpMM with the transpose: X[q,:] = sum_{e=(i,j), j = cols[q]} s_e * Y[i,:]. */
/* A direct scatter over the nonzeros in CSR order; it builds no transpose.  */
/* ------------------------------------------------------------------------- */
int oracle_spmm_t(int64_t M, int64_t N, int64_t K,
                  const int32_t* rowptr, const int32_t* colidx,
                  const double* vals, const double* vals2, int abs_mode,
                  int dty, const void* Y, int64_t ldy, const float* y_scale,
                  int64_t ncols, const int64_t* cols, double* X)
{
    int64_t count = cols ? ncols : N;
    int64_t* slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    if (!slot) return 3;
    for (int64_t j = 0; j < N; ++j) slot[j] = cols ? -1 : j;
    for (int64_t q = 0; cols && q < count; ++q) {
        if (cols[q] < 0 || cols[q] >= N) { free(slot); return 1; }
        slot[cols[q]] = q;
    }
    for (int64_t q = 0; q < count * K; ++q) X[q] = 0.0;
    for (int64_t i = 0; i < M; ++i) {
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            int64_t j = colidx[e];
            if (j < 0 || j >= N) { free(slot); return 2; }
            int64_t q = slot[j];
            if (q < 0) continue;
            double s = sval(vals, vals2, e);
            for (int64_t k = 0; k < K; ++k) {
                double t = s * elem(dty, Y, i * ldy + k, y_scale, i);
                X[q * K + k] += abs_mode ? fabs(t) : t;
            }
        }
    }
    free(slot);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Transpose by a stable counting sort on the column index.                  */
/* colptr[N+1], rowidx[nnz]: the CSC pattern; perm[p] = CSR slot of CSC slot */
/* p.  Within a column the entries keep their CSR (row-major) order.         */
/* ------------------------------------------------------------------------- */
int oracle_transpose(int64_t M, int64_t N, const int32_t* rowptr, const int32_t* colidx,
                     int32_t* colptr, int32_t* rowidx, int32_t* perm)
{
    int64_t nnz = rowptr[M];
    int64_t* cursor = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    if (!cursor) return 3;
    for (int64_t e = 0; e < nnz; ++e) {
        if (colidx[e] < 0 || colidx[e] >= N) { free(cursor); return 2; }
        cursor[colidx[e] + 1]++;
    }
    for (int64_t j = 0; j < N; ++j) cursor[j + 1] += cursor[j];
    for (int64_t j = 0; j <= N; ++j) colptr[j] = (int32_t)cursor[j];
    for (int64_t i = 0; i < M; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            int64_t p = cursor[colidx[e]]++;
            rowidx[p] = (int32_t)i;
            perm[p] = (int32_t)e;
        }
    free(cursor);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Merge path: walk d steps of the merge of the row-end offsets              */
/* rowptr[1..M] with the nonzero indices 0..nnz-1.  A row end is taken first */
/* when it is <= the next nonzero index (row r is finished once all of its   */
/* nonzeros were consumed).  Returns (rows finished, nonzeros consumed).     */
/* ------------------------------------------------------------------------- */
void oracle_merge_path(int64_t M, const int32_t* rowptr, int64_t d, int64_t* r_out, int64_t* e_out)
{
    int64_t r = 0, e = 0, nnz = rowptr[M];
    for (int64_t step = 0; step < d; ++step) {
        if (r < M && rowptr[r + 1] <= e) r++;
        else if (e < nnz) e++;
        else r++;
    }
    *r_out = r;
    *e_out = e;
}

/* ------------------------------------------------------------------------- */
/* COO -> CSR.  S given by coordinates (Sec. 3.1: the nonzeros s_ij of an    */
/* M x N matrix) is put in row-major order: entries ordered by (row, column),*/
/* ties in input order, by two stable counting sorts (column, then row).     */
/* dedup 0 keeps every entry; 1 keeps the first entry (in input order) of    */
/* each repeated (row, column); 2 keeps one entry whose value is the sum of  */
/* the repeated entries' values (in double).  vals / vals_out may be NULL.   */
/* Writes rowptr[M+1], colidx / vals_out[nnz_out]; returns 1 on an index out */
/* of range, 3 on allocation failure.                                        */
/* ------------------------------------------------------------------------- */
int oracle_coo_to_csr(int64_t M, int64_t N, int64_t nnz, const int32_t* rows, const int32_t* cols,
                      const double* vals, int dedup, int32_t* rowptr, int32_t* colidx, double* vals_out,
                      int64_t* nnz_out)
{
    int64_t* by_col = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t* cnt = (int64_t*)calloc((size_t)((M > N ? M : N) + 1), sizeof(int64_t));
    if (!by_col || !order || !cnt) { free(by_col); free(order); free(cnt); return 3; }
    for (int64_t e = 0; e < nnz; ++e)
        if (rows[e] < 0 || rows[e] >= M || cols[e] < 0 || cols[e] >= N) {
            free(by_col); free(order); free(cnt);
            return 1;
        }
    /* stable counting sort by column */
    for (int64_t e = 0; e < nnz; ++e) cnt[cols[e] + 1]++;
    for (int64_t j = 0; j < N; ++j) cnt[j + 1] += cnt[j];
    for (int64_t e = 0; e < nnz; ++e) by_col[cnt[cols[e]]++] = e;
    /* stable counting sort of that order by row */
    memset(cnt, 0, sizeof(int64_t) * (size_t)((M > N ? M : N) + 1));
    for (int64_t e = 0; e < nnz; ++e) cnt[rows[e] + 1]++;
    for (int64_t i = 0; i < M; ++i) cnt[i + 1] += cnt[i];
    for (int64_t q = 0; q < nnz; ++q) {
        int64_t e = by_col[q];
        order[cnt[rows[e]]++] = e;
    }
    /* emit, merging repeats */
    int64_t n = 0;
    for (int64_t i = 0; i <= M; ++i) rowptr[i] = 0;
    for (int64_t q = 0; q < nnz; ++q) {
        int64_t e = order[q];
        int repeat = q > 0 && rows[order[q - 1]] == rows[e] && cols[order[q - 1]] == cols[e];
        if (dedup && repeat) {
            if (dedup == 2 && vals && vals_out) vals_out[n - 1] += vals[e];
            continue;
        }
        colidx[n] = cols[e];
        if (vals_out) vals_out[n] = vals ? vals[e] : 1.0;
        rowptr[rows[e] + 1]++;
        n++;
    }
    for (int64_t i = 0; i < M; ++i) rowptr[i + 1] += rowptr[i];
    *nnz_out = n;
    free(by_col); free(order); free(cnt);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Reverse Cuthill-McKee order of a square pattern (Cuthill & McKee 1969,    */
/* reversed as George 1971 proposed), on the symmetric graph with an edge    */
/* i - j for every stored (i, j), i != j (repeats count in the degree).      */
/* Components are started, in turn, from the unvisited vertex of smallest    */
/* (degree, index); a vertex's unvisited neighbours are queued by (degree,   */
/* index).  perm[p] = vertex at position p of the reversed visiting order.   */
/* ------------------------------------------------------------------------- */
static const int64_t* g_rcm_deg;
static int rcm_cmp(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    if (g_rcm_deg[x] != g_rcm_deg[y]) return g_rcm_deg[x] < g_rcm_deg[y] ? -1 : 1;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int oracle_rcm(int64_t M, const int32_t* rowptr, const int32_t* colidx, int32_t* perm)
{
    int64_t nnz = rowptr[M];
    int64_t* deg = (int64_t*)calloc((size_t)M + 1, sizeof(int64_t));
    int64_t* start = (int64_t*)calloc((size_t)M + 1, sizeof(int64_t));
    int64_t* adj = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * nnz + 1));
    int64_t* fill = (int64_t*)calloc((size_t)M + 1, sizeof(int64_t));
    int64_t* byd = (int64_t*)malloc(sizeof(int64_t) * (size_t)(M + 1));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(M + 1));
    char* seen = (char*)calloc((size_t)M + 1, 1);
    if (!deg || !start || !adj || !fill || !byd || !order || !seen) {
        free(deg); free(start); free(adj); free(fill); free(byd); free(order); free(seen);
        return 3;
    }
    for (int64_t i = 0; i < M; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            int64_t j = colidx[e];
            if (j < 0 || j >= M) { free(deg); free(start); free(adj); free(fill); free(byd); free(order); free(seen); return 2; }
            if (j != i) { deg[i]++; deg[j]++; }
        }
    for (int64_t i = 0; i < M; ++i) start[i + 1] = start[i] + deg[i];
    for (int64_t i = 0; i < M; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            int64_t j = colidx[e];
            if (j == i) continue;
            adj[start[i] + fill[i]++] = j;
            adj[start[j] + fill[j]++] = i;
        }
    g_rcm_deg = deg;
    for (int64_t i = 0; i < M; ++i) byd[i] = i;
    qsort(byd, (size_t)M, sizeof(int64_t), rcm_cmp);
    int64_t head = 0, tail = 0, next_start = 0;
    while (tail < M) {
        while (seen[byd[next_start]]) next_start++;
        int64_t s = byd[next_start];
        seen[s] = 1;
        order[tail++] = s;
        while (head < tail) {
            int64_t v = order[head++];
            int64_t first = tail;
            for (int64_t q = start[v]; q < start[v + 1]; ++q) {
                int64_t w = adj[q];
                if (!seen[w]) { seen[w] = 1; order[tail++] = w; }
            }
            qsort(order + first, (size_t)(tail - first), sizeof(int64_t), rcm_cmp);
        }
    }
    for (int64_t p = 0; p < M; ++p) perm[p] = (int32_t)order[M - 1 - p];
    free(deg); free(start); free(adj); free(fill); free(byd); free(order); free(seen);
    return 0;
}
