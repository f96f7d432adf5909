/*
 * hec_oracle.c -- the CPU oracle for the level-scheduled HEC triangular solver.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, serial, slow and deliberately obvious FP64 code on CSR
 * matrices.  It exists so the CUDA path can be checked against an independent statement of
 * the mathematics.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it; the product library never links, includes or calls anything here, and nothing
 * here includes or calls the product.
 *
 * Conventions: 0-based int32 indices; every CSR row is sorted by ascending column (Sec. 2:
 * "each row of L and U is sorted in ascending order").  Functions return 0 on success and a
 * negative code on malformed input:
 *   -1 entry on the wrong side of the diagonal, -2 missing diagonal, -3 zero pivot,
 *   -4 unsorted row / bad column, -5 bad argument, -6 out of memory.
 *
 * Every function cites the passage of the paper (Chen, Liu, Yang, "Parallel Triangular
 * Solvers on GPU", arXiv 1606.00541) or the textbook definition it restates.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EXPORT __attribute__((visibility("default")))

enum { OR_ERR_SIDE = -1, OR_ERR_NODIAG = -2, OR_ERR_PIVOT = -3, OR_ERR_UNSORTED = -4,
       OR_ERR_ARG = -5, OR_ERR_OOM = -6 };

/* ------------------------------------------------------------------------------------- */
/* Input checks (Sec. 2: rows sorted ascending)                                            */
/* ------------------------------------------------------------------------------------- */

/* uplo: 0 lower, 1 upper.  Checks sortedness, triangularity and a nonzero diagonal. */
OR_EXPORT int or_check_triangular(int n, const int* rp, const int* ci, const double* v, int uplo)
{
    if (n < 0) return OR_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        int has_diag = 0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int j = ci[p];
            if (j < 0 || j >= n) return OR_ERR_UNSORTED;
            if (p > rp[i] && ci[p - 1] >= j) return OR_ERR_UNSORTED;
            if (uplo == 0 && j > i) return OR_ERR_SIDE;
            if (uplo == 1 && j < i) return OR_ERR_SIDE;
            if (j == i) {
                has_diag = 1;
                if (v && v[p] == 0.0) return OR_ERR_PIVOT;
            }
        }
        if (!has_diag) return OR_ERR_NODIAG;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Forward and back substitution (Eq. 1: L y = b, then U x = y)                            */
/* ------------------------------------------------------------------------------------- */

/* Forward substitution: for i ascending, y_i = (b_i - sum_{j<i} L_ij y_j) / L_ii, the sum
 * taken in ascending j.  This is the exact result that any level schedule reaches. */
OR_EXPORT int or_lower_solve(int n, const int* rp, const int* ci, const double* v,
                             const double* b, double* y)
{
    for (int i = 0; i < n; ++i) {
        double s = b[i], d = 0.0;
        int has_diag = 0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int j = ci[p];
            if (j < i) s -= v[p] * y[j];
            else if (j == i) { d = v[p]; has_diag = 1; }
            else return OR_ERR_SIDE;
        }
        if (!has_diag) return OR_ERR_NODIAG;
        if (d == 0.0) return OR_ERR_PIVOT;
        y[i] = s / d;
    }
    return 0;
}

/* Back substitution: for i descending, x_i = (y_i - sum_{j>i} U_ij x_j) / U_ii. */
OR_EXPORT int or_upper_solve(int n, const int* rp, const int* ci, const double* v,
                             const double* y, double* x)
{
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i], d = 0.0;
        int has_diag = 0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int j = ci[p];
            if (j > i) s -= v[p] * x[j];
            else if (j == i) { d = v[p]; has_diag = 1; }
            else return OR_ERR_SIDE;
        }
        if (!has_diag) return OR_ERR_NODIAG;
        if (d == 0.0) return OR_ERR_PIVOT;
        x[i] = s / d;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Levels (Eq. 2), level sets and the map m (Eq. 3), upper factor by reversal (Sec. 2.2)   */
/* ------------------------------------------------------------------------------------- */

/* Eq. 2 with the diagonal excluded from the dependencies: the paper level of row i is
 * 1 + max l(j) over the off-diagonal entries L_ij (j < i), l(j) starting at 0, so a row with
 * no off-diagonal entry gets paper level 1.  The level returned here is the paper level minus
 * one (0-based).
 *
 * For the upper factor the paper turns U x = b into a lower problem by reversing the index
 * order.  With 0-based indices that reversal is t(i) = n-1-i: row t of the reversed matrix
 * is row n-1-t of U and its dependencies are the columns j > i of U.  level[i] is returned for
 * the ORIGINAL row i in both cases.  Returns the number of levels (>= 0) or a negative code. */
OR_EXPORT int or_levels(int n, const int* rp, const int* ci, int uplo, int* level)
{
    if (n < 0 || (uplo != 0 && uplo != 1)) return OR_ERR_ARG;
    int* pl = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1)); /* paper level, 1-based */
    if (!pl) return OR_ERR_OOM;
    for (int i = 0; i < n; ++i) pl[i] = 0; /* "l(i) is zero initially" */
    int nlev = 0;
    for (int t = 0; t < n; ++t) {
        int i = uplo == 0 ? t : n - 1 - t; /* visit rows in the order of the lower problem */
        int mx = 0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int j = ci[p];
            int dep = uplo == 0 ? (j < i) : (j > i);
            if (dep && pl[j] > mx) mx = pl[j];
        }
        pl[i] = 1 + mx;
        if (pl[i] > nlev) nlev = pl[i];
    }
    for (int i = 0; i < n; ++i) level[i] = pl[i] - 1;
    free(pl);
    return nlev;
}

/* Eq. 3.  S_k = rows of level k, each set in ascending order of the lower problem's index
 * (for U that index is t = n-1-i); N_k = |S_k|; m(i) = N_0 + ... + N_{k-1} + p_k(i), with
 * p_k(i) the 0-based position of i in S_k.  Outputs perm[i] = m(i) for the original row i,
 * iperm (its inverse) and level_ptr[k] = N_0 + ... + N_{k-1}, k = 0..nlev. */
OR_EXPORT int or_level_map(int n, const int* level, int nlev, int uplo,
                           int* perm, int* iperm, int* level_ptr)
{
    if (n < 0 || nlev < 0) return OR_ERR_ARG;
    int* N = (int*)calloc((size_t)nlev + 1, sizeof(int));
    int* fill = (int*)calloc((size_t)nlev + 1, sizeof(int));
    if (!N || !fill) { free(N); free(fill); return OR_ERR_OOM; }
    for (int i = 0; i < n; ++i) {
        if (level[i] < 0 || level[i] >= nlev) { free(N); free(fill); return OR_ERR_ARG; }
        N[level[i]]++;
    }
    level_ptr[0] = 0;
    for (int k = 0; k < nlev; ++k) level_ptr[k + 1] = level_ptr[k] + N[k];
    for (int t = 0; t < n; ++t) { /* ascending index of the lower problem */
        int i = uplo == 0 ? t : n - 1 - t;
        int k = level[i];
        int pk = fill[k]++; /* position of i in S_k */
        perm[i] = level_ptr[k] + pk;
    }
    for (int i = 0; i < n; ++i) iperm[perm[i]] = i;
    free(N);
    free(fill);
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Value rounding for reduced-precision factor storage                                     */
/* ------------------------------------------------------------------------------------- */

/* FP64 -> FP32, round to nearest, ties to even (the C conversion under the default mode). */
OR_EXPORT uint32_t or_round_f32_bits(double d)
{
    float f = (float)d;
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* FP64 -> BF16 (8 significant bits, FP32 exponent range), round to nearest, ties to even,
 * taken directly from the double (no intermediate FP32 rounding).  Written from the
 * definition: scale d so that one bf16 unit in the last place is 1, round to the nearest
 * integer with ties to even (nearbyint under the default mode), scale back.  Returns the
 * 16-bit pattern. */
OR_EXPORT uint32_t or_round_bf16_bits(double d)
{
    if (isnan(d)) return 0x7FC0u;
    uint32_t sign = signbit(d) ? 0x8000u : 0u;
    double a = fabs(d);
    if (isinf(a)) return sign | 0x7F80u;
    if (a == 0.0) return sign;
    int e;
    frexp(a, &e);            /* a = m * 2^e, 0.5 <= m < 1, so the leading bit has weight 2^(e-1) */
    int lead = e - 1;
    if (lead < -126) lead = -126;          /* subnormal range: fixed spacing 2^-133 */
    int ulp_exp = lead - 7;                /* 8 significant bits */
    double q = nearbyint(ldexp(a, -ulp_exp)); /* exact scaling, RNE rounding */
    double r = ldexp(q, ulp_exp);
    if (r >= ldexp(1.0, 128)) return sign | 0x7F80u; /* overflow to infinity */
    /* encode r: it is exactly representable in bf16 */
    float f = (float)r;
    uint32_t u;
    memcpy(&u, &f, 4);
    return sign | ((u >> 16) & 0x7FFFu);
}

/* Array form of or_round_bf16_bits. */
OR_EXPORT void or_round_bf16_array(long n, const double* in, uint16_t* out)
{
    for (long i = 0; i < n; ++i) out[i] = (uint16_t)or_round_bf16_bits(in[i]);
}

static double bf16_bits_to_double(uint32_t h)
{
    uint32_t u = (h & 0xFFFFu) << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double f32_bits_to_double(uint32_t u)
{
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* ------------------------------------------------------------------------------------- */
/* HEC format (Sec. 2.1): column-major ELL slab + CSR tail holding at least the diagonal   */
/* ------------------------------------------------------------------------------------- */

/* The paper leaves the ELL width rule open.  The rule used throughout: the largest w such
 * that at least ceil(0.65 n) rows have w or more entries eligible for the slab (so at most
 * 35% of every slab column is padding).  count[i] = eligible entries of row i. */
OR_EXPORT int or_ell_width_rule(int n, const int* count)
{
    if (n <= 0) return 0;
    long need = (65L * n + 99) / 100; /* ceil(0.65 n) in exact integer arithmetic */
    int best = 0;
    for (int w = 1;; ++w) {
        long rows = 0;
        for (int i = 0; i < n; ++i) if (count[i] >= w) rows++;
        if (rows >= need) best = w; else break;
    }
    return best;
}

OR_EXPORT int or_round_up32(int n) { return (n + 31) / 32 * 32; }

static void store_val(void* dst, long idx, double v, int vdt)
{
    if (vdt == 0) ((double*)dst)[idx] = v;
    else if (vdt == 1) ((uint32_t*)dst)[idx] = or_round_f32_bits(v);
    else ((uint16_t*)dst)[idx] = (uint16_t)or_round_bf16_bits(v);
}

static double load_val(const void* src, long idx, int vdt)
{
    if (vdt == 0) return ((const double*)src)[idx];
    if (vdt == 1) return f32_bits_to_double(((const uint32_t*)src)[idx]);
    return bf16_bits_to_double(((const uint16_t*)src)[idx]);
}

/* Size query for HEC packing.  tri = 1: triangular factor (uplo 0/1) reordered by perm, the
 * diagonal held back for the tail; tri = 0: general matrix in its own order (perm ignored),
 * every entry eligible for the slab.  w < 0 selects the width rule.  Outputs the width and
 * the tail length. */
OR_EXPORT int or_hec_sizes(int n, const int* rp, const int* ci, int tri, int w_req,
                           int* w_out, long* tail_nnz)
{
    (void)ci;
    int* cnt = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
    if (!cnt) return OR_ERR_OOM;
    for (int i = 0; i < n; ++i) {
        int c = rp[i + 1] - rp[i];
        if (tri) c -= 1; /* the diagonal always goes to the tail */
        cnt[i] = c;
    }
    int w = w_req >= 0 ? w_req : or_ell_width_rule(n, cnt);
    long t = 0;
    for (int i = 0; i < n; ++i) {
        int over = cnt[i] > w ? cnt[i] - w : 0;
        t += over + (tri ? 1 : 0);
    }
    free(cnt);
    *w_out = w;
    *tail_nnz = t;
    return 0;
}

/* Alg. 1, steps 3-4: reorder L to L' (L_ij -> L'_{m(i) m(j)}) and convert L' to HEC.
 * Reading used where the paper is silent: each row of L' is re-sorted by ascending new
 * column; its first w off-diagonal entries go to ELL slots 0..w-1 (entry k of row r stored at
 * k*ld + r, ld = round_up(n,32)); unused slots, and all slots of rows n..ld-1, hold column -1
 * and value +0.0; the remaining off-diagonals follow in the tail in ascending new column, and
 * the diagonal is the last tail entry of its row.  For tri = 0 (a general matrix, no
 * reordering) the row keeps its CSR order, the first w entries go to the slab and the rest to
 * the tail, which may then be empty for a row.  vdt: 0 FP64, 1 FP32, 2 BF16 (values rounded
 * once, to nearest even).  The caller sizes ell_* as w*ld and the tail from or_hec_sizes. */
OR_EXPORT int or_hec_pack(int n, const int* rp, const int* ci, const double* v, int tri, int uplo,
                          const int* perm, const int* iperm, int w, int vdt,
                          int* ell_col, void* ell_val, int* tptr, int* tcol, void* tval)
{
    if (n < 0 || w < 0 || vdt < 0 || vdt > 2) return OR_ERR_ARG;
    int ld = or_round_up32(n);
    for (long s = 0; s < (long)w * ld; ++s) { ell_col[s] = -1; store_val(ell_val, s, 0.0, vdt); }
    int maxlen = 0;
    for (int i = 0; i < n; ++i) if (rp[i + 1] - rp[i] > maxlen) maxlen = rp[i + 1] - rp[i];
    int* rc = (int*)malloc(sizeof(int) * (size_t)(maxlen + 1));
    double* rv = (double*)malloc(sizeof(double) * (size_t)(maxlen + 1));
    if (!rc || !rv) { free(rc); free(rv); return OR_ERR_OOM; }
    tptr[0] = 0;
    for (int r = 0; r < n; ++r) {
        int i = tri ? iperm[r] : r; /* original row stored as new row r */
        int cnt = 0;
        double diag = 0.0;
        int has_diag = 0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int j = ci[p];
            if (tri && j == i) { diag = v[p]; has_diag = 1; continue; }
            if (tri && (uplo == 0 ? j > i : j < i)) { free(rc); free(rv); return OR_ERR_SIDE; }
            rc[cnt] = tri ? perm[j] : j;
            rv[cnt] = v[p];
            cnt++;
        }
        if (tri && !has_diag) { free(rc); free(rv); return OR_ERR_NODIAG; }
        if (tri) { /* insertion sort by new column */
            for (int a = 1; a < cnt; ++a) {
                int c = rc[a]; double x = rv[a]; int b = a - 1;
                while (b >= 0 && rc[b] > c) { rc[b + 1] = rc[b]; rv[b + 1] = rv[b]; --b; }
                rc[b + 1] = c; rv[b + 1] = x;
            }
        }
        int t = tptr[r];
        for (int k = 0; k < cnt; ++k) {
            if (k < w) {
                ell_col[(long)k * ld + r] = rc[k];
                store_val(ell_val, (long)k * ld + r, rv[k], vdt);
            } else {
                tcol[t] = rc[k];
                store_val(tval, t, rv[k], vdt);
                t++;
            }
        }
        if (tri) { tcol[t] = r; store_val(tval, t, diag, vdt); t++; }
        tptr[r + 1] = t;
    }
    free(rc);
    free(rv);
    return 0;
}

/* Inverse of or_hec_pack: rebuild the CSR of the ORIGINAL matrix (original row and column
 * numbers, rows sorted ascending) from HEC, values widened back to FP64.  out_rp has n+1
 * entries; out_ci/out_v are sized for nnz.  Used by round-trip checks. */
OR_EXPORT int or_hec_unpack(int n, int w, const int* ell_col, const void* ell_val, const int* tptr,
                            const int* tcol, const void* tval, int tri, const int* iperm, int vdt,
                            int* out_rp, int* out_ci, double* out_v)
{
    int ld = or_round_up32(n);
    int* len = (int*)calloc((size_t)n + 1, sizeof(int));
    if (!len) return OR_ERR_OOM;
    for (int r = 0; r < n; ++r) {
        int i = tri ? iperm[r] : r;
        int c = 0;
        for (int k = 0; k < w; ++k) if (ell_col[(long)k * ld + r] >= 0) c++;
        c += tptr[r + 1] - tptr[r];
        len[i] = c;
    }
    out_rp[0] = 0;
    for (int i = 0; i < n; ++i) out_rp[i + 1] = out_rp[i] + len[i];
    for (int r = 0; r < n; ++r) {
        int i = tri ? iperm[r] : r;
        int q = out_rp[i];
        for (int k = 0; k < w; ++k) {
            long s = (long)k * ld + r;
            if (ell_col[s] < 0) continue;
            out_ci[q] = tri ? iperm[ell_col[s]] : ell_col[s];
            out_v[q] = load_val(ell_val, s, vdt);
            q++;
        }
        for (int p = tptr[r]; p < tptr[r + 1]; ++p) {
            out_ci[q] = tri ? iperm[tcol[p]] : tcol[p];
            out_v[q] = load_val(tval, p, vdt);
            q++;
        }
        /* restore ascending original column order */
        int b0 = out_rp[i], e0 = out_rp[i + 1];
        for (int a = b0 + 1; a < e0; ++a) {
            int c = out_ci[a]; double x = out_v[a]; int b = a - 1;
            while (b >= b0 && out_ci[b] > c) { out_ci[b + 1] = out_ci[b]; out_v[b + 1] = out_v[b]; --b; }
            out_ci[b + 1] = c; out_v[b + 1] = x;
        }
    }
    free(len);
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* SpMV and incomplete factorizations (Sec. 3)                                             */
/* ------------------------------------------------------------------------------------- */

/* y = A x, each row summed in CSR order. */
OR_EXPORT void or_spmv(int n, const int* rp, const int* ci, const double* v, const double* x, double* y)
{
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) s += v[p] * x[ci[p]];
        y[i] = s;
    }
}

/* Split an in-place LU (on a pattern that contains every diagonal) into L (unit lower, the
 * 1.0 diagonal stored explicitly so every row of L has its diagonal, as the HEC tail needs)
 * and U (upper with its diagonal).  Output arrays sized by the caller: L and U each get at
 * most nnz + n entries. */
static void split_lu(int n, const int* rp, const int* ci, const double* lu,
                     int* Lrp, int* Lci, double* Lv, int* Urp, int* Uci, double* Uv)
{
    int lq = 0, uq = 0;
    Lrp[0] = 0; Urp[0] = 0;
    for (int i = 0; i < n; ++i) {
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int j = ci[p];
            if (j < i) { Lci[lq] = j; Lv[lq] = lu[p]; lq++; }
        }
        Lci[lq] = i; Lv[lq] = 1.0; lq++;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int j = ci[p];
            if (j >= i) { Uci[uq] = j; Uv[uq] = lu[p]; uq++; }
        }
        Lrp[i + 1] = lq; Urp[i + 1] = uq;
    }
}

/* Numeric incomplete LU restricted to a given pattern (IKJ Gaussian elimination, Saad's
 * "ILU(0)" algorithm, Sec. 3): for each row i, for each k < i in the pattern of row i in
 * ascending order: a_ik <- a_ik / a_kk; then a_ij <- a_ij - a_ik a_kj for every j > k that
 * is in the pattern of both row i and row k.  The pattern must hold every diagonal.  lu is
 * overwritten with the factors on the pattern. */
static int ilu_on_pattern(int n, const int* rp, const int* ci, double* lu)
{
    int* pos = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int* dg = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!pos || !dg) { free(pos); free(dg); return OR_ERR_OOM; }
    for (int j = 0; j < n; ++j) pos[j] = -1;
    for (int i = 0; i < n; ++i) {
        dg[i] = -1;
        for (int p = rp[i]; p < rp[i + 1]; ++p) if (ci[p] == i) dg[i] = p;
        if (dg[i] < 0) { free(pos); free(dg); return OR_ERR_NODIAG; }
    }
    for (int i = 0; i < n; ++i) {
        for (int p = rp[i]; p < rp[i + 1]; ++p) pos[ci[p]] = p;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int k = ci[p];
            if (k >= i) break;
            double piv = lu[dg[k]];
            if (piv == 0.0) { free(pos); free(dg); return OR_ERR_PIVOT; }
            lu[p] = lu[p] / piv;
            for (int q = dg[k] + 1; q < rp[k + 1]; ++q) {
                int j = ci[q];
                if (pos[j] >= 0) lu[pos[j]] -= lu[p] * lu[q];
            }
        }
        if (lu[dg[i]] == 0.0) { free(pos); free(dg); return OR_ERR_PIVOT; }
        for (int p = rp[i]; p < rp[i + 1]; ++p) pos[ci[p]] = -1;
    }
    free(pos);
    free(dg);
    return 0;
}

/* ILU(0) (Sec. 3: "if no fill-in is allowed").  L and U output arrays hold nnz(A) + n
 * entries at most; Lrp/Urp have n+1 entries. */
OR_EXPORT int or_ilu0(int n, const int* rp, const int* ci, const double* v,
                      int* Lrp, int* Lci, double* Lv, int* Urp, int* Uci, double* Uv)
{
    long nnz = rp[n];
    double* lu = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    if (!lu) return OR_ERR_OOM;
    memcpy(lu, v, sizeof(double) * (size_t)nnz);
    int rc = ilu_on_pattern(n, rp, ci, lu);
    if (rc == 0) split_lu(n, rp, ci, lu, Lrp, Lci, Lv, Urp, Uci, Uv);
    free(lu);
    return rc;
}

/* Symbolic ILU(k) (Sec. 3, "k is the fill-in level"): level of fill lev(i,j) = 0 on the
 * pattern of A; eliminating row i with pivot k (processed in ascending order, including
 * fill created earlier in the same row) gives fill lev(i,j) = min(lev(i,j), lev(i,k) +
 * lev(k,j) + 1) for j > k in row k of the factor; entries with lev <= K are kept.  Pass
 * out_rp only (out_ci NULL) to count: out_rp[n] is then the nnz.  Call again with out_ci to
 * fill the sorted pattern. */
OR_EXPORT int or_iluk_symbolic(int n, const int* rp, const int* ci, int K,
                               int* out_rp, int* out_ci)
{
    if (n < 0 || K < 0) return OR_ERR_ARG;
    /* Per-row factor pattern + levels, kept for use by later rows. */
    int** rows = (int**)calloc((size_t)(n > 0 ? n : 1), sizeof(int*));
    int** levs = (int**)calloc((size_t)(n > 0 ? n : 1), sizeof(int*));
    int* rlen = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
    int* lev = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1)); /* dense work: level or -1 */
    int* next = (int*)malloc(sizeof(int) * (size_t)(n + 1));        /* sorted linked list */
    if (!rows || !levs || !rlen || !lev || !next) goto oom;
    for (int j = 0; j < n; ++j) lev[j] = -1;
    out_rp[0] = 0;
    for (int i = 0; i < n; ++i) {
        /* list head is index n; columns linked in ascending order */
        int head = n;
        next[head] = -1;
        int tail = head;
        int has_diag = 0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int j = ci[p];
            lev[j] = 0;
            next[tail] = j; next[j] = -1; tail = j;
            if (j == i) has_diag = 1;
        }
        if (!has_diag) { /* the factor pattern always holds the diagonal */
            int prev = head;
            while (next[prev] != -1 && next[prev] < i) prev = next[prev];
            next[i] = next[prev]; next[prev] = i; lev[i] = 0;
        }
        for (int k = next[head]; k != -1 && k < i; k = next[k]) {
            int lik = lev[k];
            /* row k of the factor: its U part, columns > k */
            int prev = k;
            for (int q = 0; q < rlen[k]; ++q) {
                int j = rows[k][q];
                if (j <= k) continue;
                int nl = lik + levs[k][q] + 1;
                if (nl > K) continue;
                if (lev[j] < 0) { /* new fill: insert in sorted position after prev */
                    while (next[prev] != -1 && next[prev] < j) prev = next[prev];
                    next[j] = next[prev]; next[prev] = j;
                    lev[j] = nl;
                } else if (nl < lev[j]) {
                    lev[j] = nl;
                }
                prev = j; /* j is in the list now and later columns of row k are larger */
            }
        }
        int len = 0;
        for (int j = next[head]; j != -1; j = next[j]) len++;
        rows[i] = (int*)malloc(sizeof(int) * (size_t)(len > 0 ? len : 1));
        levs[i] = (int*)malloc(sizeof(int) * (size_t)(len > 0 ? len : 1));
        if (!rows[i] || !levs[i]) goto oom;
        int q = 0;
        for (int j = next[head]; j != -1; j = next[j]) { rows[i][q] = j; levs[i][q] = lev[j]; q++; }
        rlen[i] = len;
        for (int j = next[head]; j != -1; j = next[j]) lev[j] = -1;
        out_rp[i + 1] = out_rp[i] + len;
        if (out_ci) memcpy(out_ci + out_rp[i], rows[i], sizeof(int) * (size_t)len);
    }
    for (int i = 0; i < n; ++i) { free(rows[i]); free(levs[i]); }
    free(rows); free(levs); free(rlen); free(lev); free(next);
    return 0;
oom:
    if (rows) for (int i = 0; i < n; ++i) free(rows[i]);
    if (levs) for (int i = 0; i < n; ++i) free(levs[i]);
    free(rows); free(levs); free(rlen); free(lev); free(next);
    return OR_ERR_OOM;
}

/* ILU(k) numeric: the ILU(0) elimination on the ILU(k) pattern, with A's values scattered
 * into it (fill starts at 0).  prp/pci is the pattern from or_iluk_symbolic. */
OR_EXPORT int or_iluk_numeric(int n, const int* rp, const int* ci, const double* v,
                              const int* prp, const int* pci,
                              int* Lrp, int* Lci, double* Lv, int* Urp, int* Uci, double* Uv)
{
    long nnz = prp[n];
    double* lu = (double*)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
    if (!lu) return OR_ERR_OOM;
    for (int i = 0; i < n; ++i) {
        int q = prp[i];
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            while (q < prp[i + 1] && pci[q] < ci[p]) q++;
            if (q < prp[i + 1] && pci[q] == ci[p]) lu[q] = v[p];
            else { free(lu); return OR_ERR_UNSORTED; }
        }
    }
    int rc = ilu_on_pattern(n, prp, pci, lu);
    if (rc == 0) split_lu(n, prp, pci, lu, Lrp, Lci, Lv, Urp, Uci, Uv);
    free(lu);
    return rc;
}

/* ILUT(p, tol), Saad's dual-threshold incomplete LU (Sec. 3: dropping by value tol and by a
 * maximum number p of nonzeros per row).  Reading used: tau_i = tol * ||a_i,:||_2; while
 * row i is eliminated (pivots k < i in ascending order, fill included), a multiplier w_k with
 * |w_k| < tau_i is dropped and not used; afterwards every off-diagonal with |w_j| < tau_i is
 * dropped, then the p largest magnitudes are kept in the strict lower part and the p largest
 * in the strict upper part (ties to the smaller column); the diagonal is always kept.  L is
 * unit lower with its 1.0 diagonal stored.  Call with Lci == NULL to get the sizes in
 * Lrp[n], Urp[n] (the factorization is run either way). */
OR_EXPORT int or_ilut(int n, const int* rp, const int* ci, const double* v, int p_keep, double tol,
                      int* Lrp, int* Lci, double* Lv, int* Urp, int* Uci, double* Uv)
{
    if (n < 0 || p_keep < 0 || tol < 0) return OR_ERR_ARG;
    double* w = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int* in = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int* next = (int*)malloc(sizeof(int) * (size_t)(n + 1));
    int* cand = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    /* U rows kept so far (needed by later rows) */
    int** Ur = (int**)calloc((size_t)(n > 0 ? n : 1), sizeof(int*));
    double** Uw = (double**)calloc((size_t)(n > 0 ? n : 1), sizeof(double*));
    int* Ul = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
    int** Lr = (int**)calloc((size_t)(n > 0 ? n : 1), sizeof(int*));
    double** Lw = (double**)calloc((size_t)(n > 0 ? n : 1), sizeof(double*));
    int* Ll = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
    int rc = 0;
    if (!w || !in || !next || !cand || !Ur || !Uw || !Ul || !Lr || !Lw || !Ll) { rc = OR_ERR_OOM; goto done; }
    for (int j = 0; j < n; ++j) in[j] = 0;
    for (int i = 0; i < n; ++i) {
        double nrm = 0.0;
        int head = n;
        next[head] = -1;
        int tail = head;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int j = ci[p];
            w[j] = v[p]; in[j] = 1;
            next[tail] = j; next[j] = -1; tail = j;
            nrm += v[p] * v[p];
        }
        double tau = tol * sqrt(nrm);
        if (!in[i]) { /* keep a structural diagonal slot */
            int prev = head;
            while (next[prev] != -1 && next[prev] < i) prev = next[prev];
            next[i] = next[prev]; next[prev] = i; in[i] = 1; w[i] = 0.0;
        }
        for (int k = next[head]; k != -1 && k < i; k = next[k]) {
            double dk = Uw[k][0]; /* diagonal of U row k is its first entry */
            w[k] = w[k] / dk;
            if (fabs(w[k]) < tau) { w[k] = 0.0; continue; } /* dropped multiplier */
            int prev = k;
            for (int q = 1; q < Ul[k]; ++q) {
                int j = Ur[k][q];
                if (!in[j]) {
                    while (next[prev] != -1 && next[prev] < j) prev = next[prev];
                    next[j] = next[prev]; next[prev] = j; in[j] = 1; w[j] = 0.0;
                }
                w[j] -= w[k] * Uw[k][q];
                prev = j;
            }
        }
        if (w[i] == 0.0) { rc = OR_ERR_PIVOT; }
        /* gather candidates of the strict lower / strict upper parts that survive tau */
        int nl = 0, nu = 0;
        for (int j = next[head]; j != -1; j = next[j]) {
            if (j == i) continue;
            if (w[j] == 0.0 || fabs(w[j]) < tau) continue;
            if (j < i) cand[nl++] = j;
        }
        int lcount = nl;
        for (int j = next[head]; j != -1; j = next[j]) {
            if (j <= i) continue;
            if (w[j] == 0.0 || fabs(w[j]) < tau) continue;
            cand[lcount + nu++] = j;
        }
        /* keep the p largest magnitudes in each part; ties go to the smaller column. Simple
         * selection: repeatedly pick the best remaining candidate. */
        for (int part = 0; part < 2; ++part) {
            int* c = part == 0 ? cand : cand + lcount;
            int m = part == 0 ? nl : nu;
            int keep = m < p_keep ? m : p_keep;
            for (int a = 0; a < keep; ++a) {
                int best = a;
                for (int b = a + 1; b < m; ++b) {
                    double fb = fabs(w[c[b]]), fbest = fabs(w[c[best]]);
                    if (fb > fbest || (fb == fbest && c[b] < c[best])) best = b;
                }
                int t = c[a]; c[a] = c[best]; c[best] = t;
            }
            /* sort the kept ones by column */
            for (int a = 1; a < keep; ++a) {
                int t = c[a]; int b = a - 1;
                while (b >= 0 && c[b] > t) { c[b + 1] = c[b]; --b; }
                c[b + 1] = t;
            }
            if (part == 0) nl = keep; else nu = keep;
        }
        Ll[i] = nl;
        Lr[i] = (int*)malloc(sizeof(int) * (size_t)(nl + 1));
        Lw[i] = (double*)malloc(sizeof(double) * (size_t)(nl + 1));
        Ul[i] = nu + 1;
        Ur[i] = (int*)malloc(sizeof(int) * (size_t)(nu + 1));
        Uw[i] = (double*)malloc(sizeof(double) * (size_t)(nu + 1));
        if (!Lr[i] || !Lw[i] || !Ur[i] || !Uw[i]) { rc = OR_ERR_OOM; goto done; }
        for (int a = 0; a < nl; ++a) { Lr[i][a] = cand[a]; Lw[i][a] = w[cand[a]]; }
        Ur[i][0] = i; Uw[i][0] = w[i];
        for (int a = 0; a < nu; ++a) { Ur[i][a + 1] = cand[lcount + a]; Uw[i][a + 1] = w[cand[lcount + a]]; }
        for (int j = next[head]; j != -1; j = next[j]) { in[j] = 0; w[j] = 0.0; }
        if (rc) goto done;
    }
    Lrp[0] = 0; Urp[0] = 0;
    for (int i = 0; i < n; ++i) {
        Lrp[i + 1] = Lrp[i] + Ll[i] + 1;
        Urp[i + 1] = Urp[i] + Ul[i];
        if (Lci) {
            int q = Lrp[i];
            for (int a = 0; a < Ll[i]; ++a) { Lci[q] = Lr[i][a]; Lv[q] = Lw[i][a]; q++; }
            Lci[q] = i; Lv[q] = 1.0;
            q = Urp[i];
            for (int a = 0; a < Ul[i]; ++a) { Uci[q] = Ur[i][a]; Uv[q] = Uw[i][a]; q++; }
        }
    }
done:
    for (int i = 0; i < n; ++i) {
        if (Ur) free(Ur[i]);
        if (Uw) free(Uw[i]);
        if (Lr) free(Lr[i]);
        if (Lw) free(Lw[i]);
    }
    free(w); free(in); free(next); free(cand); free(Ur); free(Uw); free(Ul); free(Lr); free(Lw); free(Ll);
    return rc;
}

/* ------------------------------------------------------------------------------------- */
/* Restricted Additive Schwarz (Sec. 3, Eq. 4)                                              */
/* ------------------------------------------------------------------------------------- */

/* Extended subdomains with overlap 1: for subdomain s, ext(s) = owned(s) united with every
 * column j of a row i owned by s ("extended according to the topology of the graph"), in
 * ascending global index.  part[i] = owning subdomain of row i (0..ns-1).  Outputs
 * ext_ptr[ns+1] and ext_idx (call with ext_idx NULL first to get ext_ptr[ns]). */
OR_EXPORT int or_ras_extend(int n, const int* rp, const int* ci, const int* part, int ns,
                            int* ext_ptr, int* ext_idx)
{
    char* mark = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!mark) return OR_ERR_OOM;
    ext_ptr[0] = 0;
    for (int s = 0; s < ns; ++s) {
        for (int i = 0; i < n; ++i) {
            if (part[i] != s) continue;
            mark[i] = 1;
            for (int p = rp[i]; p < rp[i + 1]; ++p) mark[ci[p]] = 1;
        }
        int c = 0;
        for (int i = 0; i < n; ++i) {
            if (mark[i]) {
                if (ext_idx) ext_idx[ext_ptr[s] + c] = i;
                c++;
                mark[i] = 0;
            }
        }
        ext_ptr[s + 1] = ext_ptr[s] + c;
    }
    free(mark);
    return 0;
}

/* A_s = A restricted to ext(s) (rows and columns), renumbered locally.  Output CSR arrays
 * sized by the caller (at most nnz(A) entries). */
OR_EXPORT int or_submatrix(int n, const int* rp, const int* ci, const double* v,
                           int m, const int* idx, int* srp, int* sci, double* sv)
{
    int* loc = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!loc) return OR_ERR_OOM;
    for (int j = 0; j < n; ++j) loc[j] = -1;
    for (int q = 0; q < m; ++q) loc[idx[q]] = q;
    srp[0] = 0;
    int c = 0;
    for (int q = 0; q < m; ++q) {
        int i = idx[q];
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int lj = loc[ci[p]];
            if (lj < 0) continue;
            sci[c] = lj; sv[c] = v[p]; c++;
        }
        srp[q + 1] = c;
    }
    free(loc);
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Preconditioners as callbacks, and FGMRES (Sec. 4 uses GMRES(20) in FP64)                 */
/* ------------------------------------------------------------------------------------- */

typedef int (*or_prec_fn)(void* ctx, const double* v, double* z);

typedef struct {
    int n;
    const int *Lrp, *Lci; const double* Lv;
    const int *Urp, *Uci; const double* Uv;
    double* tmp;
} or_ilu_ctx;

/* z = U^-1 L^-1 v (Eq. 1). */
static int ilu_prec(void* c, const double* v, double* z)
{
    or_ilu_ctx* k = (or_ilu_ctx*)c;
    int rc = or_lower_solve(k->n, k->Lrp, k->Lci, k->Lv, v, k->tmp);
    if (rc) return rc;
    return or_upper_solve(k->n, k->Urp, k->Uci, k->Uv, k->tmp, z);
}

OR_EXPORT int or_ilu_apply(int n, const int* Lrp, const int* Lci, const double* Lv,
                           const int* Urp, const int* Uci, const double* Uv,
                           const double* v, double* z)
{
    double* tmp = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!tmp) return OR_ERR_OOM;
    or_ilu_ctx k = {n, Lrp, Lci, Lv, Urp, Uci, Uv, tmp};
    int rc = ilu_prec(&k, v, z);
    free(tmp);
    return rc;
}

/* RAS apply (Sec. 3): z = sum_s R0_s^T U_s^-1 L_s^-1 R_s v, where R_s gathers the extended
 * rows of subdomain s and R0_s^T writes back only the rows that s owns.  The factors of all
 * subdomains are given as one block-diagonal pair (Eq. 4): local row q of subdomain s is
 * block row ext_ptr[s] + q, and ext_idx maps block rows to global rows. */
typedef struct {
    int n, ns;
    const int *ext_ptr, *ext_idx, *part;
    const int *Lrp, *Lci; const double* Lv;
    const int *Urp, *Uci; const double* Uv;
    double *r, *y, *t;
} or_ras_ctx;

static int ras_prec(void* c, const double* v, double* z)
{
    or_ras_ctx* k = (or_ras_ctx*)c;
    for (int i = 0; i < k->n; ++i) z[i] = 0.0;
    for (int s = 0; s < k->ns; ++s) {
        int b = k->ext_ptr[s], m = k->ext_ptr[s + 1] - b;
        for (int q = 0; q < m; ++q) k->r[q] = v[k->ext_idx[b + q]];
        /* the diagonal block s of the block-diagonal factors, rebased to local numbering */
        for (int q = 0; q < m; ++q) {
            double s1 = k->r[q], d = 0.0;
            int row = b + q;
            for (int p = k->Lrp[row]; p < k->Lrp[row + 1]; ++p) {
                int j = k->Lci[p] - b;
                if (j < q) s1 -= k->Lv[p] * k->t[j]; else if (j == q) d = k->Lv[p];
            }
            if (d == 0.0) return OR_ERR_PIVOT;
            k->t[q] = s1 / d;
        }
        for (int q = m - 1; q >= 0; --q) {
            double s1 = k->t[q], d = 0.0;
            int row = b + q;
            for (int p = k->Urp[row]; p < k->Urp[row + 1]; ++p) {
                int j = k->Uci[p] - b;
                if (j > q) s1 -= k->Uv[p] * k->y[j]; else if (j == q) d = k->Uv[p];
            }
            if (d == 0.0) return OR_ERR_PIVOT;
            k->y[q] = s1 / d;
        }
        for (int q = 0; q < m; ++q) {
            int g = k->ext_idx[b + q];
            if (k->part[g] == s) z[g] = k->y[q];
        }
    }
    return 0;
}

OR_EXPORT int or_ras_apply(int n, int ns, const int* ext_ptr, const int* ext_idx, const int* part,
                           const int* Lrp, const int* Lci, const double* Lv,
                           const int* Urp, const int* Uci, const double* Uv,
                           const double* v, double* z)
{
    int mx = 0;
    for (int s = 0; s < ns; ++s) if (ext_ptr[s + 1] - ext_ptr[s] > mx) mx = ext_ptr[s + 1] - ext_ptr[s];
    double* buf = (double*)malloc(sizeof(double) * 3 * (size_t)(mx > 0 ? mx : 1));
    if (!buf) return OR_ERR_OOM;
    or_ras_ctx k = {n, ns, ext_ptr, ext_idx, part, Lrp, Lci, Lv, Urp, Uci, Uv, buf, buf + mx, buf + 2 * mx};
    int rc = ras_prec(&k, v, z);
    free(buf);
    return rc;
}

static double dot(int n, const double* a, const double* b)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Right-preconditioned flexible GMRES(m) (Saad's FGMRES), modified Gram-Schmidt, Givens
 * rotations.  x holds x0 on entry and the solution on exit.  Stops when the Arnoldi residual
 * estimate |g_{j+1}| <= rtol ||b|| and then confirms with the true residual; restarts
 * otherwise.  max_iters caps the inner iterations.  info[0] = iterations, info[1] = final
 * true relative residual, info[2] = restarts.  hist (may be NULL, max_iters+1 long) receives
 * the estimate |g_{j+1}|/||b|| per iteration.  Returns 0 when converged, 1 when not. */
static int fgmres(int n, const int* rp, const int* ci, const double* v, or_prec_fn prec, void* ctx,
                  const double* b, double* x, int m, double rtol, int max_iters,
                  double* info, double* hist)
{
    size_t N = (size_t)(n > 0 ? n : 1);
    double* V = (double*)malloc(sizeof(double) * N * (size_t)(m + 1));
    double* Z = (double*)malloc(sizeof(double) * N * (size_t)m);
    double* H = (double*)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    double* cs = (double*)malloc(sizeof(double) * (size_t)m);
    double* sn = (double*)malloc(sizeof(double) * (size_t)m);
    double* g = (double*)malloc(sizeof(double) * (size_t)(m + 1));
    double* yv = (double*)malloc(sizeof(double) * (size_t)m);
    double* r = (double*)malloc(sizeof(double) * N);
    if (!V || !Z || !H || !cs || !sn || !g || !yv || !r) {
        free(V); free(Z); free(H); free(cs); free(sn); free(g); free(yv); free(r);
        return OR_ERR_OOM;
    }
    double bn = sqrt(dot(n, b, b));
    int its = 0, restarts = 0, converged = 0, rc = 0;
    double relres = 1.0;
    if (bn == 0.0) { for (int i = 0; i < n; ++i) x[i] = 0.0; converged = 1; relres = 0.0; }
    while (!converged && its < max_iters) {
        or_spmv(n, rp, ci, v, x, r);
        for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
        double beta = sqrt(dot(n, r, r));
        relres = beta / bn;
        if (relres <= rtol) { converged = 1; break; }
        for (int i = 0; i < n; ++i) V[i] = r[i] / beta;
        g[0] = beta;
        for (int a = 1; a <= m; ++a) g[a] = 0.0;
        int j = 0;
        for (; j < m && its < max_iters; ++j) {
            double* vj = V + (size_t)j * N;
            double* zj = Z + (size_t)j * N;
            double* w = V + (size_t)(j + 1) * N;
            rc = prec(ctx, vj, zj);
            if (rc) goto out;
            or_spmv(n, rp, ci, v, zj, w);
            for (int a = 0; a <= j; ++a) { /* modified Gram-Schmidt */
                double* va = V + (size_t)a * N;
                double h = dot(n, w, va);
                H[a * m + j] = h;
                for (int i = 0; i < n; ++i) w[i] -= h * va[i];
            }
            double hn = sqrt(dot(n, w, w));
            H[(j + 1) * m + j] = hn;
            if (hn != 0.0) for (int i = 0; i < n; ++i) w[i] /= hn;
            for (int a = 0; a < j; ++a) { /* previous rotations */
                double h0 = H[a * m + j], h1 = H[(a + 1) * m + j];
                H[a * m + j] = cs[a] * h0 + sn[a] * h1;
                H[(a + 1) * m + j] = -sn[a] * h0 + cs[a] * h1;
            }
            double h0 = H[j * m + j], h1 = H[(j + 1) * m + j];
            double den = sqrt(h0 * h0 + h1 * h1);
            cs[j] = den == 0.0 ? 1.0 : h0 / den;
            sn[j] = den == 0.0 ? 0.0 : h1 / den;
            H[j * m + j] = cs[j] * h0 + sn[j] * h1;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            its++;
            if (hist) hist[its] = fabs(g[j + 1]) / bn;
            if (fabs(g[j + 1]) <= rtol * bn || hn == 0.0) { j++; break; }
        }
        /* solve the j x j upper triangular system and update x = x + Z y */
        for (int a = j - 1; a >= 0; --a) {
            double s = g[a];
            for (int c = a + 1; c < j; ++c) s -= H[a * m + c] * yv[c];
            yv[a] = s / H[a * m + a];
        }
        for (int a = 0; a < j; ++a) {
            double* za = Z + (size_t)a * N;
            for (int i = 0; i < n; ++i) x[i] += yv[a] * za[i];
        }
        restarts++;
    }
    if (!converged) {
        or_spmv(n, rp, ci, v, x, r);
        for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
        relres = bn > 0 ? sqrt(dot(n, r, r)) / bn : 0.0;
        converged = relres <= rtol;
    }
out:
    if (info) { info[0] = its; info[1] = relres; info[2] = restarts; }
    if (hist) hist[0] = 1.0;
    free(V); free(Z); free(H); free(cs); free(sn); free(g); free(yv); free(r);
    if (rc) return rc;
    return converged ? 0 : 1;
}

static int identity_prec(void* c, const double* v, double* z)
{
    int n = *(const int*)c;
    for (int i = 0; i < n; ++i) z[i] = v[i];
    return 0;
}

/* FGMRES with no preconditioner (z = v): plain restarted GMRES. */
OR_EXPORT int or_fgmres_identity(int n, const int* rp, const int* ci, const double* v,
                                 const double* b, double* x, int m, double rtol, int max_iters,
                                 double* info, double* hist)
{
    int nn = n;
    return fgmres(n, rp, ci, v, identity_prec, &nn, b, x, m, rtol, max_iters, info, hist);
}

/* FGMRES preconditioned by z = U^-1 L^-1 v. */
OR_EXPORT int or_fgmres_ilu(int n, const int* rp, const int* ci, const double* v,
                            const int* Lrp, const int* Lci, const double* Lv,
                            const int* Urp, const int* Uci, const double* Uv,
                            const double* b, double* x, int m, double rtol, int max_iters,
                            double* info, double* hist)
{
    double* tmp = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!tmp) return OR_ERR_OOM;
    or_ilu_ctx k = {n, Lrp, Lci, Lv, Urp, Uci, Uv, tmp};
    int rc = fgmres(n, rp, ci, v, ilu_prec, &k, b, x, m, rtol, max_iters, info, hist);
    free(tmp);
    return rc;
}

/* FGMRES preconditioned by RAS (block-diagonal factors as in or_ras_apply). */
OR_EXPORT int or_fgmres_ras(int n, const int* rp, const int* ci, const double* v,
                            int ns, const int* ext_ptr, const int* ext_idx, const int* part,
                            const int* Lrp, const int* Lci, const double* Lv,
                            const int* Urp, const int* Uci, const double* Uv,
                            const double* b, double* x, int m, double rtol, int max_iters,
                            double* info, double* hist)
{
    int mx = 0;
    for (int s = 0; s < ns; ++s) if (ext_ptr[s + 1] - ext_ptr[s] > mx) mx = ext_ptr[s + 1] - ext_ptr[s];
    double* buf = (double*)malloc(sizeof(double) * 3 * (size_t)(mx > 0 ? mx : 1));
    if (!buf) return OR_ERR_OOM;
    or_ras_ctx k = {n, ns, ext_ptr, ext_idx, part, Lrp, Lci, Lv, Urp, Uci, Uv, buf, buf + mx, buf + 2 * mx};
    int rc = fgmres(n, rp, ci, v, ras_prec, &k, b, x, m, rtol, max_iters, info, hist);
    free(buf);
    return rc;
}
