// Symmetric Gauss-Seidel smoother on the level-scheduled triangular sweeps.
//
// The paper names smoothers (Gauss-Seidel in AMG) as another use of the triangular solver
// (Sec. 1).  With the splitting A = L_s + D + U_s (strict lower part, diagonal, strict upper
// part) one symmetric sweep is
//     forward:  (D + L_s) x' = b - U_s x
//     backward: (D + U_s) x'' = b - L_s x'
// and each triangular solve is the level-scheduled HEC sweep of Alg. 2 (level scheduling only
// reorders independent rows, so every sweep equals the sequential Gauss-Seidel sweep up to
// rounding).  The handle keeps the two triangles as solve plans, the two strict parts as FP64
// HEC matrices for the residual products, and one n x max_nrhs work vector.
#include <algorithm>

#include "internal.cuh"

struct hec_sgs {
    int n = 0, max_nrhs = 1;
    hec_csr* tri[4] = {};         // D + L_s, D + U_s, U_s, L_s (device CSR)
    hec_levels* lv[2] = {};       // analyses of D + L_s (uplo 0) and D + U_s (uplo 1)
    hec_matrix* H[2] = {};        // their HEC forms
    sptrsv_plan* plan[2] = {};    // their solve plans
    hec_matrix* strict[2] = {};   // U_s and L_s as general-mode FP64 HEC (SpMV)
    double* r = nullptr;          // [n * max_nrhs] right-hand side of the current sweep
};

namespace {
void free_sgs(hec_sgs* S) {
    if (!S) return;
    for (auto* p : S->plan) sptrsv_plan_destroy(p);
    for (auto* h : S->H) hec_matrix_destroy(h);
    for (auto* h : S->strict) hec_matrix_destroy(h);
    for (auto* l : S->lv) hec_levels_destroy(l);
    for (auto* t : S->tri) hec_csr_destroy(t);
    hec::dfree(S->r);
    delete S;
}
}  // namespace

using namespace hec;

HEC_API hec_status sgs_create(int n, const int* rowptr, const int* col, const double* val, hec_dtype vdt,
                              int max_nrhs, hec_sgs** out, void* stream) {
    clear_error();
    if (!out || n < 1 || max_nrhs < 1 || max_nrhs > 16 || !rowptr || !col || !val ||
        (vdt != HEC_F64 && vdt != HEC_F32 && vdt != HEC_BF16))
        return set_error(HEC_ERR_INVALID_ARG, "sgs_create: need n >= 1, 1 <= max_nrhs <= 16 and device CSR arrays");
    *out = nullptr;
    hec_sgs* S = new hec_sgs();
    S->n = n;
    S->max_nrhs = max_nrhs;
    hec_status st = HEC_OK;
    auto fail = [&](hec_status e) {
        free_sgs(S);
        return e;
    };
    // triangles: (uplo, strict) = (0, 0) D + L_s, (1, 0) D + U_s, (1, 1) U_s, (0, 1) L_s
    const int tri_uplo[4] = {0, 1, 1, 0}, tri_strict[4] = {0, 0, 1, 1};
    for (int i = 0; i < 4; ++i)
        if ((st = csr_triangle(n, rowptr, col, val, tri_uplo[i], tri_strict[i], &S->tri[i], stream))) return fail(st);
    for (int i = 0; i < 2; ++i) {
        const hec_csr* T = S->tri[i];
        if ((st = sptrsv_analyze(n, T->rowptr, T->col, i, &S->lv[i], stream))) return fail(st);
        if ((st = hec_from_csr(n, T->rowptr, T->col, T->val, S->lv[i], -1, vdt, &S->H[i], stream))) return fail(st);
        if ((st = sptrsv_plan_create(S->H[i], S->lv[i], max_nrhs, nullptr, &S->plan[i]))) return fail(st);
        const hec_csr* P = S->tri[2 + i];
        if ((st = hec_from_csr(n, P->rowptr, P->col, P->val, nullptr, -1, HEC_F64, &S->strict[i], stream)))
            return fail(st);
    }
    if ((st = dalloc(&S->r, (size_t)n * max_nrhs))) return fail(st);
    *out = S;
    return HEC_OK;
}

HEC_API hec_status sgs_smooth(const hec_sgs* sg, int nrhs, const double* b, int ldb, double* x, int ldx, int sweeps,
                              void* stream) {
    clear_error();
    if (!sg || nrhs < 1 || nrhs > sg->max_nrhs || ldb < nrhs || ldx < nrhs || !b || !x || sweeps < 0)
        return set_error(HEC_ERR_INVALID_ARG, "sgs_smooth: bad argument");
    cudaStream_t s = S(stream);
    const size_t row_bytes = sizeof(double) * (size_t)nrhs;
    for (int it = 0; it < sweeps; ++it) {
        for (int i = 0; i < 2; ++i) {
            // r = b - (U_s x | L_s x'), then the triangle (D + L_s | D + U_s) solved into x
            HEC_CUDA(cudaMemcpy2DAsync(sg->r, row_bytes, b, sizeof(double) * (size_t)ldb, row_bytes, (size_t)sg->n,
                                       cudaMemcpyDeviceToDevice, s));
            HEC_CHECK(spmv_impl(sg->strict[i], nrhs, -1.0, x, ldx, 1.0, sg->r, nrhs, s));
            HEC_CHECK(sweep(sg->plan[i], nrhs, sg->r, nrhs, sg->lv[i]->iperm, x, ldx, sg->lv[i]->iperm, s));
        }
    }
    return HEC_OK;
}

HEC_API hec_status sgs_sync_status(const hec_sgs* sg, void* stream) {
    if (!sg) return set_error(HEC_ERR_INVALID_ARG, "sgs_sync_status: NULL");
    const hec_status a = hec_sync_status(sg->plan[0], stream);
    const hec_status c = hec_sync_status(sg->plan[1], stream);
    return a != HEC_OK ? a : c;
}

HEC_API hec_status sgs_destroy(hec_sgs* S) {
    free_sgs(S);
    return HEC_OK;
}
