// HEC packing (Sec. 2.1; Alg. 1 steps 3-4) and its inverse.
//
// One thread per new row r of L': it reads original row i = iperm[r], maps every column j to
// perm[j], ranks the off-diagonals by new column (a row's rank of an entry is the number of
// entries of the row with a smaller new column, so no sort is needed), and writes slot `rank`
// of the row: slab slots first, then the tail, then the diagonal last.  All of this is integer
// work plus one rounding per value and matches the serial construction bit for bit.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace hec {
hec_status validate_csr(int n, const int* rp, const int* col, int uplo, cudaStream_t s);

namespace {

// FP64 -> BF16 rounded to nearest even directly from the FP64 value: round to FP32 with
// round-to-odd (truncate, then set the last bit when inexact), then FP32 -> BF16 to nearest
// even.  FP32 keeps 16 more bits than BF16, so the two-step result equals the direct one
// (Boldo & Melquiond, "Emulation of FMA and correctly rounded sums: proved algorithms using
// rounding to odd", IEEE TC 2008).
__device__ __forceinline__ __nv_bfloat16 f64_to_bf16_rne(double d) {
    float f = __double2float_rz(d);
    if ((double)f != d && !isnan(d)) f = __uint_as_float(__float_as_uint(f) | 1u);
    return __float2bfloat16_rn(f);
}

template <typename VT> __device__ __forceinline__ VT cvt(double d);
template <> __device__ __forceinline__ double cvt<double>(double d) { return d; }
template <> __device__ __forceinline__ float cvt<float>(double d) { return __double2float_rn(d); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(double d) { return f64_to_bf16_rne(d); }

template <typename VT> __device__ __forceinline__ double widen(VT v);
template <> __device__ __forceinline__ double widen<double>(double v) { return v; }
template <> __device__ __forceinline__ double widen<float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double widen<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// eligible entries per new row (off-diagonals in triangular mode)
__global__ void k_row_counts(int n, const int* __restrict__ rp, const int* __restrict__ iperm, int tri, int* cnt,
                             int* maxcnt) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    int c = 0;
    if (r < n) {
        int i = tri ? iperm[r] : r;
        c = rp[i + 1] - rp[i] - (tri ? 1 : 0);
        cnt[r] = c;
    }
    for (int o = 16; o; o >>= 1) c = max(c, __shfl_xor_sync(0xffffffffu, c, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxcnt, c);
}

// histogram of the row counts: few distinct values, so each block counts the small ones in shared
// memory and adds its totals once (a global atomic per row would serialise on a handful of bins)
__global__ void k_count_hist(int n, const int* __restrict__ cnt, int nbins, int* hist) {
    __shared__ int sh[64];
    for (int t = threadIdx.x; t < 64; t += blockDim.x) sh[t] = 0;
    __syncthreads();
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int c = cnt[r];
        if (c < 64) atomicAdd(sh + c, 1);
        else atomicAdd(hist + c, 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 64 && t < nbins; t += blockDim.x)
        if (sh[t]) atomicAdd(hist + t, sh[t]);
}

__global__ void k_tail_len(int n, const int* __restrict__ cnt, int w, int tri, int* tlen) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) tlen[r] = max(0, cnt[r] - w) + (tri ? 1 : 0);
}

template <typename VT>
__global__ void k_pack(int n, int ld, int w, int tri, const int* __restrict__ rp, const int* __restrict__ col,
                       const double* __restrict__ val, const int* __restrict__ perm, const int* __restrict__ iperm,
                       const int* __restrict__ tptr, int* ell_col, VT* ell_val, int* tcol, VT* tval) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ld) return;
    if (r >= n) {
        for (int k = 0; k < w; ++k) {
            ell_col[(long)k * ld + r] = -1;
            ell_val[(long)k * ld + r] = cvt<VT>(0.0);
        }
        return;
    }
    int i = tri ? iperm[r] : r;
    int a = rp[i], b = rp[i + 1];
    int t0 = tptr[r];
    int cnt = 0;
    for (int p = a; p < b; ++p) {
        int j = col[p];
        if (tri && j == i) {
            tval[tptr[r + 1] - 1] = cvt<VT>(val[p]);
            tcol[tptr[r + 1] - 1] = r;
            continue;
        }
        int nc = tri ? perm[j] : j;
        int rank = 0;
        if (tri) {
            for (int q = a; q < b; ++q) {
                int jq = col[q];
                if (jq != i && perm[jq] < nc) rank++;
            }
        } else {
            rank = p - a;
        }
        if (rank < w) {
            ell_col[(long)rank * ld + r] = nc;
            ell_val[(long)rank * ld + r] = cvt<VT>(val[p]);
        } else {
            tcol[t0 + rank - w] = nc;
            tval[t0 + rank - w] = cvt<VT>(val[p]);
        }
        cnt++;
    }
    for (int k = cnt; k < w; ++k) {
        ell_col[(long)k * ld + r] = -1;
        ell_val[(long)k * ld + r] = cvt<VT>(0.0);
    }
}

// ---- HEC -> CSR of the original matrix ----
__global__ void k_unpack_len(int n, int ld, int w, int tri, const int* __restrict__ ell_col, const int* __restrict__ tptr,
                             const int* __restrict__ iperm, int* len) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int c = tptr[r + 1] - tptr[r];
    for (int k = 0; k < w; ++k) c += ell_col[(long)k * ld + r] >= 0;
    len[tri ? iperm[r] : r] = c;
}

template <typename VT>
__global__ void k_unpack(int n, int ld, int w, int tri, const int* __restrict__ ell_col, const VT* __restrict__ ell_val,
                         const int* __restrict__ tptr, const int* __restrict__ tcol, const VT* __restrict__ tval,
                         const int* __restrict__ iperm, const int* __restrict__ orp, int* oci, double* ov) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int i = tri ? iperm[r] : r;
    int base = orp[i];
    int m = orp[i + 1] - base;
    // gather this row's original columns, then place each by its rank among them
    auto orig = [&](int e, int& c, double& v) {
        if (e < w) {
            int s = 0, k = 0;
            for (; k < w; ++k) {
                if (ell_col[(long)k * ld + r] >= 0) {
                    if (s == e) break;
                    s++;
                }
            }
            c = ell_col[(long)k * ld + r];
            v = widen<VT>(ell_val[(long)k * ld + r]);
        } else {
            int p = tptr[r] + (e - w);
            c = tcol[p];
            v = widen<VT>(tval[p]);
        }
        c = tri ? iperm[c] : c;
    };
    int nell = 0;
    for (int k = 0; k < w; ++k) nell += ell_col[(long)k * ld + r] >= 0;
    for (int e = 0; e < m; ++e) {
        int idx_e = e < nell ? e : w + (e - nell);
        int ce;
        double ve;
        orig(idx_e, ce, ve);
        int rank = 0;
        for (int f = 0; f < m; ++f) {
            int idx_f = f < nell ? f : w + (f - nell);
            int cf;
            double vf;
            orig(idx_f, cf, vf);
            if (cf < ce) rank++;
        }
        oci[base + rank] = ce;
        ov[base + rank] = ve;
    }
}

template <typename VT>
hec_status launch_pack(hec_matrix* M, const int* rp, const int* col, const double* val, const int* perm,
                       const int* iperm, cudaStream_t s) {
    int grid = (M->ld + 127) / 128;
    if (grid == 0) return HEC_OK;
    k_pack<VT><<<grid, 128, 0, s>>>(M->n, M->ld, M->w, M->tri, rp, col, val, perm, iperm, M->tptr, M->ell_col,
                                    (VT*)M->ell_val, M->tcol, (VT*)M->tval);
    HEC_LAUNCHED();
    return HEC_OK;
}

size_t vsize(hec_dtype d) { return d == HEC_F64 ? 8 : d == HEC_F32 ? 4 : 2; }

}  // namespace

void free_matrix(hec_matrix* M) {
    if (!M) return;
    dfree(M->ell_col);
    dfree(M->ell_val);
    dfree(M->tptr);
    dfree(M->tcol);
    dfree(M->tval);
    delete M;
}

}  // namespace hec

using namespace hec;

HEC_API hec_status hec_from_csr(int n, const int* rowptr, const int* col, const double* val, const hec_levels* lv,
                                int ell_width, hec_dtype vdt, hec_matrix** out, void* stream) {
    clear_error();
    if (!out || n < 0 || (n > 0 && (!rowptr || !col || !val)) || ell_width < -1 ||
        (vdt != HEC_F64 && vdt != HEC_F32 && vdt != HEC_BF16))
        return set_error(HEC_ERR_INVALID_ARG, "hec_from_csr: bad argument");
    if (lv && lv->n != n) return set_error(HEC_ERR_INVALID_ARG, "hec_from_csr: level analysis has another size");
    *out = nullptr;
    cudaStream_t s = S(stream);
    const int tri = lv ? 1 : 0;
    HEC_CHECK(validate_csr(n, rowptr, col, tri ? lv->uplo : -1, s));
    hec_matrix* M = new hec_matrix();
    M->n = n;
    M->ld = (n + 31) / 32 * 32;
    M->tri = tri;
    M->uplo = tri ? lv->uplo : 0;
    M->vdt = vdt;
    M->lv = lv;
    int* cnt = nullptr;
    int* small = nullptr;  // [0] max count, [1] tail total
    hec_status st = HEC_OK;
    auto fail = [&](hec_status e) {
        dfree(cnt);
        dfree(small);
        free_matrix(M);
        return e;
    };
    if ((st = dalloc(&cnt, (size_t)n + 1)) || (st = dalloc(&small, 2))) return fail(st);
    if ((st = dalloc(&M->tptr, (size_t)n + 1))) return fail(st);
    cudaMemsetAsync(small, 0, 2 * sizeof(int), s);
    const int* iperm = tri ? lv->iperm : nullptr;
    const int* perm = tri ? lv->perm : nullptr;
    int g = (n + 255) / 256;
    if (n > 0) {
        k_row_counts<<<g, 256, 0, s>>>(n, rowptr, iperm, tri, cnt, small);
        count_launch();
    }
    int w = ell_width;
    if (w < 0) {
        int maxcnt = 0;
        if (cudaMemcpyAsync(&maxcnt, small, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "hec_from_csr: count"));
        int* hist = nullptr;
        if ((st = dalloc(&hist, (size_t)maxcnt + 1))) return fail(st);
        cudaMemsetAsync(hist, 0, sizeof(int) * ((size_t)maxcnt + 1), s);
        if (n > 0) {
            k_count_hist<<<std::min(g, 4 * num_sms()), 256, 0, s>>>(n, cnt, maxcnt + 1, hist);
            count_launch();
        }
        std::vector<int> h((size_t)maxcnt + 1);
        cudaError_t e = cudaMemcpyAsync(h.data(), hist, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        dfree(hist);
        if (e != cudaSuccess) return fail(cuda_error(e, "hec_from_csr: histogram"));
        // largest w with #rows(count >= w) >= ceil(0.65 n)
        long long need = (long long)((65LL * n + 99) / 100);
        long long atleast = 0;
        w = 0;
        for (int c = maxcnt; c >= 1; --c) {
            atleast += h[c];
            if (n > 0 && atleast >= need) { w = c; break; }
        }
    }
    M->w = w;
    if (n > 0) {
        k_tail_len<<<g, 256, 0, s>>>(n, cnt, w, tri, cnt);
        count_launch();
    }
    if ((st = exclusive_scan_i32(cnt, M->tptr, n, true, s))) return fail(st);
    int tn = 0;
    if (cudaMemcpyAsync(&tn, M->tptr + n, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(cuda_error(cudaGetLastError(), "hec_from_csr: tail size"));
    M->tail_nnz = tn;
    size_t vs = vsize(vdt);
    if ((st = dalloc(&M->ell_col, (size_t)w * M->ld)) || (st = dmalloc(&M->ell_val, vs * (size_t)w * M->ld + 16)) ||
        (st = dalloc(&M->tcol, (size_t)tn)) || (st = dmalloc(&M->tval, vs * (size_t)tn + 16)))
        return fail(st);
    if (vdt == HEC_F64) st = launch_pack<double>(M, rowptr, col, val, perm, iperm, s);
    else if (vdt == HEC_F32) st = launch_pack<float>(M, rowptr, col, val, perm, iperm, s);
    else st = launch_pack<__nv_bfloat16>(M, rowptr, col, val, perm, iperm, s);
    if (st) return fail(st);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_error(e, "hec_from_csr: pack"));
    dfree(cnt);
    dfree(small);
    *out = M;
    return HEC_OK;
}

HEC_API hec_status hec_matrix_get(const hec_matrix* A, hec_matrix_info* info) {
    if (!A || !info) return set_error(HEC_ERR_INVALID_ARG, "hec_matrix_get: NULL");
    info->n = A->n;
    info->ld = A->ld;
    info->w = A->w;
    info->tri = A->tri;
    info->uplo = A->uplo;
    info->vdt = A->vdt;
    info->tail_nnz = A->tail_nnz;
    info->ell_col = A->ell_col;
    info->ell_val = A->ell_val;
    info->tptr = A->tptr;
    info->tcol = A->tcol;
    info->tval = A->tval;
    return HEC_OK;
}

HEC_API hec_status hec_to_csr(const hec_matrix* A, const hec_levels* lv, int* rowptr, int* col, double* val, void* stream) {
    clear_error();
    if (!A || !rowptr || (A->tri && !lv) || (lv && lv->n != A->n))
        return set_error(HEC_ERR_INVALID_ARG, "hec_to_csr: bad argument");
    cudaStream_t s = S(stream);
    int n = A->n;
    int* len = nullptr;
    HEC_CHECK(dalloc(&len, (size_t)n + 1));
    const int* iperm = A->tri ? lv->iperm : nullptr;
    int g = (n + 255) / 256;
    if (n > 0) {
        k_unpack_len<<<g, 256, 0, s>>>(n, A->ld, A->w, A->tri, A->ell_col, A->tptr, iperm, len);
        count_launch();
    }
    hec_status st = exclusive_scan_i32(len, rowptr, n, true, s);
    if (st == HEC_OK && n > 0) {
        if (A->vdt == HEC_F64)
            k_unpack<double><<<g, 256, 0, s>>>(n, A->ld, A->w, A->tri, A->ell_col, (const double*)A->ell_val, A->tptr,
                                               A->tcol, (const double*)A->tval, iperm, rowptr, col, val);
        else if (A->vdt == HEC_F32)
            k_unpack<float><<<g, 256, 0, s>>>(n, A->ld, A->w, A->tri, A->ell_col, (const float*)A->ell_val, A->tptr,
                                              A->tcol, (const float*)A->tval, iperm, rowptr, col, val);
        else
            k_unpack<__nv_bfloat16><<<g, 256, 0, s>>>(n, A->ld, A->w, A->tri, A->ell_col,
                                                      (const __nv_bfloat16*)A->ell_val, A->tptr, A->tcol,
                                                      (const __nv_bfloat16*)A->tval, iperm, rowptr, col, val);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(e, "hec_to_csr");
    }
    dfree(len);
    return st;
}

HEC_API hec_status hec_matrix_destroy(hec_matrix* A) {
    free_matrix(A);
    return HEC_OK;
}
