// Incomplete LU factorization on the GPU: ILU(0), ILU(1) and ILU(k) (Sec. 3); the ILU(k) pattern for
// k >= 2 comes from iluk.cu.
//
// Row i of the factors needs the finished U rows of every q < i in its lower pattern, which is
// the same dependency structure as the triangular solve with L.  The numeric kernel therefore
// runs rows in the level order of the lower pattern with the same persistent, point-to-point
// scheme as the sweeps: a row waits (acquire) for the completion flag of each pivot row it
// uses, eliminates, and publishes its own flag (release) after its values are written.
//
// ILU(1)'s pattern adds to A the entries (i, j) reachable as i -> q -> j through an original
// entry a_iq (q < i) and an original entry a_qj (j > q): fill of level 1.  Each row's pattern is
// the sorted union of its own columns and the upper parts of its pivot rows, built by a k-way
// merge of those sorted lists (no dependency between rows, so this step is fully parallel).
#include <algorithm>

#include "internal.cuh"
#include "sync.cuh"

namespace hec {
hec_status validate_csr(int n, const int* rp, const int* col, int uplo, cudaStream_t s);
hec_status iluk_pattern(int n, const int* rp, const int* ci, int k, int** prp, int** pci, long long* nnz,
                        cudaStream_t s);
hec_status compute_levels(int n, const int* rp, const int* col, int dep_side, hec_levels* lv, cudaStream_t s);
void free_levels(hec_levels* lv);

namespace {

__global__ void k_find_diag(int n, const int* __restrict__ rp, const int* __restrict__ col, int* dg, int* code) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int d = -1;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
        if (col[p] == i) d = p;
    dg[i] = d;
    if (d < 0) atomicCAS(code, 0, HEC_ERR_MISSING_DIAG);
}

// lu holds A's values on the pattern; on return the factors in place.  done[] zeroed.
// One warp per row, rows taken in the level order of the lower pattern (order[t]); the row's
// columns and values sit in shared memory (rows longer than kIluCap are worked in place in
// global memory).  For each pivot k < i in ascending order: every lane acquires row k's
// completion flag, l_ik = a_ik / u_kk, and the lanes split row k's upper entries, each finding
// its column in row i by binary search and applying a_ij <- fma(-l_ik, u_kj, a_ij).  Every entry
// receives the same operations in the same order as in a serial IKJ elimination.
constexpr int kIluCap = 256;
constexpr int kIluWarps = 8;

__device__ __forceinline__ int lower_bound_i(const int* c, int lo, int hi, int v) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (c[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kIluWarps * 32) k_ilu_numeric(int n, const int* __restrict__ rp,
                                                                const int* __restrict__ col, const int* __restrict__ dg,
                                                                const int* __restrict__ order, double* lu, int* done,
                                                                int* status, long long budget) {
    __shared__ int s_col[kIluWarps][kIluCap];
    __shared__ double s_val[kIluWarps][kIluCap];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int W = gridDim.x * kIluWarps;
    for (int t = blockIdx.x * kIluWarps + wl; t < n; t += W) {
        const int i = __ldg(order + t);
        const int a = __ldg(rp + i), di = __ldg(dg + i), e = __ldg(rp + i + 1);
        const int len = e - a, dpos = di - a;
        const bool sm = len <= kIluCap;
        const int* rc = sm ? s_col[wl] : col + a;
        double* rv = sm ? s_val[wl] : lu + a;
        if (sm) {
            for (int q = lane; q < len; q += 32) {
                s_col[wl][q] = __ldg(col + a + q);
                s_val[wl][q] = lu[a + q];
            }
        }
        __syncwarp();
        bool bad = false;
        for (int p = 0; p < dpos; ++p) {
            const int k = rc[p];
            // every lane acquires row k (bounded), so its reads of row k are ordered after the release
            bool ready = ld_acquire_i32(done + k) != 0;
            if (!__all_sync(full, ready)) {
                const long long t0 = clock64();
                for (unsigned it = 1; !__all_sync(full, ready); ++it) {
                    ready = ld_acquire_i32(done + k) != 0;
                    if ((it & 63u) == 0u && __any_sync(full, clock64() - t0 > budget || ld_relaxed_u32(status) != 0u)) {
                        if (lane == 0) record(status, HEC_ERR_TIMEOUT);
                        bad = true;
                        break;
                    }
                }
            }
            if (bad) break;
            const int dk = __ldg(dg + k), ek = __ldg(rp + k + 1);
            const double piv = lu[dk];
            if (piv == 0.0) {
                if (lane == 0) record(status, HEC_ERR_ZERO_PIVOT);
                continue;
            }
            const double lik = rv[p] / piv;
            __syncwarp();
            if (lane == 0) rv[p] = lik;
            for (int qb = dk + 1; qb < ek; qb += 32) {
                const int q = qb + lane;
                if (q < ek) {
                    const int j = __ldg(col + q);
                    const int pos = lower_bound_i(rc, p + 1, len, j);
                    if (pos < len && rc[pos] == j) rv[pos] = fma(-lik, lu[q], rv[pos]);
                }
            }
            __syncwarp();
        }
        if (sm)
            for (int q = lane; q < len; q += 32) lu[a + q] = s_val[wl][q];
        __syncwarp();
        if (lane == 0) {
            if (rv[dpos] == 0.0) record(status, HEC_ERR_ZERO_PIVOT);
            __threadfence();
            st_release_i32(done + i, 1);
        }
        __syncwarp();
    }
}

__global__ void k_split_len(int n, const int* __restrict__ rp, const int* __restrict__ dg, int* llen, int* ulen) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    llen[i] = dg[i] - rp[i] + 1;
    ulen[i] = rp[i + 1] - dg[i];
}

__global__ void k_split(int n, const int* __restrict__ rp, const int* __restrict__ col, const int* __restrict__ dg,
                        const double* __restrict__ lu, const int* __restrict__ lrp, int* lci, double* lv,
                        const int* __restrict__ urp, int* uci, double* uv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int ql = lrp[i];
    for (int p = rp[i]; p < dg[i]; ++p, ++ql) {
        lci[ql] = col[p];
        lv[ql] = lu[p];
    }
    lci[ql] = i;
    lv[ql] = 1.0;
    int qu = urp[i];
    for (int p = dg[i]; p < rp[i + 1]; ++p, ++qu) {
        uci[qu] = col[p];
        uv[qu] = lu[p];
    }
}

// ILU(1) pattern: the sorted union of row i's columns and, for each q < i in row i, the columns
// j > q of row q.  k-way merge over at most kMaxLists sorted lists.
constexpr int kMaxLists = 64;

template <bool kFill>
__global__ void k_ilu1_pattern(int n, const int* __restrict__ rp, const int* __restrict__ col,
                               const int* __restrict__ prp, int* pci, int* plen, int* code) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int head[kMaxLists], end[kMaxLists];
    int nl = 0;
    head[nl] = rp[i];
    end[nl] = rp[i + 1];
    nl++;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        int q = col[p];
        if (q >= i) break;
        if (nl >= kMaxLists) {
            atomicCAS(code, 0, HEC_ERR_INVALID_ARG);
            return;
        }
        int a = rp[q], b = rp[q + 1];
        while (a < b && col[a] <= q) ++a;  // upper part of row q
        head[nl] = a;
        end[nl] = b;
        nl++;
    }
    int cnt = 0, last = -1;
    int out = kFill ? prp[i] : 0;
    while (true) {
        int best = 0x7fffffff;
        for (int l = 0; l < nl; ++l)
            if (head[l] < end[l]) best = min(best, col[head[l]]);
        if (best == 0x7fffffff) break;
        for (int l = 0; l < nl; ++l)
            if (head[l] < end[l] && col[head[l]] == best) head[l]++;
        if (best != last) {
            if (kFill) pci[out + cnt] = best;
            cnt++;
            last = best;
        }
    }
    if (!kFill) plen[i] = cnt;
}

// scatter A's values into the (sorted, superset) pattern; fill entries start at 0
__global__ void k_scatter_vals(int n, const int* __restrict__ rp, const int* __restrict__ col,
                               const double* __restrict__ val, const int* __restrict__ prp,
                               const int* __restrict__ pci, double* pv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int q = prp[i];
    const int e = prp[i + 1];
    for (int p = prp[i]; p < e; ++p) pv[p] = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        while (q < e && pci[q] < col[p]) ++q;
        pv[q] = val[p];
    }
}

hec_status read_code(int* dcode, cudaStream_t s, int* h) {
    HEC_CUDA(cudaMemcpyAsync(h, dcode, sizeof(int), cudaMemcpyDeviceToHost, s));
    HEC_CUDA(cudaStreamSynchronize(s));
    return HEC_OK;
}

}  // namespace

void free_csr(hec_csr* M) {
    if (!M) return;
    dfree(M->rowptr);
    dfree(M->col);
    dfree(M->val);
    delete M;
}

}  // namespace hec

using namespace hec;

HEC_API hec_status hec_csr_get(const hec_csr* M, int* n, long long* nnz, const int** rowptr, const int** col,
                               const double** val) {
    if (!M) return set_error(HEC_ERR_INVALID_ARG, "hec_csr_get: NULL");
    if (n) *n = M->n;
    if (nnz) *nnz = M->nnz;
    if (rowptr) *rowptr = M->rowptr;
    if (col) *col = M->col;
    if (val) *val = M->val;
    return HEC_OK;
}

namespace hec {
namespace {
// keep (i, j) when j <= i (uplo 0) or j >= i (uplo 1), the diagonal excluded when strict
__device__ __forceinline__ bool keep_entry(int i, int j, int uplo, int strict) {
    return uplo == 0 ? (strict ? j < i : j <= i) : (strict ? j > i : j >= i);
}
__global__ void k_tri_count(int n, const int* __restrict__ rp, const int* __restrict__ col, int uplo, int strict,
                            int* __restrict__ len) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) c += keep_entry(i, col[p], uplo, strict);
    len[i] = c;
}
__global__ void k_tri_fill(int n, const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
                           int uplo, int strict, const int* __restrict__ orp, int* __restrict__ ocol,
                           double* __restrict__ oval) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int o = orp[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p)
        if (keep_entry(i, col[p], uplo, strict)) {
            ocol[o] = col[p];
            oval[o] = val[p];
            ++o;
        }
}
}  // namespace
}  // namespace hec

HEC_API hec_status csr_triangle(int n, const int* rowptr, const int* col, const double* val, int uplo, int strict,
                                hec_csr** out, void* stream) {
    clear_error();
    if (!out || n < 0 || (uplo != 0 && uplo != 1) || (n > 0 && (!rowptr || !col || !val)))
        return set_error(HEC_ERR_INVALID_ARG, "csr_triangle: bad argument");
    *out = nullptr;
    cudaStream_t s = S(stream);
    HEC_CHECK(validate_csr(n, rowptr, col, -1, s));
    hec_csr* T = new hec_csr();
    T->n = n;
    int* len = nullptr;
    hec_status st = HEC_OK;
    auto fail = [&](hec_status e) {
        dfree(len);
        free_csr(T);
        return e;
    };
    if ((st = dalloc(&len, (size_t)n + 1)) || (st = dalloc(&T->rowptr, (size_t)n + 1))) return fail(st);
    const int g = std::max(1, (n + 255) / 256);
    if (n > 0) k_tri_count<<<g, 256, 0, s>>>(n, rowptr, col, uplo, strict, len);
    count_launch();
    if ((st = exclusive_scan_i32(len, T->rowptr, n, true, s))) return fail(st);
    int nnz = 0;
    HEC_CUDA(cudaMemcpyAsync(&nnz, T->rowptr + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    HEC_CUDA(cudaStreamSynchronize(s));
    T->nnz = nnz;
    if ((st = dalloc(&T->col, (size_t)std::max(nnz, 1))) || (st = dalloc(&T->val, (size_t)std::max(nnz, 1))))
        return fail(st);
    if (n > 0) k_tri_fill<<<g, 256, 0, s>>>(n, rowptr, col, val, uplo, strict, T->rowptr, T->col, T->val);
    count_launch();
    HEC_CUDA(cudaGetLastError());
    dfree(len);
    *out = T;
    return HEC_OK;
}

HEC_API hec_status hec_csr_destroy(hec_csr* M) {
    free_csr(M);
    return HEC_OK;
}

HEC_API hec_status ilu_factor(int n, const int* rowptr, const int* col, const double* val, int k, hec_csr** Lout,
                              hec_csr** Uout, void* stream) {
    clear_error();
    if (!Lout || !Uout || n < 0 || k < 0 || (n > 0 && (!rowptr || !col || !val)))
        return set_error(HEC_ERR_INVALID_ARG, "ilu_factor: bad argument (k must be >= 0)");
    *Lout = *Uout = nullptr;
    cudaStream_t s = S(stream);
    HEC_CHECK(validate_csr(n, rowptr, col, -1, s));
    int *dg = nullptr, *code = nullptr, *done = nullptr, *prp = nullptr, *pci = nullptr, *plen = nullptr;
    double* lu = nullptr;
    hec_levels* lv = nullptr;
    hec_csr *L = new hec_csr(), *U = new hec_csr();
    hec_status st = HEC_OK;
    auto cleanup = [&]() {
        dfree(dg); dfree(code); dfree(done); dfree(plen); dfree(lu);
        if (prp != rowptr) dfree(prp);
        if (pci != col) dfree(pci);
        free_levels(lv);
    };
    auto fail = [&](hec_status e) {
        cleanup();
        free_csr(L);
        free_csr(U);
        return e;
    };
    const int g = (n + 255) / 256;
    if ((st = dalloc(&code, 2))) return fail(st);
    HEC_CUDA(cudaMemsetAsync(code, 0, 2 * sizeof(int), s));
    int hcode = 0;
    long long pnnz = 0;
    // ---- pattern ----
    if (k == 0) {
        prp = const_cast<int*>(rowptr);
        pci = const_cast<int*>(col);
        int h = 0;
        if (n > 0) HEC_CUDA(cudaMemcpy(&h, rowptr + n, sizeof(int), cudaMemcpyDeviceToHost));
        pnnz = h;
        if ((st = dalloc(&lu, (size_t)pnnz))) return fail(st);
        HEC_CUDA(cudaMemcpyAsync(lu, val, sizeof(double) * (size_t)pnnz, cudaMemcpyDeviceToDevice, s));
    } else if (k >= 2) {
        if (n > 0) {
            if ((st = iluk_pattern(n, rowptr, col, k, &prp, &pci, &pnnz, s))) return fail(st);
            if ((st = dalloc(&lu, (size_t)pnnz))) return fail(st);
            k_scatter_vals<<<g, 256, 0, s>>>(n, rowptr, col, val, prp, pci, lu);
            count_launch();
        }
    } else {
        if ((st = dalloc(&plen, (size_t)n + 1)) || (st = dalloc(&prp, (size_t)n + 1))) return fail(st);
        if (n > 0) {
            k_ilu1_pattern<false><<<g, 256, 0, s>>>(n, rowptr, col, nullptr, nullptr, plen, code);
            count_launch();
        }
        if ((st = read_code(code, s, &hcode))) return fail(st);
        if (hcode) return fail(set_error(HEC_ERR_INVALID_ARG, "ilu_factor: a row has more than 63 pivots (ILU(1) limit)"));
        if ((st = exclusive_scan_i32(plen, prp, n, true, s))) return fail(st);
        int h = 0;
        HEC_CUDA(cudaMemcpy(&h, prp + n, sizeof(int), cudaMemcpyDeviceToHost));
        pnnz = h;
        if ((st = dalloc(&pci, (size_t)pnnz)) || (st = dalloc(&lu, (size_t)pnnz))) return fail(st);
        if (n > 0) {
            k_ilu1_pattern<true><<<g, 256, 0, s>>>(n, rowptr, col, prp, pci, nullptr, code);
            k_scatter_vals<<<g, 256, 0, s>>>(n, rowptr, col, val, prp, pci, lu);
            count_launch(2);
        }
    }
    if (n == 0) {
        if ((st = dalloc(&L->rowptr, 1)) || (st = dalloc(&U->rowptr, 1))) return fail(st);
        cudaMemset(L->rowptr, 0, sizeof(int));
        cudaMemset(U->rowptr, 0, sizeof(int));
        cleanup();
        *Lout = L;
        *Uout = U;
        return HEC_OK;
    }
    // ---- diagonal positions, levels of the lower pattern ----
    if ((st = dalloc(&dg, (size_t)n))) return fail(st);
    k_find_diag<<<g, 256, 0, s>>>(n, prp, pci, dg, code);
    count_launch();
    if ((st = read_code(code, s, &hcode))) return fail(st);
    if (hcode) return fail(set_error(HEC_ERR_MISSING_DIAG, "ilu_factor: a row has no diagonal entry"));
    lv = new hec_levels();
    if ((st = compute_levels(n, prp, pci, 0, lv, s))) return fail(st);
    // ---- numeric elimination in level order ----
    if ((st = dalloc(&done, (size_t)n))) return fail(st);
    HEC_CUDA(cudaMemsetAsync(done, 0, sizeof(int) * (size_t)n, s));
    {
        const int threads = kIluWarps * 32;
        int per_sm = max_coop_blocks((const void*)k_ilu_numeric, threads, 0);
        if (per_sm <= 0) return fail(set_error(HEC_ERR_CUDA, "factor kernel cannot be resident"));
        int blocks = std::max(1, std::min(per_sm * num_sms(), (n + kIluWarps - 1) / kIluWarps));
        long long budget = 4000000000LL;
        int nn = n;
        int* status = code + 1;
        void* args[] = {&nn, &prp, &pci, &dg, &lv->iperm, &lu, &done, &status, &budget};
        HEC_CUDA(cudaLaunchCooperativeKernel((const void*)k_ilu_numeric, dim3(blocks), dim3(threads), args, 0, s));
        count_launch();
    }
    int hs[2] = {0, 0};
    HEC_CUDA(cudaMemcpyAsync(hs, code, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    HEC_CUDA(cudaStreamSynchronize(s));
    if (hs[1] == HEC_ERR_ZERO_PIVOT) return fail(set_error(HEC_ERR_ZERO_PIVOT, "ilu_factor: zero pivot"));
    if (hs[1]) return fail(set_error((hec_status)hs[1], "ilu_factor: dependency wait timed out"));
    // ---- split into L (unit lower, diagonal stored) and U ----
    int *llen = nullptr, *ulen = nullptr;
    if ((st = dalloc(&llen, (size_t)n + 1)) || (st = dalloc(&ulen, (size_t)n + 1))) {
        dfree(llen);
        return fail(st);
    }
    k_split_len<<<g, 256, 0, s>>>(n, prp, dg, llen, ulen);
    count_launch();
    L->n = U->n = n;
    if ((st = dalloc(&L->rowptr, (size_t)n + 1)) || (st = dalloc(&U->rowptr, (size_t)n + 1)) ||
        (st = exclusive_scan_i32(llen, L->rowptr, n, true, s)) || (st = exclusive_scan_i32(ulen, U->rowptr, n, true, s))) {
        dfree(llen); dfree(ulen);
        return fail(st);
    }
    dfree(llen);
    dfree(ulen);
    int ln = 0, un = 0;
    HEC_CUDA(cudaMemcpy(&ln, L->rowptr + n, sizeof(int), cudaMemcpyDeviceToHost));
    HEC_CUDA(cudaMemcpy(&un, U->rowptr + n, sizeof(int), cudaMemcpyDeviceToHost));
    L->nnz = ln;
    U->nnz = un;
    if ((st = dalloc(&L->col, (size_t)ln)) || (st = dalloc(&L->val, (size_t)ln)) || (st = dalloc(&U->col, (size_t)un)) ||
        (st = dalloc(&U->val, (size_t)un)))
        return fail(st);
    k_split<<<g, 256, 0, s>>>(n, prp, pci, dg, lu, L->rowptr, L->col, L->val, U->rowptr, U->col, U->val);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_error(e, "ilu_factor: split"));
    cleanup();
    *Lout = L;
    *Uout = U;
    return HEC_OK;
}
