// ILUT(p, tol) on the GPU (Sec. 3 names ILUT; the dual-threshold rule is Saad's): for row i,
// tau_i = tol * ||a_i||_2; the row's entries k < i are eliminated in ascending column order,
// w_k <- w_k / u_kk, a multiplier with |w_k| < tau_i is dropped, otherwise w_j <- w_j - w_k u_kj
// for the entries j > k of U row k (creating fill); then entries below tau_i are dropped and
// the p largest magnitudes are kept in the strict lower and in the strict upper part (ties to
// the smaller column), the diagonal always.  L is unit lower with its 1.0 diagonal stored.
//
// GB300 design: one cooperative persistent launch; row i belongs to warp i mod W and a warp
// takes its rows in increasing order, so the smallest unfinished row can always proceed.  A
// warp keeps its row as a sorted (column, value) list in shared memory; merging U row k is a
// warp-parallel binary search plus a ballot-ranked insertion of the fill.  A finished row is
// written into fixed slots (p strictly lower, 1 + p upper entries) and published with a release
// store of its U length; a row that needs U row k waits for that flag (acquire, bounded).  The
// arithmetic is the definition's, operation by operation and without fused multiply-adds
// (w_j - (w_k * u_kj), the norm summed in row order), so the drop decisions match any IEEE
// FP64 implementation that performs the same operations in the same order.
#include <algorithm>

#include "internal.cuh"
#include "sync.cuh"

namespace hec {
void free_csr(hec_csr* M);
hec_status validate_csr(int n, const int* rp, const int* col, int uplo, cudaStream_t s);

namespace {

constexpr unsigned kAll = 0xffffffffu;
// working-list capacity per warp and warps per block, tried in this order when a row's fill
// outgrows the list (24 bytes per entry and warp: two column and two value buffers)
constexpr int kCaps[4] = {120, 240, 1984, 9000};
constexpr int kWarpsFor[4] = {8, 8, 4, 1};

struct IlutParams {
    int n, p;
    double tol;
    const int* __restrict__ rp;
    const int* __restrict__ ci;
    const double* __restrict__ v;
    int* lcol;     // [n * p]
    double* lval;
    int* llen;     // [n]
    int* ucol;     // [n * (p + 1)], diagonal first
    double* uval;
    int* ulen;     // [n], 0 until the row is published
    int* status;
    long long budget;
    int cap;       // entries of a row's working list
};

__device__ __forceinline__ int ld_acquire_flag(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ldcg_i(const int* p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg_d(const double* p) { return __ldcg(p); }

// position of the first entry with column >= c in cols[lo, hi)
__device__ __forceinline__ int lower_bound(const int* cols, int lo, int hi, int c) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cols[mid] < c) lo = mid + 1; else hi = mid;
    }
    return lo;
}

}  // namespace
}  // namespace hec

namespace hec {
namespace {

// publish U row i: its length is the flag later rows wait on (release after the warp's stores)
__device__ __forceinline__ void ilut_publish(const IlutParams& P, int i, int lane, int nu1) {
    __syncwarp();
    if (lane == 0) {
        __threadfence();
        st_release_i32(P.ulen + i, nu1);
    }
    __syncwarp();
}

// One strict part of a finished row, list positions [b0, b1): the entries with w != 0 and
// |w| >= tau are the candidates; the p largest magnitudes are kept (ties to the smaller column)
// and written to out_col / out_val in column order.  The candidates are first compacted, in
// column order, into the warp's spare buffer; up to 64 of them are ranked with shuffles (two per
// lane), more by a scan of the compacted list.  Returns the number kept.
__device__ __forceinline__ int ilut_select(const int* col, const double* val, int b0, int b1, double tau, int p,
                                           int lane, int* scol, double* sval, int* out_col, double* out_val) {
    const unsigned lt = (1u << lane) - 1u;
    int m = 0;
    for (int bb = b0; bb < b1; bb += 32) {
        const int b = bb + lane;
        bool c = false;
        if (b < b1) {
            const double v = val[b];
            c = v != 0.0 && !(fabs(v) < tau);
        }
        const unsigned cm = __ballot_sync(kAll, c);
        if (c) {
            scol[m + __popc(cm & lt)] = col[b];
            sval[m + __popc(cm & lt)] = val[b];
        }
        m += __popc(cm);
    }
    __syncwarp();
    if (m == 0 || p == 0) return 0;
    int kept = 0;
    if (m <= 64) {
        const bool h0 = lane < m, h1 = lane + 32 < m;
        const double a0 = h0 ? fabs(sval[lane]) : 0.0, a1 = h1 ? fabs(sval[lane + 32]) : 0.0;
        int r0 = 0, r1 = 0;  // candidates ahead of this lane's two (larger, or equal with a smaller column)
        for (int t = 0; t < m; ++t) {
            const double at = __shfl_sync(kAll, t < 32 ? a0 : a1, t & 31);
            r0 += (at > a0 || (at == a0 && t < lane)) ? 1 : 0;
            r1 += (at > a1 || (at == a1 && t < lane + 32)) ? 1 : 0;
        }
        const bool k0 = h0 && r0 < p, k1 = h1 && r1 < p;
        const unsigned m0 = __ballot_sync(kAll, k0), m1 = __ballot_sync(kAll, k1);
        if (k0) { out_col[__popc(m0 & lt)] = scol[lane]; out_val[__popc(m0 & lt)] = sval[lane]; }
        if (k1) {
            out_col[__popc(m0) + __popc(m1 & lt)] = scol[lane + 32];
            out_val[__popc(m0) + __popc(m1 & lt)] = sval[lane + 32];
        }
        kept = __popc(m0) + __popc(m1);
    } else {
        for (int eb = 0; eb < m; eb += 32) {
            const int e = eb + lane;
            bool k = false;
            if (e < m) {
                const double ae = fabs(sval[e]);
                int rank = 0;
                for (int t = 0; t < m && rank < p; ++t) {
                    const double at = fabs(sval[t]);
                    rank += (at > ae || (at == ae && t < e)) ? 1 : 0;
                }
                k = rank < p;
            }
            const unsigned km = __ballot_sync(kAll, k);
            if (k) { out_col[kept + __popc(km & lt)] = scol[e]; out_val[kept + __popc(km & lt)] = sval[e]; }
            kept += __popc(km);
        }
    }
    __syncwarp();
    return kept;
}

// a row that cannot be factored (error recorded): diagonal 1.0 only, so later rows still finish
__device__ __forceinline__ void ilut_fail(const IlutParams& P, int i, int lane, int code) {
    if (lane == 0) {
        record(P.status, code);
        P.ucol[(long)i * (P.p + 1)] = i;
        P.uval[(long)i * (P.p + 1)] = 1.0;
        P.llen[i] = 0;
    }
    ilut_publish(P, i, lane, 1);
}

__global__ void __launch_bounds__(256) k_ilut(IlutParams P) {
    // per warp: values [2][cap] (8-byte aligned first), columns [2][cap], the merge's new columns [32]
    extern __shared__ __align__(16) unsigned char ilut_smem[];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    const int cap = P.cap;
    double* wv = (double*)(ilut_smem + (size_t)wl * (24 * (size_t)cap + 128));
    int* wc = (int*)(wv + 2 * cap);
    int* s_newp = wc + 2 * cap;
    const int W = gridDim.x * nwb;
    const int up = P.p + 1;
    for (int i = blockIdx.x * nwb + wl; i < P.n; i += W) {
        int cur = 0;
        int* col = wc;
        double* val = wv;
        const int a0 = __ldg(P.rp + i);
        int len = __ldg(P.rp + i + 1) - a0;
        if (len + 1 > cap) { ilut_fail(P, i, lane, HEC_ERR_OUT_OF_BOUNDS); continue; }
        for (int e = lane; e < len; e += 32) {
            col[e] = __ldg(P.ci + a0 + e);
            val[e] = __ldg(P.v + a0 + e);
        }
        __syncwarp();
        // tau = tol * ||a_i||_2, the squares summed in row order
        double tau = 0.0;
        if (lane == 0) {
            double nrm = 0.0;
            for (int e = 0; e < len; ++e) nrm = __dadd_rn(nrm, __dmul_rn(val[e], val[e]));
            tau = __dmul_rn(P.tol, __dsqrt_rn(nrm));
        }
        tau = __shfl_sync(kAll, tau, 0);
        // a structural diagonal slot when the row has none
        {
            const int dpos = lower_bound(col, 0, len, i);
            if (dpos == len || col[dpos] != i) {
                int* ncol = (wc + (cur ^ 1) * cap);
                double* nval = (wv + (cur ^ 1) * cap);
                for (int e = lane; e < len; e += 32) {
                    ncol[e + (e >= dpos)] = col[e];
                    nval[e + (e >= dpos)] = val[e];
                }
                if (lane == 0) { ncol[dpos] = i; nval[dpos] = 0.0; }
                __syncwarp();
                cur ^= 1; col = ncol; val = nval; ++len;
            }
        }
        int failed = 0;  // the error code of a row that cannot be finished
        for (int pos = 0; pos < len && col[pos] < i; ++pos) {
            const int k = col[pos];
            int ul = 0;
            if (lane == 0) {
                ul = ld_acquire_flag(P.ulen + k);
                if (ul == 0) {
                    const long long t0 = clock64();
                    for (unsigned it = 1; (ul = ld_acquire_flag(P.ulen + k)) == 0; ++it)
                        if ((it & 63u) == 0u && (clock64() - t0 > P.budget || ld_relaxed_u32(P.status) != 0u)) {
                            ul = -1;
                            break;
                        }
                }
            }
            ul = __shfl_sync(kAll, ul, 0);
            if (ul < 0) { failed = HEC_ERR_TIMEOUT; break; }
            // U row k's first 32 entries in one batch of loads; u_kk is its first entry
            int j0 = 0;
            double u0 = 0.0;
            if (lane < ul) {
                j0 = ldcg_i(P.ucol + (long)k * up + lane);
                u0 = ldcg_d(P.uval + (long)k * up + lane);
            }
            const double wk = __ddiv_rn(val[pos], __shfl_sync(kAll, u0, 0));
            __syncwarp();
            if (fabs(wk) < tau) {  // dropped multiplier
                if (lane == 0) val[pos] = 0.0;
                __syncwarp();
                continue;
            }
            if (lane == 0) val[pos] = wk;
            __syncwarp();
            // w_j -= w_k * u_kj for the entries j > k of U row k (q >= 1), 32 at a time
            for (int qb = 0; qb < ul; qb += 32) {
                const int q = qb + lane;
                const bool has = q >= 1 && q < ul;
                int j = j0;
                double u = u0;
                if (qb > 0 && has) {
                    j = ldcg_i(P.ucol + (long)k * up + q);
                    u = ldcg_d(P.uval + (long)k * up + q);
                }
                const int at = has ? lower_bound(col, pos + 1, len, j) : len;
                const bool found = has && at < len && col[at] == j;
                const double prod = __dmul_rn(wk, u);
                if (found) val[at] = __dsub_rn(val[at], prod);
                const unsigned newm = __ballot_sync(kAll, has && !found);
                const int nnew = __popc(newm);
                __syncwarp();
                if (nnew == 0) continue;
                if (len + nnew > cap) { failed = HEC_ERR_OUT_OF_BOUNDS; break; }
                const int rk = __popc(newm & ((1u << lane) - 1u));
                if (has && !found) s_newp[rk] = j;
                __syncwarp();
                int* ncol = (wc + (cur ^ 1) * cap);
                double* nval = (wv + (cur ^ 1) * cap);
                for (int e = lane; e < len; e += 32) {
                    const int c = col[e];
                    int sh = 0;
                    for (int t = 0; t < nnew; ++t) sh += s_newp[t] < c;
                    ncol[e + sh] = c;
                    nval[e + sh] = val[e];
                }
                if (has && !found) {  // a fill entry: 0 - w_k u_kj
                    ncol[at + rk] = j;
                    nval[at + rk] = __dsub_rn(0.0, prod);
                }
                __syncwarp();
                cur ^= 1; col = ncol; val = nval; len += nnew;
            }
            if (failed) break;
        }
        if (failed) {
            ilut_fail(P, i, lane, failed);
            continue;
        }
        // drop below tau, keep the p largest of each strict part (ties to the smaller column); the
        // upper part first, so the rows waiting for U row i are released before the lower part
        const int dp = lower_bound(col, 0, len, i);
        const double wd = val[dp];
        if (wd == 0.0) { ilut_fail(P, i, lane, HEC_ERR_ZERO_PIVOT); continue; }
        int* scol = wc + (cur ^ 1) * cap;
        double* sval = wv + (cur ^ 1) * cap;
        const int nu = ilut_select(col, val, dp + 1, len, tau, P.p, lane, scol, sval, P.ucol + (long)i * up + 1,
                                   P.uval + (long)i * up + 1);
        if (lane == 0) {
            P.ucol[(long)i * up] = i;
            P.uval[(long)i * up] = wd;
        }
        ilut_publish(P, i, lane, nu + 1);
        const int nl = ilut_select(col, val, 0, dp, tau, P.p, lane, scol, sval, P.lcol + (long)i * P.p,
                                   P.lval + (long)i * P.p);
        if (lane == 0) P.llen[i] = nl;
    }
}

// CSR of L (kept strict entries, then the unit diagonal) and U (diagonal first) from the slots
__global__ void k_ilut_rowlen(int n, const int* __restrict__ llen, const int* __restrict__ ulen, int* lrl, int* url) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        lrl[i] = llen[i] + 1;
        url[i] = ulen[i];
    }
}

__global__ void k_ilut_pack(int n, int p, const int* __restrict__ lrp, const int* __restrict__ llen,
                            const int* __restrict__ lcol, const double* __restrict__ lval, int* Lc, double* Lv,
                            const int* __restrict__ urp, const int* __restrict__ ucol, const double* __restrict__ uval,
                            int* Uc, double* Uv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l0 = lrp[i], nl = llen[i];
    for (int a = 0; a < nl; ++a) {
        Lc[l0 + a] = lcol[(long)i * p + a];
        Lv[l0 + a] = lval[(long)i * p + a];
    }
    Lc[l0 + nl] = i;
    Lv[l0 + nl] = 1.0;
    const int u0 = urp[i], nu = urp[i + 1] - u0;
    for (int a = 0; a < nu; ++a) {
        Uc[u0 + a] = ucol[(long)i * (p + 1) + a];
        Uv[u0 + a] = uval[(long)i * (p + 1) + a];
    }
}

}  // namespace
}  // namespace hec

using namespace hec;

HEC_API hec_status ilut_factor(int n, const int* rowptr, const int* col, const double* val, int p, double tol,
                               hec_csr** Lout, hec_csr** Uout, void* stream) {
    clear_error();
    if (!Lout || !Uout || n < 0 || p < 0 || !(tol >= 0.0) || (n > 0 && (!rowptr || !col || !val)))
        return set_error(HEC_ERR_INVALID_ARG, "ilut_factor: bad argument (need p >= 0, tol >= 0)");
    *Lout = *Uout = nullptr;
    cudaStream_t s = S(stream);
    HEC_CHECK(validate_csr(n, rowptr, col, -1, s));
    hec_csr *L = new hec_csr(), *U = new hec_csr();
    int *lcol = nullptr, *llen = nullptr, *ucol = nullptr, *ulen = nullptr, *status = nullptr, *lrl = nullptr,
        *url = nullptr;
    double *lval = nullptr, *uval = nullptr;
    auto cleanup = [&]() {
        dfree(lcol); dfree(llen); dfree(ucol); dfree(ulen); dfree(status); dfree(lrl);
        dfree(url); dfree(lval); dfree(uval);
    };
    auto fail = [&](hec_status e) {
        cleanup();
        free_csr(L);
        free_csr(U);
        return e;
    };
    hec_status st = HEC_OK;
    const size_t ln = (size_t)n * p + 1, un = (size_t)n * (p + 1) + 1;
    if ((st = dalloc(&lcol, ln)) || (st = dalloc(&lval, ln)) || (st = dalloc(&llen, (size_t)n + 1)) ||
        (st = dalloc(&ucol, un)) || (st = dalloc(&uval, un)) || (st = dalloc(&ulen, (size_t)n + 1)) ||
        (st = dalloc(&status, 1)) || (st = dalloc(&lrl, (size_t)n + 1)) || (st = dalloc(&url, (size_t)n + 1)) ||
        (st = dalloc(&L->rowptr, (size_t)n + 1)) || (st = dalloc(&U->rowptr, (size_t)n + 1)))
        return fail(st);
    if (cudaMemsetAsync(ulen, 0, sizeof(int) * ((size_t)n + 1), s) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess)
        return fail(cuda_error(cudaGetLastError(), "ilut_factor: memset"));
    L->n = U->n = n;
    if (n > 0) {
        IlutParams P;
        P.n = n; P.p = p; P.tol = tol; P.rp = rowptr; P.ci = col; P.v = val;
        P.lcol = lcol; P.lval = lval; P.llen = llen; P.ucol = ucol; P.uval = uval; P.ulen = ulen;
        P.status = status;
        P.budget = 4000000000LL;  // about two seconds of SM cycles per wait
        const void* k = (const void*)k_ilut;
        int h = 0, cap = 0;
        // a larger working list (fewer warps per block) only when a row's fill outgrew the last one
        for (int t = 0; t < 4; ++t) {
            cap = kCaps[t];
            const int warps = kWarpsFor[t];
            const size_t smem = (size_t)warps * (24 * (size_t)cap + 128);
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return fail(cuda_error(cudaGetLastError(), "ilut_factor: shared memory"));
            const int per_sm = max_coop_blocks(k, warps * 32, smem);
            if (per_sm <= 0) return fail(set_error(HEC_ERR_CUDA, "ilut_factor: kernel cannot be resident"));
            const int blocks = (int)std::max(1L, std::min((long)per_sm * num_sms(), ((long)n + warps - 1) / warps));
            if (t > 0 && (cudaMemsetAsync(ulen, 0, sizeof(int) * ((size_t)n + 1), s) != cudaSuccess ||
                          cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess))
                return fail(cuda_error(cudaGetLastError(), "ilut_factor: memset"));
            P.cap = cap;
            void* args[] = {&P};
            if (cudaLaunchCooperativeKernel(k, dim3(blocks), dim3(warps * 32), args, smem, s) != cudaSuccess)
                return fail(cuda_error(cudaGetLastError(), "ilut_factor: launch"));
            count_launch();
            if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return fail(cuda_error(cudaGetLastError(), "ilut_factor"));
            if (h != HEC_ERR_OUT_OF_BOUNDS) break;
        }
        if (h == HEC_ERR_ZERO_PIVOT) return fail(set_error(HEC_ERR_ZERO_PIVOT, "ilut_factor: zero pivot"));
        if (h == HEC_ERR_OUT_OF_BOUNDS)
            return fail(set_error(HEC_ERR_OUT_OF_BOUNDS, "ilut_factor: a row's working fill exceeds " +
                                                             std::to_string(cap) + " entries"));
        if (h) return fail(set_error((hec_status)h, "ilut_factor: a dependency wait timed out"));
        const int g = (n + 255) / 256;
        k_ilut_rowlen<<<g, 256, 0, s>>>(n, llen, ulen, lrl, url);
        count_launch();
    }
    if ((st = exclusive_scan_i32(lrl, L->rowptr, n, true, s)) || (st = exclusive_scan_i32(url, U->rowptr, n, true, s)))
        return fail(st);
    int hl = 0, hu = 0;
    if (cudaMemcpy(&hl, L->rowptr + n, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&hu, U->rowptr + n, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(cuda_error(cudaGetLastError(), "ilut_factor: nnz"));
    L->nnz = hl;
    U->nnz = hu;
    if ((st = dalloc(&L->col, (size_t)hl)) || (st = dalloc(&L->val, (size_t)hl)) || (st = dalloc(&U->col, (size_t)hu)) ||
        (st = dalloc(&U->val, (size_t)hu)))
        return fail(st);
    if (n > 0) {
        k_ilut_pack<<<(n + 255) / 256, 256, 0, s>>>(n, p, L->rowptr, llen, lcol, lval, L->col, L->val, U->rowptr, ucol,
                                                   uval, U->col, U->val);
        count_launch();
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(cuda_error(cudaGetLastError(), "ilut_factor: pack"));
    cleanup();
    *Lout = L;
    *Uout = U;
    return HEC_OK;
}
