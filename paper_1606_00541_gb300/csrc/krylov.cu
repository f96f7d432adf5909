// SpMV on HEC and the FP64 FGMRES(m) outer solver (the paper's experiments use GMRES(20) in
// FP64, Sec. 4; this library uses the flexible variant so that any preconditioner stage may
// change between iterations).
//
// Vectors of nrhs right-hand sides are row-major n x K (K = nrhs).  Reductions are
// deterministic: every block writes its partial sums and a second kernel adds them in a fixed
// order.  Each inner iteration runs: z_j = M^-1 v_j (ilu_apply), w = A z_j (SpMV), classical
// Gram-Schmidt twice (h = V^T w; w -= V h), ||w||, and the small Hessenberg update on the host.
#include <chrono>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace hec {
namespace {

constexpr int kThreads = 256;
constexpr int kDotGroup = 8;  // dot products per block row of the multi-dot

template <int KP>
__global__ void __launch_bounds__(kThreads) k_spmv(int n, int ld, int w, const int* __restrict__ ell_col,
                                                   const double* __restrict__ ell_val, const int* __restrict__ tptr,
                                                   const int* __restrict__ tcol, const double* __restrict__ tval,
                                                   int K, double alpha, const double* __restrict__ x, int ldx,
                                                   double beta, double* __restrict__ y, int ldy) {
    constexpr int RPB = kThreads / KP;
    const int q = threadIdx.x % KP;
    const int r = blockIdx.x * RPB + threadIdx.x / KP;
    if (r >= n || q >= K) return;
    double acc = 0.0;
    for (int k = 0; k < w; ++k) {
        const long s = (long)k * ld + r;
        const int c = __ldg(ell_col + s);
        if (c < 0) break;
        acc = fma(__ldg(ell_val + s), __ldg(x + (long)c * ldx + q), acc);
    }
    const int t1 = __ldg(tptr + r + 1);
    for (int t = __ldg(tptr + r); t < t1; ++t) acc = fma(__ldg(tval + t), __ldg(x + (long)__ldg(tcol + t) * ldx + q), acc);
    double* yp = y + (long)r * ldy + q;
    *yp = beta == 0.0 ? alpha * acc : fma(beta, *yp, alpha * acc);
}

// dst (dense n x K) = src (n x K with leading dimension lds)
__global__ void k_copy(long total, int K, const double* __restrict__ src, int lds, double* __restrict__ dst, int ldd) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long st = (long)gridDim.x * blockDim.x;
    for (; e < total; e += st) {
        long r = e / K;
        int q = (int)(e - r * K);
        dst[r * ldd + q] = src[r * lds + q];
    }
}

// partial[g][blk][q] for the dot products <V_a, w>, a = a0 + g, over this block's rows
template <int KP>
__global__ void __launch_bounds__(kThreads) k_multidot(int n, int K, const double* __restrict__ V, long vstride,
                                                       int count, const double* __restrict__ w,
                                                       double* __restrict__ partial) {
    constexpr int RPB = kThreads / KP;
    __shared__ double red[kThreads / 32][kDotGroup][KP];
    const int q = threadIdx.x % KP;
    const int a0 = blockIdx.y * kDotGroup;
    const int na = min(kDotGroup, count - a0);
    double acc[kDotGroup];
#pragma unroll
    for (int g = 0; g < kDotGroup; ++g) acc[g] = 0.0;
    if (q < K) {
        for (long r = (long)blockIdx.x * RPB + threadIdx.x / KP; r < n; r += (long)gridDim.x * RPB) {
            const double wv = w[r * K + q];
#pragma unroll
            for (int g = 0; g < kDotGroup; ++g)
                if (g < na) acc[g] = fma(V[(long)(a0 + g) * vstride + r * K + q], wv, acc[g]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int g = 0; g < kDotGroup; ++g) {
        double v = acc[g];
#pragma unroll
        for (int o = 16; o >= KP; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane < KP) red[warp][g][lane] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDotGroup * KP) {
        const int g = threadIdx.x / KP, qq = threadIdx.x % KP;
        double s = 0.0;
        for (int wi = 0; wi < kThreads / 32; ++wi) s += red[wi][g][qq];
        if (g < na && qq < K) partial[((long)(a0 + g) * gridDim.x + blockIdx.x) * K + qq] = s;
    }
}

// out[a][q] = sum over blocks of partial[a][blk][q] (+ out when accumulate)
__global__ void k_reduce(int count, int nblk, int K, const double* __restrict__ partial, double* out, int accumulate) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= count * K) return;
    int a = idx / K, q = idx % K;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[((long)a * nblk + b) * K + q];
    out[idx] = accumulate ? out[idx] + s : s;
}

// w -= sum_a V_a h[a]   (classical Gram-Schmidt update)
__global__ void k_cgs_update(long total, int K, const double* __restrict__ V, long vstride, int count,
                             const double* __restrict__ h, double* __restrict__ w) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long st = (long)gridDim.x * blockDim.x;
    for (; e < total; e += st) {
        int q = (int)(e % K);
        double s = w[e];
        for (int a = 0; a < count; ++a) s = fma(-V[(long)a * vstride + e], h[a * K + q], s);
        w[e] = s;
    }
}

__global__ void k_scale(long total, int K, double* __restrict__ v, const double* __restrict__ f) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long st = (long)gridDim.x * blockDim.x;
    for (; e < total; e += st) v[e] *= f[e % K];
}

// x (ldx) += sum_a Z_a y[a]
__global__ void k_update_x(long total, int K, const double* __restrict__ Z, long zstride, int count,
                           const double* __restrict__ y, double* __restrict__ x, int ldx) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long st = (long)gridDim.x * blockDim.x;
    for (; e < total; e += st) {
        long r = e / K;
        int q = (int)(e - r * K);
        double s = 0.0;
        for (int a = 0; a < count; ++a) s = fma(Z[(long)a * zstride + e], y[a * K + q], s);
        x[r * ldx + q] += s;
    }
}

int grid_for(long total) { return (int)std::max(1L, std::min((long)num_sms() * 8, (total + kThreads - 1) / kThreads)); }

// Dots <V_a, w> for a < count, per right-hand side, into dev_out[count][K].
struct Dots {
    double* partial = nullptr;
    int nblk = 0;
    int cap = 0;
    hec_status init(int maxcount, int K) {
        nblk = num_sms() * 2;
        cap = maxcount;
        return dalloc(&partial, (size_t)maxcount * nblk * K);
    }
    ~Dots() { cudaFree(partial); }
    template <int KP>
    hec_status run_kp(int n, int K, const double* V, long vstride, int count, const double* w, double* out, bool acc,
                      cudaStream_t s) {
        dim3 g(nblk, (count + kDotGroup - 1) / kDotGroup);
        k_multidot<KP><<<g, kThreads, 0, s>>>(n, K, V, vstride, count, w, partial);
        count_launch();
        k_reduce<<<(count * K + 127) / 128, 128, 0, s>>>(count, nblk, K, partial, out, acc ? 1 : 0);
        HEC_LAUNCHED();
        return HEC_OK;
    }
    hec_status run(int n, int K, const double* V, long vstride, int count, const double* w, double* out, bool acc,
                   cudaStream_t s) {
        if (K <= 1) return run_kp<1>(n, K, V, vstride, count, w, out, acc, s);
        if (K <= 2) return run_kp<2>(n, K, V, vstride, count, w, out, acc, s);
        if (K <= 4) return run_kp<4>(n, K, V, vstride, count, w, out, acc, s);
        if (K <= 8) return run_kp<8>(n, K, V, vstride, count, w, out, acc, s);
        return run_kp<16>(n, K, V, vstride, count, w, out, acc, s);
    }
};

}  // namespace

hec_status spmv_impl(const hec_matrix* A, int K, double alpha, const double* x, int ldx, double beta, double* y,
                     int ldy, cudaStream_t s) {
    if (A->n == 0) return HEC_OK;
    auto go = [&](auto kp) -> hec_status {
        constexpr int KP = decltype(kp)::value;
        int blocks = (int)(((long)A->n * KP + kThreads - 1) / kThreads);
        k_spmv<KP><<<blocks, kThreads, 0, s>>>(A->n, A->ld, A->w, A->ell_col, (const double*)A->ell_val, A->tptr,
                                               A->tcol, (const double*)A->tval, K, alpha, x, ldx, beta, y, ldy);
        HEC_LAUNCHED();
        return HEC_OK;
    };
    if (K <= 1) return go(std::integral_constant<int, 1>());
    if (K <= 2) return go(std::integral_constant<int, 2>());
    if (K <= 4) return go(std::integral_constant<int, 4>());
    if (K <= 8) return go(std::integral_constant<int, 8>());
    return go(std::integral_constant<int, 16>());
}

}  // namespace hec

using namespace hec;

HEC_API hec_status spmv(const hec_matrix* A, int nrhs, double alpha, const double* x, int ldx, double beta, double* y,
                        int ldy, void* stream) {
    clear_error();
    if (!A || A->tri || A->vdt != HEC_F64 || nrhs < 1 || nrhs > 16 || ldx < nrhs || ldy < nrhs ||
        (A->n > 0 && (!x || !y)))
        return set_error(HEC_ERR_INVALID_ARG, "spmv: need a general-mode FP64 HEC matrix and 1 <= nrhs <= 16");
    return spmv_impl(A, nrhs, alpha, x, ldx, beta, y, ldy, S(stream));
}

HEC_API hec_status fgmres_solve(const hec_matrix* A, const ilu_precond* M, int nrhs, const double* b, int ldb,
                                double* x, int ldx, int restart, double rtol, int max_iters, hec_fgmres_info* info,
                                void* stream) {
    clear_error();
    auto t_start = std::chrono::steady_clock::now();
    if (!A || A->tri || A->vdt != HEC_F64 || nrhs < 1 || nrhs > 16 || ldb < nrhs || ldx < nrhs || restart < 1 ||
        restart > 256 || !(rtol > 0) || max_iters < 0 || (M && (M->n_glob != A->n || M->max_nrhs < nrhs)))
        return set_error(HEC_ERR_INVALID_ARG, "fgmres_solve: bad argument");
    cudaStream_t s = S(stream);
    const int n = A->n, K = nrhs, m = restart;
    const long nk = (long)n * K;
    hec_fgmres_info inf{};
    if (n == 0) {
        inf.converged = 1;
        if (info) *info = inf;
        return HEC_OK;
    }
    double *V = nullptr, *Z = nullptr, *dh = nullptr, *dsc = nullptr;
    hec_status st = HEC_OK;
    Dots dots;
    if ((st = dalloc(&V, (size_t)(m + 1) * nk)) || (st = dalloc(&Z, (size_t)m * nk)) ||
        (st = dalloc(&dh, (size_t)(2 * (m + 1) + 4) * K)) || (st = dots.init(m + 1, K))) {
        cudaFree(V); cudaFree(Z); cudaFree(dh);
        return st;
    }
    double* dh2 = dh + (size_t)(m + 1) * K;  // second Gram-Schmidt pass
    dsc = dh2 + (size_t)(m + 1) * K;         // [K] scale factors, [K] norms
    double* dnorm = dsc + K;
    std::vector<double> H((size_t)(m + 1) * m * K), cs((size_t)m * K), sn((size_t)m * K), g((size_t)(m + 1) * K);
    std::vector<double> bnorm(K), hcol((size_t)(m + 1) * K), nrm(K), yv((size_t)m * K), f(K);
    std::vector<int> jq(K), conv(K, 0);
    const int gb = grid_for(nk);
    auto fail = [&](hec_status e) {
        cudaFree(V); cudaFree(Z); cudaFree(dh);
        return e;
    };
    auto norms = [&](const double* v, double* host) -> hec_status {
        HEC_CHECK(dots.run(n, K, v, nk, 1, v, dnorm, false, s));
        HEC_CUDA(cudaMemcpyAsync(host, dnorm, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
        HEC_CUDA(cudaStreamSynchronize(s));
        for (int q = 0; q < K; ++q) host[q] = std::sqrt(std::max(host[q], 0.0));
        return HEC_OK;
    };
    auto check_sweeps = [&]() -> hec_status {
        if (!M) return HEC_OK;
        hec_status a = hec_sync_status(M->L, stream);
        hec_status c = hec_sync_status(M->U, stream);
        return a != HEC_OK ? a : c;
    };
    // ||b||
    k_copy<<<gb, kThreads, 0, s>>>(nk, K, b, ldb, V, K);
    count_launch();
    if ((st = norms(V, bnorm.data()))) return fail(st);
    int its = 0, restarts = 0;
    double worst = 0.0;
    bool all_conv = false;
    while (true) {
        // r = b - A x, beta = ||r||, v_0 = r / beta
        k_copy<<<gb, kThreads, 0, s>>>(nk, K, b, ldb, V, K);
        count_launch();
        // V currently holds b; subtract A x (x may have a leading dimension != K)
        if (ldx == K) {
            if ((st = spmv_impl(A, K, -1.0, x, ldx, 1.0, V, K, s))) return fail(st);
        } else {
            if ((st = spmv_impl(A, K, -1.0, x, ldx, 1.0, V, K, s))) return fail(st);
        }
        if ((st = norms(V, nrm.data()))) return fail(st);
        all_conv = true;
        worst = 0.0;
        for (int q = 0; q < K; ++q) {
            double rel = bnorm[q] > 0 ? nrm[q] / bnorm[q] : 0.0;
            worst = std::max(worst, rel);
            conv[q] = rel <= rtol;
            all_conv = all_conv && conv[q];
            f[q] = nrm[q] > 0 ? 1.0 / nrm[q] : 0.0;
            std::fill(&g[0] + 0, &g[0] + 0, 0.0);
            for (int a = 0; a <= m; ++a) g[(size_t)a * K + q] = 0.0;
            g[q] = nrm[q];
            jq[q] = 0;
        }
        if (all_conv || its >= max_iters) break;
        HEC_CUDA(cudaMemcpyAsync(dsc, f.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
        k_scale<<<gb, kThreads, 0, s>>>(nk, K, V, dsc);
        count_launch();
        std::vector<int> active(K);
        for (int q = 0; q < K; ++q) active[q] = !conv[q];
        int j = 0;
        for (; j < m && its < max_iters; ++j) {
            double* vj = V + (long)j * nk;
            double* zj = Z + (long)j * nk;
            double* wv = V + (long)(j + 1) * nk;
            if (M) {
                if ((st = ilu_apply(M, K, vj, K, zj, K, stream))) return fail(st);
            } else {
                HEC_CUDA(cudaMemcpyAsync(zj, vj, sizeof(double) * nk, cudaMemcpyDeviceToDevice, s));
            }
            if ((st = spmv_impl(A, K, 1.0, zj, K, 0.0, wv, K, s))) return fail(st);
            // classical Gram-Schmidt, twice
            if ((st = dots.run(n, K, V, nk, j + 1, wv, dh, false, s))) return fail(st);
            k_cgs_update<<<gb, kThreads, 0, s>>>(nk, K, V, nk, j + 1, dh, wv);
            count_launch();
            if ((st = dots.run(n, K, V, nk, j + 1, wv, dh2, false, s))) return fail(st);
            k_cgs_update<<<gb, kThreads, 0, s>>>(nk, K, V, nk, j + 1, dh2, wv);
            count_launch();
            HEC_CUDA(cudaMemcpyAsync(hcol.data(), dh, sizeof(double) * (j + 1) * K, cudaMemcpyDeviceToHost, s));
            std::vector<double> h2((size_t)(j + 1) * K);
            HEC_CUDA(cudaMemcpyAsync(h2.data(), dh2, sizeof(double) * (j + 1) * K, cudaMemcpyDeviceToHost, s));
            if ((st = norms(wv, nrm.data()))) return fail(st);
            its++;
            bool any_active = false;
            for (int q = 0; q < K; ++q) {
                f[q] = 0.0;
                if (!active[q]) continue;
                for (int a = 0; a <= j; ++a) H[((size_t)a * m + j) * K + q] = hcol[a * K + q] + h2[a * K + q];
                double hn = nrm[q];
                H[((size_t)(j + 1) * m + j) * K + q] = hn;
                f[q] = hn > 0 ? 1.0 / hn : 0.0;
                for (int a = 0; a < j; ++a) {
                    double h0 = H[((size_t)a * m + j) * K + q], h1 = H[((size_t)(a + 1) * m + j) * K + q];
                    H[((size_t)a * m + j) * K + q] = cs[a * K + q] * h0 + sn[a * K + q] * h1;
                    H[((size_t)(a + 1) * m + j) * K + q] = -sn[a * K + q] * h0 + cs[a * K + q] * h1;
                }
                double h0 = H[((size_t)j * m + j) * K + q], h1 = hn;
                double den = std::sqrt(h0 * h0 + h1 * h1);
                double c = den == 0.0 ? 1.0 : h0 / den, sv = den == 0.0 ? 0.0 : h1 / den;
                cs[j * K + q] = c;
                sn[j * K + q] = sv;
                H[((size_t)j * m + j) * K + q] = c * h0 + sv * h1;
                double gj = g[(size_t)j * K + q];
                g[(size_t)(j + 1) * K + q] = -sv * gj;
                g[(size_t)j * K + q] = c * gj;
                jq[q] = j + 1;
                if (std::fabs(g[(size_t)(j + 1) * K + q]) <= rtol * bnorm[q] || hn == 0.0) active[q] = 0;
                else any_active = true;
            }
            if (!any_active) { j++; break; }
            HEC_CUDA(cudaMemcpyAsync(dsc, f.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
            k_scale<<<gb, kThreads, 0, s>>>(nk, K, wv, dsc);
            count_launch();
        }
        // back substitution on the rotated Hessenberg, x += Z y
        std::fill(yv.begin(), yv.end(), 0.0);
        int jmax = 0;
        for (int q = 0; q < K; ++q) {
            int jj = jq[q];
            jmax = std::max(jmax, jj);
            for (int a = jj - 1; a >= 0; --a) {
                double sacc = g[(size_t)a * K + q];
                for (int c = a + 1; c < jj; ++c) sacc -= H[((size_t)a * m + c) * K + q] * yv[c * K + q];
                double d = H[((size_t)a * m + a) * K + q];
                yv[a * K + q] = d != 0.0 ? sacc / d : 0.0;
            }
        }
        if (jmax > 0) {
            HEC_CUDA(cudaMemcpyAsync(dh, yv.data(), sizeof(double) * jmax * K, cudaMemcpyHostToDevice, s));
            k_update_x<<<gb, kThreads, 0, s>>>(nk, K, Z, nk, jmax, dh, x, ldx);
            count_launch();
        }
        restarts++;
        if ((st = check_sweeps())) return fail(st);
    }
    if ((st = check_sweeps())) return fail(st);
    inf.iterations = its;
    inf.restarts = restarts;
    inf.converged = all_conv ? 1 : 0;
    inf.rel_residual = worst;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (info) *info = inf;
    cudaFree(V); cudaFree(Z); cudaFree(dh);
    if (!all_conv) return set_error(HEC_ERR_NOT_CONVERGED, "fgmres_solve: max_iters reached before rtol");
    return HEC_OK;
}
