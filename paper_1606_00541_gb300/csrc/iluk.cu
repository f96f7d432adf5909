// ILU(k) pattern for any level of fill k on the GPU (Sec. 3: ILU(k), "k is the fill-in level").
//
// The level-of-fill rule: entries of A have level 0; eliminating pivot q of row i (q < i, in
// ascending order, fill pivots included) gives entry (i, j), j > q in U row q, the level
// lev(i, q) + lev(q, j) + 1, and the entry keeps the smallest level it receives; entries with
// level <= k are kept.  Row i therefore needs the final upper pattern (with levels) of every
// pivot row, which is the dependency structure of the factorization itself.
//
// GB300 design, as the GPU ILUT: one cooperative persistent launch; row i belongs to warp
// i mod W and a warp takes its rows in increasing order, so the smallest unfinished row can
// always proceed.  A warp keeps its row as a sorted (column, level) list in shared memory;
// merging the upper part of pivot row q is a warp-parallel binary search plus a ballot-ranked
// insertion of the new columns.  A finished row is written to fixed slots of `cap` entries and
// published with a release store (1 + the position of its diagonal); a row that needs pivot row q
// waits for that flag (acquire, bounded).  A row whose pattern outgrows `cap` records
// OUT_OF_BOUNDS and the host retries with a larger list.  The numeric factorization then runs on
// the pattern (factor.cu).
#include <algorithm>

#include "internal.cuh"
#include "sync.cuh"

namespace hec {
namespace {

constexpr unsigned kAllLanes = 0xffffffffu;
// working-list capacity per warp and warps per block, tried in this order
constexpr int kKCaps[4] = {64, 256, 1024, 4096};
constexpr int kKWarps[4] = {8, 8, 4, 2};

struct IlukParams {
    int n, k;
    const int* __restrict__ rp;
    const int* __restrict__ ci;
    int* pcol;     // [n * cap] the row's final pattern, ascending
    int* plev;     // [n * cap] its levels of fill
    int* plen;     // [n] pattern length
    int* ready;    // [n] 0 until the row is published, then 1 + the diagonal's position
    int* status;
    long long budget;
    int cap;
};

__device__ __forceinline__ int k_lower_bound(const int* cols, int lo, int hi, int c) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cols[mid] < c) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int acquire_i32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// write row i's list to its slots and publish it (release after the warp's stores)
__device__ __forceinline__ void iluk_publish(const IlukParams& P, int i, int lane, const int* col, const int* lev,
                                             int len) {
    const long base = (long)i * P.cap;
    for (int e = lane; e < len; e += 32) {
        P.pcol[base + e] = col[e];
        P.plev[base + e] = lev[e];
    }
    const int dpos = k_lower_bound(col, 0, len, i);
    __syncwarp();
    if (lane == 0) {
        P.plen[i] = len;
        __threadfence();
        st_release_i32(P.ready + i, dpos + 1);
    }
    __syncwarp();
}

// a row that cannot be finished (error recorded): its diagonal only, so later rows still finish
__device__ __forceinline__ void iluk_fail(const IlukParams& P, int i, int lane, int code) {
    if (lane == 0) {
        record(P.status, code);
        P.pcol[(long)i * P.cap] = i;
        P.plev[(long)i * P.cap] = 0;
        P.plen[i] = 1;
        __threadfence();
        st_release_i32(P.ready + i, 1);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(256) k_iluk_symbolic(IlukParams P) {
    // per warp: columns [2][cap], levels [2][cap], the merge's new columns and levels [32] each
    extern __shared__ __align__(16) int iluk_smem[];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    const int cap = P.cap;
    int* wc = iluk_smem + (size_t)wl * (4 * (size_t)cap + 64);
    int* wlv = wc + 2 * cap;
    int* s_newc = wlv + 2 * cap;
    int* s_newl = s_newc + 32;
    const int W = gridDim.x * nwb;
    for (int i = blockIdx.x * nwb + wl; i < P.n; i += W) {
        int cur = 0;
        int* col = wc;
        int* lev = wlv;
        const int a0 = __ldg(P.rp + i);
        int len = __ldg(P.rp + i + 1) - a0;
        if (len > cap) { iluk_fail(P, i, lane, HEC_ERR_OUT_OF_BOUNDS); continue; }
        for (int e = lane; e < len; e += 32) {
            col[e] = __ldg(P.ci + a0 + e);
            lev[e] = 0;
        }
        __syncwarp();
        int failed = 0;
        for (int pos = 0; pos < len && col[pos] < i; ++pos) {
            const int q = col[pos];
            const int liq = lev[pos];
            int d1 = 0;  // 1 + the diagonal's position in row q
            if (lane == 0) {
                d1 = acquire_i32(P.ready + q);
                if (d1 == 0) {
                    const long long t0 = clock64();
                    for (unsigned it = 1; (d1 = acquire_i32(P.ready + q)) == 0; ++it)
                        if ((it & 63u) == 0u && (clock64() - t0 > P.budget || ld_relaxed_u32(P.status) != 0u)) {
                            d1 = -1;
                            break;
                        }
                }
            }
            d1 = __shfl_sync(kAllLanes, d1, 0);
            if (d1 < 0) { failed = HEC_ERR_TIMEOUT; break; }
            const int qlen = __ldcg(P.plen + q);
            const long qb = (long)q * cap;
            // the entries j > q of row q, 32 at a time: level liq + lev(q, j) + 1 when within k
            for (int eb = d1; eb < qlen; eb += 32) {
                const int e = eb + lane;
                int j = 0, nl = 0x7fffffff;
                if (e < qlen) {
                    j = __ldcg(P.pcol + qb + e);
                    nl = liq + __ldcg(P.plev + qb + e) + 1;
                }
                const bool has = e < qlen && nl <= P.k;
                const int at = has ? k_lower_bound(col, pos + 1, len, j) : len;
                const bool found = has && at < len && col[at] == j;
                if (found && nl < lev[at]) lev[at] = nl;
                const unsigned newm = __ballot_sync(kAllLanes, has && !found);
                const int nnew = __popc(newm);
                __syncwarp();
                if (nnew == 0) continue;
                if (len + nnew > cap) { failed = HEC_ERR_OUT_OF_BOUNDS; break; }
                const int rk = __popc(newm & ((1u << lane) - 1u));
                if (has && !found) {
                    s_newc[rk] = j;
                    s_newl[rk] = nl;
                }
                __syncwarp();
                int* ncol = wc + (cur ^ 1) * cap;
                int* nlev = wlv + (cur ^ 1) * cap;
                for (int x = lane; x < len; x += 32) {
                    const int c = col[x];
                    int sh = 0;
                    for (int t = 0; t < nnew; ++t) sh += s_newc[t] < c;
                    ncol[x + sh] = c;
                    nlev[x + sh] = lev[x];
                }
                if (has && !found) {
                    ncol[at + rk] = j;
                    nlev[at + rk] = nl;
                }
                __syncwarp();
                cur ^= 1;
                col = ncol;
                lev = nlev;
                len += nnew;
            }
            if (failed) break;
        }
        if (failed) {
            iluk_fail(P, i, lane, failed);
            continue;
        }
        iluk_publish(P, i, lane, col, lev, len);
    }
}

__global__ void k_iluk_pack(int n, int cap, const int* __restrict__ prp, const int* __restrict__ pcol, int* pci) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = prp[i], m = prp[i + 1] - o;
    for (int e = 0; e < m; ++e) pci[o + e] = pcol[(long)i * cap + e];
}

}  // namespace

// The ILU(k) pattern of A (n x n, rows ascending) as CSR: *prp (n + 1) and *pci (*nnz entries),
// allocated here.  Synchronizes `s`.
hec_status iluk_pattern(int n, const int* rp, const int* ci, int k, int** prp, int** pci, long long* nnz,
                        cudaStream_t s) {
    *prp = *pci = nullptr;
    *nnz = 0;
    int *pcol = nullptr, *plev = nullptr, *plen = nullptr, *ready = nullptr, *status = nullptr;
    auto cleanup = [&]() { dfree(pcol); dfree(plev); dfree(plen); dfree(ready); dfree(status); };
    auto fail = [&](hec_status e) {
        cleanup();
        dfree(*prp);
        dfree(*pci);
        *prp = *pci = nullptr;
        return e;
    };
    hec_status st = HEC_OK;
    if ((st = dalloc(&plen, (size_t)n + 1)) || (st = dalloc(&ready, (size_t)n + 1)) || (st = dalloc(&status, 1)) ||
        (st = dalloc(prp, (size_t)n + 1)))
        return fail(st);
    IlukParams P;
    P.n = n; P.k = k; P.rp = rp; P.ci = ci; P.plen = plen; P.ready = ready; P.status = status;
    P.budget = 4000000000LL;  // about two seconds of SM cycles per wait
    const void* kern = (const void*)k_iluk_symbolic;
    int h = 0, cap = 0;
    for (int t = 0; t < 4; ++t) {
        cap = kKCaps[t];
        const int warps = kKWarps[t];
        dfree(pcol);
        dfree(plev);
        pcol = plev = nullptr;
        if ((st = dalloc(&pcol, (size_t)n * cap)) || (st = dalloc(&plev, (size_t)n * cap))) return fail(st);
        const size_t smem = (size_t)warps * (16 * (size_t)cap + 256);
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "ilu_factor: shared memory"));
        const int per_sm = max_coop_blocks(kern, warps * 32, smem);
        if (per_sm <= 0) return fail(set_error(HEC_ERR_CUDA, "ilu_factor: symbolic kernel cannot be resident"));
        const int blocks = (int)std::max(1L, std::min((long)per_sm * num_sms(), ((long)n + warps - 1) / warps));
        if (cudaMemsetAsync(ready, 0, sizeof(int) * ((size_t)n + 1), s) != cudaSuccess ||
            cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "ilu_factor: memset"));
        P.pcol = pcol;
        P.plev = plev;
        P.cap = cap;
        void* args[] = {&P};
        if (cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(warps * 32), args, smem, s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "ilu_factor: symbolic launch"));
        count_launch();
        if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "ilu_factor: symbolic"));
        if (h != HEC_ERR_OUT_OF_BOUNDS) break;
    }
    if (h == HEC_ERR_OUT_OF_BOUNDS)
        return fail(set_error(HEC_ERR_OUT_OF_BOUNDS, "ilu_factor: a row's ILU(k) pattern exceeds " +
                                                         std::to_string(cap) + " entries"));
    if (h) return fail(set_error((hec_status)h, "ilu_factor: a dependency wait of the symbolic phase timed out"));
    if ((st = exclusive_scan_i32(plen, *prp, n, true, s))) return fail(st);
    int hn = 0;
    HEC_CUDA(cudaMemcpy(&hn, *prp + n, sizeof(int), cudaMemcpyDeviceToHost));
    if ((st = dalloc(pci, (size_t)hn))) return fail(st);
    k_iluk_pack<<<(n + 255) / 256, 256, 0, s>>>(n, cap, *prp, pcol, *pci);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_error(e, "ilu_factor: pattern"));
    *nnz = hn;
    cleanup();
    return HEC_OK;
}

}  // namespace hec
