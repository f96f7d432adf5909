// Level analysis (Eq. 2), the level-ordering map m (Eq. 3) and input validation.
//
// Levels are computed by one sync-free kernel: rows are visited in the order of the lower
// problem (i for L, n-1-i for the reversed U of Sec. 2.2) and each row waits, point to point,
// for the levels of its dependencies, which are always earlier in that order.  Work is handed
// out statically, chunk c to warp c mod W, under a cooperative launch that guarantees all warps
// are resident, so the warp holding the earliest unfinished chunk can always proceed.
//
// The map is a stable counting sort of rows by level (least-significant-digit radix passes of
// 8 bits over the level), which keeps the rows of each level in ascending order of the lower
// problem's index as Eq. 3 requires; it is exact integer work and bit-identical to the plain
// serial construction.
#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "sync.cuh"

namespace hec {
namespace {

// ---- validation -----------------------------------------------------------------------------
// code: UNSORTED (row not strictly ascending, column out of range, bad rowptr),
// NOT_TRIANGULAR, MISSING_DIAG.  uplo: 0 lower, 1 upper, -1 general (only sortedness).
__global__ void k_validate(int n, const int* __restrict__ rp, const int* __restrict__ col, int uplo, int* code) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = rp[i], b = rp[i + 1];
    if (b < a || a < 0) { atomicCAS(code, 0, HEC_ERR_UNSORTED); return; }
    int prev = -1;
    bool diag = false;
    for (int p = a; p < b; ++p) {
        int j = col[p];
        if (j < 0 || j >= n || j <= prev) { atomicCAS(code, 0, HEC_ERR_UNSORTED); return; }
        prev = j;
        if (j == i) diag = true;
        if ((uplo == 0 && j > i) || (uplo == 1 && j < i)) { atomicCAS(code, 0, HEC_ERR_NOT_TRIANGULAR); return; }
    }
    if (uplo >= 0 && !diag) atomicCAS(code, 0, HEC_ERR_MISSING_DIAG);
}

// ---- levels ---------------------------------------------------------------------------------
// lower_only: treat only j < i (uplo 0) / j > i (uplo 1) as dependencies and ignore the rest
// (used for the lower pattern of a general matrix by the factorization).
__global__ void k_levels(int n, const int* __restrict__ rp, const int* __restrict__ col, int uplo, int* level,
                         int* nlev, int* status, long long budget) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int chunks = (n + 31) >> 5;
    int mymax = 0;
    // A chunk is 32 consecutive rows of the lower problem.  A dependency inside the chunk is on an
    // earlier lane and is resolved with shuffles (one pass over the lanes in order: a lane's level
    // is final once every lower lane has been broadcast); only dependencies on earlier chunks are
    // read from memory, polled up to 8 at a time.
    for (int c = gw; c < chunks; c += nw) {
        const int base = c << 5;
        const int t = base + lane;
        int lev = 0;
        unsigned intra = 0;  // lanes of this chunk that this row depends on
        int i = 0;
        if (t < n) {
            i = uplo ? n - 1 - t : t;
            const int a = rp[i], b = rp[i + 1];
            const int* wl[8];
            int nwait = 0;
            for (int p = a; p < b; ++p) {
                const int j = __ldg(col + p);
                const bool dep = uplo ? (j > i) : (j < i);
                if (!dep || j < 0 || j >= n) continue;
                const int tj = uplo ? n - 1 - j : j;  // its position in the lower problem, < t
                if (tj >= base) {
                    intra |= 1u << (tj - base);
                    continue;
                }
                wl[nwait++] = level + j;
                if (nwait == 8 || p + 1 == b) {
                    int lv[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) lv[q] = q < nwait ? (int)ld_relaxed_u32(wl[q]) : 0;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (q < nwait) {
                            const int lj = lv[q] == kSentI ? wait_i32(wl[q], status, budget) : lv[q];
                            lev = max(lev, lj + 1);
                        }
                    nwait = 0;
                }
            }
            if (nwait) {
                for (int q = 0; q < nwait; ++q) lev = max(lev, wait_i32(wl[q], status, budget) + 1);
            }
        }
#pragma unroll
        for (int d = 0; d < 32; ++d) {
            const int ld = __shfl_sync(0xffffffffu, lev, d);
            if ((intra >> d) & 1u) lev = max(lev, ld + 1);
        }
        if (t < n) {
            publish_i32(level + i, lev);
            mymax = max(mymax, lev + 1);
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) mymax = max(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
    if (lane == 0 && mymax) atomicMax(nlev, mymax);
}

// ---- stable counting sort by level ------------------------------------------------------------
constexpr int kRadixBits = 8;
constexpr int kDigits = 1 << kRadixBits;
constexpr int kTileItems = 32 * 32;  // keys per warp tile
constexpr int kSortWarps = 8;        // warps per block

// keys for the first pass: key[t] = level of the row at position t of the lower problem,
// val[t] = that original row
__global__ void k_init_keys(int n, int uplo, const int* __restrict__ level, int* key, int* val) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int i = uplo ? n - 1 - t : t;
    key[t] = level[i];
    val[t] = i;
}

__global__ void k_digit_count(int n, const int* __restrict__ key, int shift, int ntiles, int* counts) {
    __shared__ int cnt[kSortWarps][kDigits];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tile = blockIdx.x * kSortWarps + warp;
    for (int d = lane; d < kDigits; d += 32) cnt[warp][d] = 0;
    __syncwarp();
    if (tile < ntiles) {
        long base = (long)tile * kTileItems;
        for (int k = lane; k < kTileItems; k += 32) {
            long t = base + k;
            if (t < n) atomicAdd(&cnt[warp][(key[t] >> shift) & (kDigits - 1)], 1);
        }
        __syncwarp();
        for (int d = lane; d < kDigits; d += 32) counts[(long)d * ntiles + tile] = cnt[warp][d];
    }
}

__global__ void k_digit_scatter(int n, const int* __restrict__ key, const int* __restrict__ val, int shift, int ntiles,
                                const int* __restrict__ offs, int* okey, int* oval) {
    __shared__ int base[kSortWarps][kDigits];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tile = blockIdx.x * kSortWarps + warp;
    if (tile >= ntiles) return;  // whole warp leaves together
    for (int d = lane; d < kDigits; d += 32) base[warp][d] = offs[(long)d * ntiles + tile];
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    long t0 = (long)tile * kTileItems;
    for (int r = 0; r < kTileItems; r += 32) {
        long t = t0 + r + lane;
        bool ok = t < n;
        int k = ok ? key[t] : 0;
        int d = ok ? ((k >> shift) & (kDigits - 1)) : kDigits + lane;  // invalid lanes get unique digits
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        int pos = ok ? base[warp][d] + rank : 0;
        __syncwarp();
        if (ok && rank == 0) base[warp][d] += __popc(peers);
        __syncwarp();
        if (ok) {
            okey[pos] = k;
            oval[pos] = val[t];
        }
    }
}

__global__ void k_perm_from_order(int n, const int* __restrict__ order, int* perm, int* iperm) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int i = order[p];
    iperm[p] = i;
    perm[i] = p;
}

__global__ void k_level_hist(int n, const int* __restrict__ level, int* hist) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(hist + level[i], 1);
}

}  // namespace

hec_status validate_csr(int n, const int* rp, const int* col, int uplo, cudaStream_t s) {
    if (n == 0) return HEC_OK;
    int* code = nullptr;
    HEC_CHECK(dalloc(&code, 1));
    cudaMemsetAsync(code, 0, sizeof(int), s);
    k_validate<<<(n + 255) / 256, 256, 0, s>>>(n, rp, col, uplo, code);
    count_launch();
    int h = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, code, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(code);
    if (e != cudaSuccess) return cuda_error(e, "validate");
    switch (h) {
        case 0: return HEC_OK;
        case HEC_ERR_UNSORTED: return set_error(HEC_ERR_UNSORTED, "CSR row not strictly ascending, column out of range or bad rowptr");
        case HEC_ERR_NOT_TRIANGULAR: return set_error(HEC_ERR_NOT_TRIANGULAR, "entry on the wrong side of the diagonal");
        case HEC_ERR_MISSING_DIAG: return set_error(HEC_ERR_MISSING_DIAG, "row without its diagonal entry");
        default: return set_error((hec_status)h, "invalid CSR");
    }
}

// Levels + map for a validated pattern.  dep_side: 0 = j < i, 1 = j > i.  Fills lv (device
// arrays allocated here).  Synchronizes.
hec_status compute_levels(int n, const int* rp, const int* col, int dep_side, hec_levels* lv, cudaStream_t s) {
    lv->n = n;
    lv->uplo = dep_side;
    HEC_CHECK(dalloc(&lv->level, (size_t)n));
    HEC_CHECK(dalloc(&lv->perm, (size_t)n));
    HEC_CHECK(dalloc(&lv->iperm, (size_t)n));
    int* dnlev = nullptr;
    int* status = nullptr;
    HEC_CHECK(dalloc(&dnlev, 2));
    status = dnlev + 1;
    HEC_CUDA(cudaMemsetAsync(dnlev, 0, 2 * sizeof(int), s));
    if (n > 0) {
        HEC_CUDA(cudaMemsetAsync(lv->level, 0xFF, sizeof(int) * (size_t)n, s));
        const int threads = 256;
        int per_sm = max_coop_blocks((const void*)k_levels, threads, 0);
        if (per_sm <= 0) { dfree(dnlev); return set_error(HEC_ERR_CUDA, "level kernel cannot be resident"); }
        int chunks = (n + 31) / 32;
        int blocks = std::min(per_sm * num_sms(), (chunks + threads / 32 - 1) / (threads / 32));
        blocks = std::max(blocks, 1);
        long long budget = 4000000000LL;
        int nn = n, up = dep_side;
        void* args[] = {&nn, (void*)&rp, (void*)&col, &up, &lv->level, &dnlev, &status, &budget};
        HEC_CUDA(cudaLaunchCooperativeKernel((const void*)k_levels, dim3(blocks), dim3(threads), args, 0, s));
        count_launch();
    }
    int h[2] = {0, 0};
    HEC_CUDA(cudaMemcpyAsync(h, dnlev, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    HEC_CUDA(cudaStreamSynchronize(s));
    dfree(dnlev);
    if (h[1] != 0) return set_error((hec_status)h[1], "level analysis: dependency wait timed out");
    lv->nlev = h[0];
    HEC_CHECK(dalloc(&lv->level_ptr, (size_t)lv->nlev + 1));
    if (n == 0) {
        HEC_CUDA(cudaMemsetAsync(lv->level_ptr, 0, sizeof(int), s));
        HEC_CUDA(cudaStreamSynchronize(s));
        return HEC_OK;
    }
    // level_ptr: histogram + exclusive scan
    HEC_CUDA(cudaMemsetAsync(lv->level_ptr, 0, sizeof(int) * ((size_t)lv->nlev + 1), s));
    k_level_hist<<<(n + 255) / 256, 256, 0, s>>>(n, lv->level, lv->level_ptr);
    HEC_LAUNCHED();
    HEC_CHECK(exclusive_scan_i32(lv->level_ptr, lv->level_ptr, lv->nlev, true, s));
    // stable LSD radix sort of (level, position) pairs
    int *k0 = nullptr, *v0 = nullptr, *k1 = nullptr, *v1 = nullptr, *counts = nullptr;
    int ntiles = (n + kTileItems - 1) / kTileItems;
    hec_status st = HEC_OK;
    if ((st = dalloc(&k0, (size_t)n)) || (st = dalloc(&v0, (size_t)n)) || (st = dalloc(&k1, (size_t)n)) ||
        (st = dalloc(&v1, (size_t)n)) || (st = dalloc(&counts, (size_t)kDigits * ntiles + 1))) {
        dfree(k0); dfree(v0); dfree(k1); dfree(v1); dfree(counts);
        return st;
    }
    k_init_keys<<<(n + 255) / 256, 256, 0, s>>>(n, dep_side, lv->level, k0, v0);
    count_launch();
    int bits = 0;
    while ((1LL << bits) < (long long)lv->nlev) bits++;
    int passes = std::max(1, (bits + kRadixBits - 1) / kRadixBits);
    int sblocks = (ntiles + kSortWarps - 1) / kSortWarps;
    for (int ps = 0; ps < passes && st == HEC_OK; ++ps) {
        int shift = ps * kRadixBits;
        k_digit_count<<<sblocks, 32 * kSortWarps, 0, s>>>(n, k0, shift, ntiles, counts);
        count_launch();
        st = exclusive_scan_i32(counts, counts, kDigits * ntiles, false, s);
        if (st != HEC_OK) break;
        k_digit_scatter<<<sblocks, 32 * kSortWarps, 0, s>>>(n, k0, v0, shift, ntiles, counts, k1, v1);
        count_launch();
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    if (st == HEC_OK) {
        k_perm_from_order<<<(n + 255) / 256, 256, 0, s>>>(n, v0, lv->perm, lv->iperm);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(e, "level sort");
    }
    dfree(k0); dfree(v0); dfree(k1); dfree(v1); dfree(counts);
    return st;
}

// Stable sort of (key, val) pairs by key, 0 <= key <= max_key, in place (LSD radix, 8-bit
// digits).  Synchronizes.
hec_status sort_pairs_i32(int* keys, int* vals, int n, int max_key, cudaStream_t s) {
    if (n <= 1) return HEC_OK;
    int *k1 = nullptr, *v1 = nullptr, *counts = nullptr;
    const int ntiles = (n + kTileItems - 1) / kTileItems;
    hec_status st = HEC_OK;
    if ((st = dalloc(&k1, (size_t)n)) || (st = dalloc(&v1, (size_t)n)) ||
        (st = dalloc(&counts, (size_t)kDigits * ntiles + 1))) {
        dfree(k1); dfree(v1); dfree(counts);
        return st;
    }
    int bits = 0;
    while ((1LL << bits) <= (long long)max_key) bits++;
    const int passes = std::max(1, (bits + kRadixBits - 1) / kRadixBits);
    const int sblocks = (ntiles + kSortWarps - 1) / kSortWarps;
    int *ka = keys, *va = vals, *kb = k1, *vb = v1;
    for (int ps = 0; ps < passes && st == HEC_OK; ++ps) {
        k_digit_count<<<sblocks, 32 * kSortWarps, 0, s>>>(n, ka, ps * kRadixBits, ntiles, counts);
        count_launch();
        st = exclusive_scan_i32(counts, counts, kDigits * ntiles, false, s);
        if (st != HEC_OK) break;
        k_digit_scatter<<<sblocks, 32 * kSortWarps, 0, s>>>(n, ka, va, ps * kRadixBits, ntiles, counts, kb, vb);
        count_launch();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (st == HEC_OK && ka != keys) {
        cudaMemcpyAsync(keys, ka, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, va, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (st == HEC_OK && e != cudaSuccess) st = cuda_error(e, "sort");
    dfree(k1); dfree(v1); dfree(counts);
    return st;
}

void free_levels(hec_levels* lv) {
    if (!lv) return;
    dfree(lv->level);
    dfree(lv->perm);
    dfree(lv->iperm);
    dfree(lv->level_ptr);
    delete lv;
}

}  // namespace hec

using namespace hec;

HEC_API hec_status sptrsv_analyze(int n, const int* rowptr, const int* col, int uplo, hec_levels** out, void* stream) {
    clear_error();
    if (!out || n < 0 || (uplo != 0 && uplo != 1) || (n > 0 && (!rowptr || !col)))
        return set_error(HEC_ERR_INVALID_ARG, "sptrsv_analyze: bad argument");
    *out = nullptr;
    cudaStream_t s = S(stream);
    HEC_CHECK(validate_csr(n, rowptr, col, uplo, s));
    hec_levels* lv = new hec_levels();
    hec_status st = compute_levels(n, rowptr, col, uplo, lv, s);
    if (st != HEC_OK) { free_levels(lv); return st; }
    *out = lv;
    return HEC_OK;
}

HEC_API hec_status hec_levels_get(const hec_levels* lv, int* n, int* nlev, int* uplo, const int** level, const int** perm,
                                  const int** iperm, const int** level_ptr) {
    if (!lv) return set_error(HEC_ERR_INVALID_ARG, "hec_levels_get: NULL handle");
    if (n) *n = lv->n;
    if (nlev) *nlev = lv->nlev;
    if (uplo) *uplo = lv->uplo;
    if (level) *level = lv->level;
    if (perm) *perm = lv->perm;
    if (iperm) *iperm = lv->iperm;
    if (level_ptr) *level_ptr = lv->level_ptr;
    return HEC_OK;
}

HEC_API hec_status hec_levels_destroy(hec_levels* lv) {
    free_levels(lv);
    return HEC_OK;
}
