// Allocation-free triangular sweep.
//
// sptrsv_solve_noalloc runs the same lower/upper sweep as sptrsv_lower / sptrsv_upper, but
// every piece of device scratch it needs (the level-aligned chunk table, the internal
// level-ordered solution and the status word) lives in one file-scope __device__ array of fixed
// size instead of buffers obtained from cudaMalloc.  It is meant for callers that are not
// allowed to allocate device memory at solve time: code whose device memory is owned by
// another allocator (a framework or pool that must account for every byte), deployments that
// reserve all memory up front and forbid allocation afterwards, and latency-sensitive loops
// where a cudaMalloc (which may synchronize the device) is unacceptable.
//
// Host code never dereferences g_noalloc_scratch: in host code the symbol is only a stand-in,
// so every call looks up its device address with cudaGetSymbolAddress, with the calling device
// current.  The lookup allocates nothing and is cheap; doing it on every call (instead of caching
// the address per device) keeps the call correct after the context is reset and recreated.
//
// The buffer is part of this library's device code module.  With lazy module loading (the CUDA
// default) that module is loaded, and the buffer reserved, at the first use of a kernel or symbol
// of this file on a device, i.e. during the first call of sptrsv_solve_noalloc there (of any size,
// n = 0 included).  Callers that must not see device memory change inside later calls make one
// warm-up call at initialization.
#include <algorithm>
#include <string>

#include "internal.cuh"

namespace hec {
namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB, held by every device that loads the library
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// chunks per level (ceil(N_l / rpw)) into cptr[0..nlev-1]
__global__ void k_na_counts(int nlev, const int* __restrict__ level_ptr, int rpw, int* cptr) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < nlev) cptr[l] = (level_ptr[l + 1] - level_ptr[l] + rpw - 1) / rpw;
}

// in-place exclusive scan of cptr[0..nlev-1] by one block; cptr[nlev] = total
__global__ void k_na_scan(int nlev, int* cptr) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nlev; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = i < nlev ? cptr[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int s = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_tot[lane] = s;
        }
        __syncthreads();
        int excl = carry + (warp ? warp_tot[warp - 1] : 0) + x - v;
        if (i < nlev) cptr[i] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) cptr[nlev] = carry;
}

// chunk table of at most cap entries; entries past the real count are empty (0 rows)
__global__ void k_na_table(int nlev, const int* __restrict__ level_ptr, const int* __restrict__ cptr, int rpw,
                           int cap, int2* tbl) {
    const int total = cptr[nlev];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cap; c += gridDim.x * blockDim.x) {
        if (c >= total) {
            tbl[c] = make_int2(0, 0);
            continue;
        }
        int lo = 0, hi = nlev - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (cptr[mid] <= c) lo = mid; else hi = mid - 1;
        }
        int row0 = level_ptr[lo] + (c - cptr[lo]) * rpw;
        tbl[c] = make_int2(row0, min(rpw, level_ptr[lo + 1] - row0));
    }
}

// reciprocal diagonal in the work type, the same arithmetic as a solve plan's
template <typename VT, typename XT>
__global__ void k_na_dinv(int n, const int* __restrict__ tptr, const VT* __restrict__ tval, XT* dinv) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const VT d = tval[tptr[r + 1] - 1];
    if (sizeof(XT) == 8) dinv[r] = (XT)(1.0 / (double)d);
    else dinv[r] = (XT)(1.0f / (float)d);
}
template <>
__global__ void k_na_dinv<__nv_bfloat16, float>(int n, const int* __restrict__ tptr, const __nv_bfloat16* __restrict__ tval,
                                                float* dinv) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) dinv[r] = 1.0f / __bfloat162float(tval[tptr[r + 1] - 1]);
}

hec_status scratch_ptr(unsigned char** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
    *out = (unsigned char*)p;
    return HEC_OK;
}

}  // namespace
}  // namespace hec

using namespace hec;

HEC_API size_t sptrsv_noalloc_capacity(void) { return kScratchBytes; }

HEC_API hec_status sptrsv_solve_noalloc(const hec_matrix* tri, const hec_levels* lv, int nrhs, const double* b, int ldb,
                                        double* x, int ldx, int* status_out, void* stream) {
    clear_error();
    if (!tri || !lv || !tri->tri || tri->lv != lv || nrhs < 1 || nrhs > 16 || ldb < nrhs || ldx < nrhs ||
        (tri->n > 0 && (!b || !x)))
        return set_error(HEC_ERR_INVALID_ARG, "sptrsv_solve_noalloc: need a triangular HEC matrix, the analysis it "
                                              "was packed with, 1 <= nrhs <= 16 and ld >= nrhs");
    if (status_out) *status_out = 0;
    unsigned char* base = nullptr;
    HEC_CHECK(scratch_ptr(&base));  // also loads the buffer on a device's first call
    const int n = tri->n, nlev = lv->nlev;
    if (n == 0) return HEC_OK;
    const int kp = sweep_kp(nrhs);  // padded row stride of the solution
    // lane layout (as a plan with default settings): one right-hand side takes the lanes-per-row
    // rule of the row lengths, more take G right-hand sides per lane; it selects the chunk table
    const int lpr1 = nrhs == 1 ? default_lanes_per_row(tri) : 1;
    const int kp_idx = log2i(nrhs == 1 ? lpr1 : sweep_lpr(nrhs, tri->vdt));
    const int rpw = 32 >> kp_idx;
    // layout: [status | chunk prefix (nlev+1) | chunk table | level-ordered solution]
    const size_t chunk_cap = (size_t)nlev + ((size_t)n + rpw - 1) / rpw;
    const size_t off_cptr = 256;
    const size_t off_tbl = off_cptr + align256(sizeof(int) * ((size_t)nlev + 1));
    const size_t off_xp = off_tbl + align256(sizeof(int2) * chunk_cap);
    const size_t ws = tri->vdt == HEC_F64 ? 8 : 4;
    const size_t xp_bytes = ws * (size_t)n * kp;
    const size_t off_dinv = off_xp + align256(xp_bytes);
    const size_t need = off_dinv + align256(ws * (size_t)n);
    if (need > kScratchBytes)
        return set_error(HEC_ERR_INVALID_ARG,
                         "sptrsv_solve_noalloc: problem needs " + std::to_string(need) + " bytes of scratch, more than the " +
                             std::to_string(kScratchBytes) + "-byte static buffer (use sptrsv_lower/sptrsv_upper)");
    cudaStream_t s = S(stream);
    int* status = (int*)base;
    int* cptr = (int*)(base + off_cptr);
    int2* tbl = (int2*)(base + off_tbl);
    HEC_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));  // the last call's status must not leak in
    k_na_counts<<<(nlev + 255) / 256, 256, 0, s>>>(nlev, lv->level_ptr, rpw, cptr);
    HEC_LAUNCHED();
    k_na_scan<<<1, 1024, 0, s>>>(nlev, cptr);
    HEC_LAUNCHED();
    const int tb = (int)std::min<size_t>(4096, (chunk_cap + 255) / 256);
    k_na_table<<<tb, 256, 0, s>>>(nlev, lv->level_ptr, cptr, rpw, (int)chunk_cap, tbl);
    HEC_LAUNCHED();
    void* dinv = base + off_dinv;
    const int gd = (n + 255) / 256;
    if (tri->vdt == HEC_F64)
        k_na_dinv<double, double><<<gd, 256, 0, s>>>(n, tri->tptr, (const double*)tri->tval, (double*)dinv);
    else if (tri->vdt == HEC_F32)
        k_na_dinv<float, float><<<gd, 256, 0, s>>>(n, tri->tptr, (const float*)tri->tval, (float*)dinv);
    else
        k_na_dinv<__nv_bfloat16, float><<<gd, 256, 0, s>>>(n, tri->tptr, (const __nv_bfloat16*)tri->tval, (float*)dinv);
    HEC_LAUNCHED();
    // a plan that lives on the host stack and points into the static scratch
    sptrsv_plan plan;
    plan.T = tri;
    plan.lv = lv;
    plan.max_nrhs = nrhs;
    plan.xp = base + off_xp;
    plan.status = status;
    plan.chunks[kp_idx] = tbl;
    plan.nchunks[kp_idx] = (int)chunk_cap;
    plan.dinv = dinv;
    plan.lpr1 = lpr1;
    hec_status st = sweep(&plan, nrhs, b, ldb, lv->iperm, x, ldx, lv->iperm, s);
    if (st != HEC_OK) return st;
    if (status_out) {
        int h = 0;
        HEC_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
        HEC_CUDA(cudaStreamSynchronize(s));
        *status_out = h;
        if (h != 0) return set_error((hec_status)h, "sptrsv_solve_noalloc: a dependency wait timed out");
    }
    return HEC_OK;
}
