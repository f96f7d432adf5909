// Device-side check of a solve plan: every index the sweep kernels follow, verified before a
// sweep trusts it.
//
// The sweeps read slab and tail columns, chunk tables and permutations without bounds checks (a
// check per gathered index would sit on the dependency chain).  sptrsv_plan_check verifies, on
// the device and without touching any solution memory, what the kernels rely on:
//   1. the level map: perm and iperm are inverse permutations of [0, n), level_ptr is
//      non-decreasing from 0 to n;
//   2. the HEC factor (level-ordered numbering): tail row pointers non-decreasing from 0 to
//      tail_nnz with at least one entry a row; slab columns in [-1, n), padding (-1) only after a
//      row's entries, tail off-diagonals only after a full slab; every off-diagonal column
//      belongs to an earlier level than its row (so every wait is on a row the schedule computes
//      first); the last tail entry of each row is its diagonal, and nonzero;
//   3. every chunk table the plan built: chunks in order, each inside one level, of 1 to the
//      table's rows per warp step, covering [0, n) exactly;
//   4. a partition, when set: rowg a permutation of [0, n), part_row non-decreasing from 0 to n,
//      each part's chunks inside the part, level-aligned and covering it, and the repacked factor
//      with columns in [-1, n) whose dependencies lie in earlier levels of the level order.
// The first failure found (the lowest check number, then the lowest row) is reported as
// HEC_ERR_OUT_OF_BOUNDS with a message naming the check and the row.  The plan is not changed.
#include <algorithm>
#include <string>

#include "internal.cuh"

namespace hec {
namespace {

// result word: (check << 27) | min(row, 2^27 - 1); 0xFFFFFFFF = all checks passed
__device__ __forceinline__ void fail(unsigned* res, int check, long long row) {
    const unsigned code = ((unsigned)check << 27) | (unsigned)min(row, (long long)((1u << 27) - 1));
    atomicMin(res, code);
}

__device__ __forceinline__ bool is_zero(double v) { return v == 0.0; }
__device__ __forceinline__ bool is_zero(float v) { return v == 0.0f; }
__device__ __forceinline__ bool is_zero(__nv_bfloat16 v) { return __bfloat162float(v) == 0.0f; }

// level of level-ordered row r: the l with level_ptr[l] <= r < level_ptr[l + 1]
__device__ __forceinline__ int level_of(int r, const int* __restrict__ lp, int nlev) {
    int lo = 0, hi = nlev - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (lp[mid] <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_check_levels(int n, int nlev, const int* __restrict__ perm, const int* __restrict__ iperm,
                               const int* __restrict__ lp, unsigned* res) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = perm[i];
        if (p < 0 || p >= n || iperm[p] != i) fail(res, 1, i);
    }
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l <= nlev; l += gridDim.x * blockDim.x) {
        const int v = lp[l];
        if ((l == 0 && v != 0) || (l == nlev && v != n) || (l > 0 && v < lp[l - 1])) fail(res, 1, l);
    }
}

// one thread per row of a triangular HEC factor in the numbering `lp` orders by level; rowlev
// (may be NULL) maps a row to the row whose level counts (the partitioned layout's rowg)
template <typename VT>
__global__ void k_check_hec(int n, int ld, int w, long long tail_nnz, const int* __restrict__ ec, const VT* __restrict__ ev,
                            const int* __restrict__ tp, const int* __restrict__ tc, const VT* __restrict__ tv,
                            const int* __restrict__ lp, int nlev, const int* __restrict__ rowlev, int check,
                            unsigned* res) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int t0 = tp[r], t1 = tp[r + 1];
        if ((r == 0 && t0 != 0) || (r == n - 1 && (long long)t1 != tail_nnz) || t1 <= t0 || t0 < 0 ||
            (long long)t1 > tail_nnz) {
            fail(res, check, r);
            continue;
        }
        const int lr = level_of(rowlev ? rowlev[r] : r, lp, nlev);
        bool pad = false;
        for (int k = 0; k < w; ++k) {
            const int c = ec[(long)k * ld + r];
            if (c == -1) { pad = true; continue; }
            if (pad || c < 0 || c >= n || level_of(rowlev ? rowlev[c] : c, lp, nlev) >= lr) fail(res, check, r);
        }
        if (pad && t1 - t0 > 1) fail(res, check, r);  // overflow entries while the slab has room
        for (int e = t0; e < t1 - 1; ++e) {
            const int c = tc[e];
            if (c < 0 || c >= n || level_of(rowlev ? rowlev[c] : c, lp, nlev) >= lr) fail(res, check, r);
        }
        if (tc[t1 - 1] != r || is_zero(tv[t1 - 1])) fail(res, check, r);
    }
}

// chunks (first row, rows) of at most rpw rows, in order, each inside one level of `lp` (over the
// rows mapped by rowlev when given), covering [lo, hi)
__global__ void k_check_chunks(int nchunks, const int2* __restrict__ ch, int rpw, int lo, int hi,
                               const int* __restrict__ lp, int nlev, const int* __restrict__ rowlev, int check,
                               unsigned* res) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += gridDim.x * blockDim.x) {
        const int2 k = ch[c];
        const int next = c + 1 < nchunks ? ch[c + 1].x : hi;
        if ((c == 0 && k.x != lo) || k.y < 1 || k.y > rpw || k.x < lo || k.x + k.y > hi || next != k.x + k.y) {
            fail(res, check, c);
            continue;
        }
        const int a = rowlev ? rowlev[k.x] : k.x, b = rowlev ? rowlev[k.x + k.y - 1] : k.x + k.y - 1;
        if (level_of(a, lp, nlev) != level_of(b, lp, nlev)) fail(res, check, c);
    }
}

__global__ void k_check_perm(int n, const int* __restrict__ p, unsigned* seen, unsigned* res, int check) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int v = p[i];
        if (v < 0 || v >= n) fail(res, check, i);
        else if (atomicOr(seen + (v >> 5), 1u << (v & 31)) & (1u << (v & 31))) fail(res, check, i);
    }
}

__global__ void k_check_parts(int nparts, int n, const int* __restrict__ part_row, const int* __restrict__ part_chunk,
                              int nchunks, unsigned* res) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q <= nparts; q += gridDim.x * blockDim.x) {
        const int r = part_row[q], c = part_chunk[q];
        if ((q == 0 && (r != 0 || c != 0)) || (q == nparts && (r != n || c != nchunks)) ||
            (q > 0 && (r < part_row[q - 1] || c < part_chunk[q - 1])))
            fail(res, 7, q);
    }
}

// every part's chunks lie inside the part: the chunk starting a part begins at its first row
__global__ void k_check_part_chunks(int nparts, const int* __restrict__ part_row, const int* __restrict__ part_chunk,
                                    const int2* __restrict__ ch, unsigned* res) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nparts; q += gridDim.x * blockDim.x) {
        const int c0 = part_chunk[q], c1 = part_chunk[q + 1];
        if (c1 > c0 && (ch[c0].x != part_row[q] || ch[c1 - 1].x + ch[c1 - 1].y != part_row[q + 1])) fail(res, 7, q);
        if (c1 == c0 && part_row[q] != part_row[q + 1]) fail(res, 7, q);
    }
}

const char* kCheckName[] = {"", "level map (perm, iperm, level_ptr)", "HEC factor (rows, columns, levels, diagonal)",
                            "chunk table", "partition row map (rowg)", "partitioned factor", "partition chunk table",
                            "partition tables (part_row, part_chunk)"};

template <typename VT>
void launch_check_hec(const hec_matrix* T, const int* ec, const void* ev, const int* tp, const int* tc, const void* tv,
                      const hec_levels* lv, const int* rowlev, int check, unsigned* res, cudaStream_t s) {
    const int g = std::min(4096, (T->n + 255) / 256);
    k_check_hec<VT><<<g, 256, 0, s>>>(T->n, T->ld, T->w, T->tail_nnz, ec, (const VT*)ev, tp, tc, (const VT*)tv,
                                      lv->level_ptr, lv->nlev, rowlev, check, res);
    count_launch();
}

void check_hec(const hec_matrix* T, const int* ec, const void* ev, const int* tp, const int* tc, const void* tv,
               const hec_levels* lv, const int* rowlev, int check, unsigned* res, cudaStream_t s) {
    if (T->vdt == HEC_F64) launch_check_hec<double>(T, ec, ev, tp, tc, tv, lv, rowlev, check, res, s);
    else if (T->vdt == HEC_F32) launch_check_hec<float>(T, ec, ev, tp, tc, tv, lv, rowlev, check, res, s);
    else launch_check_hec<__nv_bfloat16>(T, ec, ev, tp, tc, tv, lv, rowlev, check, res, s);
}

}  // namespace
}  // namespace hec

using namespace hec;

HEC_API hec_status sptrsv_plan_check(const sptrsv_plan* p, void* stream) {
    clear_error();
    if (!p) return set_error(HEC_ERR_INVALID_ARG, "sptrsv_plan_check: NULL plan");
    const hec_matrix* T = p->T;
    const hec_levels* lv = p->lv;
    const int n = T->n;
    if (n == 0) return HEC_OK;
    cudaStream_t s = S(stream);
    unsigned* res = nullptr;
    unsigned* seen = nullptr;
    HEC_CHECK(dalloc(&res, 1));
    hec_status st = dalloc(&seen, (size_t)(n + 31) / 32);
    if (st) { dfree(res); return st; }
    auto finish = [&](hec_status e) { dfree(res); dfree(seen); return e; };
    if (cudaMemsetAsync(res, 0xff, sizeof(unsigned), s) != cudaSuccess) return finish(cuda_error(cudaGetLastError(), "memset"));
    const int g = std::min(4096, (n + 255) / 256);
    k_check_levels<<<g, 256, 0, s>>>(n, lv->nlev, lv->perm, lv->iperm, lv->level_ptr, res);
    count_launch();
    check_hec(T, T->ell_col, T->ell_val, T->tptr, T->tcol, T->tval, lv, nullptr, 2, res, s);
    for (int i = 0; i < 5; ++i)
        if (p->chunks[i] && p->nchunks[i] > 0) {
            k_check_chunks<<<std::min(4096, (p->nchunks[i] + 255) / 256), 256, 0, s>>>(
                p->nchunks[i], p->chunks[i], 32 >> i, 0, n, lv->level_ptr, lv->nlev, nullptr, 3, res);
            count_launch();
        }
    if (const hec_part_data* P = p->part) {
        cudaMemsetAsync(seen, 0, sizeof(unsigned) * ((size_t)(n + 31) / 32), s);
        k_check_perm<<<g, 256, 0, s>>>(n, P->rowg, seen, res, 4);
        k_check_parts<<<(P->nparts + 256) / 256, 256, 0, s>>>(P->nparts, n, P->part_row, P->part_chunk, P->nchunks, res);
        count_launch(2);
        unsigned h = 0;
        HEC_CUDA(cudaMemcpyAsync(&h, res, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        HEC_CUDA(cudaStreamSynchronize(s));
        if (h == 0xffffffffu) {  // the maps are sound: the repacked factor and the chunks per part
            check_hec(T, P->ell_col, P->ell_val, P->tptr, P->tcol, P->tval, lv, P->rowg, 5, res, s);
            k_check_chunks<<<std::min(4096, (P->nchunks + 255) / 256), 256, 0, s>>>(
                P->nchunks, P->chunks, 32, 0, n, lv->level_ptr, lv->nlev, P->rowg, 6, res);
            k_check_part_chunks<<<(P->nparts + 255) / 256, 256, 0, s>>>(P->nparts, P->part_row, P->part_chunk,
                                                                        P->chunks, res);
            count_launch(2);
        }
    }
    unsigned h = 0;
    HEC_CUDA(cudaMemcpyAsync(&h, res, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return finish(cuda_error(e, "sptrsv_plan_check"));
    if (h == 0xffffffffu) return finish(HEC_OK);
    const int check = (int)(h >> 27), where = (int)(h & ((1u << 27) - 1));
    return finish(set_error(HEC_ERR_OUT_OF_BOUNDS, std::string("sptrsv_plan_check: ") +
                                                       (check > 0 && check < 8 ? kCheckName[check] : "?") +
                                                       " fails at index " + std::to_string(where)));
}
