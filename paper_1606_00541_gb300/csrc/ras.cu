// Restricted Additive Schwarz setup (Sec. 3, Eq. 4) on the GPU.
//
// Each subdomain s owns the rows i with part[i] == s.  Its extended set adds every column of an
// owned row (overlap 1: the subdomain "extended according to the topology of the graph"), in
// ascending global index; with overlap 0 it is the owned set itself, which gives block ILU(0)
// (block Jacobi with ILU(0) blocks).  A_s = A restricted to the extended rows and columns, and all A_s are
// assembled as ONE block-diagonal matrix diag(A_1, ..., A_s) over the n_ext extended rows, so
// that a single ILU(0), a single level analysis and a single pair of sweeps serve every
// subdomain at once (Eq. 4).  ext2glob maps extended rows to global rows and owned marks the
// rows a subdomain writes back (the "restricted" prolongation).
//
// Construction: (subdomain, global row) pairs are emitted for every owned row and its columns,
// sorted with the stable radix sort used by the level analysis, and de-duplicated; the local
// column of an entry is found by binary search in its subdomain's sorted extended set.
#include <algorithm>

#include "internal.cuh"

struct hec_ras {
    int n = 0, nsub = 0, n_ext = 0;
    int* ext_ptr = nullptr;        // [nsub+1]
    int* ext2glob = nullptr;       // [n_ext]
    unsigned char* owned = nullptr;// [n_ext]
    hec_csr* A_ext = nullptr;      // block-diagonal, n_ext x n_ext
};

namespace hec {
hec_status validate_csr(int n, const int* rp, const int* col, int uplo, cudaStream_t s);
hec_status sort_pairs_i32(int* keys, int* vals, int n, int max_key, cudaStream_t s);
void free_csr(hec_csr* M);

namespace {

__global__ void k_check_part(int n, const int* __restrict__ part, int nsub, int* code) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (part[i] < 0 || part[i] >= nsub)) atomicCAS(code, 0, 1);
}

__global__ void k_pair_counts(int n, const int* __restrict__ rp, int overlap, int* cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cnt[i] = 1 + (overlap ? rp[i + 1] - rp[i] : 0);
}

__global__ void k_pairs(int n, const int* __restrict__ rp, const int* __restrict__ col, const int* __restrict__ part,
                        int overlap, const int* __restrict__ off, int* keys, int* vals) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int base = part[i] * n;
    int o = off[i];
    keys[o] = base + i;
    vals[o] = o;
    ++o;
    if (!overlap) return;
    for (int p = rp[i]; p < rp[i + 1]; ++p, ++o) {
        keys[o] = base + col[p];
        vals[o] = o;
    }
}

__global__ void k_first_flags(int m, const int* __restrict__ keys, int* flag) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) flag[k] = (k == 0 || keys[k] != keys[k - 1]) ? 1 : 0;
}

__global__ void k_compact(int m, int n, const int* __restrict__ keys, const int* __restrict__ flag,
                          const int* __restrict__ pos, const int* __restrict__ part, int* ext2glob, int* sub,
                          unsigned char* owned) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m || !flag[k]) return;
    const int e = pos[k];
    const int s = keys[k] / n, g = keys[k] - s * n;
    ext2glob[e] = g;
    sub[e] = s;
    owned[e] = part[g] == s ? 1 : 0;
}

// ext_ptr[s] = first extended row of subdomain s (lower bound in the sorted sub array)
__global__ void k_ext_ptr(int nsub, int n_ext, const int* __restrict__ sub, int* ext_ptr) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s > nsub) return;
    int lo = 0, hi = n_ext;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (sub[mid] < s) lo = mid + 1; else hi = mid;
    }
    ext_ptr[s] = lo;
}

template <bool kFill>
__global__ void k_sub_rows(int n_ext, const int* __restrict__ rp, const int* __restrict__ col,
                           const double* __restrict__ val, const int* __restrict__ ext2glob,
                           const int* __restrict__ sub, const int* __restrict__ ext_ptr, int* len,
                           const int* __restrict__ orp, int* oci, double* ov) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_ext) return;
    const int g = ext2glob[e], s = sub[e];
    const int lo = ext_ptr[s], hi = ext_ptr[s + 1];
    int c = 0, o = kFill ? orp[e] : 0;
    for (int p = rp[g]; p < rp[g + 1]; ++p) {
        int idx = -1;
        const int cc = col[p];
        int a = lo, b = hi;  // lower bound of cc in ext2glob[lo, hi)
        while (a < b) {
            int mid = (a + b) >> 1;
            if (ext2glob[mid] < cc) a = mid + 1; else b = mid;
        }
        if (a < hi && ext2glob[a] == cc) idx = a;
        if (idx < 0) continue;
        if (kFill) {
            oci[o + c] = idx;
            ov[o + c] = val[p];
        }
        c++;
    }
    if (!kFill) len[e] = c;
}

}  // namespace

void free_ras(hec_ras* R) {
    if (!R) return;
    dfree(R->ext_ptr);
    dfree(R->ext2glob);
    dfree(R->owned);
    free_csr(R->A_ext);
    delete R;
}

}  // namespace hec

using namespace hec;

HEC_API hec_status ras_setup_overlap(int n, const int* rowptr, const int* col, const double* val, const int* part,
                                     int nsub, int overlap, hec_ras** out, void* stream) {
    clear_error();
    if (!out || n <= 0 || nsub < 1 || !rowptr || !col || !val || !part || (long long)nsub * n > 0x7fffffffLL ||
        (overlap != 0 && overlap != 1))
        return set_error(HEC_ERR_INVALID_ARG,
                         "ras_setup: bad argument (nsub * n must stay below 2^31, overlap 0 or 1)");
    *out = nullptr;
    cudaStream_t s = S(stream);
    HEC_CHECK(validate_csr(n, rowptr, col, -1, s));
    hec_ras* R = new hec_ras();
    R->n = n;
    R->nsub = nsub;
    R->A_ext = new hec_csr();
    int *code = nullptr, *cnt = nullptr, *off = nullptr, *keys = nullptr, *vals = nullptr, *flag = nullptr,
        *pos = nullptr, *sub = nullptr, *len = nullptr;
    hec_status st = HEC_OK;
    auto cleanup = [&]() {
        dfree(code); dfree(cnt); dfree(off); dfree(keys); dfree(vals); dfree(flag);
        dfree(pos); dfree(sub); dfree(len);
    };
    auto fail = [&](hec_status e) {
        cleanup();
        free_ras(R);
        return e;
    };
    const int g = (n + 255) / 256;
    if ((st = dalloc(&code, 1))) return fail(st);
    cudaMemsetAsync(code, 0, sizeof(int), s);
    k_check_part<<<g, 256, 0, s>>>(n, part, nsub, code);
    count_launch();
    int h = 0;
    HEC_CUDA(cudaMemcpyAsync(&h, code, sizeof(int), cudaMemcpyDeviceToHost, s));
    HEC_CUDA(cudaStreamSynchronize(s));
    if (h) return fail(set_error(HEC_ERR_INVALID_ARG, "ras_setup: part[] outside [0, nsub)"));
    // (subdomain, row) pairs of every owned row and its columns
    if ((st = dalloc(&cnt, (size_t)n + 1)) || (st = dalloc(&off, (size_t)n + 1))) return fail(st);
    k_pair_counts<<<g, 256, 0, s>>>(n, rowptr, overlap, cnt);
    count_launch();
    if ((st = exclusive_scan_i32(cnt, off, n, true, s))) return fail(st);
    int m = 0;
    HEC_CUDA(cudaMemcpy(&m, off + n, sizeof(int), cudaMemcpyDeviceToHost));
    if ((st = dalloc(&keys, (size_t)m)) || (st = dalloc(&vals, (size_t)m)) || (st = dalloc(&flag, (size_t)m + 1)) ||
        (st = dalloc(&pos, (size_t)m + 1)))
        return fail(st);
    k_pairs<<<g, 256, 0, s>>>(n, rowptr, col, part, overlap, off, keys, vals);
    count_launch();
    if ((st = sort_pairs_i32(keys, vals, m, nsub * n - 1, s))) return fail(st);
    const int gm = (m + 255) / 256;
    k_first_flags<<<gm, 256, 0, s>>>(m, keys, flag);
    count_launch();
    if ((st = exclusive_scan_i32(flag, pos, m, true, s))) return fail(st);
    HEC_CUDA(cudaMemcpy(&R->n_ext, pos + m, sizeof(int), cudaMemcpyDeviceToHost));
    const int ne = R->n_ext;
    if ((st = dalloc(&R->ext2glob, (size_t)ne)) || (st = dalloc(&sub, (size_t)ne)) ||
        (st = dalloc(&R->owned, (size_t)ne)) || (st = dalloc(&R->ext_ptr, (size_t)nsub + 1)))
        return fail(st);
    k_compact<<<gm, 256, 0, s>>>(m, n, keys, flag, pos, part, R->ext2glob, sub, R->owned);
    k_ext_ptr<<<(nsub + 1 + 255) / 256, 256, 0, s>>>(nsub, ne, sub, R->ext_ptr);
    count_launch(2);
    // block-diagonal A_ext: count, scan, fill
    hec_csr* C = R->A_ext;
    C->n = ne;
    const int ge = (ne + 255) / 256;
    if ((st = dalloc(&len, (size_t)ne + 1)) || (st = dalloc(&C->rowptr, (size_t)ne + 1))) return fail(st);
    k_sub_rows<false><<<ge, 256, 0, s>>>(ne, rowptr, col, val, R->ext2glob, sub, R->ext_ptr, len, nullptr, nullptr,
                                         nullptr);
    count_launch();
    if ((st = exclusive_scan_i32(len, C->rowptr, ne, true, s))) return fail(st);
    int nnz = 0;
    HEC_CUDA(cudaMemcpy(&nnz, C->rowptr + ne, sizeof(int), cudaMemcpyDeviceToHost));
    C->nnz = nnz;
    if ((st = dalloc(&C->col, (size_t)nnz)) || (st = dalloc(&C->val, (size_t)nnz))) return fail(st);
    k_sub_rows<true><<<ge, 256, 0, s>>>(ne, rowptr, col, val, R->ext2glob, sub, R->ext_ptr, nullptr, C->rowptr, C->col,
                                        C->val);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_error(e, "ras_setup"));
    cleanup();
    *out = R;
    return HEC_OK;
}

HEC_API hec_status ras_setup(int n, const int* rowptr, const int* col, const double* val, const int* part, int nsub,
                             hec_ras** out, void* stream) {
    return ras_setup_overlap(n, rowptr, col, val, part, nsub, 1, out, stream);
}

HEC_API hec_status hec_ras_get(const hec_ras* R, int* n_ext, const int** ext_ptr, const int** ext2glob,
                               const unsigned char** owned, const hec_csr** A_ext) {
    if (!R) return set_error(HEC_ERR_INVALID_ARG, "hec_ras_get: NULL");
    if (n_ext) *n_ext = R->n_ext;
    if (ext_ptr) *ext_ptr = R->ext_ptr;
    if (ext2glob) *ext2glob = R->ext2glob;
    if (owned) *owned = R->owned;
    if (A_ext) *A_ext = R->A_ext;
    return HEC_OK;
}

HEC_API hec_status hec_ras_destroy(hec_ras* R) {
    free_ras(R);
    return HEC_OK;
}
