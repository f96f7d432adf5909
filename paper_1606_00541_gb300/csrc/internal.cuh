// Internal declarations shared by the libhec translation units.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>

#include "../../include/hec.h"

#define HEC_API extern "C" __attribute__((visibility("default")))

namespace hec {

// ---- errors ------------------------------------------------------------------------------
hec_status set_error(hec_status s, const std::string& msg);
hec_status cuda_error(cudaError_t e, const char* what);
void clear_error();
void count_launch(long long k = 1);

#define HEC_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return ::hec::cuda_error(e_, #call);      \
    } while (0)

#define HEC_CHECK(st)                          \
    do {                                       \
        hec_status s_ = (st);                  \
        if (s_ != HEC_OK) return s_;           \
    } while (0)

#define HEC_LAUNCHED()                                                    \
    do {                                                                  \
        ::hec::count_launch();                                            \
        cudaError_t e_ = cudaGetLastError();                              \
        if (e_ != cudaSuccess) return ::hec::cuda_error(e_, "kernel launch"); \
    } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// device allocation that reports OOM as a status, and its release (common.cu: a per-device cache of
// released blocks; dfree waits for the device before it keeps a block, as cudaFree would)
hec_status dmalloc(void** p, size_t bytes);
void dfree(void* p);
template <typename T>
hec_status dalloc(T** p, size_t count) { return dmalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16); }

int num_sms();
// measurement hooks around kernel launches (no-ops unless hec_profile_enable(1)); categories:
enum ProfCat { PROF_SWEEP = 0, PROF_SPMV = 1, PROF_GS = 2, PROF_ARNOLDI = 3, PROF_VEC = 4, PROF_FILL = 5 };
void profile_begin(cudaStream_t s, void** token, int cat = PROF_SWEEP);
void profile_end(cudaStream_t s, void* token);
// RAII bracket for one launch
struct ProfScope {
    cudaStream_t s;
    void* tok = nullptr;
    ProfScope(cudaStream_t st, int cat) : s(st) { profile_begin(s, &tok, cat); }
    ~ProfScope() { profile_end(s, tok); }
};
int max_coop_blocks(const void* kernel, int threads, size_t smem);  // resident blocks per SM

// ---- device status word codes -------------------------------------------------------------
// Written with atomicCAS(status, 0, code) so the first failure sticks.
enum : int { DEV_OK = 0, DEV_TIMEOUT = HEC_ERR_TIMEOUT, DEV_OOB = HEC_ERR_OUT_OF_BOUNDS,
             DEV_ZERO_PIVOT = HEC_ERR_ZERO_PIVOT };

// ---- exclusive scan of int32 (device) -----------------------------------------------------
// out[i] = sum_{j<i} in[i]; out[n] = total when out has n+1 entries (total_out selects).
// in and out may alias.  Uses a workspace from the scan module's own cache.
hec_status exclusive_scan_i32(const int* in, int* out, int n, bool write_total, cudaStream_t s);

// ---- opaque handle definitions ------------------------------------------------------------
}  // namespace hec

struct hec_levels {
    int n = 0, nlev = 0, uplo = 0;
    int* level = nullptr;      // [n]
    int* perm = nullptr;       // [n]
    int* iperm = nullptr;      // [n]
    int* level_ptr = nullptr;  // [nlev+1]
};

struct hec_matrix {
    int n = 0, ld = 0, w = 0, tri = 0, uplo = 0;
    hec_dtype vdt = HEC_F64;
    long long tail_nnz = 0;
    int* ell_col = nullptr;
    void* ell_val = nullptr;
    int* tptr = nullptr;
    int* tcol = nullptr;
    void* tval = nullptr;
    const hec_levels* lv = nullptr;  // analysis used to pack (borrowed), NULL in general mode
};

// Partitioned layout of a plan (see sweep.cu, "partitioned sweep"): rows in (part, level,
// global level order) order, the factor repacked in that order.
struct hec_part_data {
    int nparts = 0, nseg = 0;
    int* rowg = nullptr;       // [n] plan row -> row of the level-ordered factor
    int* part_row = nullptr;   // [nparts+1]
    int* part_seg = nullptr;   // [nparts+1]
    int* seg_start = nullptr;  // [nseg+1] first plan row of each (part, level) segment
    int* ell_col = nullptr;    // repacked HEC (columns in plan numbering)
    void* ell_val = nullptr;
    int* tptr = nullptr;
    int* tcol = nullptr;
    void* tval = nullptr;
    void* dinv = nullptr;
    void* bp = nullptr;         // [n] right-hand side of the current sweep in plan order (FP32 work only)
    int* part_chunk = nullptr;  // [nparts+1] first level-aligned chunk of each part
    int2* chunks = nullptr;     // (first plan row, rows <= 32)
    int nchunks = 0;
    int max_rows = 0;           // rows of the largest part (its shared-memory solution)
    int threads = 256;
    // Two plan-order solution buffers (the cross-part words): a sweep polls xpb[parity] and sets
    // the other one to the sentinel for the next sweep, so no fill runs between sweeps.  Sweeps of
    // one plan are stream-ordered (as for every plan), which is what makes the other buffer idle.
    void* xpb[2] = {nullptr, nullptr};
    mutable int parity = 0;
    long long id = 0;           // unique per partition build (caches of composed indices key on it)
    int* pos = nullptr;         // [n] row of the level-ordered factor -> plan row (inverse of rowg)
    int* bidx_perm = nullptr;   // [n] plan row -> row of b for sptrsv_lower / sptrsv_upper (iperm[rowg])
};

struct sptrsv_plan {
    hec_part_data* part = nullptr;  // set by sptrsv_plan_partition
    const hec_matrix* T = nullptr;
    const hec_levels* lv = nullptr;
    int max_nrhs = 1;
    int threads = 256, blocks = 0;
    long long wait_cycles = 2000000000LL;
    int skip_row = -1;         // fault injection: row never published (tests only)
    int backoff_ns = 0;        // sleep between dependency polls
    void* xp = nullptr;        // internal solution in level order, n * max_nrhs of the work type
    int* status = nullptr;     // device status word
    int2* chunks[5] = {};      // level-aligned chunk tables for 32, 16, 8, 4, 2 rows per warp step
    int nchunks[5] = {};
    void* dinv = nullptr;      // reciprocal diagonal in the work type (NULL: the kernel divides)
    int lpr1 = 1;              // lanes per row of single-right-hand-side sweeps (1, 2, 4 or 8)
    int use_part = 1;          // single-right-hand-side sweeps take the partition when there is one
};

struct ilu_precond {
    const sptrsv_plan* L = nullptr;
    const sptrsv_plan* U = nullptr;
    int n_glob = 0, n_ext = 0;
    int* l_gather = nullptr;   // [n_ext] lower sweep: new row -> row of r to read
    int* l_scatter = nullptr;  // [n_ext] lower sweep: new row -> row of the intermediate y (in U order)
    int* u_scatter = nullptr;  // [n_ext] upper sweep: new row -> row of z to write, -1 = not owned
    void* y = nullptr;         // [n_ext * max_nrhs] intermediate, already in the upper factor's order
    bool y32 = false;          // y in FP32 (both sweeps compute in FP32), else FP64
    int max_nrhs = 1;
    // composed indices for partitioned single-right-hand-side sweeps, built at the first apply
    // after a partition changes (keyed on hec_part_data::id):
    mutable int* lg_part = nullptr;     // [n_ext] plan row of L -> row of r (l_gather[rowg_L])
    mutable long long lg_part_id = 0;
    mutable int* ls_upart = nullptr;    // [n_ext] level row of L -> plan row of U (pos_U[l_scatter])
    mutable long long ls_upart_id = 0;
};

struct hec_csr {
    int n = 0;
    long long nnz = 0;
    int* rowptr = nullptr;
    int* col = nullptr;
    double* val = nullptr;
};

namespace hec {
// Lane layout of the sweep: nrhs right-hand sides are padded to KP = the next power of two; one
// right-hand side runs a lane per row, more run G per lane (4 for FP32 work, 2 for FP64) and
// KP / G lanes per row.  The level-ordered solution has a row stride of KP values, and the chunk
// table used is the one for 32 / lanes-per-row rows per warp.
inline int sweep_kp(int nrhs) {
    int kp = 1;
    while (kp < nrhs) kp <<= 1;
    return kp;
}
inline int sweep_lpr(int nrhs, hec_dtype vdt) {
    if (nrhs <= 1) return 1;
    const int kp = sweep_kp(nrhs);
    const int g = vdt == HEC_F64 ? 2 : (kp >= 4 ? 4 : 2);
    return kp / g;
}
inline int log2i(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}
// Single-right-hand-side lanes per row by row length: the one-lane kernel polls up to 8 slab
// slots and 4 tail entries per wait and waits again for every further slot; several lanes per
// row poll 3 slab slots and 2 tail entries each, all in one wait.
inline int default_lanes_per_row(const hec_matrix* T) {
    const long long over = T->tail_nnz - (long long)T->n;  // tail entries besides the diagonals
    if (T->w <= 8 && over * 2 <= (long long)T->n) return 1;
    return T->w <= 6 ? 2 : T->w <= 12 ? 4 : 8;
}

// sweep launcher shared by sptrsv_* and ilu_apply: gather[r] is the row of b feeding new row r
// (NULL = identity), scatter[r] the row of x receiving it (NULL = identity, -1 = skip).
// For a partitioned single-right-hand-side sweep, bidx (if not NULL) gives the row of b for each
// plan row directly (a gather composed with the plan's row order), and bplan says b is already in
// the plan's row order; both are ignored on the other paths.
hec_status sweep(const sptrsv_plan* p, int nrhs, const double* b, int ldb, const int* gather, double* x,
                 int ldx, const int* scatter, cudaStream_t s, bool b32 = false, bool x32 = false,
                 const int* bidx = nullptr, bool bplan = false);
// y = alpha A x + beta y for a general-mode FP64 HEC matrix (krylov.cu; no argument checks)
hec_status spmv_impl(const hec_matrix* A, int K, double alpha, const double* x, int ldx, double beta, double* y,
                     int ldy, cudaStream_t s);
}  // namespace hec
