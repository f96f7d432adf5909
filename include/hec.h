/*
 * hec.h -- C ABI of libhec: level-scheduled sparse triangular solves on the HEC format, the
 * ILU / RAS preconditioners they apply, SpMV and FGMRES, all computed by CUDA kernels on one
 * GB300 (sm_103a).
 *
 * Method: Chen, Liu, Yang, "Parallel Triangular Solvers on GPU" (arXiv 1606.00541).
 *
 * Conventions shared by every entry point
 *   - Indices are 0-based int32.  CSR inputs have rowptr[n+1], col[nnz], val[nnz]; every row is
 *     sorted by ascending column (the paper assumes this, Sec. 2).
 *   - Every array argument is a DEVICE pointer owned by the caller unless the comment says
 *     "host".  Handles (hec_levels, hec_matrix, sptrsv_plan, ilu_precond, hec_csr) own their
 *     internal device buffers and are released with the matching *_destroy.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default stream.  Compute
 *     calls are asynchronous on that stream unless their comment says they synchronize.
 *   - Dense blocks of right-hand sides are row-major n x nrhs with leading dimension ld >= nrhs
 *     (the nrhs values of one row are contiguous).
 *   - Every function returns a hec_status.  On failure hec_last_error() describes the cause
 *     (thread-local, valid until the next call on the same thread).  No exception and no abort
 *     crosses this boundary.  Device-side failures (a dependency wait that ran out of time, an
 *     index out of bounds) are recorded in a device status word of the handle and reported by
 *     hec_sync_status() and by fgmres_solve.
 *   - There is no CPU fallback: when no sm_103a device is present the calls fail with
 *     HEC_ERR_CUDA.
 */
#ifndef HEC_H
#define HEC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HEC_OK = 0,
    HEC_ERR_INVALID_ARG = 1,    /* bad size, NULL pointer, unsupported option */
    HEC_ERR_UNSORTED = 2,       /* a CSR row not strictly ascending, or a column out of range */
    HEC_ERR_NOT_TRIANGULAR = 3, /* an entry on the wrong side of the diagonal */
    HEC_ERR_MISSING_DIAG = 4,   /* a row of a triangular factor without its diagonal */
    HEC_ERR_ZERO_PIVOT = 5,     /* a zero diagonal (solve) or pivot (factorization) */
    HEC_ERR_OOM = 6,            /* device allocation failed */
    HEC_ERR_CUDA = 7,           /* a CUDA runtime error; see hec_last_error() */
    HEC_ERR_TIMEOUT = 8,        /* a device-side dependency wait exceeded its time budget */
    HEC_ERR_NOT_CONVERGED = 9,  /* FGMRES reached max_iters before rtol */
    HEC_ERR_OUT_OF_BOUNDS = 10  /* a device-side index check failed */
} hec_status;

typedef enum { HEC_F64 = 0, HEC_F32 = 1, HEC_BF16 = 2 } hec_dtype;

typedef struct hec_levels hec_levels;
typedef struct hec_matrix hec_matrix;
typedef struct sptrsv_plan sptrsv_plan;
typedef struct ilu_precond ilu_precond;
typedef struct hec_csr hec_csr;

/* Message for the last failing call on this thread ("" when none). */
const char* hec_last_error(void);

/* Device memory held for reuse.  The library keeps the blocks its handles and set-up steps release
 * (per device, up to 16 GiB a process) and hands them out again for later requests of about the
 * same size, since cudaMalloc / cudaFree cost tens to hundreds of microseconds each.  A released
 * block is cached only after the device has finished the work queued before the release (as
 * cudaFree would), so a cached block is never in use.  This call returns every cached block to the
 * CUDA runtime and the number of bytes returned; a failing cudaMalloc does the same for its device
 * before it retries. */
size_t hec_release_cached_memory(void);

/* Library version and the number of kernel launches issued by this process so far (host
 * counter, incremented by every launch the library makes). */
int hec_version(void);
long long hec_launch_count(void);

/* Kernel timing for measurement: while enabled, every launch of the library's kernel categories
 * (listed at hec_profile_read_category) is bracketed by a pair of CUDA events recorded on the
 * stream it is launched on.  hec_profile_read waits for the recorded events and returns the
 * summed device time (ms) and the number of triangular-sweep launches since the last reset
 * (reset != 0 clears the whole record).  Off by default. */
hec_status hec_profile_enable(int on);
/* Enables the record for the categories in `mask` only (bit c = category c of
 * hec_profile_read_category; 0 disables), so a timed run can bracket just the kernels it reports
 * and leave the rest of the launch stream without event records.  hec_profile_enable(on) is
 * mask = all or none. */
hec_status hec_profile_enable_categories(unsigned int mask);
hec_status hec_profile_read(double* sweep_ms, long long* sweep_launches, int reset);
/* The same record for other kernel classes (not reset): 0 sweeps, 1 SpMV, 2 Gram-Schmidt dots
 * and updates, 3 the small Arnoldi kernels, 4 vector scale/copy/update, 5 sentinel fills (with
 * the partitioned sweep's right-hand-side gather). */
hec_status hec_profile_read_category(int category, double* ms, long long* launches);

/* ---------------------------------------------------------------------------------------- */
/* Level analysis: Eq. 2 (levels), Eq. 3 (map m), Alg. 1 steps 1-2; upper factor by the       */
/* index reversal of Sec. 2.2                                                                 */
/* ---------------------------------------------------------------------------------------- */

/* Computes the level of every row of a triangular factor and the level-ordering map.
 *   uplo 0: T is lower triangular; the dependencies of row i are its columns j < i.
 *   uplo 1: T is upper triangular; it is solved as the lower problem of the reversed order
 *           t(i) = n-1-i (the paper's t(i) = n - i with 1-based indices), so the dependencies
 *           of row i are its columns j > i.
 * Level (0-based; the paper's level minus one): 0 for a row without dependencies, else
 * 1 + the largest level among its dependencies.  The diagonal is not a dependency.
 * Map: rows are ordered by level, and within a level by ascending index of the lower problem
 * (i for uplo 0, n-1-i for uplo 1); perm[i] is the position of original row i, iperm its
 * inverse, level_ptr[k] the first position of level k (level_ptr[nlev] = n).
 * The input is validated first (sorted rows, columns in range, triangular, diagonal present);
 * a malformed factor returns UNSORTED / NOT_TRIANGULAR / MISSING_DIAG.  Synchronizes `stream`
 * (the level count sizes the outputs).  n = 0 is allowed (nlev = 0). */
hec_status sptrsv_analyze(int n, const int* rowptr, const int* col, int uplo, hec_levels** out,
                          void* stream);

/* Borrowed device pointers of a level analysis (valid until hec_levels_destroy):
 * level[n], perm[n], iperm[n], level_ptr[nlev+1].  Any output pointer may be NULL. */
hec_status hec_levels_get(const hec_levels* lv, int* n, int* nlev, int* uplo, const int** level,
                          const int** perm, const int** iperm, const int** level_ptr);
hec_status hec_levels_destroy(hec_levels* lv);

/* ---------------------------------------------------------------------------------------- */
/* HEC format: Sec. 2.1 (ELL slab in column-major order + CSR tail whose rows hold at least    */
/* the diagonal), Alg. 1 steps 3-4 (reorder L to L', convert to HEC)                          */
/* ---------------------------------------------------------------------------------------- */

typedef struct {
    int n;          /* rows */
    int ld;         /* slab leading dimension = n rounded up to a multiple of 32 */
    int w;          /* slab width (entries per row in the ELL part) */
    int tri;        /* 1: triangular factor reordered by a level map; 0: general matrix */
    int uplo;       /* for tri = 1 */
    hec_dtype vdt;  /* value type of ell_val and tval */
    long long tail_nnz;
    const int* ell_col;   /* [w*ld] column of slot k of row r at k*ld + r; -1 = padding */
    const void* ell_val;  /* [w*ld] values, same layout; padding holds +0.0 */
    const int* tptr;      /* [n+1] tail row pointers */
    const int* tcol;      /* [tail_nnz] */
    const void* tval;     /* [tail_nnz] */
} hec_matrix_info;

/* Packs a CSR matrix into HEC.
 * lv != NULL (triangular mode): the factor analysed by `lv` is reordered, L'(m(i), m(j)) =
 *   L(i, j); each row of L' is sorted by new column; its first w off-diagonal entries go to
 *   slab slots 0..w-1, the rest follow in the tail in ascending new column, and the diagonal
 *   is the LAST tail entry of the row (so every tail row holds at least one entry).  Unused
 *   slots, and every slot of rows n..ld-1, hold column -1 and value +0.0.  Columns are in the
 *   new (level-ordered) numbering.  The factor must be the one `lv` was computed from.
 * lv == NULL (general mode, e.g. the matrix A for SpMV): rows and columns keep their numbering
 *   and CSR order; the first w entries of a row go to the slab, the rest to the tail, which
 *   may then be empty for a row.
 * ell_width: >= 0 fixes w; -1 applies the rule: the largest w such that at least
 *   ceil(0.65 n) rows have w or more slab-eligible entries (off-diagonals in triangular mode).
 * vdt: value storage; FP32 and BF16 values are rounded once from FP64, to nearest even
 *   (BF16 directly from the FP64 value).
 * Synchronizes `stream` (the width rule and the tail size are needed on the host). */
hec_status hec_from_csr(int n, const int* rowptr, const int* col, const double* val,
                        const hec_levels* lv, int ell_width, hec_dtype vdt, hec_matrix** out,
                        void* stream);
hec_status hec_matrix_get(const hec_matrix* A, hec_matrix_info* info /* host */);

/* Rebuilds the CSR of the ORIGINAL matrix (original numbering, rows ascending, values widened
 * to FP64) from HEC; lv must be the analysis used to pack it (NULL in general mode).
 * rowptr[n+1], col[nnz], val[nnz] are caller-allocated device arrays; nnz = the number of
 * non-padding entries.  Used for round-trip checks.  Synchronizes `stream`. */
hec_status hec_to_csr(const hec_matrix* A, const hec_levels* lv, int* rowptr, int* col,
                      double* val, void* stream);
hec_status hec_matrix_destroy(hec_matrix* A);

/* ---------------------------------------------------------------------------------------- */
/* Triangular sweeps: Alg. 2 (permute b, solve level by level, permute back) and its upper    */
/* form by reversal (Sec. 2.2)                                                                */
/* ---------------------------------------------------------------------------------------- */

typedef struct {
    int block_threads;      /* threads per block of the sweep kernel (0 = 256) */
    int blocks_per_sm;      /* resident blocks per SM (0 = as many as fit) */
    long long wait_cycles;  /* SM cycles a dependency wait may spin before HEC_ERR_TIMEOUT
                               (0 = 2e9, about one second) */
    int debug_unpublished_row; /* fault injection for tests: a new (level-ordered) row whose
                                  solution is computed but never published to its dependents,
                                  so their waits run out and the call reports HEC_ERR_TIMEOUT;
                                  0 disables it, r + 1 selects row r */
    int backoff_ns;         /* nanoseconds a warp sleeps between polls of an unpublished
                               dependency (0 = poll continuously) */
    int lanes_per_row;      /* lanes sharing a row in single-right-hand-side sweeps: 1, 2, 4 or 8;
                               0 = by row length (1 while the slab is at most 8 wide and the tail
                               holds few entries besides the diagonals, else 2 / 4 / 8 for slabs up
                               to 6 / 12 / wider).  Several lanes poll all of a long row's
                               dependencies in one wait and add their partial sums with an xor
                               butterfly (a different summation order from one lane). */
    int partitioned;        /* output of sptrsv_autotune: 1 when single-right-hand-side sweeps of
                               the plan take its partition (sptrsv_plan_partition), 0 when the
                               global schedule was faster or there is no partition; ignored as
                               an input */
} hec_tune;

/* A solve plan for one triangular factor: its HEC form and level analysis (both borrowed; they
 * must outlive the plan) plus the workspace for up to max_nrhs right-hand sides
 * (1 <= max_nrhs <= 16).  tune may be NULL for defaults. */
hec_status sptrsv_plan_create(const hec_matrix* tri, const hec_levels* lv, int max_nrhs,
                              const hec_tune* tune, sptrsv_plan** out);
hec_status sptrsv_plan_destroy(sptrsv_plan* p);

/* x = T^-1 b for the lower (sptrsv_lower) or upper (sptrsv_upper) factor of the plan.
 * b and x are n x nrhs row-major FP64 (ldb, ldx >= nrhs), in the ORIGINAL row numbering; the
 * gather b'(m(i)) = b(i) and the scatter x(i) = x'(m(i)) of Alg. 2 happen inside the sweep
 * kernel.  Each row is computed as x'_r = (b'_r - sum_c L'_rc x'_c) / L'_rr, summing the slab
 * slots then the tail in ascending new column; FP64 values are summed in FP64, FP32 and BF16
 * values in FP32 (the solution is stored back as FP64).  b and x must not overlap.  The call
 * fails with INVALID_ARG when the plan's factor has the other triangle. */
hec_status sptrsv_lower(const sptrsv_plan* p, int nrhs, const double* b, int ldb, double* x,
                        int ldx, void* stream);
hec_status sptrsv_upper(const sptrsv_plan* p, int nrhs, const double* b, int ldb, double* x,
                        int ldx, void* stream);

/* Partitioned sweep (a GB300 schedule of Alg. 2's level loop, same results up to summation
 * order): the rows are split into nparts parts, one resident thread block per part (cooperative
 * launch, so nparts <= sptrsv_partition_capacity()).  Inside a part the rows keep the global
 * level order, cut into level-aligned chunks of at most 32 rows dealt round-robin to the block's
 * warps; each row waits point to point for exactly its dependencies.  The part's solution lives
 * in shared memory (the value is its own flag), so a dependency on a row of the same part is an
 * SM-local poll, and only a dependency on another part polls the global solution through L2.
 * part: device int[n], the part of each row of the plan's factor in its ORIGINAL numbering (for
 * a RAS preconditioner, the extended rows; compact regions of the grid work best, and with one
 * part per RAS subdomain no dependency crosses a part, since the factors are block diagonal;
 * the paper partitions with METIS), or NULL for contiguous ranges of the row index.
 * threads: 128, 256, 512 or 1024 (0 = 256) per block.  Fails with INVALID_ARG when the parts
 * cannot all be resident at that block size, or when the largest part's solution (FP64 values:
 * 8 bytes a row, else 4) leaves room for fewer resident blocks than nparts.  Applies to single-
 * right-hand-side sweeps of this plan (sptrsv_lower / sptrsv_upper / ilu_apply with nrhs = 1);
 * nparts = 0 removes it.  The plan keeps its own copy of the factor in the partitioned order,
 * two plan-order solution buffers (a sweep polls one and resets the other for the next sweep),
 * and, for FP32 or BF16 values, an n-entry buffer into which each sweep first gathers its part's
 * rows of the right-hand side in that order (the upper sweep of an ilu_apply receives y already
 * in that order and skips it).  Synchronizes `stream`. */
hec_status sptrsv_plan_partition(sptrsv_plan* p, const int* part, int nparts, int threads,
                                 void* stream);
int sptrsv_partition_capacity(const sptrsv_plan* p, int threads);

/* Autotuner: times the plan's own sweep (on a zero right-hand side, nrhs columns) and keeps the
 * fastest of the candidates in the plan; `out` (host, may be NULL) receives the choice.
 * Candidates: launch shapes block_threads in {128, 256} x blocks_per_sm in {2, 4, 8, 16} (those
 * that fit 2048 threads per SM); for nrhs = 1 also lanes per row in {1, 2, 4, 8} (one thread per
 * row against several lanes sharing a long row), and, when the plan has a partition
 * (sptrsv_plan_partition), the partitioned schedule against the best global one (a plan whose
 * global schedule wins keeps its partition unused; partitioning it again re-enables it).
 * Results are cached per (rows, slab width, tail entries, levels, value type, nrhs rounded up to
 * a power of two, partition given) for the life of the process.  Synchronizes `stream`.  The
 * point-to-point sweep has no per-level barriers, so the paper's level-merging threshold has no
 * counterpart. */
hec_status sptrsv_autotune(sptrsv_plan* p, int nrhs, hec_tune* out, void* stream);

/* Checks, on the device, every index the sweep kernels follow without a bounds check (a check per
 * gathered index would sit on the dependency chain), so that a plan whose arrays were corrupted
 * is reported instead of swept: the level map (perm and iperm inverse permutations, level_ptr
 * from 0 to n); the HEC factor (tail row pointers increasing from 0 to tail_nnz, slab columns in
 * [-1, n) with padding only after a row's entries, tail off-diagonals only after a full slab,
 * every off-diagonal in an earlier level than its row, the diagonal last in the tail and
 * nonzero); every chunk table (in order, each chunk inside one level, covering [0, n)); and, for a
 * partitioned plan, the row map (a permutation), the part tables, the repacked factor and the
 * part chunks.  Returns HEC_OK, or HEC_ERR_OUT_OF_BOUNDS with hec_last_error() naming the first
 * failing check and index.  Reads only the plan; synchronizes `stream`. */
hec_status sptrsv_plan_check(const sptrsv_plan* p, void* stream);

/* Reads and clears the device status word of a plan (synchronizes `stream`).  Returns HEC_OK,
 * HEC_ERR_TIMEOUT or HEC_ERR_OUT_OF_BOUNDS as recorded by the kernels since the last call. */
hec_status hec_sync_status(const sptrsv_plan* p, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Preconditioners: ILU (Eq. 1: L y = r, U z = y) and Restricted Additive Schwarz with the     */
/* subdomain factors batched block-diagonally (Sec. 3, Eq. 4)                                 */
/* ---------------------------------------------------------------------------------------- */

/* Plain ILU: ext2glob == NULL; L and U are factors of the n x n matrix and n_glob == n.
 * RAS: L and U are block-diagonal factors of diag(A_1, ..., A_s) over n_ext extended rows;
 * ext2glob[n_ext] maps each extended row to its global row (a global row appears once per
 * subdomain that contains it) and owned[n_ext] is 1 for the rows the subdomain owns (each
 * global row owned exactly once).  ilu_apply then computes
 * z = sum_s R0_s^T U_s^-1 L_s^-1 R_s r: gather r through ext2glob, sweep L then U, and write
 * back only owned rows.  The plans (and arrays) are borrowed. */
hec_status ilu_create(const sptrsv_plan* L, const sptrsv_plan* U, int n_glob, int n_ext,
                      const int* ext2glob, const unsigned char* owned, ilu_precond** out);
hec_status ilu_destroy(ilu_precond* M);

/* z = M^-1 r; r and z are n_glob x nrhs row-major FP64 (nrhs <= the plans' max_nrhs). */
hec_status ilu_apply(const ilu_precond* M, int nrhs, const double* r, int ldr, double* z,
                     int ldz, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* SpMV on HEC (FP64 values) and the FGMRES outer solver                                      */
/* ---------------------------------------------------------------------------------------- */

/* y = alpha * A x + beta * y for a general-mode HEC matrix with FP64 values (beta = 0 ignores
 * the input y).  x and y are n x nrhs row-major with ldx, ldy >= nrhs. */
hec_status spmv(const hec_matrix* A, int nrhs, double alpha, const double* x, int ldx,
                double beta, double* y, int ldy, void* stream);

typedef struct {
    int iterations;      /* inner iterations (largest over the right-hand sides) */
    int restarts;
    int converged;       /* 1 when every right-hand side reached rtol */
    double rel_residual; /* largest true relative residual ||b - A x|| / ||b|| at exit */
    double seconds;      /* wall time of the call, host clock */
    int reorthogonalized; /* inner iterations that took a second Gram-Schmidt pass (classical mode) */
} hec_fgmres_info;

/* Gram-Schmidt variant of the Arnoldi step in fgmres_solve, process-wide (default
 * HEC_GS_CLASSICAL).  Both are FP64 and equal in exact arithmetic; the paper runs GMRES without
 * naming one (Sec. 4).
 *   HEC_GS_CLASSICAL: all inner products h = V^T w from the same w (one grid-wide reduction a
 *     step), w -= V h, and a second pass (h2 = V^T w, w -= V h2) for a right-hand side whose norm
 *     fell below 0.25 ||w|| (selective reorthogonalization); ||w - V h|| from ||w||^2 - ||h||^2
 *     when no second pass runs.  hec_fgmres_info.reorthogonalized counts the second passes.
 *   HEC_GS_MODIFIED: one projection at a time (one grid-wide reduction per projection), as the
 *     textbook modified Gram-Schmidt.
 * Returns HEC_ERR_INVALID_ARG for any other value.  Not thread-safe against a concurrent
 * fgmres_solve call (the mode is read once when a solve starts). */
enum { HEC_GS_CLASSICAL = 0, HEC_GS_MODIFIED = 1 };
hec_status hec_set_gram_schmidt(int mode);
int hec_get_gram_schmidt(void);

/* Solves A x = b by right-preconditioned flexible GMRES(restart), z_j = M^-1 v_j with the ILU
 * or RAS preconditioner M (NULL = none), FP64 throughout: SpMV, Gram-Schmidt in one persistent
 * kernel per inner iteration (classical with selective reorthogonalization by default, or
 * modified: hec_set_gram_schmidt; deterministic fixed-order grid-wide reductions), Givens
 * rotations.  Each of the nrhs right-hand sides (row-major n x nrhs, nrhs <= 16) has its
 * own Krylov space; their kernels run batched.  x holds x0 on entry (zero it for x0 = 0) and the
 * solution on exit.  Convergence: the Arnoldi estimate |g_{j+1}| <= rtol ||b|| ends a cycle,
 * then the true residual ||b - A x|| is computed and checked; max_iters bounds the inner
 * iterations.  info (host, may be NULL) receives the statistics.
 * Synchronization: the Hessenberg matrix, the rotations and the residual estimate stay on the
 * device.  Inside a restart cycle the host only reads a per-iteration "still active" flag through
 * pinned memory one iteration behind the device (an event wait, the device never idles for the
 * host); `stream` is synchronized at each restart (true residual, status of the sweeps) and at
 * exit.  Allocates its workspace (restart + 1 + restart vectors of n x nrhs) per call, from the
 * library's device memory cache; the pinned flag pair and its two events are kept per calling
 * thread and device and reused by later calls.  Returns
 * HEC_ERR_NOT_CONVERGED when max_iters is reached, HEC_ERR_TIMEOUT when a sweep's dependency
 * wait timed out. */
typedef struct hec_stage hec_stage;
hec_status fgmres_solve(const hec_matrix* A, const ilu_precond* M, const hec_stage* extra,
                        int nrhs, const double* b, int ldb, double* x, int ldx, int restart,
                        double rtol, int max_iters, hec_fgmres_info* info /* host */,
                        void* stream);
/* `extra` (may be NULL) is a learned correction stage (stage_create below) applied after M in
 * every iteration; it requires M and nrhs = 1. */

/* ---------------------------------------------------------------------------------------- */
/* Learned correction stage (not in the paper): a 4-layer 3x3x3 convolutional network, 2 -> 16 */
/* -> 16 -> 16 -> 1 channels, ReLU between layers, BF16 weights and activations with FP32      */
/* accumulation on the tensor cores, trained on (residual, error) pairs of the FP64 solver      */
/* ---------------------------------------------------------------------------------------- */

typedef struct hec_net hec_net;

/* Number of FP32 parameters: 4 layers x (27 taps x 16 in x 16 out weights + 16 biases).  Layer l
 * occupies [l * 6928, (l+1) * 6928): weight (tap, ci, co) at (tap*16 + ci)*16 + co with
 * tap = (dz*3 + dy)*3 + dx (offsets dz-1, dy-1, dx-1), then the 16 biases.  Channels the network
 * does not use (inputs 2..15 of layer 0, outputs 1..15 of layer 3) should be zero. */
int net_param_count(void);
/* params: host FP32 array of net_param_count() values (the initialization). */
hec_status net_create(const float* params, hec_net** out);
hec_status net_destroy(hec_net* net);
/* Host copies of the FP32 parameters and of the last computed gradients (either may be NULL). */
hec_status net_get_params(const hec_net* net, float* params, float* grads);
hec_status net_set_params(hec_net* net, const float* params);
/* Forward pass on a field of nx*ny*nz voxels (x fastest) made of nz/zs samples of zs planes
 * stacked along z (each sample padded with zeros at its own boundary).  x_in: device BF16,
 * channels-last, 16 channels per voxel (channels 0 and 1 used).  acts_out (may be NULL): device
 * BF16 [4][nvox][16], the outputs of the four layers (after ReLU for the first three).  out (may
 * be NULL): device FP32 [nvox], channel 0 of the last layer before rounding to BF16. */
hec_status net_forward(hec_net* net, int nx, int ny, int nz, int zs, const void* x_in,
                       void* acts_out, float* out, void* stream);
/* One training step on a minibatch laid out as in net_forward: forward, mean-squared error
 * against target (device FP32 [nvox]), backward (gradients kept, see net_get_params) and, when
 * update != 0, one Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected) with rate lr.
 * loss_out (host, may be NULL) receives the loss and then the call synchronizes `stream`. */
hec_status net_train_step(hec_net* net, int nx, int ny, int nz, int zs, const void* x_in,
                          const float* target, float lr, int update, float* loss_out,
                          void* stream);
/* The two halves of net_train_step.  net_backward: forward, mean-squared error against target
 * and backward on one minibatch (layout as net_forward); the parameter gradients are kept in the
 * net (net_get_params) and loss_out (host, may be NULL) receives the loss, after which the call
 * synchronizes `stream`.  net_adam_step: one Adam step (beta 0.9 / 0.999, eps 1e-8,
 * bias-corrected with the net's own step count) from the kept gradients with rate lr, then the
 * BF16 weight copies the forward pass uses.  net_train_step(..., update = 1) = net_backward +
 * net_adam_step. */
hec_status net_backward(hec_net* net, int nx, int ny, int nz, int zs, const void* x_in,
                        const float* target, float* loss_out, void* stream);
hec_status net_adam_step(hec_net* net, float lr, void* stream);
/* The forward pass (all four layers) runs on tcgen05 MMAs (tensor_cores = 1, the default) or on
 * the warp-level mma.sync path (0); both accumulate the same BF16 products in FP32, in a different
 * order.  The backward pass (net_backward, net_train_step) always uses mma.sync. */
hec_status net_set_engine(hec_net* net, int tensor_cores);
/* Synchronizes `stream` and returns HEC_ERR_TIMEOUT (then clears it) when a tcgen05 convolution
 * since the last call gave up waiting for its MMAs (its outputs were not written), else HEC_OK.
 * fgmres_solve checks its stage's net this way at every restart. */
hec_status net_sync_status(hec_net* net, void* stream);

/* A training sample from one residual / error pair on an n-voxel field: sigma = RMS(r) (device
 * FP64, *sigma_out), x_out = channels-last BF16 [n][16] with channel 0 = r / sigma, channel 1 =
 * aux_scale * aux, the rest 0, and target_out (may be NULL) = e / sigma in FP32 [n]. */
hec_status net_make_sample(int n, const double* r, const double* e, const double* aux,
                           double aux_scale, void* x_out, float* target_out, double* sigma_out,
                           void* stream);

/* The stage used by fgmres_solve: with z1 = M^-1 v (the ILU sweep) and r1 = v - A z1,
 * c = sigma * Net([r1 / sigma, aux_scale * aux]) with sigma = RMS(r1), alpha = <r1, A c> /
 * <A c, A c>, and z = z1 + alpha c when alpha > 0 and ||r1 - alpha A c|| < rho ||r1||, else z = z1
 * (the plain ILU result: the fallback).  sigma comes from FP64 sums; alpha and the acceptance
 * test from FP32 partial sums (they only scale the correction).  Inside fgmres_solve a stage on
 * the solver's own A also returns A z = (v - r1) + alpha A c, which replaces the solver's product.
 * A: the FP64 general-mode matrix on an nx*ny*nz grid;
 * aux: device FP64 [n] second input field (e.g. ln k), copied.  The net is borrowed. */
hec_status stage_create(hec_net* net, const hec_matrix* A, int nx, int ny, int nz,
                        const double* aux, double aux_scale, double rho, hec_stage** out);
/* One application of the stage outside the solver, as fgmres_solve applies it: v (device FP64
 * [n]) is the vector to precondition, z (device FP64 [n]) holds z1 = M^-1 v on entry (e.g. from
 * ilu_apply) and z1 or z1 + alpha c on return.  Asynchronous on `stream`; counts toward
 * stage_stats. */
hec_status stage_apply(const hec_stage* stage, const double* v, double* z, void* stream);
/* Applications and accepted corrections since creation or the last reset. */
hec_status stage_stats(const hec_stage* stage, int* applied, int* accepted, int reset);
hec_status stage_destroy(hec_stage* stage);

/* ---------------------------------------------------------------------------------------- */
/* Incomplete factorizations on the GPU (Sec. 3): ILU(k) and ILUT of a CSR matrix               */
/* ---------------------------------------------------------------------------------------- */

/* Device CSR owned by the library. */
hec_status hec_csr_get(const hec_csr* M, int* n, long long* nnz, const int** rowptr,
                       const int** col, const double** val);
hec_status hec_csr_destroy(hec_csr* M);

/* The lower (uplo 0: j <= i) or upper (uplo 1: j >= i) triangle of a CSR matrix (n x n,
 * ascending columns), without the diagonal when strict != 0, as a device CSR owned by the
 * library.  With it the sweeps run Gauss-Seidel: one forward sweep is (D + L) x' = b - U_s x,
 * one backward sweep (D + U) x'' = b - L_s x' (the smoothers the paper names as another use of
 * the triangular solver, Sec. 1).  Synchronizes `stream`. */
hec_status csr_triangle(int n, const int* rowptr, const int* col, const double* val, int uplo,
                        int strict, hec_csr** out, void* stream);
/* Symmetric Gauss-Seidel smoother on the level-scheduled sweeps (the smoothers the paper names as
 * another use of the triangular solver, Sec. 1).  With A = L_s + D + U_s (strict lower part,
 * diagonal, strict upper part of the n x n CSR matrix, ascending columns, nonzero diagonal), one
 * symmetric sweep is the forward sweep (D + L_s) x' = b - U_s x followed by the backward sweep
 * (D + U_s) x'' = b - L_s x'; each triangle is solved by the HEC sweep of Alg. 2 (level
 * scheduling reorders only independent rows, so a sweep equals sequential Gauss-Seidel up to
 * rounding).  sgs_create builds the handle: the triangles D + L_s and D + U_s analysed, packed
 * with values of type vdt and planned for up to max_nrhs (<= 16) right-hand sides; U_s and L_s
 * in FP64 for the residual products; one n x max_nrhs work vector.  Synchronizes `stream`.
 * sgs_smooth runs `sweeps` symmetric sweeps on x in place (row-major n x nrhs FP64; x holds the
 * start on entry and the result on exit; b is not modified).  Asynchronous on `stream`;
 * sgs_sync_status reads and clears the device status of the two sweeps (HEC_ERR_TIMEOUT when a
 * dependency wait ran out). */
typedef struct hec_sgs hec_sgs;
hec_status sgs_create(int n, const int* rowptr, const int* col, const double* val, hec_dtype vdt,
                      int max_nrhs, hec_sgs** out, void* stream);
hec_status sgs_smooth(const hec_sgs* sgs, int nrhs, const double* b, int ldb, double* x, int ldx,
                      int sweeps, void* stream);
hec_status sgs_sync_status(const hec_sgs* sgs, void* stream);
hec_status sgs_destroy(hec_sgs* sgs);

/* ILU(k), k >= 0 ("k is the fill-in level", Sec. 3).  The pattern: entries of A have level 0;
 * eliminating pivot q of row i (q < i, ascending, fill pivots included) gives (i, j), j > q in U
 * row q, the level lev(i, q) + lev(q, j) + 1, an entry keeps the smallest level it receives, and
 * entries with level <= k are kept.  k = 0 is the pattern of A; k = 1 is built by a merge of the
 * original rows (at most 63 pivots a row); k >= 2 by a row-dependent symbolic pass (one warp per
 * row, a row's list capped at 4096 entries: OUT_OF_BOUNDS beyond).  Each row i is then
 * eliminated IKJ-style: for the pattern columns q < i in ascending order,
 * a_iq <- a_iq / u_qq, then a_ij <- a_ij - a_iq u_qj for pattern columns j > q of both rows.
 * Rows run in the level order of the lower pattern with point-to-point completion waits.
 * Outputs L (unit lower, the 1.0 diagonal stored) and U (upper with its diagonal).  A must have
 * a nonzero diagonal in every row; ZERO_PIVOT if an eliminated pivot is zero; TIMEOUT if a
 * dependency wait runs out.  Synchronizes. */
hec_status ilu_factor(int n, const int* rowptr, const int* col, const double* val, int k,
                      hec_csr** L, hec_csr** U, void* stream);

/* ILUT(p, tol) (Sec. 3 lists ILUT among the preconditioners; the dual-threshold rule is Saad's):
 * for row i, tau_i = tol * ||a_i||_2 (squares summed in row order); the row's entries k < i,
 * including fill, are eliminated in ascending column order: w_k <- w_k / u_kk, dropped when
 * |w_k| < tau_i, else w_j <- w_j - (w_k * u_kj) for the entries j > k of U row k.  Then entries
 * with w_j = 0 or |w_j| < tau_i are dropped and the p largest magnitudes kept in the strict lower
 * and in the strict upper part (ties to the smaller column); the diagonal is always kept (a
 * missing diagonal gets a structural zero slot).  Every operation is rounded separately (no
 * fused multiply-add), in this order.  Outputs L (unit lower, the 1.0 diagonal stored last in its
 * row) and U (upper, diagonal first), columns ascending.  A's rows must be sorted ascending.
 * Errors: ZERO_PIVOT; OUT_OF_BOUNDS when a row's working fill exceeds 9000 entries; TIMEOUT if a
 * dependency wait runs out.  Synchronizes `stream`. */
hec_status ilut_factor(int n, const int* rowptr, const int* col, const double* val, int p,
                       double tol, hec_csr** L, hec_csr** U, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Restricted Additive Schwarz setup (Sec. 3; Eq. 4: the subdomain problems as one            */
/* block-diagonal system)                                                                     */
/* ---------------------------------------------------------------------------------------- */

typedef struct hec_ras hec_ras;

/* Builds the RAS subdomain system of A (n x n, CSR) for the ownership map part[n] (each row
 * owned by one subdomain in [0, nsub); the paper partitions with METIS, the caller supplies any
 * partition).  Overlap 1: subdomain s's extended set is its owned rows plus every column of an
 * owned row, in ascending global index.  Outputs (owned by the handle, see hec_ras_get):
 * ext_ptr[nsub+1] (extended rows of s are ext_ptr[s] .. ext_ptr[s+1]-1), ext2glob[n_ext] (global
 * row of each extended row), owned[n_ext] (1 when the extended row is owned by its subdomain), and
 * A_ext = diag(A_1, ..., A_s), A_s = A restricted to ext(s) x ext(s), as one block-diagonal CSR
 * matrix in the extended numbering.  Factor A_ext with ilu_factor, then pass ext2glob and owned
 * to ilu_create: ilu_apply then computes z = sum_s R0_s^T U_s^-1 L_s^-1 R_s r.  Requires
 * nsub * n < 2^31.  Synchronizes `stream`. */
hec_status ras_setup(int n, const int* rowptr, const int* col, const double* val, const int* part,
                     int nsub, hec_ras** out, void* stream);
/* The same with the overlap chosen: 1 as ras_setup; 0 keeps each subdomain to its owned rows,
 * which makes ilu_apply block ILU(0) (block Jacobi with ILU(0) blocks, the paper's BILU).  Any
 * other overlap returns HEC_ERR_INVALID_ARG. */
hec_status ras_setup_overlap(int n, const int* rowptr, const int* col, const double* val,
                             const int* part, int nsub, int overlap, hec_ras** out, void* stream);
hec_status hec_ras_get(const hec_ras* R, int* n_ext, const int** ext_ptr, const int** ext2glob,
                       const unsigned char** owned, const hec_csr** A_ext);
hec_status hec_ras_destroy(hec_ras* R);

/* ---------------------------------------------------------------------------------------- */
/* Allocation-free sweep (the paper has no counterpart: this is a deployment convenience)      */
/* ---------------------------------------------------------------------------------------- */

/* The same triangular sweep as sptrsv_lower (tri->uplo == 0) or sptrsv_upper (tri->uplo == 1),
 * for callers that must not allocate device memory when they solve: their device memory is
 * owned and accounted for by another allocator, or every byte is reserved up front and later
 * allocation is forbidden, or they cannot afford a cudaMalloc (which may synchronize the
 * device) inside a latency-critical loop.  This call allocates nothing: the scratch it needs
 * (chunk table, level-ordered solution, status word) lives in one static device buffer of
 * sptrsv_noalloc_capacity() bytes (32 MiB), which a device holds from the first call on it until
 * the process exits.  The caller still passes tri and lv (built once with sptrsv_analyze and
 * hec_from_csr) and the device arrays b and x, with the layout of sptrsv_lower.  The lane
 * layout is that of a plan with default settings (for one right-hand side the lanes-per-row rule
 * of hec_tune.lanes_per_row = 0), so the results equal those of sptrsv_lower / sptrsv_upper on a
 * default plan bit for bit.
 *   - Size limit: the scratch of a problem is, in bytes, with ws = 8 for FP64 factors and 4 for
 *     FP32 / BF16, kp = nrhs rounded up to a power of two, and rpw = 32 / (lanes per row) rows per
 *     chunk (32 for one right-hand side with one lane per row):
 *       256 + a(4 (nlev + 1)) + a(8 (nlev + ceil(n / rpw))) + a(ws n kp) + a(ws n),
 *     where a() rounds up to a multiple of 256 (status word, chunk prefix, chunk table,
 *     level-ordered solution, reciprocal diagonal).  A problem beyond the buffer is rejected with
 *     HEC_ERR_INVALID_ARG and a message giving the bytes needed; use sptrsv_lower / sptrsv_upper
 *     for those.
 *   - The buffer belongs to the library's device code.  With lazy module loading (the CUDA
 *     default) the device reserves it at the first call on that device (any size, n = 0
 *     included), not when the library is loaded: a caller that must see no change in free device
 *     memory after initialization makes one warm-up call then.  Later calls change nothing.
 *   - Every call looks up the buffer's device address (cudaGetSymbolAddress, which allocates
 *     nothing) with the calling device current; make the first call on a device before any
 *     stream capture.
 *   - All calls share the one buffer and it keeps the last call's contents; every call resets
 *     the parts that must start fresh.  Calls whose work overlaps on the GPU (different
 *     streams, or different host threads on one device) race on the buffer: serialize them.
 *   - status_out (host, may be NULL): when given, the call synchronizes `stream` and stores the
 *     device-side status (0, or HEC_ERR_TIMEOUT when a dependency wait ran out), also returned.
 *     When NULL the call is asynchronous and device-side failures are not reported. */
hec_status sptrsv_solve_noalloc(const hec_matrix* tri, const hec_levels* lv, int nrhs,
                                const double* b, int ldb, double* x, int ldx, int* status_out,
                                void* stream);
/* Bytes of the static buffer used by sptrsv_solve_noalloc. */
size_t sptrsv_noalloc_capacity(void);

#ifdef __cplusplus
}
#endif
#endif /* HEC_H */
