// Level-ordered triangular sweeps on HEC (Alg. 2; upper factor by the reversal of Sec. 2.2)
// and the ILU / RAS preconditioner apply built on them (Eq. 1, Eq. 4).
//
// GB300 design.  The paper launches one kernel per level with one thread per row.  On GB300 a
// kernel boundary (or a grid-wide barrier) costs about a microsecond, which for the 382 levels
// of a 128^3 ILU(0) factor is far more than the time to stream the factor from HBM.  Here one
// cooperative persistent launch solves every level: rows are processed in level order (the
// order of L'), chunk c of rows going to warp c mod W, and each row waits point to point only
// for the rows it actually depends on by polling their solution words (see sync.cuh).  Every
// dependency of row r lies in an earlier chunk, so with all warps resident the earliest
// unfinished chunk can always proceed.  The HEC slab is read column-major, so the consecutive
// rows of a warp read consecutive addresses; the gather of b (b'(m(i)) = b(i)) and the scatter
// of x (x(i) = x'(m(i))) of Alg. 2 are fused into the row's first load and last store.
//
// Multiple right-hand sides: lane = (row of the warp's chunk, right-hand side), with the
// right-hand sides of a row interleaved, so one slab entry serves up to 16 solves.
#include <algorithm>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include <atomic>

#include "internal.cuh"
#include "sync.cuh"

namespace hec {
namespace {

struct SweepParams {
    int n, ld, w, K;
    const int* __restrict__ ell_col;
    const void* __restrict__ ell_val;
    const int* __restrict__ tptr;
    const int* __restrict__ tcol;
    const void* __restrict__ tval;
    const double* __restrict__ b;
    int ldb;
    const int* __restrict__ gather;
    double* __restrict__ x;
    int ldx;
    const int* __restrict__ scatter;
    void* xp;
    int* status;
    long long budget;
    int skip_row;
    int backoff_ns;
    const int2* __restrict__ chunks;  // (first row, rows) of each level-aligned chunk
    int nchunks;
    const void* __restrict__ dinv;     // reciprocal diagonal in the work type (NULL: divide)
    int b32, x32;                      // b / x hold FP32 values (the ILU apply's intermediate)
};

// The right-hand side read and the solution written by a sweep: FP64 at the boundary, FP32 for
// the intermediate y of an ILU apply with FP32 / BF16 factor values (it only feeds the upper
// sweep, which computes in FP32, so keeping it in FP32 changes no result).
template <typename AT> __device__ __forceinline__ AT ld_rhs(const double* b, int b32, long i) {
    return b32 ? (AT)__ldg((const float*)b + i) : (AT)__ldg(b + i);
}
template <typename AT> __device__ __forceinline__ void st_sol(double* x, int x32, long i, AT v) {
    if (x32) ((float*)x)[i] = (float)v;
    else x[i] = (double)v;
}

template <typename XT> struct Acc { typedef float T; };
template <> struct Acc<double> { typedef double T; };

template <typename VT, typename AT> __device__ __forceinline__ AT ldv(const VT* p) { return (AT)__ldg(p); }
template <> __device__ __forceinline__ float ldv<__nv_bfloat16, float>(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
}

// a stored value widened to the work type (no load)
template <typename VT, typename AT> __device__ __forceinline__ AT widen_v(VT v) { return (AT)v; }
template <> __device__ __forceinline__ float widen_v<__nv_bfloat16, float>(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double wait_x(const double* p, int* st, long long b) { return wait_f64(p, st, b); }
__device__ __forceinline__ float wait_x(const float* p, int* st, long long b) { return wait_f32(p, st, b); }
__device__ __forceinline__ void publish_x(double* p, double v) { publish_f64(p, v); }
__device__ __forceinline__ void publish_x(float* p, float v) { publish_f32(p, v); }

// Raw word access to the internal solution (the sentinel test needs the bits).
template <typename XT> struct Word;
template <> struct Word<double> {
    typedef unsigned long long T;
    static constexpr T kSent = kSent64;
    __device__ static T load(const double* p) { return ld_relaxed_u64(p); }
    __device__ static double val(T w) { return __longlong_as_double((long long)w); }
};
template <> struct Word<float> {
    typedef unsigned int T;
    static constexpr T kSent = kSent32;
    __device__ static T load(const float* p) { return ld_relaxed_u32(p); }
    __device__ static float val(T w) { return __uint_as_float(w); }
};

constexpr unsigned kFull = 0xffffffffu;

// The warp waits, converged, until every lane's pending dependency words have been published.
// pending: bit k set = slot k of this lane still outstanding.  Polls are issued for all
// outstanding slots at once.  Returns false (and records DEV_TIMEOUT) when the budget runs out.
template <typename XT, int NS>
__device__ __forceinline__ void warp_wait(const XT* const (&addr)[NS], typename Word<XT>::T (&raw)[NS],
                                          unsigned pending, int* status, long long budget, int backoff_ns) {
    typedef Word<XT> W;
    if (!__any_sync(kFull, pending)) return;
    const long long t0 = clock64();
    // the status word as read at the previous check: its load is issued there and only used
    // here, so a check does not stall the poll loop for an L2 round trip
    unsigned failed = 0u;
    for (unsigned it = 1;; ++it) {
        if (backoff_ns) __nanosleep(backoff_ns);
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (pending & (1u << k)) {
                raw[k] = W::load(addr[k]);
                if (raw[k] != W::kSent) pending &= ~(1u << k);
            }
        }
        if (!__any_sync(kFull, pending)) return;
        if ((it & 31u) == 0u) {
            const bool give_up = (clock64() - t0 > budget) || failed != 0u;
            if (__any_sync(kFull, give_up)) {
                record(status, HEC_ERR_TIMEOUT);
#pragma unroll
                for (int k = 0; k < NS; ++k)
                    if (pending & (1u << k)) raw[k] = 0;
                return;
            }
            failed = ld_relaxed_u32(status);
        }
    }
}

constexpr int kTailBatch = 4;

// Up to NS dependencies of one lane: their solution addresses, the coefficients, and the words
// read so far.  Entries are accumulated in slot order, which is the row's column order.
template <typename XT, typename AT, int NS>
struct DepBatch {
    typedef Word<XT> W;
    const XT* addr[NS];
    typename W::T raw[NS];
    AT v[NS];
    unsigned valid, pend;
    __device__ __forceinline__ void clear(const XT* base) {
        valid = pend = 0;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            addr[k] = base;
            raw[k] = 0;
            v[k] = AT(0);
        }
    }
    __device__ __forceinline__ void set(int k, const XT* a, AT coef) {
        addr[k] = a;
        v[k] = coef;
        valid |= 1u << k;
        pend |= 1u << k;
    }
    template <typename VT>
    __device__ __forceinline__ void load_tail(const int* __restrict__ tcol, const VT* __restrict__ tv, int t0, int tb,
                                              int tl, const XT* xp, int K, int q) {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (tb + k < tl) {
                const int cc = __ldg(tcol + t0 + tb + k);
                set(k, xp + (long)cc * K + q, ldv<VT, AT>(tv + t0 + tb + k));
            }
        }
    }
    __device__ __forceinline__ void poll() {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (pend & (1u << k)) {
                raw[k] = W::load(addr[k]);
                if (raw[k] != W::kSent) pend &= ~(1u << k);
            }
        }
    }
    __device__ __forceinline__ void wait(int* status, long long budget, int backoff_ns) {
        warp_wait<XT, NS>(addr, raw, pend, status, budget, backoff_ns);
    }
    // FP64 work: slots at or beyond `w` (the same for every lane) are skipped by a uniform branch,
    // since GB300's FP64 unit spends 16 SM-cycles on a warp's FP64 instruction even with every lane
    // predicated off (FP32 work keeps the predicated form, which costs it nothing)
    __device__ __forceinline__ AT accumulate(AT acc, int w = NS) const {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (sizeof(AT) == 8 && k >= w) break;
            if (valid & (1u << k)) acc = fma(-v[k], (AT)W::val(raw[k]), acc);
        }
        return acc;
    }
};

template <typename VT, typename XT, int KP, int WMAX>
__global__ void __launch_bounds__(256) k_sweep(SweepParams p) {
    typedef typename Acc<XT>::T AT;
    typedef Word<XT> W;
    constexpr int RPW = 32 / KP;  // rows per warp step
    const int lane = threadIdx.x & 31;
    const int rsub = lane / KP, q = lane % KP;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int nchunks = p.nchunks;
    const VT* __restrict__ ev = (const VT*)p.ell_val;
    const VT* __restrict__ tv = (const VT*)p.tval;
    XT* xp = (XT*)p.xp;
    const int K = p.K;
    // A chunk is up to RPW consecutive rows of ONE level, so no row of a chunk depends on another
    // row of the same chunk and the lockstep waits below cannot wait on the warp itself.  The loop
    // trip counts are warp-uniform, so the warp stays converged throughout.
    for (int c = gw; c < nchunks; c += nw) {
        const int2 ch = __ldg(p.chunks + c);
        const int r = ch.x + rsub;
        const bool act = rsub < ch.y && q < K;
        // Everything that does not depend on other rows is loaded before the first wait, so that
        // after the last dependency arrives only arithmetic and the two stores remain.
        AT acc = AT(0), diag = AT(1);
        int t0 = 0, tl = 0, sr = -1;
        if (act) {
            const int gr = p.gather ? __ldg(p.gather + r) : r;
            acc = ld_rhs<AT>(p.b, p.b32, (long)gr * p.ldb + q);
            t0 = __ldg(p.tptr + r);
            const int t1 = __ldg(p.tptr + r + 1) - 1;
            tl = t1 - t0;
            // the diagonal is the last tail entry; with a precomputed reciprocal the division
            // leaves the critical path (one multiply after the last dependency arrives)
            diag = p.dinv ? (AT)__ldg((const XT*)p.dinv + r) : ldv<VT, AT>(tv + t1);
            sr = p.scatter ? __ldg(p.scatter + r) : r;
        }
        DepBatch<XT, AT, WMAX> slab;
        slab.clear(xp);
#pragma unroll
        for (int k = 0; k < WMAX; ++k) {
            if (act && k < p.w) {
                const long s = (long)k * p.ld + r;
                const int cc = __ldg(p.ell_col + s);
                if (cc >= 0) slab.set(k, xp + (long)cc * K + q, ldv<VT, AT>(ev + s));
            }
        }
        const int tmax = __reduce_max_sync(kFull, tl);
        DepBatch<XT, AT, kTailBatch> tail;
        tail.clear(xp);
        if (tmax > 0) tail.load_tail(p.tcol, tv, t0, 0, tl, xp, K, q);
        slab.poll();
        slab.wait(p.status, p.budget, p.backoff_ns);
        acc = slab.accumulate(acc, p.w);
        // wider slabs: the remaining slots kTailBatch at a time (same order)
        for (int kb = WMAX; kb < p.w; kb += kTailBatch) {
            DepBatch<XT, AT, kTailBatch> more;
            more.clear(xp);
#pragma unroll
            for (int j = 0; j < kTailBatch; ++j) {
                const int k = kb + j;
                if (act && k < p.w) {
                    const long s = (long)k * p.ld + r;
                    const int cc = __ldg(p.ell_col + s);
                    if (cc >= 0) more.set(j, xp + (long)cc * K + q, ldv<VT, AT>(ev + s));
                }
            }
            more.poll();
            more.wait(p.status, p.budget, p.backoff_ns);
            acc = more.accumulate(acc);
        }
        // tail overflow entries in ascending new column, kTailBatch at a time (warp-uniform count)
        for (int tb = 0; tb < tmax; tb += kTailBatch) {
            if (tb > 0) {
                tail.clear(xp);
                tail.load_tail(p.tcol, tv, t0, tb, tl, xp, K, q);
            }
            tail.poll();
            tail.wait(p.status, p.budget, p.backoff_ns);
            acc = tail.accumulate(acc);
        }
        if (act) {
            const AT xr = p.dinv ? acc * diag : acc / diag;
            if (r != p.skip_row) publish_x(xp + (long)r * K + q, (XT)xr);
            if (sr >= 0) st_sol(p.x, p.x32, (long)sr * p.ldx + q, xr);
        }
    }
}

// ---- several lanes per row (one right-hand side, long rows) --------------------------------
// LPR lanes share a row: lane `sub` of the group takes slab slots sub, sub + LPR, ... and tail
// entries sub, sub + LPR, ..., so every dependency of the row is polled in the same warp-wide
// wait (a row with w slab slots and t tail entries needs one wait for w <= LPR*SPL and
// t <= LPR*TB, where the one-lane kernel would wait once per slot beyond its register batch);
// wider slabs and longer tails take further rounds.
// The partial sums are combined by an xor butterfly, which gives every lane of the group the
// same bits; the fixed pairing makes the result deterministic (it differs from the one-lane
// kernel only in summation order).
template <typename VT, typename XT, int LPR, int SPL, int TB>
__global__ void __launch_bounds__(256) k_sweep_lpr(SweepParams p) {
    typedef typename Acc<XT>::T AT;
    constexpr int NS = SPL + TB;
    const int lane = threadIdx.x & 31;
    const int rsub = lane / LPR, sub = lane % LPR;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const VT* __restrict__ ev = (const VT*)p.ell_val;
    const VT* __restrict__ tv = (const VT*)p.tval;
    XT* xp = (XT*)p.xp;
    for (int c = gw; c < p.nchunks; c += nw) {
        const int2 ch = __ldg(p.chunks + c);
        const int r = ch.x + rsub;
        const bool act = rsub < ch.y;
        AT acc = AT(0), diag = AT(1);
        int t0 = 0, tl = 0, sr = -1;
        if (act) {
            t0 = __ldg(p.tptr + r);
            const int t1 = __ldg(p.tptr + r + 1) - 1;
            tl = t1 - t0;
            if (sub == 0) {
                const int gr = p.gather ? __ldg(p.gather + r) : r;
                acc = ld_rhs<AT>(p.b, p.b32, (long)gr * p.ldb);
                diag = p.dinv ? (AT)__ldg((const XT*)p.dinv + r) : ldv<VT, AT>(tv + t1);
                sr = p.scatter ? __ldg(p.scatter + r) : r;
            }
        }
        // slab slots of this lane, then its first tail entries, all polled in one wait
        DepBatch<XT, AT, NS> dep;
        dep.clear(xp);
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
            const int k = sub + j * LPR;
            if (act && k < p.w) {
                const long s = (long)k * p.ld + r;
                const int cc = __ldg(p.ell_col + s);
                if (cc >= 0) dep.set(j, xp + cc, ldv<VT, AT>(ev + s));
            }
        }
#pragma unroll
        for (int j = 0; j < TB; ++j) {
            const int t = sub + j * LPR;
            if (act && t < tl) dep.set(SPL + j, xp + __ldg(p.tcol + t0 + t), ldv<VT, AT>(tv + t0 + t));
        }
        dep.poll();
        dep.wait(p.status, p.budget, p.backoff_ns);
        acc = dep.accumulate(acc);
        // wider slabs: further rounds of LPR * SPL slots (p.w is the same for every lane)
        for (int kb = LPR * SPL; kb < p.w; kb += LPR * SPL) {
            DepBatch<XT, AT, SPL> more;
            more.clear(xp);
#pragma unroll
            for (int j = 0; j < SPL; ++j) {
                const int k = kb + sub + j * LPR;
                if (act && k < p.w) {
                    const long s = (long)k * p.ld + r;
                    const int cc = __ldg(p.ell_col + s);
                    if (cc >= 0) more.set(j, xp + cc, ldv<VT, AT>(ev + s));
                }
            }
            more.poll();
            more.wait(p.status, p.budget, p.backoff_ns);
            acc = more.accumulate(acc);
        }
        // longer tails: further rounds of LPR * TB entries (warp-uniform trip count)
        const int tmax = __reduce_max_sync(kFull, tl);
        for (int tb = LPR * TB; tb < tmax; tb += LPR * TB) {
            DepBatch<XT, AT, TB> more;
            more.clear(xp);
#pragma unroll
            for (int j = 0; j < TB; ++j) {
                const int t = tb + sub + j * LPR;
                if (act && t < tl) more.set(j, xp + __ldg(p.tcol + t0 + t), ldv<VT, AT>(tv + t0 + t));
            }
            more.poll();
            more.wait(p.status, p.budget, p.backoff_ns);
            acc = more.accumulate(acc);
        }
#pragma unroll
        for (int off = LPR / 2; off >= 1; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
        if (act && sub == 0) {
            const AT xr = p.dinv ? acc * diag : acc / diag;
            if (r != p.skip_row) publish_x(xp + r, (XT)xr);
            if (sr >= 0) st_sol(p.x, p.x32, (long)sr * p.ldx, xr);
        }
    }
}

// ---- several right-hand sides per lane ------------------------------------------------------
// For nrhs > 1 a lane carries G consecutive right-hand sides of one row (G = 4 for FP32 work,
// 2 for FP64) and moves them with one 16-byte (or 8-byte) relaxed vector access; LPR = KP / G
// lanes serve a row, so a warp covers 32 / LPR rows of a level.  The level-ordered solution
// is stored with a padded row stride of KP values; padded right-hand sides carry zeros.  Every
// element is a single-copy-atomic word, so a consumer checks each one against the sentinel.
template <typename XT, int G> struct VecIO;
template <> struct VecIO<float, 2> {
    __device__ static void load(const float* p, unsigned (&w)[2]) {
        asm volatile("ld.relaxed.gpu.global.v2.b32 {%0, %1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "l"(p));
    }
    __device__ static void store(float* p, const unsigned (&w)[2]) {
        asm volatile("st.relaxed.gpu.global.v2.b32 [%0], {%1, %2};" ::"l"(p), "r"(w[0]), "r"(w[1]) : "memory");
    }
};
template <> struct VecIO<float, 4> {
    __device__ static void load(const float* p, unsigned (&w)[4]) {
        asm volatile("ld.relaxed.gpu.global.v4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p));
    }
    __device__ static void store(float* p, const unsigned (&w)[4]) {
        asm volatile("st.relaxed.gpu.global.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(w[0]), "r"(w[1]),
                     "r"(w[2]), "r"(w[3]) : "memory");
    }
};
template <> struct VecIO<double, 2> {
    __device__ static void load(const double* p, unsigned long long (&w)[2]) {
        asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(w[0]), "=l"(w[1]) : "l"(p));
    }
    __device__ static void store(double* p, const unsigned long long (&w)[2]) {
        asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(w[0]), "l"(w[1]) : "memory");
    }
};

template <typename XT, typename AT, int NS, int G>
struct DepBatchV {
    typedef Word<XT> W;
    typedef typename W::T WT;
    const XT* addr[NS];
    WT raw[NS][G];
    AT v[NS];
    unsigned valid, pend;
    __device__ __forceinline__ void clear(const XT* base) {
        valid = pend = 0;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            addr[k] = base;
            v[k] = AT(0);
#pragma unroll
            for (int g = 0; g < G; ++g) raw[k][g] = 0;
        }
    }
    __device__ __forceinline__ void set(int k, const XT* a, AT coef) {
        addr[k] = a;
        v[k] = coef;
        valid |= 1u << k;
        pend |= 1u << k;
    }
    __device__ __forceinline__ void poll() {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (pend & (1u << k)) {
                VecIO<XT, G>::load(addr[k], raw[k]);
                bool ready = true;
#pragma unroll
                for (int g = 0; g < G; ++g) ready = ready && raw[k][g] != W::kSent;
                if (ready) pend &= ~(1u << k);
            }
        }
    }
    __device__ __forceinline__ void wait(int* status, long long budget, int backoff_ns) {
        if (!__any_sync(kFull, pend)) return;
        const long long t0 = clock64();
        unsigned failed = 0u;  // the status word as read at the previous check
        for (unsigned it = 1;; ++it) {
            if (backoff_ns) __nanosleep(backoff_ns);
            poll();
            if (!__any_sync(kFull, pend)) return;
            if ((it & 31u) == 0u) {
                const bool give_up = (clock64() - t0 > budget) || failed != 0u;
                failed = ld_relaxed_u32(status);
                if (__any_sync(kFull, give_up)) {
                    record(status, HEC_ERR_TIMEOUT);
#pragma unroll
                    for (int k = 0; k < NS; ++k)
#pragma unroll
                        for (int g = 0; g < G; ++g)
                            if (pend & (1u << k)) raw[k][g] = 0;
                    return;
                }
            }
        }
    }
    __device__ __forceinline__ void accumulate(AT (&acc)[G]) const {
#pragma unroll
        for (int k = 0; k < NS; ++k)
            if (valid & (1u << k))
#pragma unroll
                for (int g = 0; g < G; ++g) acc[g] = fma(-v[k], (AT)W::val(raw[k][g]), acc[g]);
    }
};

// One lane's share of a row of a chunk of the multi-right-hand-side sweep, everything but the
// dependencies' values: its G right-hand sides (gathered through p.gather), the reciprocal
// diagonal (the diagonal itself when the plan has none), the tail range, the scatter row and the
// first WMAX slab slots.  Loaded for the warp's
// next chunk while it works on the current one, so a chunk's HBM loads overlap the wait of the
// chunk before it.
template <typename VT, typename XT, typename AT, int G, int WMAX>
struct VecRow {
    AT b[G];
    AT d;
    int t0, tl, sr;
    int cc[WMAX];
    VT v[WMAX];
    __device__ __forceinline__ void load(const SweepParams& p, int2 ch, int rsub, int q0) {
#pragma unroll
        for (int g = 0; g < G; ++g) b[g] = AT(0);
        d = AT(1);
        t0 = tl = 0;
        sr = -1;
#pragma unroll
        for (int k = 0; k < WMAX; ++k) {
            cc[k] = -1;
            v[k] = VT(0.0f);
        }
        if (rsub < ch.y) {
            const int r = ch.x + rsub;
            const int gr = p.gather ? __ldg(p.gather + r) : r;
#pragma unroll
            for (int g = 0; g < G; ++g)
                if (q0 + g < p.K) b[g] = ld_rhs<AT>(p.b, p.b32, (long)gr * p.ldb + q0 + g);
            t0 = __ldg(p.tptr + r);
            const int t1 = __ldg(p.tptr + r + 1) - 1;
            tl = t1 - t0;
            d = p.dinv ? (AT)__ldg((const XT*)p.dinv + r) : ldv<VT, AT>((const VT*)p.tval + t1);
            sr = p.scatter ? __ldg(p.scatter + r) : r;
#pragma unroll
            for (int k = 0; k < WMAX; ++k) {
                if (k < p.w) {
                    const long s = (long)k * p.ld + r;
                    cc[k] = __ldg(p.ell_col + s);
                    v[k] = __ldg((const VT*)p.ell_val + s);
                }
            }
        }
    }
};

template <typename VT, typename XT, int LPR, int G, int WMAX>
__global__ void __launch_bounds__(256) k_sweep_vec(SweepParams p) {
    typedef typename Acc<XT>::T AT;
    typedef Word<XT> W;
    constexpr int KS = LPR * G;   // padded row stride of the level-ordered solution
    const int lane = threadIdx.x & 31;
    const int rsub = lane / LPR, q0 = (lane % LPR) * G;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const VT* __restrict__ ev = (const VT*)p.ell_val;
    const VT* __restrict__ tv = (const VT*)p.tval;
    XT* xp = (XT*)p.xp;
    const int K = p.K;
    // chunk entries run two chunks ahead of the warp, row data one chunk ahead
    int2 ch_a = gw < p.nchunks ? __ldg(p.chunks + gw) : make_int2(0, 0);
    int2 ch_b = gw + nw < p.nchunks ? __ldg(p.chunks + gw + nw) : make_int2(0, 0);
    VecRow<VT, XT, AT, G, WMAX> nxt, row;
    nxt.load(p, ch_a, rsub, q0);
    for (int c = gw; c < p.nchunks; c += nw) {
        const int2 ch = ch_a;
        ch_a = ch_b;
        if (c + 2 * nw < p.nchunks) ch_b = __ldg(p.chunks + c + 2 * nw);
        row = nxt;
        nxt.load(p, c + nw < p.nchunks ? ch_a : make_int2(0, 0), rsub, q0);
        const int r = ch.x + rsub;
        const bool act = rsub < ch.y;
        AT acc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g] = row.b[g];
        const AT diag = row.d;
        const int t0 = row.t0, tl = row.tl, sr = row.sr;
        DepBatchV<XT, AT, WMAX, G> slab;
        slab.clear(xp);
#pragma unroll
        for (int k = 0; k < WMAX; ++k)
            if (act && row.cc[k] >= 0) slab.set(k, xp + (long)row.cc[k] * KS + q0, widen_v<VT, AT>(row.v[k]));
        slab.poll();
        slab.wait(p.status, p.budget, p.backoff_ns);
        slab.accumulate(acc);
        // wider slabs: the remaining slots kTailBatch at a time, in slot order
        for (int kb = WMAX; kb < p.w; kb += kTailBatch) {
            DepBatchV<XT, AT, kTailBatch, G> more;
            more.clear(xp);
#pragma unroll
            for (int j = 0; j < kTailBatch; ++j) {
                const int k = kb + j;
                if (act && k < p.w) {
                    const long s = (long)k * p.ld + r;
                    const int cc = __ldg(p.ell_col + s);
                    if (cc >= 0) more.set(j, xp + (long)cc * KS + q0, ldv<VT, AT>(ev + s));
                }
            }
            more.poll();
            more.wait(p.status, p.budget, p.backoff_ns);
            more.accumulate(acc);
        }
        const int tmax = __reduce_max_sync(kFull, tl);
        for (int tb = 0; tb < tmax; tb += kTailBatch) {
            DepBatchV<XT, AT, kTailBatch, G> tail;
            tail.clear(xp);
#pragma unroll
            for (int k = 0; k < kTailBatch; ++k) {
                if (tb + k < tl) {
                    const int cc = __ldg(p.tcol + t0 + tb + k);
                    tail.set(k, xp + (long)cc * KS + q0, ldv<VT, AT>(tv + t0 + tb + k));
                }
            }
            tail.poll();
            tail.wait(p.status, p.budget, p.backoff_ns);
            tail.accumulate(acc);
        }
        if (act) {
            typename W::T outw[G];
            AT xr[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                xr[g] = p.dinv ? acc[g] * diag : acc[g] / diag;
                const XT xv = q0 + g < K ? (XT)xr[g] : XT(0);
                typename W::T wv;
                if (sizeof(XT) == 8) wv = (typename W::T)__double_as_longlong((double)xv);
                else wv = (typename W::T)__float_as_uint((float)xv);
                if (wv == W::kSent) wv = sizeof(XT) == 8 ? (typename W::T)0x7FF8000000000000ull : (typename W::T)0x7FC00000u;
                outw[g] = wv;
            }
            // publish first (the next level waits on it), then the scatter to the caller's x
            if (r != p.skip_row) VecIO<XT, G>::store(xp + (long)r * KS + q0, outw);
            if (sr >= 0)
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (q0 + g < K) st_sol(p.x, p.x32, (long)sr * p.ldx + q0 + g, xr[g]);
        }
    }
}

// ---- partitioned sweep ---------------------------------------------------------------------
// The rows are split into parts, one resident CTA per part.  Inside a part the rows keep the
// global level order and are cut into level-aligned chunks of at most 32 rows; chunk c of the
// part goes to warp c mod (warps per CTA), so, as in the plain sweep, each row waits point to
// point for exactly its dependencies and warps run ahead to later levels.  The part's own
// solution values live in shared memory (sentinel-filled at start, the value is its own flag),
// so a dependency inside the part is an SM-local poll of a few tens of cycles; only a dependency
// on another part polls the global solution through L2.  With parts that are compact regions of
// the grid, a long dependency chain crosses a part boundary only a few times.  Every wait is on
// a row of lower global level and every warp walks its rows in increasing level, so the lowest
// unfinished row can always proceed (all CTAs are resident: cooperative launch).
struct PartParams {
    int n, ld, w;
    const int* __restrict__ ell_col;
    const void* __restrict__ ell_val;
    const int* __restrict__ tptr;
    const int* __restrict__ tcol;
    const void* __restrict__ tval;
    const void* __restrict__ dinv;
    const int* __restrict__ rowg;
    const int* __restrict__ part_row;
    const int* __restrict__ part_chunk;
    const int2* __restrict__ chunks;
    void* bp;  // b gathered into plan order in the work type (by each part, in the sweep's prologue)
    const double* __restrict__ b;
    int ldb;
    const int* __restrict__ gather;
    double* __restrict__ x;
    int ldx;
    const int* __restrict__ scatter;
    void* xp;       // plan-order solution words polled by this sweep (set to the sentinel before it)
    void* xp_next;  // the other buffer: set to the sentinel here for the next sweep
    const int* __restrict__ bidx;  // plan row -> row of b (NULL: gather[rowg] or rowg)
    int bplan;                     // b already in plan order
    int* status;
    long long budget;
    int skip_row;
    int b32, x32;  // b / x hold FP32 values (the ILU apply's intermediate)
};

// Volatile shared-memory word loads by shared-window address, so a local poll is always a
// shared-memory load whatever the compiler can infer about the pointer.
__device__ __forceinline__ unsigned int ld_shared_u32(unsigned int a) {
    unsigned int v;
    asm volatile("ld.volatile.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ unsigned long long ld_shared_u64(unsigned int a) {
    unsigned long long v;
    asm volatile("ld.volatile.shared.b64 %0, [%1];" : "=l"(v) : "r"(a));
    return v;
}

// dependencies of one lane, each either in this part's shared memory (shared-window byte
// address) or in the global solution (row index)
template <typename XT, typename AT, int NS>
struct DepBatchP {
    typedef Word<XT> W;
    typedef typename W::T WT;
    unsigned int where[NS];
    WT raw[NS];
    AT v[NS];
    unsigned valid, pend, local;
    __device__ __forceinline__ void clear() {
        valid = pend = local = 0;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            where[k] = 0;
            raw[k] = 0;
            v[k] = AT(0);
        }
    }
    // sbase: shared-window address of the part's solution, whose rows are lo .. hi-1
    __device__ __forceinline__ void set(int k, unsigned int sbase, int cc, int lo, int hi, AT coef) {
        v[k] = coef;
        valid |= 1u << k;
        pend |= 1u << k;
        if (cc >= lo && cc < hi) {
            where[k] = sbase + (unsigned int)(cc - lo) * (unsigned int)sizeof(WT);
            local |= 1u << k;
        } else {
            where[k] = (unsigned int)cc;
        }
    }
    __device__ __forceinline__ void poll(const XT* xp) {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (pend & (1u << k)) {
                if (local & (1u << k))
                    raw[k] = sizeof(WT) == 8 ? (WT)ld_shared_u64(where[k]) : (WT)ld_shared_u32(where[k]);
                else
                    raw[k] = W::load(xp + where[k]);
                if (raw[k] != W::kSent) pend &= ~(1u << k);
            }
        }
    }
    __device__ __forceinline__ void wait(const XT* xp, int* status, long long budget) {
        if (!__any_sync(kFull, pend)) return;
        const long long t0 = clock64();
        unsigned failed = 0u;  // the status word as read at the previous check
        // First spin on one word a lane: its latest outstanding local dependency (the largest
        // row index, so the highest level; rows are in level order).  One shared load per
        // iteration instead of one per slot keeps the polls of the waiting warps from crowding
        // the shared-memory pipe that the producers' stores and the other polls go through.
        // A warp with an outstanding dependency in another part keeps polling every slot, so
        // the L2 round trip of that poll overlaps the local waits.
        unsigned int last = 0u;
        const unsigned lp = pend & local;
#pragma unroll
        for (int k = 0; k < NS; ++k)
            if ((lp & (1u << k)) && where[k] > last) last = where[k];
        if (__any_sync(kFull, lp != 0u) && !__any_sync(kFull, (pend & ~local) != 0u)) {
            for (unsigned it = 1;; ++it) {
                const WT lv = lp == 0u ? (WT)0 : (sizeof(WT) == 8 ? (WT)ld_shared_u64(last) : (WT)ld_shared_u32(last));
                if (__all_sync(kFull, lp == 0u || lv != W::kSent)) {
                    // the spun-on word is published: it is that dependency's value, so only the
                    // lane's other outstanding words need the poll below
#pragma unroll
                    for (int k = 0; k < NS; ++k)
                        if ((lp & (1u << k)) && where[k] == last) {
                            raw[k] = lv;
                            pend &= ~(1u << k);
                        }
                    break;
                }
                if ((it & 63u) == 0u) {
                    const bool give_up = (clock64() - t0 > budget) || failed != 0u;
                    failed = ld_relaxed_u32(status);
                    if (__any_sync(kFull, give_up)) break;  // the loop below records the failure
                }
            }
        }
        for (unsigned it = 1;; ++it) {
            poll(xp);
            if (!__any_sync(kFull, pend)) return;
            if ((it & 63u) == 0u) {
                const bool give_up = (clock64() - t0 > budget) || failed != 0u;
                failed = ld_relaxed_u32(status);
                if (__any_sync(kFull, give_up)) {
                    record(status, HEC_ERR_TIMEOUT);
#pragma unroll
                    for (int k = 0; k < NS; ++k)
                        if (pend & (1u << k)) raw[k] = 0;
                    return;
                }
            }
        }
    }
    // FP64 work: slots at or beyond `w` (the same for every lane) are skipped by a uniform branch,
    // since GB300's FP64 unit spends 16 SM-cycles on a warp's FP64 instruction even with every lane
    // predicated off (FP32 work keeps the predicated form, which costs it nothing)
    __device__ __forceinline__ AT accumulate(AT acc, int w = NS) const {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (sizeof(AT) == 8 && k >= w) break;
            if (valid & (1u << k)) acc = fma(-v[k], (AT)W::val(raw[k]), acc);
        }
        return acc;
    }
};

// One lane's row of a chunk of the partitioned sweep: everything but the dependencies, loaded
// for the warp's next chunk while it waits on the current one.  The loads are all one step from
// the row index (the right-hand side is gathered into plan order in the sweep's prologue) and
// nothing here uses a loaded value: widening, the tail length and the scatter index are derived
// when the chunk is processed, so issuing the prefetch never stalls the warp.  Slab values are
// loaded whether or not the slot is padding (padding is in bounds and zero).

template <typename VT, typename XT, typename AT, int NP>
struct PartRow {
    AT b;            // right-hand side
    XT d;            // reciprocal diagonal
    int g, t0, t1;   // factor row (-1: idle lane), tail range [t0, t1) with the diagonal last
    int cc[NP > 0 ? NP : 1];
    VT v[NP > 0 ? NP : 1];
    __device__ __forceinline__ void load(const PartParams& p, int2 ch, int lane, bool have) {
        b = AT(0);
        d = XT(1);
        g = -1;
        t0 = 0;
        t1 = 1;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            cc[k] = -1;
            v[k] = VT(0.0f);
        }
        if (have && lane < ch.y) {
            const int r = ch.x + lane;
            g = __ldg(p.rowg + r);
            if (p.bplan) {
                b = ld_rhs<AT>(p.b, p.b32, (long)r * p.ldb);
            } else if (sizeof(AT) == 4) {
                b = __ldcg((const AT*)p.bp + r);  // written by this block in the prologue: not the read-only path
            } else {  // FP64: gathered here (the row is loaded when its chunk starts)
                const int gr = p.bidx ? __ldg(p.bidx + r) : p.gather ? __ldg(p.gather + g) : g;
                b = ld_rhs<AT>(p.b, p.b32, (long)gr * p.ldb);
            }
            t0 = __ldg(p.tptr + r);
            t1 = __ldg(p.tptr + r + 1);
            d = __ldg((const XT*)p.dinv + r);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                if (k < p.w) {
                    const long s = (long)k * p.ld + r;
                    cc[k] = __ldg(p.ell_col + s);
                    v[k] = __ldg((const VT*)p.ell_val + s);
                }
            }
        }
    }
};

template <typename VT, typename XT, int WMAX>
__global__ void __launch_bounds__(1024, 1) k_sweep_part(PartParams p) {
    typedef typename Acc<XT>::T AT;
    typedef Word<XT> W;
    typedef typename W::T WT;
    // slab slots carried in the prefetched row: all four of a narrow FP32 slab, fewer where the
    // registers of a 1024-thread block (64 a thread) would otherwise spill
    constexpr int NP = WMAX > 4 ? 0 : sizeof(AT) == 8 ? 2 : WMAX;
    // FP32 work: the next chunk's row is loaded while the current one waits, and the right-hand
    // side is gathered into plan order in the prologue.  FP64 work: a level is long enough (FP64
    // arithmetic on the chain) that loading the row, right-hand side gather included, when the
    // chunk starts costs nothing, while a gathering step before the sweep would.
    constexpr bool PF = sizeof(AT) == 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WT* sxp = (WT*)smem_raw;
    const unsigned int sbase = (unsigned int)__cvta_generic_to_shared(smem_raw);
    const int part = blockIdx.x;
    const int lo = __ldg(p.part_row + part), hi = __ldg(p.part_row + part + 1);
    // Prologue: the part's rows of the shared solution set to the sentinel and, for FP32 work, the
    // part's rows of the right-hand side gathered into plan order (read back only by this block).
    // The global buffer this sweep polls was set to the sentinel by the previous sweep of the plan
    // (see the epilogue), so no grid-wide synchronisation is needed.
    {
        for (int i = threadIdx.x; i < hi - lo; i += blockDim.x) sxp[i] = W::kSent;
        if (PF && !p.bplan) {
            // kPro rows a thread at a time, each dependent load issued for all of them before the
            // next, so a batch costs one memory round trip per step of the index chain
            constexpr int kPro = 8;
            AT* bp = (AT*)p.bp;
            for (int i0 = 0; i0 < hi - lo; i0 += kPro * (int)blockDim.x) {
                int gi[kPro];
                AT bv[kPro];
#pragma unroll
                for (int u = 0; u < kPro; ++u) {
                    const int i = i0 + u * (int)blockDim.x + (int)threadIdx.x;
                    gi[u] = i < hi - lo ? __ldg((p.bidx ? p.bidx : p.rowg) + lo + i) : -1;
                }
                if (p.gather && !p.bidx) {
#pragma unroll
                    for (int u = 0; u < kPro; ++u) gi[u] = gi[u] >= 0 ? __ldg(p.gather + gi[u]) : -1;
                }
#pragma unroll
                for (int u = 0; u < kPro; ++u) bv[u] = gi[u] >= 0 ? ld_rhs<AT>(p.b, p.b32, (long)gi[u] * p.ldb) : AT(0);
#pragma unroll
                for (int u = 0; u < kPro; ++u) {
                    const int i = i0 + u * (int)blockDim.x + (int)threadIdx.x;
                    if (i < hi - lo) bp[lo + i] = bv[u];
                }
            }
        }
        __syncthreads();
    }
    const int c0 = __ldg(p.part_chunk + part), c1 = __ldg(p.part_chunk + part + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const VT* __restrict__ ev = (const VT*)p.ell_val;
    const VT* __restrict__ tv = (const VT*)p.tval;
    XT* xp = (XT*)p.xp;
    // chunk entries run two chunks ahead of the warp, row data one chunk ahead
    int2 ch_a = c0 + warp < c1 ? __ldg(p.chunks + c0 + warp) : make_int2(0, 0);
    int2 ch_b = c0 + warp + nwarps < c1 ? __ldg(p.chunks + c0 + warp + nwarps) : make_int2(0, 0);
    PartRow<VT, XT, AT, NP> nxt, row;
    if (PF) nxt.load(p, ch_a, lane, c0 + warp < c1);
    for (int c = c0 + warp; c < c1; c += nwarps) {
        const int2 ch = ch_a;
        ch_a = ch_b;
        if (c + 2 * nwarps < c1) ch_b = __ldg(p.chunks + c + 2 * nwarps);
        if (PF) {
            row = nxt;
            nxt.load(p, ch_a, lane, c + nwarps < c1);
        } else {
            row.load(p, ch, lane, true);
        }
        const int r = ch.x + lane;
        const bool act = lane < ch.y;
        AT acc = row.b;
        const AT diag = (AT)row.d;
        const int t0 = row.t0, tl = row.t1 - 1 - row.t0;
        const int sr = row.g < 0 ? -1 : p.scatter ? __ldg(p.scatter + row.g) : row.g;
        DepBatchP<XT, AT, WMAX> slab;
        slab.clear();
#pragma unroll
        for (int k = 0; k < WMAX; ++k) {
            if (k < NP) {
                if (row.cc[k] >= 0) slab.set(k, sbase, row.cc[k], lo, hi, widen_v<VT, AT>(row.v[k]));
            } else if (act && k < p.w) {
                const long s = (long)k * p.ld + r;
                const int cc = __ldg(p.ell_col + s);
                if (cc >= 0) slab.set(k, sbase, cc, lo, hi, ldv<VT, AT>(ev + s));
            }
        }
        const int tmax = __reduce_max_sync(kFull, tl);
        slab.poll(xp);
        slab.wait(xp, p.status, p.budget);
        acc = slab.accumulate(acc, p.w);
        for (int kb = WMAX; kb < p.w; kb += kTailBatch) {  // wider slabs, kTailBatch slots at a time
            DepBatchP<XT, AT, kTailBatch> more;
            more.clear();
#pragma unroll
            for (int j = 0; j < kTailBatch; ++j) {
                const int k = kb + j;
                if (act && k < p.w) {
                    const long s = (long)k * p.ld + r;
                    const int cc = __ldg(p.ell_col + s);
                    if (cc >= 0) more.set(j, sbase, cc, lo, hi, ldv<VT, AT>(ev + s));
                }
            }
            more.poll(xp);
            more.wait(xp, p.status, p.budget);
            acc = more.accumulate(acc);
        }
        for (int tb = 0; tb < tmax; tb += kTailBatch) {
            DepBatchP<XT, AT, kTailBatch> tail;
            tail.clear();
#pragma unroll
            for (int k = 0; k < kTailBatch; ++k)
                if (tb + k < tl)
                    tail.set(k, sbase, __ldg(p.tcol + t0 + tb + k), lo, hi, ldv<VT, AT>(tv + t0 + tb + k));
            tail.poll(xp);
            tail.wait(xp, p.status, p.budget);
            acc = tail.accumulate(acc);
        }
        const AT xr = acc * diag;
        const bool pub = act && r != p.skip_row;
        if (pub) {
            WT wv = sizeof(XT) == 8 ? (WT)__double_as_longlong((double)(XT)xr) : (WT)__float_as_uint((float)(XT)xr);
            if (wv == W::kSent) wv = sizeof(XT) == 8 ? (WT)0x7FF8000000000000ull : (WT)0x7FC00000u;
            *(volatile WT*)(sxp + (r - lo)) = wv;  // consumers in this part
        }
        if (pub) publish_x(xp + r, (XT)xr);  // consumers in other parts
        if (act && sr >= 0) st_sol(p.x, p.x32, (long)sr * p.ldx, xr);
    }
    // Epilogue: the part's rows of the other global buffer, which the next sweep of this plan
    // polls, set to the sentinel (nothing reads that buffer during this sweep; done last, it stays
    // off the dependency chain).
    WT* nxp = (WT*)p.xp_next;
    for (int i = threadIdx.x; i < hi - lo; i += blockDim.x) nxp[lo + i] = W::kSent;
}

template <typename XT>
__global__ void k_fill_sentinel(XT* xp, long count) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long st = (long)gridDim.x * blockDim.x;
    for (; i < count; i += st) {
        if (sizeof(XT) == 8) ((unsigned long long*)xp)[i] = kSent64;
        else ((unsigned int*)xp)[i] = kSent32;
    }
}

std::mutex g_occ_mu;
std::unordered_map<const void*, int> g_occ[9];  // per block size (threads / 32)

int occupancy(const void* k, int threads) {
    std::lock_guard<std::mutex> g(g_occ_mu);
    auto& tbl = g_occ[(threads / 32) % 9];
    auto it = tbl.find(k);
    if (it != tbl.end()) return it->second;
    int nb = max_coop_blocks(k, threads, 0);
    tbl[k] = nb;
    return nb;
}

template <typename VT, typename XT, int KP, int WMAX>
hec_status launch_sweep(const sptrsv_plan* pl, SweepParams& sp, cudaStream_t s) {
    const void* k = (const void*)k_sweep<VT, XT, KP, WMAX>;
    const int threads = pl->threads;
    int per_sm = occupancy(k, threads);
    if (per_sm <= 0) return set_error(HEC_ERR_CUDA, "sweep kernel cannot be resident");
    if (pl->blocks > 0) per_sm = std::min(per_sm, pl->blocks);
    constexpr int kp_idx = KP == 1 ? 0 : KP == 2 ? 1 : KP == 4 ? 2 : KP == 8 ? 3 : 4;
    if (!pl->chunks[kp_idx]) return set_error(HEC_ERR_INVALID_ARG, "sweep: nrhs above the plan's max_nrhs");
    sp.chunks = pl->chunks[kp_idx];
    sp.nchunks = pl->nchunks[kp_idx];
    long nchunks = sp.nchunks;
    long want = (nchunks + threads / 32 - 1) / (threads / 32);
    int blocks = (int)std::max(1L, std::min((long)per_sm * num_sms(), want));
    long count = (long)sp.n * sp.K;
    int fb = (int)std::min(4096L, std::max(1L, (count + 255) / 256));
    {
        ProfScope ps_(s, PROF_FILL);
        k_fill_sentinel<XT><<<fb, 256, 0, s>>>((XT*)sp.xp, count);
    }
    HEC_LAUNCHED();
    void* args[] = {&sp};
    void* tok = nullptr;
    profile_begin(s, &tok);
    HEC_CUDA(cudaLaunchCooperativeKernel(k, dim3(blocks), dim3(threads), args, 0, s));
    profile_end(s, tok);
    count_launch();
    return HEC_OK;
}

template <typename VT, typename XT, int LPR, int G, int WMAX>
hec_status launch_sweep_vec(const sptrsv_plan* pl, SweepParams& sp, cudaStream_t s) {
    const void* k = (const void*)k_sweep_vec<VT, XT, LPR, G, WMAX>;
    const int threads = pl->threads;
    int per_sm = occupancy(k, threads);
    if (per_sm <= 0) return set_error(HEC_ERR_CUDA, "sweep kernel cannot be resident");
    if (pl->blocks > 0) per_sm = std::min(per_sm, pl->blocks);
    constexpr int idx = LPR == 1 ? 0 : LPR == 2 ? 1 : LPR == 4 ? 2 : LPR == 8 ? 3 : 4;
    if (!pl->chunks[idx]) return set_error(HEC_ERR_INVALID_ARG, "sweep: nrhs above the plan's max_nrhs");
    sp.chunks = pl->chunks[idx];
    sp.nchunks = pl->nchunks[idx];
    const long want = ((long)sp.nchunks + threads / 32 - 1) / (threads / 32);
    const int blocks = (int)std::max(1L, std::min((long)per_sm * num_sms(), want));
    const long count = (long)sp.n * LPR * G;
    const int fb = (int)std::min(4096L, std::max(1L, (count + 255) / 256));
    {
        ProfScope ps_(s, PROF_FILL);
        k_fill_sentinel<XT><<<fb, 256, 0, s>>>((XT*)sp.xp, count);
    }
    HEC_LAUNCHED();
    void* args[] = {&sp};
    void* tok = nullptr;
    profile_begin(s, &tok);
    HEC_CUDA(cudaLaunchCooperativeKernel(k, dim3(blocks), dim3(threads), args, 0, s));
    profile_end(s, tok);
    count_launch();
    return HEC_OK;
}

template <typename VT, typename XT, int LPR>
hec_status launch_sweep_lpr(const sptrsv_plan* pl, SweepParams& sp, cudaStream_t s) {
    const void* k = (const void*)k_sweep_lpr<VT, XT, LPR, 3, 2>;
    const int threads = pl->threads;
    int per_sm = occupancy(k, threads);
    if (per_sm <= 0) return set_error(HEC_ERR_CUDA, "sweep kernel cannot be resident");
    if (pl->blocks > 0) per_sm = std::min(per_sm, pl->blocks);
    constexpr int idx = LPR == 2 ? 1 : LPR == 4 ? 2 : 3;
    if (!pl->chunks[idx]) return set_error(HEC_ERR_INVALID_ARG, "sweep: no chunk table for the plan's lanes per row");
    sp.chunks = pl->chunks[idx];
    sp.nchunks = pl->nchunks[idx];
    const long want = ((long)sp.nchunks + threads / 32 - 1) / (threads / 32);
    const int blocks = (int)std::max(1L, std::min((long)per_sm * num_sms(), want));
    const long count = sp.n;
    const int fb = (int)std::min(4096L, std::max(1L, (count + 255) / 256));
    {
        ProfScope ps_(s, PROF_FILL);
        k_fill_sentinel<XT><<<fb, 256, 0, s>>>((XT*)sp.xp, count);
    }
    HEC_LAUNCHED();
    void* args[] = {&sp};
    void* tok = nullptr;
    profile_begin(s, &tok);
    HEC_CUDA(cudaLaunchCooperativeKernel(k, dim3(blocks), dim3(threads), args, 0, s));
    profile_end(s, tok);
    count_launch();
    return HEC_OK;
}

// one right-hand side: lane per row; more: G right-hand sides per lane, LPR lanes per row
template <typename VT, typename XT, int WMAX>
hec_status dispatch_k(const sptrsv_plan* pl, SweepParams& sp, cudaStream_t s) {
    constexpr int G = sizeof(XT) == 8 ? 2 : 4;
    if (sp.K <= 1) return launch_sweep<VT, XT, 1, WMAX>(pl, sp, s);
    if (sp.K <= 2) return launch_sweep_vec<VT, XT, 1, 2, WMAX>(pl, sp, s);
    if (sp.K <= 4) return launch_sweep_vec<VT, XT, 4 / G, G, WMAX>(pl, sp, s);
    if (sp.K <= 8) return launch_sweep_vec<VT, XT, 8 / G, G, WMAX>(pl, sp, s);
    return launch_sweep_vec<VT, XT, 16 / G, G, WMAX>(pl, sp, s);
}

// slab slots held in registers: 4 covers the 5- and 7-point ILU(0) factors, 8 the wider ones
template <typename VT, typename XT>
hec_status dispatch_w(const sptrsv_plan* pl, SweepParams& sp, cudaStream_t s) {
    if (sp.K <= 1 && pl->lpr1 > 1) {  // long rows: several lanes per row (one wait per row)
        if (pl->lpr1 == 2) return launch_sweep_lpr<VT, XT, 2>(pl, sp, s);
        if (pl->lpr1 == 4) return launch_sweep_lpr<VT, XT, 4>(pl, sp, s);
        return launch_sweep_lpr<VT, XT, 8>(pl, sp, s);
    }
    if (sp.w <= 4) return dispatch_k<VT, XT, 4>(pl, sp, s);
    return dispatch_k<VT, XT, 8>(pl, sp, s);
}

size_t work_size(hec_dtype d) { return d == HEC_F64 ? 8 : 4; }

// dinv[r] = 1 / diagonal of new row r, in the work type (FP64 for FP64 factors, else FP32)
template <typename VT, typename XT>
__global__ void k_dinv(int n, const int* __restrict__ tptr, const VT* __restrict__ tval, XT* dinv) {
    typedef typename Acc<XT>::T AT;
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) dinv[r] = (XT)(AT(1) / ldv<VT, AT>(tval + tptr[r + 1] - 1));
}

hec_status build_dinv(sptrsv_plan* p) {
    const hec_matrix* T = p->T;
    HEC_CHECK(dmalloc(&p->dinv, work_size(T->vdt) * (size_t)T->n + 16));
    if (T->n == 0) return HEC_OK;
    const int g = (T->n + 255) / 256;
    if (T->vdt == HEC_F64) k_dinv<double, double><<<g, 256>>>(T->n, T->tptr, (const double*)T->tval, (double*)p->dinv);
    else if (T->vdt == HEC_F32) k_dinv<float, float><<<g, 256>>>(T->n, T->tptr, (const float*)T->tval, (float*)p->dinv);
    else k_dinv<__nv_bfloat16, float><<<g, 256>>>(T->n, T->tptr, (const __nv_bfloat16*)T->tval, (float*)p->dinv);
    HEC_LAUNCHED();
    HEC_CUDA(cudaStreamSynchronize(0));
    return HEC_OK;
}

// Level-aligned chunks of at most rpw rows: level l contributes ceil(N_l / rpw) chunks.
__global__ void k_chunk_counts(int nlev, const int* __restrict__ level_ptr, int rpw, int* cnt) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < nlev) cnt[l] = (level_ptr[l + 1] - level_ptr[l] + rpw - 1) / rpw;
}

__global__ void k_chunk_table(int nlev, const int* __restrict__ level_ptr, const int* __restrict__ cptr, int rpw,
                              int nchunks, int2* tbl) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    int lo = 0, hi = nlev - 1;  // last level l with cptr[l] <= c
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (cptr[mid] <= c) lo = mid; else hi = mid - 1;
    }
    int row0 = level_ptr[lo] + (c - cptr[lo]) * rpw;
    tbl[c] = make_int2(row0, min(rpw, level_ptr[lo + 1] - row0));
}

// the chunk tables of the lane layouts in `needed` (bit i: 32 >> i rows per warp step) that the
// plan does not have yet
hec_status build_chunks(sptrsv_plan* p, unsigned needed) {
    const hec_levels* lv = p->lv;
    const int nlev = lv->nlev;
    int* cptr = nullptr;
    HEC_CHECK(dalloc(&cptr, (size_t)nlev + 1));
    hec_status st = HEC_OK;
    cudaStream_t s = 0;
    for (int i = 0; i < 5 && st == HEC_OK; ++i) {
        const int rpw = 32 >> i;
        if (!(needed & (1u << i)) || p->chunks[i]) continue;
        if (nlev > 0) {
            k_chunk_counts<<<(nlev + 255) / 256, 256, 0, s>>>(nlev, lv->level_ptr, rpw, cptr);
            count_launch();
        }
        if ((st = exclusive_scan_i32(cptr, cptr, nlev, true, s))) break;
        int nc = 0;
        if (cudaMemcpy(&nc, cptr + nlev, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "chunk table");
            break;
        }
        if ((st = dalloc(&p->chunks[i], (size_t)nc))) break;
        p->nchunks[i] = nc;
        if (nc > 0) {
            k_chunk_table<<<(nc + 255) / 256, 256, 0, s>>>(nlev, lv->level_ptr, cptr, rpw, nc, p->chunks[i]);
            count_launch();
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(e, "chunk table");
    }
    dfree(cptr);
    return st;
}

}  // namespace

namespace {
template <typename VT, typename XT, int WMAX>
hec_status launch_part(const sptrsv_plan* pl, PartParams& pp, cudaStream_t s) {
    const hec_part_data* P = pl->part;
    const void* k = (const void*)k_sweep_part<VT, XT, WMAX>;
    void* args[] = {&pp};
    void* tok = nullptr;
    const size_t smem = (size_t)P->max_rows * sizeof(XT);
    profile_begin(s, &tok);
    HEC_CUDA(cudaLaunchCooperativeKernel(k, dim3(P->nparts), dim3(P->threads), args, smem, s));
    profile_end(s, tok);
    count_launch();
    P->parity ^= 1;  // launched: the next sweep polls the buffer this one sets to the sentinel
    return HEC_OK;
}

template <typename VT, typename XT>
hec_status dispatch_part(const sptrsv_plan* pl, PartParams& pp, cudaStream_t s) {
    if (pp.w <= 4) return launch_part<VT, XT, 4>(pl, pp, s);
    return launch_part<VT, XT, 8>(pl, pp, s);
}

template <typename VT, typename XT>
const void* part_kernel(int w) {
    return w <= 4 ? (const void*)k_sweep_part<VT, XT, 4> : (const void*)k_sweep_part<VT, XT, 8>;
}
}  // namespace

hec_status sweep(const sptrsv_plan* pl, int nrhs, const double* b, int ldb, const int* gather, double* x, int ldx,
                 const int* scatter, cudaStream_t s, bool b32, bool x32, const int* bidx, bool bplan) {
    const hec_matrix* T = pl->T;
    if (T->n == 0) return HEC_OK;
    if (pl->part && pl->use_part && nrhs == 1) {
        const hec_part_data* P = pl->part;
        PartParams pp;
        pp.n = T->n;
        pp.ld = T->ld;
        pp.w = T->w;
        pp.ell_col = P->ell_col;
        pp.ell_val = P->ell_val;
        pp.tptr = P->tptr;
        pp.tcol = P->tcol;
        pp.tval = P->tval;
        pp.dinv = P->dinv;
        pp.rowg = P->rowg;
        pp.part_row = P->part_row;
        pp.part_chunk = P->part_chunk;
        pp.chunks = P->chunks;
        pp.bp = P->bp;
        pp.b = b;
        pp.ldb = ldb;
        pp.gather = gather;
        pp.x = x;
        pp.ldx = ldx;
        pp.scatter = scatter;
        pp.xp = P->xpb[P->parity];
        pp.xp_next = P->xpb[P->parity ^ 1];
        pp.bidx = bidx ? bidx : (gather && gather == pl->lv->iperm ? P->bidx_perm : nullptr);
        pp.bplan = bplan;
        pp.status = pl->status;
        pp.budget = pl->wait_cycles;
        pp.skip_row = pl->skip_row;
        pp.b32 = b32;
        pp.x32 = x32;
        switch (T->vdt) {
            case HEC_F64: return dispatch_part<double, double>(pl, pp, s);
            case HEC_F32: return dispatch_part<float, float>(pl, pp, s);
            default: return dispatch_part<__nv_bfloat16, float>(pl, pp, s);
        }
    }
    SweepParams sp;
    sp.n = T->n;
    sp.ld = T->ld;
    sp.w = T->w;
    sp.K = nrhs;
    sp.ell_col = T->ell_col;
    sp.ell_val = T->ell_val;
    sp.tptr = T->tptr;
    sp.tcol = T->tcol;
    sp.tval = T->tval;
    sp.b = b;
    sp.ldb = ldb;
    sp.gather = gather;
    sp.x = x;
    sp.ldx = ldx;
    sp.scatter = scatter;
    sp.xp = pl->xp;
    sp.status = pl->status;
    sp.budget = pl->wait_cycles;
    sp.skip_row = pl->skip_row;
    sp.backoff_ns = pl->backoff_ns;
    sp.dinv = pl->dinv;
    sp.b32 = b32;
    sp.x32 = x32;
    switch (T->vdt) {
        case HEC_F64: return dispatch_w<double, double>(pl, sp, s);
        case HEC_F32: return dispatch_w<float, float>(pl, sp, s);
        default: return dispatch_w<__nv_bfloat16, float>(pl, sp, s);
    }
}

namespace {
__global__ void k_ilu_maps(int n, const int* __restrict__ iperm_l, const int* __restrict__ perm_u,
                           const int* __restrict__ iperm_u, const int* __restrict__ ext2glob,
                           const unsigned char* __restrict__ owned, int* lg, int* ls, int* us) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int il = iperm_l[r];
    lg[r] = ext2glob ? ext2glob[il] : il;  // lower sweep reads r at the global row of its extended row
    ls[r] = perm_u[il];                    // and writes y straight into the upper factor's order
    int iu = iperm_u[r];
    us[r] = ext2glob ? (owned[iu] ? ext2glob[iu] : -1) : iu;  // upper sweep writes owned rows only
}
// out[i] = outer[inner[i]] (-1 stays -1)
__global__ void k_compose(int n, const int* __restrict__ inner, const int* __restrict__ outer, int* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = inner[i];
    out[i] = k >= 0 ? outer[k] : -1;
}
// The composed indices of partitioned sweeps of M: for the lower factor's partition, the row of r
// of each plan row (so the sweep's gather is one load); for the upper factor's, the plan row of U
// that receives each row of y (so the lower sweep writes y in the order the upper sweep reads it).
hec_status ilu_compose(const ilu_precond* M, const hec_part_data* P, bool lower, cudaStream_t s) {
    int*& out = lower ? M->lg_part : M->ls_upart;
    long long& id = lower ? M->lg_part_id : M->ls_upart_id;
    if (id == P->id) return HEC_OK;
    if (!out) HEC_CHECK(dalloc(&out, (size_t)M->n_ext));
    const int n = M->n_ext;
    if (lower) k_compose<<<(n + 255) / 256, 256, 0, s>>>(n, P->rowg, M->l_gather, out);
    else k_compose<<<(n + 255) / 256, 256, 0, s>>>(n, M->l_scatter, P->pos, out);
    count_launch();
    HEC_CUDA(cudaGetLastError());
    id = P->id;
    return HEC_OK;
}
}  // namespace

void free_part(hec_part_data* P) {
    if (!P) return;
    dfree(P->rowg); dfree(P->part_row); dfree(P->part_seg); dfree(P->seg_start);
    dfree(P->ell_col); dfree(P->ell_val); dfree(P->tptr); dfree(P->tcol); dfree(P->tval); dfree(P->dinv);
    dfree(P->bp); dfree(P->part_chunk); dfree(P->chunks);
    dfree(P->xpb[0]); dfree(P->xpb[1]); dfree(P->pos); dfree(P->bidx_perm);
    delete P;
}

void free_plan(sptrsv_plan* p) {
    if (!p) return;
    dfree(p->xp);
    dfree(p->status);
    for (int i = 0; i < 5; ++i) dfree(p->chunks[i]);
    dfree(p->dinv);
    free_part(p->part);
    delete p;
}

hec_status sort_pairs_i32(int* keys, int* vals, int n, int max_key, cudaStream_t s);

namespace {
// part id of each level-ordered row g (from the caller's map of original rows, or contiguous
// ranges of the original index), and the identity payload for the sort
__global__ void k_part_keys(int n, const int* __restrict__ iperm, const int* __restrict__ part, int nparts, int* key,
                            int* val, int* bad) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int i = iperm[g];
    const int pk = part ? part[i] : (int)((long long)i * nparts / n);
    if (pk < 0 || pk >= nparts) atomicCAS(bad, 0, 1);
    key[g] = min(max(pk, 0), nparts - 1);
    val[g] = g;
}
// rows per part: a block counts parts below 1024 in shared memory and adds its totals once (one
// global atomic per row would serialise on the few parts a stretch of sorted keys covers)
__global__ void k_hist(int n, const int* __restrict__ key, int nparts, int* cnt) {
    __shared__ int sh[1024];
    for (int t = threadIdx.x; t < 1024; t += blockDim.x) sh[t] = 0;
    __syncthreads();
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int k = key[r];
        if (k < 1024) atomicAdd(sh + k, 1);
        else atomicAdd(cnt + k, 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 1024 && t < nparts; t += blockDim.x)
        if (sh[t]) atomicAdd(cnt + t, sh[t]);
}
// segment starts: a new segment where the part or the level changes
__global__ void k_seg_flags(int n, const int* __restrict__ key, const int* __restrict__ rowg,
                            const int* __restrict__ iperm, const int* __restrict__ level, int* flag, int* sigma) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int g = rowg[r];
    sigma[g] = r;
    int f = 1;
    if (r > 0) {
        const int g0 = rowg[r - 1];
        f = (key[r] != key[r - 1]) || (level[iperm[g]] != level[iperm[g0]]);
    }
    flag[r] = f;
}
__global__ void k_seg_table(int n, const int* __restrict__ flag, const int* __restrict__ segidx, int nseg, int* seg_start) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n && flag[r]) seg_start[segidx[r]] = r;
    if (r == 0) seg_start[nseg] = n;
}
__global__ void k_part_seg(int nparts, int n, int nseg, const int* __restrict__ part_row, const int* __restrict__ segidx,
                           int* part_seg) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > nparts) return;
    const int r = part_row[p];
    part_seg[p] = r < n ? segidx[r] : nseg;
}
__global__ void k_gather_idx(int m, const int* __restrict__ idx, const int* __restrict__ src, int* dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) dst[i] = src[idx[i]];
}
__global__ void k_tail_len_perm(int n, const int* __restrict__ rowg, const int* __restrict__ tptr, int* len) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) len[r] = tptr[rowg[r] + 1] - tptr[rowg[r]];
}
// plan row r takes level-ordered row g = rowg[r]; columns renumbered by sigma and re-sorted
template <typename VT>
__global__ void k_repack(int n, int ld, int w, const int* __restrict__ rowg, const int* __restrict__ sigma,
                         const int* __restrict__ ec, const VT* __restrict__ ev, const int* __restrict__ tp,
                         const int* __restrict__ tc, const VT* __restrict__ tv, const int* __restrict__ ntp, int* nec,
                         VT* nev, int* ntc, VT* ntv) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ld) return;
    if (r >= n) {
        for (int k = 0; k < w; ++k) {
            nec[(long)k * ld + r] = -1;
            nev[(long)k * ld + r] = (VT)0.0f;
        }
        return;
    }
    const int g = rowg[r];
    int nell = 0;
    for (int k = 0; k < w; ++k) nell += ec[(long)k * ld + g] >= 0;
    const int t0 = tp[g], tcnt = tp[g + 1] - t0 - 1;  // overflow entries, the diagonal excluded
    const int cnt = nell + tcnt;
    auto col_of = [&](int e) { return sigma[e < nell ? ec[(long)e * ld + g] : tc[t0 + e - nell]]; };
    auto val_of = [&](int e) { return e < nell ? ev[(long)e * ld + g] : tv[t0 + e - nell]; };
    const int nt0 = ntp[r];
    for (int e = 0; e < cnt; ++e) {
        const int c = col_of(e);
        int rank = 0;
        for (int f = 0; f < cnt; ++f) rank += col_of(f) < c;
        if (rank < w) {
            nec[(long)rank * ld + r] = c;
            nev[(long)rank * ld + r] = val_of(e);
        } else {
            ntc[nt0 + rank - w] = c;
            ntv[nt0 + rank - w] = val_of(e);
        }
    }
    for (int k = cnt; k < w; ++k) {
        nec[(long)k * ld + r] = -1;
        nev[(long)k * ld + r] = (VT)0.0f;
    }
    ntc[ntp[r + 1] - 1] = r;
    ntv[ntp[r + 1] - 1] = tv[tp[g + 1] - 1];
}
template <typename XT>
__global__ void k_perm_dinv(int n, const int* __restrict__ rowg, const XT* __restrict__ d, XT* nd) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) nd[r] = d[rowg[r]];
}
// pos = inverse of rowg; bidx[r] = iperm[rowg[r]] (the row of b of plan row r in sptrsv_lower/upper)
__global__ void k_part_pos(int n, const int* __restrict__ rowg, const int* __restrict__ iperm, int* pos, int* bidx) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int g = rowg[r];
    pos[g] = r;
    bidx[r] = iperm[g];
}
std::atomic<long long> g_part_id{0};
}  // namespace

hec_status build_partition(sptrsv_plan* p, const int* part, int nparts, cudaStream_t s) {
    const hec_matrix* T = p->T;
    const hec_levels* lv = p->lv;
    const int n = T->n;
    hec_part_data* P = new hec_part_data();
    P->nparts = nparts;
    int *key = nullptr, *flag = nullptr, *segidx = nullptr, *sigma = nullptr, *len = nullptr, *bad = nullptr;
    hec_status st = HEC_OK;
    auto done = [&](hec_status e) {
        dfree(key); dfree(flag); dfree(segidx); dfree(sigma); dfree(len); dfree(bad);
        if (e != HEC_OK) free_part(P);
        return e;
    };
    const int g = (n + 255) / 256;
    if ((st = dalloc(&key, n)) || (st = dalloc(&P->rowg, n)) || (st = dalloc(&bad, 1)) ||
        (st = dalloc(&P->part_row, (size_t)nparts + 1)) || (st = dalloc(&flag, (size_t)n + 1)) ||
        (st = dalloc(&segidx, (size_t)n + 1)) || (st = dalloc(&sigma, n)) || (st = dalloc(&len, (size_t)n + 1)) ||
        (st = dalloc(&P->part_seg, (size_t)nparts + 1)))
        return done(st);
    cudaMemsetAsync(bad, 0, sizeof(int), s);
    k_part_keys<<<g, 256, 0, s>>>(n, lv->iperm, part, nparts, key, P->rowg, bad);
    count_launch();
    int hbad = 0;
    HEC_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    HEC_CUDA(cudaStreamSynchronize(s));
    if (hbad) return done(set_error(HEC_ERR_INVALID_ARG, "sptrsv_plan_partition: part[] outside [0, nparts)"));
    if ((st = sort_pairs_i32(key, P->rowg, n, nparts - 1, s))) return done(st);
    HEC_CUDA(cudaMemsetAsync(P->part_row, 0, sizeof(int) * ((size_t)nparts + 1), s));
    k_hist<<<std::min(g, 4 * num_sms()), 256, 0, s>>>(n, key, nparts, P->part_row);
    k_seg_flags<<<g, 256, 0, s>>>(n, key, P->rowg, lv->iperm, lv->level, flag, sigma);
    count_launch(2);
    if ((st = exclusive_scan_i32(P->part_row, P->part_row, nparts, true, s))) return done(st);
    if ((st = exclusive_scan_i32(flag, segidx, n, true, s))) return done(st);
    HEC_CUDA(cudaMemcpy(&P->nseg, segidx + n, sizeof(int), cudaMemcpyDeviceToHost));
    if ((st = dalloc(&P->seg_start, (size_t)P->nseg + 1))) return done(st);
    k_seg_table<<<g, 256, 0, s>>>(n, flag, segidx, P->nseg, P->seg_start);
    k_part_seg<<<(nparts + 256) / 256, 256, 0, s>>>(nparts, n, P->nseg, P->part_row, segidx, P->part_seg);
    k_tail_len_perm<<<g, 256, 0, s>>>(n, P->rowg, T->tptr, len);
    count_launch(3);
    if ((st = dalloc(&P->tptr, (size_t)n + 1)) || (st = exclusive_scan_i32(len, P->tptr, n, true, s))) return done(st);
    // level-aligned chunks of at most 32 rows inside each (part, level) segment
    {
        int* cseg = nullptr;
        if ((st = dalloc(&cseg, (size_t)P->nseg + 1)) || (st = dalloc(&P->part_chunk, (size_t)nparts + 1))) {
            dfree(cseg);
            return done(st);
        }
        k_chunk_counts<<<(P->nseg + 255) / 256, 256, 0, s>>>(P->nseg, P->seg_start, 32, cseg);
        count_launch();
        if ((st = exclusive_scan_i32(cseg, cseg, P->nseg, true, s))) { dfree(cseg); return done(st); }
        cudaMemcpy(&P->nchunks, cseg + P->nseg, sizeof(int), cudaMemcpyDeviceToHost);
        if ((st = dalloc(&P->chunks, (size_t)P->nchunks))) { dfree(cseg); return done(st); }
        k_chunk_table<<<(P->nchunks + 255) / 256, 256, 0, s>>>(P->nseg, P->seg_start, cseg, 32, P->nchunks, P->chunks);
        k_gather_idx<<<(nparts + 256) / 256, 256, 0, s>>>(nparts + 1, P->part_seg, cseg, P->part_chunk);
        count_launch(2);
        cudaError_t ce = cudaStreamSynchronize(s);
        dfree(cseg);
        if (ce != cudaSuccess) return done(cuda_error(ce, "partition chunks"));
        std::vector<int> pr((size_t)nparts + 1);
        HEC_CUDA(cudaMemcpy(pr.data(), P->part_row, sizeof(int) * pr.size(), cudaMemcpyDeviceToHost));
        for (int q = 0; q < nparts; ++q) P->max_rows = std::max(P->max_rows, pr[q + 1] - pr[q]);
    }
    const size_t vs = T->vdt == HEC_F64 ? 8 : T->vdt == HEC_F32 ? 4 : 2;
    const size_t ws = T->vdt == HEC_F64 ? 8 : 4;
    if ((st = dalloc(&P->ell_col, (size_t)T->w * T->ld)) || (st = dmalloc(&P->ell_val, vs * (size_t)T->w * T->ld + 16)) ||
        (st = dalloc(&P->tcol, (size_t)T->tail_nnz)) || (st = dmalloc(&P->tval, vs * (size_t)T->tail_nnz + 16)) ||
        (st = dmalloc(&P->dinv, ws * (size_t)n + 16)) || (ws == 4 && (st = dmalloc(&P->bp, ws * (size_t)n + 16))) ||
        (st = dmalloc(&P->xpb[0], ws * (size_t)n + 16)) || (st = dmalloc(&P->xpb[1], ws * (size_t)n + 16)) ||
        (st = dalloc(&P->pos, n)) || (st = dalloc(&P->bidx_perm, n)))
        return done(st);
    P->id = ++g_part_id;
    k_part_pos<<<g, 256, 0, s>>>(n, P->rowg, lv->iperm, P->pos, P->bidx_perm);
    count_launch();
    {
        // the buffer the first sweep polls; every sweep sets the other one for its successor
        const int fb = std::min(4096, std::max(1, g));
        if (ws == 8) k_fill_sentinel<double><<<fb, 256, 0, s>>>((double*)P->xpb[0], n);
        else k_fill_sentinel<float><<<fb, 256, 0, s>>>((float*)P->xpb[0], n);
        count_launch();
    }
    const int gl = (T->ld + 255) / 256;
    if (T->vdt == HEC_F64) {
        k_repack<double><<<gl, 256, 0, s>>>(n, T->ld, T->w, P->rowg, sigma, T->ell_col, (const double*)T->ell_val, T->tptr,
                                            T->tcol, (const double*)T->tval, P->tptr, P->ell_col, (double*)P->ell_val,
                                            P->tcol, (double*)P->tval);
        k_perm_dinv<double><<<g, 256, 0, s>>>(n, P->rowg, (const double*)p->dinv, (double*)P->dinv);
    } else if (T->vdt == HEC_F32) {
        k_repack<float><<<gl, 256, 0, s>>>(n, T->ld, T->w, P->rowg, sigma, T->ell_col, (const float*)T->ell_val, T->tptr,
                                           T->tcol, (const float*)T->tval, P->tptr, P->ell_col, (float*)P->ell_val, P->tcol,
                                           (float*)P->tval);
        k_perm_dinv<float><<<g, 256, 0, s>>>(n, P->rowg, (const float*)p->dinv, (float*)P->dinv);
    } else {
        k_repack<__nv_bfloat16><<<gl, 256, 0, s>>>(n, T->ld, T->w, P->rowg, sigma, T->ell_col,
                                                   (const __nv_bfloat16*)T->ell_val, T->tptr, T->tcol,
                                                   (const __nv_bfloat16*)T->tval, P->tptr, P->ell_col,
                                                   (__nv_bfloat16*)P->ell_val, P->tcol, (__nv_bfloat16*)P->tval);
        k_perm_dinv<float><<<g, 256, 0, s>>>(n, P->rowg, (const float*)p->dinv, (float*)P->dinv);
    }
    count_launch(2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return done(cuda_error(e, "sptrsv_plan_partition"));
    free_part(p->part);
    p->part = P;
    return done(HEC_OK);
}

// resident blocks of the partitioned kernel for `smem` bytes of shared solution per block
int part_capacity(const sptrsv_plan* p, int threads, size_t smem) {
    const void* k = p->T->vdt == HEC_F64 ? part_kernel<double, double>(p->T->w)
                    : p->T->vdt == HEC_F32 ? part_kernel<float, float>(p->T->w)
                                           : part_kernel<__nv_bfloat16, float>(p->T->w);
    if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return max_coop_blocks(k, threads, smem) * num_sms();
}

}  // namespace hec

using namespace hec;

HEC_API hec_status sptrsv_plan_create(const hec_matrix* tri, const hec_levels* lv, int max_nrhs, const hec_tune* tune,
                                      sptrsv_plan** out) {
    clear_error();
    if (!out || !tri || !lv || !tri->tri || tri->lv != lv || max_nrhs < 1 || max_nrhs > 16)
        return set_error(HEC_ERR_INVALID_ARG,
                         "sptrsv_plan_create: need a triangular HEC matrix, the analysis it was packed with, 1 <= max_nrhs <= 16");
    *out = nullptr;
    sptrsv_plan* p = new sptrsv_plan();
    p->T = tri;
    p->lv = lv;
    p->max_nrhs = max_nrhs;
    if (tune) {
        if (tune->block_threads) p->threads = tune->block_threads;
        if (tune->blocks_per_sm) p->blocks = tune->blocks_per_sm;
        if (tune->wait_cycles) p->wait_cycles = tune->wait_cycles;
        if (tune->debug_unpublished_row > 0) p->skip_row = tune->debug_unpublished_row - 1;
        if (tune->backoff_ns > 0) p->backoff_ns = tune->backoff_ns;
    }
    p->lpr1 = default_lanes_per_row(tri);
    if (tune && tune->lanes_per_row) p->lpr1 = tune->lanes_per_row;
    if (p->lpr1 != 1 && p->lpr1 != 2 && p->lpr1 != 4 && p->lpr1 != 8) {
        delete p;
        return set_error(HEC_ERR_INVALID_ARG, "sptrsv_plan_create: lanes_per_row must be 0, 1, 2, 4 or 8");
    }
    if (p->threads % 32 || p->threads < 32 || p->threads > 256) {
        delete p;
        return set_error(HEC_ERR_INVALID_ARG, "sptrsv_plan_create: block_threads must be a multiple of 32 in [32, 256]");
    }
    hec_status st = dmalloc(&p->xp, work_size(tri->vdt) * (size_t)tri->n * sweep_kp(max_nrhs) + 16);
    if (st == HEC_OK) st = dalloc(&p->status, 1);
    if (st == HEC_OK && cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) st = cuda_error(cudaGetLastError(), "memset");
    unsigned needed = 1u << log2i(p->lpr1);  // only the lane layouts this plan can be called with
    for (int k = 1; k <= max_nrhs; ++k) needed |= 1u << log2i(sweep_lpr(k, tri->vdt));
    if (st == HEC_OK) st = build_chunks(p, needed);
    if (st == HEC_OK) st = build_dinv(p);
    if (st != HEC_OK) { free_plan(p); return st; }
    *out = p;
    return HEC_OK;
}

HEC_API hec_status sptrsv_plan_partition(sptrsv_plan* p, const int* part, int nparts, int threads, void* stream) {
    clear_error();
    if (!p) return set_error(HEC_ERR_INVALID_ARG, "sptrsv_plan_partition: NULL plan");
    if (nparts == 0) {
        free_part(p->part);
        p->part = nullptr;
        return HEC_OK;
    }
    if (threads == 0) threads = 256;
    if (nparts < 1 || (threads != 128 && threads != 256 && threads != 512 && threads != 1024) || p->T->n == 0)
        return set_error(HEC_ERR_INVALID_ARG, "sptrsv_plan_partition: need nparts >= 1, threads 128, 256, 512 or 1024");
    const int cap0 = part_capacity(p, threads, 0);
    if (nparts > cap0)
        return set_error(HEC_ERR_INVALID_ARG, "sptrsv_plan_partition: " + std::to_string(nparts) +
                                                  " parts cannot all be resident (at most " + std::to_string(cap0) + ")");
    sptrsv_plan tmp;  // build into a scratch holder, keep the old partition on failure
    tmp.T = p->T;
    tmp.lv = p->lv;
    tmp.dinv = p->dinv;
    hec_status st = build_partition(&tmp, part, nparts, S(stream));
    tmp.dinv = nullptr;
    if (st != HEC_OK) return st;
    const size_t ws = p->T->vdt == HEC_F64 ? 8 : 4;
    const size_t smem = (size_t)tmp.part->max_rows * ws;
    const int cap = smem <= 227 * 1024 ? part_capacity(p, threads, smem) : 0;
    if (nparts > cap) {
        free_part(tmp.part);
        tmp.part = nullptr;
        return set_error(HEC_ERR_INVALID_ARG, "sptrsv_plan_partition: the largest part (" +
                                                  std::to_string(smem) + " bytes of shared solution) leaves room for " +
                                                  std::to_string(cap) + " resident parts, fewer than " +
                                                  std::to_string(nparts));
    }
    free_part(p->part);
    p->part = tmp.part;
    tmp.part = nullptr;
    p->part->threads = threads;
    p->use_part = 1;
    return HEC_OK;
}

HEC_API int sptrsv_partition_capacity(const sptrsv_plan* p, int threads) {
    if (!p) return 0;
    return part_capacity(p, threads ? threads : 256, 0);
}

HEC_API hec_status sptrsv_plan_destroy(sptrsv_plan* p) {
    free_plan(p);
    return HEC_OK;
}

static hec_status sweep_api(const sptrsv_plan* p, int uplo, int nrhs, const double* b, int ldb, double* x, int ldx,
                            void* stream) {
    clear_error();
    if (!p || p->T->uplo != uplo || nrhs < 1 || nrhs > p->max_nrhs || ldb < nrhs || ldx < nrhs ||
        (p->T->n > 0 && (!b || !x)))
        return set_error(HEC_ERR_INVALID_ARG, uplo ? "sptrsv_upper: bad argument" : "sptrsv_lower: bad argument");
    return sweep(p, nrhs, b, ldb, p->lv->iperm, x, ldx, p->lv->iperm, S(stream));
}

HEC_API hec_status sptrsv_lower(const sptrsv_plan* p, int nrhs, const double* b, int ldb, double* x, int ldx,
                                void* stream) {
    return sweep_api(p, 0, nrhs, b, ldb, x, ldx, stream);
}

HEC_API hec_status sptrsv_upper(const sptrsv_plan* p, int nrhs, const double* b, int ldb, double* x, int ldx,
                                void* stream) {
    return sweep_api(p, 1, nrhs, b, ldb, x, ldx, stream);
}

// ---- autotuner ------------------------------------------------------------------------------
// The free parameters of the point-to-point sweep, searched on the plan's own factor:
//  - residency (block size x blocks per SM): too few resident warps and a level's rows are not
//    all in flight; too many and far-ahead warps only add polling traffic;
//  - for one right-hand side, lanes per row (1, 2, 4 or 8): one lane per row (thread per row)
//    against several lanes sharing a row's dependencies and a shuffle reduction (the
//    thread-versus-warp choice by row length);
//  - for one right-hand side on a plan given a partition, the partitioned schedule against the
//    best global one.
// The point-to-point sweep has no per-level barriers, so the paper's level-merging threshold has
// no counterpart.  Results are cached per matrix signature (rows, slab width, tail entries,
// levels, value type, right-hand sides, whether a partition was given) so identical factors are
// tuned once per process.
namespace {
struct TuneKey {
    int n, w, nlev, vdt, kp, parted;
    long long tail;
    bool operator==(const TuneKey& o) const {
        return n == o.n && w == o.w && nlev == o.nlev && vdt == o.vdt && kp == o.kp && parted == o.parted &&
               tail == o.tail;
    }
};
struct TuneKeyHash {
    size_t operator()(const TuneKey& k) const {
        return std::hash<long long>()(((long long)k.n * 1315423911LL) ^ (k.tail * 2654435761LL) ^ (k.nlev * 97) ^
                                      (k.w * 31 + k.vdt * 7 + k.kp * 3 + k.parted));
    }
};
struct TuneChoice {
    int threads, blocks, lpr1, use_part;
};
std::mutex g_tune_mu;
std::unordered_map<TuneKey, TuneChoice, TuneKeyHash> g_tune_cache;

void apply_choice(sptrsv_plan* p, const TuneChoice& c, hec_tune* out) {
    p->threads = c.threads;
    p->blocks = c.blocks;
    p->lpr1 = c.lpr1;
    p->use_part = c.use_part;
    if (out) {
        *out = hec_tune{};
        out->block_threads = c.threads;
        out->blocks_per_sm = c.blocks;
        out->lanes_per_row = c.lpr1;
        out->partitioned = (p->part && c.use_part) ? 1 : 0;
    }
}
}  // namespace

HEC_API hec_status sptrsv_autotune(sptrsv_plan* p, int nrhs, hec_tune* out, void* stream) {
    clear_error();
    if (!p || nrhs < 1 || nrhs > p->max_nrhs) return set_error(HEC_ERR_INVALID_ARG, "sptrsv_autotune: bad argument");
    cudaStream_t s = S(stream);
    const hec_matrix* T = p->T;
    int kp = 1;
    while (kp < nrhs) kp <<= 1;
    const int parted = (nrhs == 1 && p->part) ? 1 : 0;
    TuneKey key{T->n, T->w, p->lv->nlev, (int)T->vdt, kp, parted, T->tail_nnz};
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            if (nrhs == 1) HEC_CHECK(build_chunks(p, 1u << log2i(it->second.lpr1)));
            apply_choice(p, it->second, out);
            return HEC_OK;
        }
    }
    double* b = nullptr;
    double* x = nullptr;
    const size_t cnt = (size_t)std::max(T->n, 1) * nrhs;
    HEC_CHECK(dalloc(&b, cnt));
    hec_status st = dalloc(&x, cnt);
    if (st) { dfree(b); return st; }
    cudaMemsetAsync(b, 0, sizeof(double) * cnt, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const TuneChoice saved{p->threads, p->blocks, p->lpr1, p->use_part};
    // one warm-up and three timed sweeps of the plan as it is set
    auto time_it = [&](float* ms) -> hec_status {
        hec_status r = sweep(p, nrhs, b, nrhs, p->lv->iperm, x, nrhs, p->lv->iperm, s);
        if (r) return r;
        cudaEventRecord(e0, s);
        for (int k = 0; k < 3 && r == HEC_OK; ++k) r = sweep(p, nrhs, b, nrhs, p->lv->iperm, x, nrhs, p->lv->iperm, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        *ms = 0.f;
        cudaEventElapsedTime(ms, e0, e1);
        return r;
    };
    float best = 1e30f;
    TuneChoice bc = saved;
    const int cand_t[2] = {128, 256};
    const int cand_b[4] = {2, 4, 8, 16};
    const int cand_l[4] = {1, 2, 4, 8};
    for (int li = 0; li < (nrhs == 1 ? 4 : 1) && st == HEC_OK; ++li) {
        const int lpr = nrhs == 1 ? cand_l[li] : saved.lpr1;
        if (nrhs == 1 && (st = build_chunks(p, 1u << log2i(lpr)))) break;
        for (int ti = 0; ti < 2 && st == HEC_OK; ++ti) {
            for (int bi = 0; bi < 4 && st == HEC_OK; ++bi) {
                if (cand_t[ti] * cand_b[bi] > 2048) continue;
                const TuneChoice c{cand_t[ti], cand_b[bi], lpr, 0};
                apply_choice(p, c, nullptr);
                float ms = 0.f;
                st = time_it(&ms);
                if (st == HEC_OK && ms < best) { best = ms; bc = c; }
            }
        }
    }
    if (st == HEC_OK && parted) {  // the partitioned schedule (its launch shape is the partition's)
        const TuneChoice c{bc.threads, bc.blocks, bc.lpr1, 1};
        apply_choice(p, c, nullptr);
        float ms = 0.f;
        st = time_it(&ms);
        if (st == HEC_OK && ms < best) { best = ms; bc = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(b);
    dfree(x);
    if (st) { apply_choice(p, saved, nullptr); return st; }
    apply_choice(p, bc, out);
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[key] = bc;
    }
    return hec_sync_status(p, stream);
}

HEC_API hec_status hec_sync_status(const sptrsv_plan* p, void* stream) {
    if (!p) return set_error(HEC_ERR_INVALID_ARG, "hec_sync_status: NULL");
    int h = 0;
    cudaStream_t s = S(stream);
    HEC_CUDA(cudaMemcpyAsync(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    HEC_CUDA(cudaMemsetAsync(p->status, 0, sizeof(int), s));
    HEC_CUDA(cudaStreamSynchronize(s));
    if (h == 0) return HEC_OK;
    return set_error((hec_status)h, h == HEC_ERR_TIMEOUT ? "a dependency wait timed out" : "device-side check failed");
}

HEC_API hec_status ilu_create(const sptrsv_plan* L, const sptrsv_plan* U, int n_glob, int n_ext, const int* ext2glob,
                              const unsigned char* owned, ilu_precond** out) {
    clear_error();
    if (!out || !L || !U || L->T->uplo != 0 || U->T->uplo != 1 || L->T->n != n_ext || U->T->n != n_ext || n_glob < 0 ||
        (!ext2glob && n_glob != n_ext) || (ext2glob && !owned))
        return set_error(HEC_ERR_INVALID_ARG, "ilu_create: bad argument");
    *out = nullptr;
    ilu_precond* M = new ilu_precond();
    M->L = L;
    M->U = U;
    M->n_glob = n_glob;
    M->n_ext = n_ext;
    M->max_nrhs = std::min(L->max_nrhs, U->max_nrhs);
    // the intermediate y in FP32 when both sweeps compute in FP32 (FP32 / BF16 values)
    M->y32 = L->T->vdt != HEC_F64 && U->T->vdt != HEC_F64;
    hec_status st = HEC_OK;
    if ((st = dalloc(&M->l_gather, (size_t)n_ext)) || (st = dalloc(&M->l_scatter, (size_t)n_ext)) ||
        (st = dalloc(&M->u_scatter, (size_t)n_ext)) ||
        (st = dmalloc(&M->y, (M->y32 ? sizeof(float) : sizeof(double)) * (size_t)n_ext * M->max_nrhs + 16))) {
        ilu_destroy(M);
        return st;
    }
    if (n_ext > 0) {
        k_ilu_maps<<<(n_ext + 255) / 256, 256>>>(n_ext, L->lv->iperm, U->lv->perm, U->lv->iperm, ext2glob, owned,
                                                  M->l_gather, M->l_scatter, M->u_scatter);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            ilu_destroy(M);
            return cuda_error(e, "ilu_create");
        }
    }
    *out = M;
    return HEC_OK;
}

HEC_API hec_status ilu_destroy(ilu_precond* M) {
    if (!M) return HEC_OK;
    dfree(M->l_gather);
    dfree(M->l_scatter);
    dfree(M->u_scatter);
    dfree(M->y);
    dfree(M->lg_part);
    dfree(M->ls_upart);
    delete M;
    return HEC_OK;
}

HEC_API hec_status ilu_apply(const ilu_precond* M, int nrhs, const double* r, int ldr, double* z, int ldz, void* stream) {
    clear_error();
    if (!M || nrhs < 1 || nrhs > M->max_nrhs || ldr < nrhs || ldz < nrhs || (M->n_glob > 0 && (!r || !z)))
        return set_error(HEC_ERR_INVALID_ARG, "ilu_apply: bad argument");
    cudaStream_t s = S(stream);
    // partitioned single-right-hand-side sweeps take composed indices: L gathers r with one load
    // a row, and writes y straight into U's plan order, which U then reads in order
    const bool lpart = M->L->part && M->L->use_part && nrhs == 1 && M->n_ext > 0;
    const bool upart = M->U->part && M->U->use_part && nrhs == 1 && M->n_ext > 0;
    if (lpart) HEC_CHECK(ilu_compose(M, M->L->part, true, s));
    if (upart) HEC_CHECK(ilu_compose(M, M->U->part, false, s));
    // L y = r: gather r, write y already permuted into the upper factor's level (or plan) order
    HEC_CHECK(sweep(M->L, nrhs, r, ldr, M->l_gather, (double*)M->y, nrhs, upart ? M->ls_upart : M->l_scatter, s,
                    false, M->y32, lpart ? M->lg_part : nullptr));
    // U z = y: y is read in order, z is written back (owned rows only for RAS)
    return sweep(M->U, nrhs, (const double*)M->y, nrhs, nullptr, z, ldz, M->u_scatter, s, M->y32, false, nullptr,
                 upart);
}
