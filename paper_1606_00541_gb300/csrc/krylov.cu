// SpMV on HEC and the FP64 FGMRES(m) outer solver (the paper's experiments use GMRES(20) in
// FP64, Sec. 4; this library uses the flexible variant so that any preconditioner stage may
// change between iterations).
//
// Vectors of nrhs right-hand sides are row-major n x K (K = nrhs); each right-hand side has its
// own Krylov space and the kernels run them batched.  Reductions are deterministic: every block
// writes its partial sums and a second kernel adds them in a fixed order.
//
// Each inner iteration is a fixed sequence of launches with no host round trip:
//   z_j = M^-1 v_j (ilu_apply), w = A z_j (SpMV),
//   one persistent cooperative kernel (k_arnoldi_mgs): modified Gram-Schmidt against v_0..v_j
//     (one pass and one grid-wide reduction per projection), ||w||, the Hessenberg column with
//     its Givens rotations and the convergence test, and w /= h_{j+1,j}.
// The host stays one iteration ahead of the device and reads a per-iteration "still active"
// flag through pinned memory, so the GPU never waits for the host inside a restart cycle.  The
// host synchronizes once per restart to check the true residual.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <type_traits>
#include <vector>

#include <cooperative_groups.h>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace hec {
namespace {

int g_gs_mode = HEC_GS_CLASSICAL;  // process-wide Gram-Schmidt variant (hec_set_gram_schmidt)
constexpr int kThreads = 256;
constexpr int kMgsThreads = 1024;  // the persistent Arnoldi kernel: few, large blocks, so that the
                                   // per-projection sum over the blocks' partials stays short
constexpr int kDotGroup = 8;  // dot products per block row of the multi-dot

// y = alpha A x + beta y for K right-hand sides (x, y row-major with leading dimensions ldx,
// ldy).  Each thread takes RPT rows (strided by the block's row count, so loads stay coalesced)
// for one right-hand side; the rows' chains of FMAs are independent, which keeps more loads and
// FP64 operations in flight.  Each row sums its ELL slots, then its tail, in order.
template <int KP, int RPT>
__global__ void __launch_bounds__(kThreads) k_spmv(int n, int ld, int w, const int* __restrict__ ell_col,
                                                   const double* __restrict__ ell_val, const int* __restrict__ tptr,
                                                   const int* __restrict__ tcol, const double* __restrict__ tval,
                                                   int K, double alpha, const double* __restrict__ x, int ldx,
                                                   double beta, double* __restrict__ y, int ldy) {
    constexpr int RPB = kThreads / KP;
    const int q = threadIdx.x % KP;
    const int rb = blockIdx.x * RPB * RPT + threadIdx.x / KP;
    if (q >= K || rb >= n) return;
    double acc[RPT];
    int row[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        acc[i] = 0.0;
        row[i] = rb + i * RPB < n ? rb + i * RPB : -1;
    }
    // padding (col -1) only ends a row; predicating it instead of leaving the loop lets the
    // loads of all slots issue together
#pragma unroll 4
    for (int k = 0; k < w; ++k) {
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            if (row[i] < 0) continue;
            const long s = (long)k * ld + row[i];
            const int c = __ldg(ell_col + s);
            if (c >= 0) acc[i] = fma(__ldg(ell_val + s), __ldg(x + (long)c * ldx + q), acc[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        if (row[i] < 0) continue;
        const int t1 = __ldg(tptr + row[i] + 1);
        for (int t = __ldg(tptr + row[i]); t < t1; ++t)
            acc[i] = fma(__ldg(tval + t), __ldg(x + (long)__ldg(tcol + t) * ldx + q), acc[i]);
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        if (row[i] < 0) continue;
        double* yp = y + (long)row[i] * ldy + q;
        *yp = beta == 0.0 ? (alpha == 1.0 ? acc[i] : alpha * acc[i]) : fma(beta, *yp, alpha * acc[i]);
    }
}

// y = alpha A x + beta y for one right-hand side, persistent: a grid of resident blocks, each
// thread takes rows r, r + (threads of the grid), ... and loads the next row's slab and tail range
// while its current row's x gathers are in flight, so a thread keeps the loads of two rows
// outstanding instead of waiting on one row's column loads, then its gathers, in turn.  The
// per-row arithmetic is k_spmv's (slab slots in order, then the tail), so the results are the same
// bit for bit.  GB300's FP64 unit spends 16 SM-cycles on a warp's FP64 instruction whether its
// lanes are on or off, so the kernel is instantiated for the exact slab width WMAX (no FMA issued
// for slots beyond it) and the final scaling is chosen by the template MODE (0: y = Ax,
// 1: y = alpha Ax, 2: y = alpha Ax + beta y) rather than by predicated arithmetic.
template <int WMAX, int MODE>
__global__ void __launch_bounds__(kThreads, 4) k_spmv1(int n, int ld, int w, const int* __restrict__ ell_col,
                                                    const double* __restrict__ ell_val, const int* __restrict__ tptr,
                                                    const int* __restrict__ tcol, const double* __restrict__ tval,
                                                    double alpha, const double* __restrict__ x, double beta,
                                                    double* __restrict__ y) {
    const long st = (long)gridDim.x * blockDim.x;
    long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
    int c[WMAX], t0 = 0, t1 = 0;
    double v[WMAX];
    auto load = [&](long rr) {
#pragma unroll
        for (int k = 0; k < WMAX; ++k) {
            c[k] = -1;
            v[k] = 0.0;
            if (k < w && rr < n) {
                c[k] = __ldg(ell_col + (long)k * ld + rr);
                v[k] = __ldg(ell_val + (long)k * ld + rr);
            }
        }
        if (rr < n) {
            t0 = __ldg(tptr + rr);
            t1 = __ldg(tptr + rr + 1);
        }
    };
    load(r);
    while (r < n) {
        int cc[WMAX];
        double vv[WMAX];
#pragma unroll
        for (int k = 0; k < WMAX; ++k) {
            cc[k] = c[k];
            vv[k] = v[k];
        }
        const int a0 = t0, a1 = t1;
        const long rn = r + st;
        load(rn);
        double xs[WMAX];
#pragma unroll
        for (int k = 0; k < WMAX; ++k) xs[k] = cc[k] >= 0 ? __ldg(x + cc[k]) : 0.0;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < WMAX; ++k)
            if (cc[k] >= 0) acc = fma(vv[k], xs[k], acc);
        for (int t = a0; t < a1; ++t) acc = fma(__ldg(tval + t), __ldg(x + __ldg(tcol + t)), acc);
        if (MODE == 0) y[r] = acc;
        else if (MODE == 1) y[r] = alpha * acc;
        else y[r] = fma(beta, y[r], alpha * acc);
        r = rn;
    }
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

// partial[a][blk][q] = this block's share of <V_a, w> for a < count, and of <w, w> at index
// count when `self` is set.  A gate flag of 0 skips the work (re-orthogonalization pass).
template <int KP>
__global__ void __launch_bounds__(kThreads) k_multidot(int n, int K, const double* __restrict__ V, long vstride,
                                                       int count, int self, const double* __restrict__ w,
                                                       double* __restrict__ partial, const int* gate) {
    if (gate && *gate == 0) return;
    constexpr int RPB = kThreads / KP;
    __shared__ double red[kThreads / 32][kDotGroup][KP];
    const int q = threadIdx.x % KP;
    const int a0 = blockIdx.y * kDotGroup;
    const int total = count + self;
    const int na = min(kDotGroup, total - a0);
    double acc[kDotGroup];
#pragma unroll
    for (int g = 0; g < kDotGroup; ++g) acc[g] = 0.0;
    if (q < K) {
        for (long r = (long)blockIdx.x * RPB + threadIdx.x / KP; r < n; r += (long)gridDim.x * RPB) {
            const double wv = w[r * K + q];
#pragma unroll
            for (int g = 0; g < kDotGroup; ++g) {
                if (g < na) {
                    const int a = a0 + g;
                    const double va = a < count ? V[(long)a * vstride + r * K + q] : wv;
                    acc[g] = fma(va, wv, acc[g]);
                }
            }
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

// out[a][q] = sum over blocks of partial[a][blk][q]: one warp per output, fixed order
__global__ void k_reduce(int count, int nblk, int K, const double* __restrict__ partial, double* __restrict__ out,
                         const int* gate) {
    if (gate && *gate == 0) return;
    const int idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (idx >= count * K) return;
    const int a = idx / K, q = idx % K;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += partial[((long)a * nblk + b) * K + q];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[idx] = s;
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

// Arnoldi state of one restart cycle, all on the device.
struct ArnoldiState {
    double* H;     // [(m+1) * m * K]  column j, row a at (a*m + j)*K + q
    double* cs;    // [m*K]
    double* sn;    // [m*K]
    double* g;     // [(m+1)*K]
    double* y;     // [m*K]
    double* h1;    // [(m+2)*K]  first pass dots, then <w,w> before the pass at index j+1
    double* h2;    // [(m+1)*K]  second pass dots
    double* n1;    // [K]  ||w||^2 after the first pass
    double* n2;    // [K]  ||w||^2 after the second pass
    double* f;     // [K]  scale for w
    double* bnorm; // [K]
    int* active;   // [K]
    int* jq;       // [K]  columns used by each right-hand side in this cycle
    int* reorth;   // [1]  Arnoldi steps that took a second Gram-Schmidt pass in this solve
    int* any;      // [1]  some right-hand side still active after this iteration
};

// Hessenberg column j of right-hand side q: the projections h_a = hq[a * hs] (+ h2q[a * hs] when
// a second Gram-Schmidt pass ran), a <= j, and the norm hn of the orthogonalized vector; the
// previous Givens rotations are applied with a running carry, then the new rotation, the residual
// estimate g and the convergence test.  Returns the scale 1 / hn of the next basis vector (0 once
// the right-hand side finishes) and sets *live.  gj and act are g_j and the active flag as they
// stood when the Arnoldi step began.  Only a caller with `write` set stores the column, the
// rotation, g, the column count, the active flag and the scale; every caller computes the same
// result from the same inputs.  With `negated` the arrays hold -h (and -h2).
__device__ double arnoldi_col(const ArnoldiState& st, int K, int j, int m, double rtol, int q, const double* hq,
                              const double* h2q, int hs, double hn, double gj, bool act, bool write, bool* live,
                              bool negated = false) {
    *live = false;
    if (!act) {
        if (write) st.f[q] = 0.0;
        return 0.0;
    }
    // negated: hq and h2q hold -h and -h2 (negation and the sum of two negated values are exact)
    auto hval = [&](int a) {
        const double v = h2q ? hq[a * hs] + h2q[a * hs] : hq[a * hs];
        return negated ? -v : v;
    };
    double* H = st.H;
    double t = hval(0);
    for (int a = 0; a < j; ++a) {
        const double c = st.cs[a * K + q], s = st.sn[a * K + q];
        const double h1 = hval(a + 1);
        const double r = c * t + s * h1;
        t = -s * t + c * h1;
        if (write) H[((size_t)a * m + j) * K + q] = r;
    }
    const double den = sqrt(t * t + hn * hn);
    const double c = den == 0.0 ? 1.0 : t / den, s = den == 0.0 ? 0.0 : hn / den;
    const double gnext = -s * gj;
    const bool done = fabs(gnext) <= rtol * st.bnorm[q] || hn == 0.0 || j + 1 >= m;
    const double f = (!done && hn > 0.0) ? 1.0 / hn : 0.0;
    if (write) {
        H[((size_t)j * m + j) * K + q] = c * t + s * hn;
        H[((size_t)(j + 1) * m + j) * K + q] = hn;
        st.cs[j * K + q] = c;
        st.sn[j * K + q] = s;
        st.g[(j + 1) * K + q] = gnext;
        st.g[j * K + q] = c * gj;
        st.jq[q] = j + 1;
        if (done) st.active[q] = 0;
        st.f[q] = f;
    }
    *live = !done;
    return f;
}

// One Arnoldi step after w = A z_j, as one cooperative persistent launch: modified
// Gram-Schmidt against v_0..v_j (h_a = <v_a, w>; w -= h_a v_a, one grid-wide reduction per a),
// ||w||, the Hessenberg column with its rotations and the convergence test (block 0), and
// w /= h_{j+1,j}.  FP64 throughout.  Reductions are deterministic: each block writes its partial
// sum, and every block adds all partials in the same fixed order (double-buffered by step).
template <int KP>
__global__ void __launch_bounds__(kMgsThreads) k_arnoldi_mgs(int n, int K, int j, int m, double rtol,
                                                          const double* __restrict__ V, long vstride, double* w,
                                                          double* partial, ArnoldiState st) {
    cg::grid_group grid = cg::this_grid();
    constexpr int RPB = kMgsThreads / KP;
    __shared__ double red[kMgsThreads / 32][KP];
    __shared__ double hsh[KP];
    __shared__ int any;
    const int q = threadIdx.x % KP;
    const bool qa = q < K;
    const long r0 = (long)blockIdx.x * RPB + threadIdx.x / KP;
    const long rs = (long)gridDim.x * RPB;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nb = gridDim.x;
    // sum over the grid of each thread's acc for its right-hand side; the result lands in hsh[q]
    auto reduce_all = [&](double acc, int buf) {
#pragma unroll
        for (int o = 16; o >= KP; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane < KP) red[warp][lane] = acc;
        __syncthreads();
        if (threadIdx.x < KP) {
            double s = 0.0;
            for (int wi = 0; wi < kMgsThreads / 32; ++wi) s += red[wi][threadIdx.x];
            partial[((long)buf * nb + blockIdx.x) * KP + threadIdx.x] = s;
        }
        grid.sync();
        // every block adds the blocks' partial sums in the same fixed order, warp qq for right-hand
        // side qq
        if (warp < KP) {
            double s = 0.0;
            for (int b = lane; b < nb; b += 32) s += partial[((long)buf * nb + b) * KP + warp];
#pragma unroll
            for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) hsh[warp] = s;
        }
        __syncthreads();
    };
    // h_0 = <v_0, w>; then one pass per projection a: w -= h_a v_a, and in the same pass the next
    // inner product <v_{a+1}, w> (or <w, w> after the last), taken on the updated entries; the
    // per-entry order of operations is modified Gram-Schmidt's
    {
        double acc = 0.0;
        if (qa)
            for (long r = r0; r < n; r += rs) acc = fma(V[r * K + q], w[r * K + q], acc);
        reduce_all(acc, 0);
    }
    for (int a = 0; a <= j; ++a) {
        const double* va = V + (long)a * vstride;
        const double h = hsh[q];
        if (blockIdx.x == 0 && threadIdx.x < K) st.h1[a * K + threadIdx.x] = hsh[threadIdx.x];
        double acc = 0.0;
        if (qa) {
            if (a < j) {
                const double* vn = va + vstride;
                for (long r = r0; r < n; r += rs) {
                    const double wr = fma(-h, va[r * K + q], w[r * K + q]);
                    w[r * K + q] = wr;
                    acc = fma(vn[r * K + q], wr, acc);
                }
            } else {
                for (long r = r0; r < n; r += rs) {
                    const double wr = fma(-h, va[r * K + q], w[r * K + q]);
                    w[r * K + q] = wr;
                    acc = fma(wr, wr, acc);
                }
            }
        }
        reduce_all(acc, (a + 1) & 1);
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) any = 0;
        __syncthreads();
        if (threadIdx.x < K) {
            const int qq = threadIdx.x;
            bool live;
            arnoldi_col(st, K, j, m, rtol, qq, st.h1 + qq, nullptr, K, sqrt(fmax(hsh[qq], 0.0)), st.g[j * K + qq],
                        st.active[qq] != 0, true, &live);
            if (live) atomicOr(&any, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) *st.any = any;
    }
    grid.sync();
    const double f = qa ? st.f[q] : 0.0;
    if (qa)
        for (long r = r0; r < n; r += rs) w[r * K + q] *= f;
}

// --- Classical Gram-Schmidt with selective reorthogonalization -------------------------------
//
// In exact arithmetic classical and modified Gram-Schmidt give the same Hessenberg column and
// basis vector.  Classical Gram-Schmidt takes all inner products h = V^T w from the same w, so the
// Arnoldi step needs one grid-wide reduction instead of one per projection, with the same count of
// FP64 operations.  Its weakness is the loss of orthogonality when the projection cancels most of
// w; the remedy is a second pass (Daniel, Gragg, Kaufman and Stewart 1976; "twice is enough",
// Giraud, Langou and Rozloznik 2005) taken only for right-hand sides whose norm fell below
// eta ||w||.  The norm after the pass follows from Pythagoras, ||w - V h||^2 = ||w||^2 - ||h||^2;
// the pass itself keeps ||w - V h||^2 >= eta^2 ||w||^2 whenever the formula is used, so it loses
// at most a few units of rounding to cancellation.

constexpr int kCgsGroup = 8;  // inner products accumulated in one pass over a thread's rows
// Second pass when ||w - V h|| < eta ||w||.  The textbook choice 1/sqrt(2) asks for it in nearly
// every step of ILU(0)-FGMRES on the log-normal FV matrices (a step keeps about 0.4 of ||w||, since
// A M^-1 is close to the identity), which doubles the FP64 work; 0.25 asks for it in 2 of 137 steps
// at 128^3 with the same iterations and residuals as modified Gram-Schmidt.
constexpr double kCgsEta = 0.25;

// Block sum of acc[0..G) for each right-hand side: the block's partial for projection a0 + g lands
// in partial[((a0 + g) * nb + block) * KP + q] for g < na.  red is [32][G][KP] shared memory.
// Inside a warp the G sums are reduced by recursive halving: at each of the first H lane bits a lane
// keeps half of its values and adds its partner's copy of that half, so a lane adds 4 + 2 + 1
// values instead of 3 x 8, then the remaining lane bits (those above log2 KP) are summed on the one
// value left.  GB300 issues FP64 additions at the FP64 FMA rate, so this halves the warp's FP64
// instructions per reduction.  The order of the additions is fixed, and every block uses it.
template <int KP, int G>
__device__ __forceinline__ void block_partials(double (&acc)[G], double (*red)[G][KP], int a0, int na,
                                               double* partial, int nb) {
    static_assert(G == 8, "the halving below is written for 8 sums");
    constexpr int LK = KP == 1 ? 0 : KP == 2 ? 1 : KP == 4 ? 2 : KP == 8 ? 3 : 4;
    constexpr int B = 5 - LK;           // lane bits that hold rows of the same right-hand side
    constexpr int H = B < 3 ? B : 3;    // halving steps
    constexpr int R = G >> H;           // values a lane holds after them
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double v[G];
#pragma unroll
    for (int g = 0; g < G; ++g) v[g] = acc[g];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int o = 16 >> h;
        const bool up = (lane & o) != 0;
        const int half = G >> (h + 1);
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const double send = up ? v[i] : v[i + half];
            const double keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = 16 >> H; o >= KP; o >>= 1) {
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    // lane L holds sums g = hb * R + i, hb = its H top lane bits (bit 4 first)
    const int hb = (lane >> (5 - H)) & ((1 << H) - 1);
    if (((lane >> LK) & ((1 << (B - H)) - 1)) == 0) {
#pragma unroll
        for (int i = 0; i < R; ++i) red[warp][hb * R + i][lane & (KP - 1)] = v[i];
    }
    __syncthreads();
    if (threadIdx.x < G * KP) {
        const int g = threadIdx.x / KP, qq = threadIdx.x % KP;
        double s = 0.0;
        for (int wi = 0; wi < kMgsThreads / 32; ++wi) s += red[wi][g][qq];
        if (g < na) partial[((long)(a0 + g) * nb + blockIdx.x) * KP + qq] = s;
    }
    __syncthreads();
}

// One group of NA inner products over this thread's rows: acc[g] += <V_{a0+g}, x>, where index np
// stands for x itself (<x, x>).  NA is exact, so no FMA of the loop is predicated off: GB300's FP64
// pipe spends the same cycles on a warp's FMA whether all of its lanes are on or none.
template <int NA, int KP>
__device__ __forceinline__ void cgs_dots_group(int n, int K, const double* __restrict__ V, long vstride,
                                               const double* x, int np, int a0, double (&acc)[kCgsGroup], long r0,
                                               long rs, int q) {
    for (long r = r0; r < n; r += rs) {
        const double xr = x[r * K + q];
#pragma unroll
        for (int g = 0; g < NA; ++g) {
            const int a = a0 + g;
            const double va = a < np ? __ldg(V + (long)a * vstride + r * K + q) : xr;
            acc[g] = fma(va, xr, acc[g]);
        }
    }
}

// Partials of <V_a, x> for a < np and, at index np, of <x, x>, over this thread's rows (r0 + i rs)
// for its right-hand side q; lanes with `on` false contribute zeros.
template <int KP>
__device__ void cgs_dots(int n, int K, const double* __restrict__ V, long vstride, const double* x, int np,
                         double* partial, int nb, double (*red)[kCgsGroup][KP], long r0, long rs, int q, bool on) {
    constexpr int G = kCgsGroup;
    for (int a0 = 0; a0 <= np; a0 += G) {
        double acc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g] = 0.0;
        const int na = min(G, np + 1 - a0);
        if (on) {
            switch (na) {
                case 1: cgs_dots_group<1, KP>(n, K, V, vstride, x, np, a0, acc, r0, rs, q); break;
                case 2: cgs_dots_group<2, KP>(n, K, V, vstride, x, np, a0, acc, r0, rs, q); break;
                case 3: cgs_dots_group<3, KP>(n, K, V, vstride, x, np, a0, acc, r0, rs, q); break;
                case 4: cgs_dots_group<4, KP>(n, K, V, vstride, x, np, a0, acc, r0, rs, q); break;
                case 5: cgs_dots_group<5, KP>(n, K, V, vstride, x, np, a0, acc, r0, rs, q); break;
                case 6: cgs_dots_group<6, KP>(n, K, V, vstride, x, np, a0, acc, r0, rs, q); break;
                case 7: cgs_dots_group<7, KP>(n, K, V, vstride, x, np, a0, acc, r0, rs, q); break;
                default: cgs_dots_group<8, KP>(n, K, V, vstride, x, np, a0, acc, r0, rs, q); break;
            }
        }
        block_partials<KP, G>(acc, red, a0, na, partial, nb);
    }
}

// hs[a * KP + q] = sum over the nb blocks of partial[a][block][q], a < count, in a fixed order
// that every block repeats exactly (so all blocks hold bitwise the same sums).
template <int KP>
__device__ void cgs_grid_sums(int count, int K, const double* partial, int nb, double* hs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int idx = warp; idx < count * KP; idx += kMgsThreads / 32) {
        const int a = idx / KP, qq = idx % KP;
        double s = 0.0;
        if (qq < K)
            for (int b = lane; b < nb; b += 32) s += partial[((long)a * nb + b) * KP + qq];
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) hs[idx] = s;
    }
    __syncthreads();
}

// One Arnoldi step after w = A z_j as one cooperative persistent launch: h = V^T w and ||w||^2
// (one grid-wide reduction), per right-hand side the choice of a second pass, w -= V h, and for
// the right-hand sides that need it h2 = V^T w, w -= V h2 (a second reduction); the Hessenberg
// column with h (+ h2), the rotations and the convergence test (stored by block 0, computed
// identically by every block), and w /= h_{j+1,j} fused into the last pass.  Dynamic shared
// memory: 2 (j + 2) KP doubles.  partial holds two regions of (m + 2) nb KP doubles.
template <int KP>
__global__ void __launch_bounds__(kMgsThreads) k_arnoldi_cgs(int n, int K, int j, int m, double rtol, double eta2,
                                                          const double* __restrict__ V, long vstride, double* w,
                                                          double* partial, ArnoldiState st) {
    cg::grid_group grid = cg::this_grid();
    constexpr int RPB = kMgsThreads / KP;
    __shared__ double red[kMgsThreads / 32][kCgsGroup][KP];
    __shared__ double psh[KP], fsh[KP];
    __shared__ int resh[KP];
    __shared__ int any;
    extern __shared__ double dyn[];
    const int np = j + 1;
    double* hs = dyn;                          // [(np + 1) * KP]: h_a, then ||w||^2 at index np
    double* h2s = dyn + (size_t)(np + 1) * KP;  // the second pass's
    const int q = threadIdx.x % KP;
    const bool qa = q < K;
    const long r0 = (long)blockIdx.x * RPB + threadIdx.x / KP;
    const long rs = (long)gridDim.x * RPB;
    const int nb = gridDim.x;
    double* part2 = partial + (size_t)(m + 2) * nb * KP;
    // block 0 rewrites g_j and the active flags after the first grid synchronisation
    double gj = 0.0;
    bool act = false;
    if (threadIdx.x < K) {
        gj = st.g[j * K + threadIdx.x];
        act = st.active[threadIdx.x] != 0;
    }
    if (threadIdx.x == 0) any = 0;

    cgs_dots<KP>(n, K, V, vstride, w, np, partial, nb, red, r0, rs, q, qa);
    grid.sync();
    cgs_grid_sums<KP>(np + 1, K, partial, nb, hs);
    if (threadIdx.x < KP) {
        int re = 0;
        double p = 0.0;
        if (threadIdx.x < K) {
            const double s = hs[np * KP + threadIdx.x];
            double hh = 0.0;
            for (int a = 0; a < np; ++a) hh = fma(hs[a * KP + threadIdx.x], hs[a * KP + threadIdx.x], hh);
            p = s - hh;
            re = act && s > 0.0 && p < eta2 * s;
        }
        psh[threadIdx.x] = p;
        resh[threadIdx.x] = re;
    }
    __syncthreads();
    bool second = false;
    for (int qq = 0; qq < K; ++qq) second = second || resh[qq] != 0;
    // the passes below subtract h: keep -h, so that each FMA takes it as it is
    for (int i = threadIdx.x; i < np * KP; i += kMgsThreads) hs[i] = -hs[i];
    __syncthreads();

    if (!second) {
        if (threadIdx.x < K) {
            bool live;
            fsh[threadIdx.x] = arnoldi_col(st, K, j, m, rtol, threadIdx.x, hs + threadIdx.x, nullptr, KP,
                                           sqrt(fmax(psh[threadIdx.x], 0.0)), gj, act, blockIdx.x == 0, &live, true);
            if (live) atomicOr(&any, 1);
        }
        __syncthreads();
        if (blockIdx.x == 0 && threadIdx.x == 0) *st.any = any;
        if (qa) {
            const double f = fsh[q];
            for (long r = r0; r < n; r += rs) {
                double wr = w[r * K + q];
#pragma unroll 4
                for (int a = 0; a < np; ++a) wr = fma(hs[a * KP + q], __ldg(V + (long)a * vstride + r * K + q), wr);
                w[r * K + q] = wr * f;
            }
        }
        return;
    }

    // w -= V h for every right-hand side, then the second pass's inner products where it is needed
    const bool re = qa && resh[q] != 0;
    if (qa)
        for (long r = r0; r < n; r += rs) {
            double wr = w[r * K + q];
#pragma unroll 4
            for (int a = 0; a < np; ++a) wr = fma(hs[a * KP + q], __ldg(V + (long)a * vstride + r * K + q), wr);
            w[r * K + q] = wr;
        }
    cgs_dots<KP>(n, K, V, vstride, w, np, part2, nb, red, r0, rs, q, re);
    grid.sync();
    cgs_grid_sums<KP>(np + 1, K, part2, nb, h2s);
    if (threadIdx.x < K) {
        const int qq = threadIdx.x;
        double hn = sqrt(fmax(psh[qq], 0.0));
        if (resh[qq]) {
            const double s2 = h2s[np * KP + qq];
            double hh = 0.0;
            for (int a = 0; a < np; ++a) hh = fma(h2s[a * KP + qq], h2s[a * KP + qq], hh);
            const double p2 = s2 - hh;
            // a second pass that still cancels most of the vector: w lies in span(V) to working
            // precision (breakdown; the Krylov space is invariant)
            hn = p2 < eta2 * s2 ? 0.0 : sqrt(p2);
        }
        psh[qq] = hn;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < np * KP; i += kMgsThreads) h2s[i] = -h2s[i];
    __syncthreads();
    if (threadIdx.x < K) {
        const int qq = threadIdx.x;
        bool live;
        fsh[qq] = arnoldi_col(st, K, j, m, rtol, qq, hs + qq, resh[qq] ? h2s + qq : nullptr, KP, psh[qq], gj, act,
                              blockIdx.x == 0, &live, true);
        if (live) atomicOr(&any, 1);
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *st.any = any;
        *st.reorth += 1;
    }
    if (qa) {
        const double f = fsh[q];
        for (long r = r0; r < n; r += rs) {
            double wr = w[r * K + q];
            if (re) {
#pragma unroll 4
                for (int a = 0; a < np; ++a) wr = fma(h2s[a * KP + q], __ldg(V + (long)a * vstride + r * K + q), wr);
            }
            w[r * K + q] = wr * f;
        }
    }
}

// y = R^-1 g on each right-hand side's rotated Hessenberg; zero beyond its column count
__global__ void k_backsolve(int K, int m, ArnoldiState st) {
    const int q = threadIdx.x;
    if (q >= K) return;
    const int jj = st.jq[q];
    for (int a = m - 1; a >= jj; --a) st.y[a * K + q] = 0.0;
    for (int a = jj - 1; a >= 0; --a) {
        double s = st.g[a * K + q];
        for (int c = a + 1; c < jj; ++c) s -= st.H[((size_t)a * m + c) * K + q] * st.y[c * K + q];
        const double d = st.H[((size_t)a * m + a) * K + q];
        st.y[a * K + q] = d != 0.0 ? s / d : 0.0;
    }
}

int grid_for(long total) { return (int)std::max(1L, std::min((long)num_sms() * 8, (total + kThreads - 1) / kThreads)); }

struct Dots {
    double* partial = nullptr;
    int nblk = 0;
    hec_status init(int maxcount, int K) {
        nblk = num_sms() * 2;
        return dalloc(&partial, (size_t)maxcount * nblk * K);
    }
    ~Dots() { dfree(partial); }
    template <int KP>
    void run_kp(int n, int K, const double* V, long vstride, int count, int self, const double* w, double* out,
                const int* gate, cudaStream_t s) {
        const int total = count + self;
        dim3 g(nblk, (total + kDotGroup - 1) / kDotGroup);
        {
            ProfScope ps_(s, PROF_GS);
            k_multidot<KP><<<g, kThreads, 0, s>>>(n, K, V, vstride, count, self, w, partial, gate);
        }
        {
            ProfScope ps_(s, PROF_GS);
            k_reduce<<<(total * K * 32 + 255) / 256, 256, 0, s>>>(total, nblk, K, partial, out, gate);
        }
        count_launch(2);
    }
    hec_status run(int n, int K, const double* V, long vstride, int count, int self, const double* w, double* out,
                   const int* gate, cudaStream_t s) {
        if (K <= 1) run_kp<1>(n, K, V, vstride, count, self, w, out, gate, s);
        else if (K <= 2) run_kp<2>(n, K, V, vstride, count, self, w, out, gate, s);
        else if (K <= 4) run_kp<4>(n, K, V, vstride, count, self, w, out, gate, s);
        else if (K <= 8) run_kp<8>(n, K, V, vstride, count, self, w, out, gate, s);
        else run_kp<16>(n, K, V, vstride, count, self, w, out, gate, s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(e, "multidot");
        return HEC_OK;
    }
};

// Launcher of the persistent Arnoldi kernels: grid = resident blocks (cooperative launch).
struct Mgs {
    double* partial = nullptr;
    int cap_blocks = 0;
    int m = 0;
    int mode = HEC_GS_CLASSICAL;
    hec_status init(int restart, int gs_mode) {
        cap_blocks = num_sms() * (2048 / kMgsThreads);
        m = restart;
        mode = gs_mode;
        // MGS: two single-slot buffers; CGS: two regions of (m + 2) projections
        return dalloc(&partial, (size_t)2 * (m + 2) * cap_blocks * 16);
    }
    ~Mgs() { dfree(partial); }
    template <int KP>
    hec_status run_kp(int n, int K, int j, double rtol, const double* V, long vstride, double* w,
                      ArnoldiState& st, cudaStream_t s) {
        const bool cgs = mode == HEC_GS_CLASSICAL;
        const void* k = cgs ? (const void*)k_arnoldi_cgs<KP> : (const void*)k_arnoldi_mgs<KP>;
        // dynamic shared memory of the classical kernel: h and h2 for up to 256 + 2 projections
        const size_t smem_max = cgs ? (size_t)2 * (256 + 2) * KP * sizeof(double) : 0;
        static int per_sm[2] = {-1, -1};  // per template instance and kernel
        int& ps = per_sm[cgs ? 1 : 0];
        if (ps < 0) {
            if (cgs) HEC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
            ps = max_coop_blocks(k, kMgsThreads, smem_max);
        }
        if (ps <= 0) return set_error(HEC_ERR_CUDA, "Arnoldi kernel cannot be resident");
        const long want = ((long)n * KP + kMgsThreads - 1) / kMgsThreads;
        int blocks = (int)std::max(1L, std::min<long>(std::min(ps * num_sms(), cap_blocks), want));
        double* part = partial;
        int mm = m;
        ProfScope ps_(s, PROF_GS);
        if (cgs) {
            double eta2 = kCgsEta * kCgsEta;
            const size_t smem = (size_t)2 * (j + 2) * KP * sizeof(double);
            void* args[] = {&n, &K, &j, &mm, &rtol, &eta2, (void*)&V, &vstride, &w, &part, &st};
            HEC_CUDA(cudaLaunchCooperativeKernel(k, dim3(blocks), dim3(kMgsThreads), args, smem, s));
        } else {
            void* args[] = {&n, &K, &j, &mm, &rtol, (void*)&V, &vstride, &w, &part, &st};
            HEC_CUDA(cudaLaunchCooperativeKernel(k, dim3(blocks), dim3(kMgsThreads), args, 0, s));
        }
        count_launch();
        return HEC_OK;
    }
    hec_status run(int n, int K, int j, double rtol, const double* V, long vstride, double* w,
                   ArnoldiState& st, cudaStream_t s) {
        if (K <= 1) return run_kp<1>(n, K, j, rtol, V, vstride, w, st, s);
        if (K <= 2) return run_kp<2>(n, K, j, rtol, V, vstride, w, st, s);
        if (K <= 4) return run_kp<4>(n, K, j, rtol, V, vstride, w, st, s);
        if (K <= 8) return run_kp<8>(n, K, j, rtol, V, vstride, w, st, s);
        return run_kp<16>(n, K, j, rtol, V, vstride, w, st, s);
    }
};

}  // namespace

hec_status spmv_impl(const hec_matrix* A, int K, double alpha, const double* x, int ldx, double beta, double* y,
                     int ldy, cudaStream_t s) {
    if (A->n == 0) return HEC_OK;
    if (K == 1 && ldx == 1 && ldy == 1 && A->w <= 8) {
        const int mode = beta == 0.0 ? (alpha == 1.0 ? 0 : 1) : 2;
        auto go1 = [&](auto wm, auto md) -> hec_status {
            constexpr int WM = decltype(wm)::value, MD = decltype(md)::value;
            const void* k = (const void*)k_spmv1<WM, MD>;
            static int per_sm = -1;  // per template instance
            if (per_sm < 0) per_sm = max_coop_blocks(k, kThreads, 0);
            const long want = ((long)A->n + kThreads - 1) / kThreads;
            const int blocks = (int)std::max(1L, std::min<long>((long)std::max(per_sm, 1) * num_sms(), want));
            {
                ProfScope ps_(s, PROF_SPMV);
                k_spmv1<WM, MD><<<blocks, kThreads, 0, s>>>(A->n, A->ld, A->w, A->ell_col, (const double*)A->ell_val,
                                                            A->tptr, A->tcol, (const double*)A->tval, alpha, x, beta, y);
            }
            HEC_LAUNCHED();
            return HEC_OK;
        };
        auto by_mode = [&](auto wm) -> hec_status {
            using M0 = std::integral_constant<int, 0>;
            using M1 = std::integral_constant<int, 1>;
            using M2 = std::integral_constant<int, 2>;
            return mode == 0 ? go1(wm, M0()) : mode == 1 ? go1(wm, M1()) : go1(wm, M2());
        };
        switch (A->w) {
            case 0:
            case 1: return by_mode(std::integral_constant<int, 1>());
            case 2: return by_mode(std::integral_constant<int, 2>());
            case 3: return by_mode(std::integral_constant<int, 3>());
            case 4: return by_mode(std::integral_constant<int, 4>());
            case 5: return by_mode(std::integral_constant<int, 5>());
            case 6: return by_mode(std::integral_constant<int, 6>());
            case 7: return by_mode(std::integral_constant<int, 7>());
            default: return by_mode(std::integral_constant<int, 8>());
        }
    }
    auto go = [&](auto kp) -> hec_status {
        constexpr int KP = decltype(kp)::value;
        constexpr int RPT = KP == 1 ? 2 : 1;
        int blocks = (int)(((long)A->n * KP + (long)kThreads * RPT - 1) / ((long)kThreads * RPT));
        {
            ProfScope ps_(s, PROF_SPMV);
            k_spmv<KP, RPT><<<blocks, kThreads, 0, s>>>(A->n, A->ld, A->w, A->ell_col, (const double*)A->ell_val, A->tptr,
                                                   A->tcol, (const double*)A->tval, K, alpha, x, ldx, beta, y, ldy);
        }
        HEC_LAUNCHED();
        return HEC_OK;
    };
    if (K <= 1) return go(std::integral_constant<int, 1>());
    if (K <= 2) return go(std::integral_constant<int, 2>());
    if (K <= 4) return go(std::integral_constant<int, 4>());
    if (K <= 8) return go(std::integral_constant<int, 8>());
    return go(std::integral_constant<int, 16>());
}

// ---- learned correction stage --------------------------------------------------------------
hec_status net_apply_field(hec_net* N, int nx, int ny, int nz, const double* r, const double* sigma,
                           const __nv_bfloat16* aux, double* c, cudaStream_t s);

namespace {
__global__ void k_f64_to_bf16_scaled(long n, const double* __restrict__ a, double scale, __nv_bfloat16* __restrict__ o) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        o[i] = __float2bfloat16_rn((float)(a[i] * scale));
}
constexpr int kStageRpt = 2;  // rows per thread of the stage's matrix products

// The stage's matrix products on one right-hand side: y = b - A x (SUB) or y = A x, plus this
// block's partial sums of y.y and y.u (u may be NULL) in part[block][0..1].  The rows sum as in
// k_spmv.  With SUB the sums (||r1||^2, hence sigma) are FP64; otherwise they only feed the step
// length alpha and its 1 % acceptance test, so they are taken in FP32, which leaves the scarce
// FP64 pipe to the product itself.
template <bool SUB>
__global__ void __launch_bounds__(kThreads, 6) k_spmv_dots(int n, int ld, int w, const int* __restrict__ ell_col,
                                                        const double* __restrict__ ell_val, const int* __restrict__ tptr,
                                                        const int* __restrict__ tcol, const double* __restrict__ tval,
                                                        const double* __restrict__ x, const double* __restrict__ b,
                                                        double* __restrict__ y, const double* __restrict__ u,
                                                        double* __restrict__ part) {
    using T = typename std::conditional<SUB, double, float>::type;
    __shared__ T red[kThreads / 32][2];
    const int rb = blockIdx.x * kThreads * kStageRpt + threadIdx.x;
    double acc[kStageRpt];
    int row[kStageRpt];
#pragma unroll
    for (int i = 0; i < kStageRpt; ++i) {
        acc[i] = 0.0;
        row[i] = rb + i * kThreads < n ? rb + i * kThreads : -1;
    }
#pragma unroll 4
    for (int k = 0; k < w; ++k) {
#pragma unroll
        for (int i = 0; i < kStageRpt; ++i) {
            if (row[i] < 0) continue;
            const long s = (long)k * ld + row[i];
            const int c = __ldg(ell_col + s);
            if (c >= 0) acc[i] = fma(__ldg(ell_val + s), __ldg(x + c), acc[i]);
        }
    }
    T syy = 0, syu = 0;
#pragma unroll
    for (int i = 0; i < kStageRpt; ++i) {
        if (row[i] < 0) continue;
        const int t1 = __ldg(tptr + row[i] + 1);
        for (int t = __ldg(tptr + row[i]); t < t1; ++t) acc[i] = fma(__ldg(tval + t), __ldg(x + __ldg(tcol + t)), acc[i]);
        const double yi = SUB ? b[row[i]] - acc[i] : acc[i];
        y[row[i]] = yi;
        const T yf = (T)yi;
        syy = fma(yf, yf, syy);
        if (u) syu = fma(yf, (T)u[row[i]], syu);
    }
    for (int o = 16; o; o >>= 1) {
        syy += __shfl_xor_sync(0xffffffffu, syy, o);
        syu += __shfl_xor_sync(0xffffffffu, syu, o);
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (lane == 0) {
        red[wp][0] = syy;
        red[wp][1] = syu;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) s += (double)red[i][threadIdx.x];
        part[2 * blockIdx.x + threadIdx.x] = s;
    }
}

// One block: the sums of the nblk partial pairs in a fixed order.  stage 0: scal[1] = ||r1||^2,
// scal[0] = sigma = sqrt(||r1||^2 / n).  stage 1: scal[3] = <Ac, Ac>, scal[2] = <r1, Ac>, then
// the decision: alpha = <r1, Ac> / <Ac, Ac> is kept in scal[4] when alpha > 0 and
// ||r1 - alpha Ac||^2 = ||r1||^2 - alpha <r1, Ac> < rho^2 ||r1||^2, else scal[4] = 0 (fallback).
constexpr int kReduceThreads = 1024;
__global__ void __launch_bounds__(kReduceThreads) k_stage_reduce(int nblk, const double* __restrict__ part, int stage,
                                                                 long n, double rho, double* scal, int* counters) {
    __shared__ double red[kReduceThreads / 32][2];
    double s0 = 0.0, s1 = 0.0;
    for (int b = threadIdx.x; b < nblk; b += kReduceThreads) {
        s0 += part[2 * b];
        s1 += part[2 * b + 1];
    }
    for (int o = 16; o; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = s0;
        red[threadIdx.x >> 5][1] = s1;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double t0 = 0.0, t1 = 0.0;
    for (int i = 0; i < kReduceThreads / 32; ++i) {
        t0 += red[i][0];
        t1 += red[i][1];
    }
    if (stage == 0) {
        scal[1] = t0;
        scal[0] = sqrt(fmax(t0, 0.0) / (double)n);
        return;
    }
    scal[3] = t0;
    scal[2] = t1;
    const double rr = scal[1];
    double coef = 0.0;
    if (t0 > 0.0) {
        const double alpha = t1 / t0;
        const double left = rr - alpha * t1;  // ||r1 - alpha Ac||^2 at the optimal alpha
        if (alpha > 0.0 && left < rho * rho * rr) coef = alpha;
    }
    scal[4] = coef;
    counters[0] += 1;
    if (coef != 0.0) counters[1] += 1;
}

// z = z1 + coef c; and, when Az is given, Az = A z = (v - r1) + coef Ac
__global__ void k_stage_finish(long n, const double* __restrict__ scal, const double* __restrict__ c,
                               const double* __restrict__ v, const double* __restrict__ r1,
                               const double* __restrict__ Ac, double* __restrict__ z, double* __restrict__ Az) {
    const double a = scal[4];
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        if (a != 0.0) z[i] = fma(a, c[i], z[i]);
        if (Az) Az[i] = a != 0.0 ? fma(a, Ac[i], v[i] - r1[i]) : v[i] - r1[i];
    }
}
}  // namespace

}  // namespace hec

// The stage: z = z1 + alpha c, c = sigma * Net([r1 / sigma, aux]), r1 = v - A z1 (z1 = the ILU
// sweep's output); plain z1 whenever the correction does not reduce ||r1|| by the factor rho.
struct hec_stage {
    hec_net* net = nullptr;
    const hec_matrix* A = nullptr;
    int nx = 0, ny = 0, nz = 0;
    double rho = 0.99;
    __nv_bfloat16* aux = nullptr;  // [n] second input channel
    double* work = nullptr;        // [3n]: r1 | Ac | c
    double* scal = nullptr;        // sigma, ||r1||^2, <r1,Ac>, <Ac,Ac>, coef
    int* counters = nullptr;       // applications, accepted corrections
    double* part = nullptr;        // per-block partial sums of the matrix products
};

namespace hec {
int stage_blocks(long n) { return (int)((n + (long)kThreads * kStageRpt - 1) / ((long)kThreads * kStageRpt)); }

// One application; z holds z1 on entry.  When Az is given it receives A z (the product FGMRES
// needs next), assembled from the two products the stage computes anyway.
hec_status stage_run(const hec_stage* S, const double* v, double* z, double* Az, cudaStream_t s) {
    const hec_matrix* A = S->A;
    const int n = A->n;
    double* r1 = S->work;
    double* Ac = S->work + n;
    double* c = S->work + 2 * (long)n;
    const int nb = stage_blocks(n);
    const double* ev = (const double*)A->ell_val;
    const double* tv = (const double*)A->tval;
    {
        ProfScope ps_(s, PROF_SPMV);  // r1 = v - A z1, ||r1||^2, sigma
        k_spmv_dots<true><<<nb, kThreads, 0, s>>>(n, A->ld, A->w, A->ell_col, ev, A->tptr, A->tcol, tv, z, v, r1, nullptr,
                                                  S->part);
        k_stage_reduce<<<1, kReduceThreads, 0, s>>>(nb, S->part, 0, n, S->rho, S->scal, S->counters);
    }
    count_launch(2);
    HEC_CHECK(net_apply_field(S->net, S->nx, S->ny, S->nz, r1, S->scal, S->aux, c, s));  // c = sigma * Net
    {
        ProfScope ps_(s, PROF_SPMV);  // Ac, <Ac, Ac>, <r1, Ac>, alpha and the decision
        k_spmv_dots<false><<<nb, kThreads, 0, s>>>(n, A->ld, A->w, A->ell_col, ev, A->tptr, A->tcol, tv, c, nullptr, Ac,
                                                   r1, S->part);
        k_stage_reduce<<<1, kReduceThreads, 0, s>>>(nb, S->part, 1, n, S->rho, S->scal, S->counters);
    }
    {
        ProfScope ps_(s, PROF_VEC);
        k_stage_finish<<<grid_for(n), kThreads, 0, s>>>(n, S->scal, c, v, r1, Ac, z, Az);
    }
    count_launch(3);
    HEC_CUDA(cudaGetLastError());
    return HEC_OK;
}
}  // namespace hec

using namespace hec;

HEC_API hec_status stage_create(hec_net* net, const hec_matrix* A, int nx, int ny, int nz, const double* aux,
                                double aux_scale, double rho, hec_stage** out) {
    clear_error();
    if (!net || !A || !out || A->tri || A->vdt != HEC_F64 || (long)nx * ny * nz != A->n || !aux || !(rho > 0.0))
        return set_error(HEC_ERR_INVALID_ARG, "stage_create: need the FP64 general-mode A on an nx*ny*nz grid");
    *out = nullptr;
    hec_stage* S = new hec_stage();
    S->net = net;
    S->A = A;
    S->nx = nx;
    S->ny = ny;
    S->nz = nz;
    S->rho = rho;
    const long n = A->n;
    hec_status st = HEC_OK;
    auto fail = [&](hec_status e) {
        dfree(S->aux); dfree(S->work); dfree(S->scal); dfree(S->counters); dfree(S->part);
        delete S;
        return e;
    };
    if ((st = dalloc(&S->aux, (size_t)n)) || (st = dalloc(&S->work, (size_t)3 * n)) || (st = dalloc(&S->scal, 8)) ||
        (st = dalloc(&S->counters, 2)) || (st = dalloc(&S->part, (size_t)2 * stage_blocks(n))))
        return fail(st);
    k_f64_to_bf16_scaled<<<grid_for(n), kThreads>>>(n, aux, aux_scale, S->aux);
    count_launch();
    if (cudaMemset(S->counters, 0, 2 * sizeof(int)) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return fail(cuda_error(cudaGetLastError(), "stage_create"));
    *out = S;
    return HEC_OK;
}

HEC_API hec_status stage_apply(const hec_stage* stage, const double* v, double* z, void* stream) {
    clear_error();
    if (!stage || !v || !z) return set_error(HEC_ERR_INVALID_ARG, "stage_apply: NULL");
    HEC_CHECK(stage_run(stage, v, z, nullptr, S(stream)));
    HEC_CUDA(cudaGetLastError());
    return HEC_OK;
}

HEC_API hec_status stage_stats(const hec_stage* S, int* applied, int* accepted, int reset) {
    if (!S) return set_error(HEC_ERR_INVALID_ARG, "stage_stats: NULL");
    int h[2] = {0, 0};
    HEC_CUDA(cudaMemcpy(h, S->counters, sizeof(h), cudaMemcpyDeviceToHost));
    if (applied) *applied = h[0];
    if (accepted) *accepted = h[1];
    if (reset) HEC_CUDA(cudaMemset(S->counters, 0, sizeof(h)));
    return HEC_OK;
}

HEC_API hec_status stage_destroy(hec_stage* S) {
    if (!S) return HEC_OK;
    dfree(S->aux);
    dfree(S->work);
    dfree(S->scal);
    dfree(S->counters);
    dfree(S->part);
    delete S;
    return HEC_OK;
}

HEC_API hec_status hec_set_gram_schmidt(int mode) {
    clear_error();
    if (mode != HEC_GS_CLASSICAL && mode != HEC_GS_MODIFIED)
        return set_error(HEC_ERR_INVALID_ARG, "hec_set_gram_schmidt: mode must be HEC_GS_CLASSICAL or HEC_GS_MODIFIED");
    g_gs_mode = mode;
    return HEC_OK;
}

HEC_API int hec_get_gram_schmidt(void) { return g_gs_mode; }

HEC_API hec_status spmv(const hec_matrix* A, int nrhs, double alpha, const double* x, int ldx, double beta, double* y,
                        int ldy, void* stream) {
    clear_error();
    if (!A || A->tri || A->vdt != HEC_F64 || nrhs < 1 || nrhs > 16 || ldx < nrhs || ldy < nrhs ||
        (A->n > 0 && (!x || !y)))
        return set_error(HEC_ERR_INVALID_ARG, "spmv: need a general-mode FP64 HEC matrix and 1 <= nrhs <= 16");
    return spmv_impl(A, nrhs, alpha, x, ldx, beta, y, ldy, S(stream));
}

namespace {
// Device and pinned workspace of one fgmres_solve call.
struct FgmresWork {
    double* V = nullptr;       // (m+1) blocks of n x K
    double* Z = nullptr;       // m blocks of n x K
    double* small = nullptr;   // Arnoldi arrays
    int* ints = nullptr;
    ~FgmresWork() {
        dfree(V);
        dfree(Z);
        dfree(small);
        dfree(ints);
    }
};
// Host-side objects of fgmres_solve, kept per thread for the device they were made on: the pinned
// pair of per-iteration "any active" flags and the two events that order their reads
// (cudaHostAlloc / cudaFreeHost cost more than the rest of a solve's host work).
struct FgmresHost {
    int dev = -1;
    int* pinned = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ~FgmresHost() { release(); }
    void release() {
        if (pinned) cudaFreeHost(pinned);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        pinned = nullptr;
        ev[0] = ev[1] = nullptr;
        dev = -1;
        cudaGetLastError();
    }
    hec_status get() {
        int d = 0;
        HEC_CUDA(cudaGetDevice(&d));
        if (d == dev && pinned) return HEC_OK;
        release();
        HEC_CUDA(cudaHostAlloc((void**)&pinned, 2 * sizeof(int), cudaHostAllocDefault));
        HEC_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
        HEC_CUDA(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
        dev = d;
        return HEC_OK;
    }
};
thread_local FgmresHost t_fgmres_host;
}  // namespace

HEC_API hec_status fgmres_solve(const hec_matrix* A, const ilu_precond* M, const hec_stage* extra, int nrhs,
                                const double* b, int ldb, double* x, int ldx, int restart, double rtol, int max_iters,
                                hec_fgmres_info* info, void* stream) {
    clear_error();
    auto t_start = std::chrono::steady_clock::now();
    if (!A || A->tri || A->vdt != HEC_F64 || nrhs < 1 || nrhs > 16 || ldb < nrhs || ldx < nrhs || restart < 1 ||
        restart > 256 || !(rtol > 0) || max_iters < 0 || (M && (M->n_glob != A->n || M->max_nrhs < nrhs)) ||
        (extra && (!M || nrhs != 1 || extra->A->n != A->n)))
        return set_error(HEC_ERR_INVALID_ARG, "fgmres_solve: bad argument (a learned stage needs M and nrhs = 1)");
    cudaStream_t s = S(stream);
    const int n = A->n, K = nrhs, m = restart;
    const long nk = (long)n * K;
    hec_fgmres_info inf{};
    if (n == 0) {
        inf.converged = 1;
        if (info) *info = inf;
        return HEC_OK;
    }
    FgmresWork W;
    Dots dots;
    Mgs mgs;
    const size_t nsmall = (size_t)K * ((size_t)(m + 1) * m + 2 * m + (m + 1) + m + (m + 2) + (m + 1) + 4);
    hec_status st = HEC_OK;
    if ((st = dalloc(&W.V, (size_t)(m + 1) * nk)) || (st = dalloc(&W.Z, (size_t)m * nk)) ||
        (st = dalloc(&W.small, nsmall)) || (st = dalloc(&W.ints, (size_t)2 * K + 2)) || (st = dots.init(m + 2, K)) ||
        (st = mgs.init(m, g_gs_mode)))
        return st;
    FgmresHost& H = t_fgmres_host;
    HEC_CHECK(H.get());
    ArnoldiState as;
    {
        double* p = W.small;
        as.H = p; p += (size_t)(m + 1) * m * K;
        as.cs = p; p += (size_t)m * K;
        as.sn = p; p += (size_t)m * K;
        as.g = p; p += (size_t)(m + 1) * K;
        as.y = p; p += (size_t)m * K;
        as.h1 = p; p += (size_t)(m + 2) * K;
        as.h2 = p; p += (size_t)(m + 1) * K;
        as.n1 = p; p += K;
        as.n2 = p; p += K;
        as.f = p; p += K;
        as.bnorm = p; p += K;
        as.active = W.ints;
        as.jq = W.ints + K;
        as.reorth = W.ints + 2 * K;
        as.any = W.ints + 2 * K + 1;
    }
    HEC_CUDA(cudaMemsetAsync(as.reorth, 0, sizeof(int), s));
    const int gb = grid_for(nk);
    std::vector<double> hb(K), hn(K), g0((size_t)(m + 1) * K), fh(K);
    std::vector<int> act(K), jq(K);
    // ||b||
    {
        ProfScope ps_(s, PROF_VEC);
        k_copy<<<gb, kThreads, 0, s>>>(nk, K, b, ldb, W.V, K);
    }
    count_launch();
    HEC_CHECK(dots.run(n, K, W.V, nk, 0, 1, W.V, as.n1, nullptr, s));
    HEC_CUDA(cudaMemcpyAsync(hb.data(), as.n1, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
    HEC_CUDA(cudaStreamSynchronize(s));
    for (int q = 0; q < K; ++q) hb[q] = std::sqrt(std::max(hb[q], 0.0));
    HEC_CUDA(cudaMemcpyAsync(as.bnorm, hb.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
    int its = 0, restarts = 0;
    double worst = 0.0;
    bool all_conv = false;
    auto check_sweeps = [&]() -> hec_status {
        if (!M) return HEC_OK;
        hec_status a = hec_sync_status(M->L, stream);
        hec_status c = hec_sync_status(M->U, stream);
        hec_status d = extra ? net_sync_status(extra->net, stream) : HEC_OK;
        return a != HEC_OK ? a : c != HEC_OK ? c : d;
    };
    while (true) {
        // r = b - A x; beta = ||r||; v_0 = r / beta (host decides on the restart)
        {
            ProfScope ps_(s, PROF_VEC);
            k_copy<<<gb, kThreads, 0, s>>>(nk, K, b, ldb, W.V, K);
        }
        count_launch();
        HEC_CHECK(spmv_impl(A, K, -1.0, x, ldx, 1.0, W.V, K, s));
        HEC_CHECK(dots.run(n, K, W.V, nk, 0, 1, W.V, as.n1, nullptr, s));
        HEC_CUDA(cudaMemcpyAsync(hn.data(), as.n1, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
        HEC_CUDA(cudaStreamSynchronize(s));
        HEC_CHECK(check_sweeps());
        all_conv = true;
        worst = 0.0;
        std::fill(g0.begin(), g0.end(), 0.0);
        for (int q = 0; q < K; ++q) {
            const double beta = std::sqrt(std::max(hn[q], 0.0));
            const double rel = hb[q] > 0 ? beta / hb[q] : 0.0;
            worst = std::max(worst, rel);
            const bool c = rel <= rtol;
            all_conv = all_conv && c;
            act[q] = c ? 0 : 1;
            fh[q] = beta > 0 ? 1.0 / beta : 0.0;
            g0[q] = beta;
            jq[q] = 0;
        }
        if (all_conv || its >= max_iters) break;
        HEC_CUDA(cudaMemcpyAsync(as.g, g0.data(), sizeof(double) * (m + 1) * K, cudaMemcpyHostToDevice, s));
        HEC_CUDA(cudaMemcpyAsync(as.f, fh.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
        HEC_CUDA(cudaMemcpyAsync(as.active, act.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
        HEC_CUDA(cudaMemcpyAsync(as.jq, jq.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
        {
            ProfScope ps_(s, PROF_VEC);
            k_scale<<<gb, kThreads, 0, s>>>(nk, K, W.V, as.f);
        }
        count_launch();
        const int jlimit = std::min(m, max_iters - its);
        int launched = 0;
        for (int j = 0; j < jlimit; ++j) {
            double* vj = W.V + (long)j * nk;
            double* zj = W.Z + (long)j * nk;
            double* wv = W.V + (long)(j + 1) * nk;
            if (M) {
                HEC_CHECK(ilu_apply(M, K, vj, K, zj, K, stream));
                // a stage on this same matrix also returns w = A z_j
                if (extra) HEC_CHECK(stage_run(extra, vj, zj, extra->A == A ? wv : nullptr, s));
            } else {
                HEC_CUDA(cudaMemcpyAsync(zj, vj, sizeof(double) * nk, cudaMemcpyDeviceToDevice, s));
            }
            if (!extra || extra->A != A) HEC_CHECK(spmv_impl(A, K, 1.0, zj, K, 0.0, wv, K, s));
            // Gram-Schmidt, ||w||, Hessenberg column, rotations, w /= h_{j+1,j}
            HEC_CHECK(mgs.run(n, K, j, rtol, W.V, nk, wv, as, s));
            HEC_CUDA(cudaMemcpyAsync(H.pinned + (j & 1), as.any, sizeof(int), cudaMemcpyDeviceToHost, s));
            HEC_CUDA(cudaEventRecord(H.ev[j & 1], s));
            launched = j + 1;
            // stay at most one iteration ahead: look at the previous iteration's flag
            if (j >= 1) {
                HEC_CUDA(cudaEventSynchronize(H.ev[(j - 1) & 1]));
                if (H.pinned[(j - 1) & 1] == 0) break;  // every right-hand side finished at j-1
            }
        }
        // y = R^-1 g, x += Z y
        {
            ProfScope ps_(s, PROF_ARNOLDI);
            k_backsolve<<<1, 32, 0, s>>>(K, m, as);
        }
        {
            ProfScope ps_(s, PROF_VEC);
            k_update_x<<<gb, kThreads, 0, s>>>(nk, K, W.Z, nk, launched, as.y, x, ldx);
        }
        count_launch(2);
        HEC_CUDA(cudaMemcpyAsync(jq.data(), as.jq, sizeof(int) * K, cudaMemcpyDeviceToHost, s));
        HEC_CUDA(cudaStreamSynchronize(s));
        its += *std::max_element(jq.begin(), jq.end());
        restarts++;
        HEC_CUDA(cudaGetLastError());
    }
    HEC_CHECK(check_sweeps());
    HEC_CUDA(cudaMemcpyAsync(&inf.reorthogonalized, as.reorth, sizeof(int), cudaMemcpyDeviceToHost, s));
    HEC_CUDA(cudaStreamSynchronize(s));
    inf.iterations = its;
    inf.restarts = restarts;
    inf.converged = all_conv ? 1 : 0;
    inf.rel_residual = worst;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (info) *info = inf;
    if (!all_conv) return set_error(HEC_ERR_NOT_CONVERGED, "fgmres_solve: max_iters reached before rtol");
    return HEC_OK;
}
