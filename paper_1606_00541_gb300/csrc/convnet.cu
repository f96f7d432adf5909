// The learned correction network: four 3x3x3 'same' convolutions (2 -> 16 -> 16 -> 16 -> 1
// channels, ReLU between layers), BF16 weights and activations with FP32 accumulation on the
// tensor cores, and its training (backward pass, MSE loss, Adam).  Not part of the paper: it is
// a flexible-preconditioner stage applied after the ILU sweep.
//
// Layout: a field on an nx x ny x nz grid (x fastest) is stored channels-last with 16 BF16
// channels per voxel (32 bytes); unused channels are zero.  Several samples may be stacked along
// z (zs planes each); the convolution treats the sample boundaries as zero padding.
//
// Convolution = implicit GEMM: for each of the 27 taps, D[voxels x 16 out] += X_shifted[voxels x
// 16 in] * W_tap[16 in x 16 out].  The forward pass runs on tcgen05 (k_conv_tc: TMA-fed slabs,
// TMEM accumulators; see there).  The mma.sync path (one m16n8k16, BF16 in, FP32 accumulate, per
// 16 voxels per 8 output channels per tap) serves the backward pass and the forward pass when the
// tensor-core engine is switched off (net_set_engine).  A k_conv forward block computes a
// 32 x 4 x 4 voxel tile from a 34 x 6 x 6 halo tile staged in shared memory together with all 27
// weight taps (the weight-gradient kernel works on 32 x 4 x 1 tiles with a 34 x 6 x 3 halo).  The data gradient is the
// same kernel run with the spatially flipped, channel-transposed weights and the ReLU mask of
// the layer applied while the halo is staged; the weight gradient is a GEMM over voxels with
// per-block partial sums reduced in a fixed order (deterministic).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace hec {
namespace {

constexpr int C = 16;                 // stored channels
constexpr int TX = 32, TY = 4;         // output tile
constexpr int HX = TX + 2, HY = TY + 2, HZ = 3;
constexpr int NTAP = 27;
constexpr int WSZ = NTAP * C * C;      // weights of one layer
constexpr int PSZ = WSZ + C;           // + bias
constexpr int NL = 4;                  // layers
constexpr int kConvThreads = 128;      // 4 warps, one output row (y) each

struct Geom {
    int nx, ny, nz, zs;  // grid; samples of zs planes stacked along z
};

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// zero the channels whose mask value is not positive (ReLU derivative)
__device__ __forceinline__ uint4 apply_mask(uint4 v, uint4 m) {
    unsigned* pv = (unsigned*)&v;
    const unsigned* pm = (const unsigned*)&m;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float m0 = __uint_as_float(pm[i] << 16), m1 = __uint_as_float(pm[i] & 0xFFFF0000u);
        unsigned keep = (m0 > 0.f ? 0x0000FFFFu : 0u) | (m1 > 0.f ? 0xFFFF0000u : 0u);
        pv[i] &= keep;
    }
    return v;
}

// Stage the 34 x 6 x 3 halo of tile (bx, by, bz) into shared memory (zero outside the grid or the
// sample), masked by `mask` when given.
__device__ __forceinline__ void load_halo(const Geom& g, const __nv_bfloat16* __restrict__ X,
                                          const __nv_bfloat16* __restrict__ mask, int bx, int by, int bz,
                                          __nv_bfloat16 (*sx)[HY][HX][C]) {
    const int sample = bz / g.zs, zl = bz - sample * g.zs;
    for (int i = threadIdx.x; i < HZ * HY * HX * 2; i += blockDim.x) {
        const int v = i >> 1, half = i & 1;
        const int hx = v % HX, hy = (v / HX) % HY, hz = v / (HX * HY);
        const int x = bx + hx - 1, y = by + hy - 1, z = zl + hz - 1;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.zs) {
            const long gi = (((long)sample * g.zs + z) * g.ny + y) * g.nx + x;
            val = __ldg((const uint4*)X + gi * 2 + half);
            if (mask) val = apply_mask(val, __ldg((const uint4*)mask + gi * 2 + half));
        }
        ((uint4*)&sx[0][0][0][0])[v * 2 + half] = val;
    }
}

// ---- forward / data-gradient convolution ----------------------------------------------------
// A block computes a 32 (x) x 4 (y) x 4 (z) output tile with 4 warps, warp w owning the z-plane w
// of the tile (32 x 4 voxels = 2 m-tiles x 4 rows).  The 34 x 6 x 6 input halo and the weight
// taps are staged in shared memory with cp.async.  Each 16-voxel A fragment of halo row (y', z')
// shifted by dx is loaded once (ldmatrix) and multiplied into the (up to) three output rows that
// read it through dy = 0, 1, 2, so every ldmatrix.x4 of A feeds 4 mma per n-tile.
// Rows of 32 bytes (one voxel, or one output channel of a weight tap) are stored with their two
// 16-byte halves swapped when bit 2 of the row index is set; any 8 consecutive rows then hit 8
// distinct bank quads and ldmatrix runs without conflicts.
constexpr int FX = 32, FY = 4, FZ = 4;                 // output tile of the forward kernel
constexpr int GX = FX + 2, GY = FY + 2, GZ = FZ + 2;   // its input halo
constexpr int kHaloBytes = GX * GY * GZ * 32;
constexpr int kFwdSmem = kHaloBytes + NTAP * C * C * 2;

__device__ __forceinline__ unsigned swz(unsigned row, unsigned half) { return row * 32u + ((half ^ ((row >> 2) & 1u)) << 4); }

__device__ __forceinline__ void cp_async16(unsigned dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], unsigned addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(unsigned& r0, unsigned& r1, unsigned addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}

// Modes of k_conv: PLAIN (16 -> NT*8 channels, 27 taps), MASKED (the input is multiplied by the
// ReLU mask of the layer while it is staged: the data-gradient pass), EXPAND (the first layer:
// only input channels 0 and 1 are read, and the halo entry at x holds channels 0-1 of the voxels
// x-1, x, x+1 in its slots 0-5, so the three dx taps become one K = 16 product and the layer
// takes 9 taps, with weights from k_weights' Wx).
enum ConvMode { PLAIN = 0, MASKED = 1, EXPAND = 2 };

// Input of k_conv: the 16-channel field X (ReLU mask for MASKED), or, for EXPAND with r given,
// the two input channels straight from the solver's vectors: channel 0 = BF16(r / sigma)
// (0 when sigma is not positive), channel 1 = aux.
struct ConvIn {
    const __nv_bfloat16* X;
    const __nv_bfloat16* mask;
    const double* r;
    const double* sigma;
    const __nv_bfloat16* aux;
};
// Outputs: Y (16-channel BF16, optional), Y0 = channel 0 in FP32 times y0_scale (optional),
// Yd = channel 0 times *yd_scale in FP64 (optional; channel 0 is first rounded to FP32).
struct ConvOut {
    __nv_bfloat16* Y;
    float* Y0;
    float y0_scale;
    double* Yd;
    const double* yd_scale;
};

// Y = conv(X, W) + bias, optional ReLU.  W is [taps][16 out][16 in] BF16.  With NT = 1 only
// output channels 0-7 are computed and channels 8-15 of Y are written as zeros (the last layer
// has one output channel).
template <int MODE, int NT>
__global__ void __launch_bounds__(kConvThreads, 4)
    k_conv(Geom g, int ztiles, ConvIn in, const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias, int relu,
           ConvOut out) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int ntap = MODE == EXPAND ? 9 : NTAP;
    const unsigned sx = (unsigned)__cvta_generic_to_shared(smem);
    const unsigned sw = sx + kHaloBytes;
    const int x0 = blockIdx.x * FX, y0 = blockIdx.y * FY;
    const int sample = blockIdx.z / ztiles, zl0 = (blockIdx.z - sample * ztiles) * FZ;
    const long sbase = (long)sample * g.zs;
    const __nv_bfloat16* __restrict__ X = in.X;
    // weights: row = tap * 16 + out channel, two 16-byte halves of input channels
    for (int i = threadIdx.x; i < ntap * C * 2; i += kConvThreads)
        cp_async16(sw + swz(i >> 1, i & 1), W + (long)i * 8, 16);
    if constexpr (MODE == EXPAND) {
        // 1) channels 0-1 of the voxels x0 - 2 .. x0 + 33 of every halo row, packed in one word
        constexpr int RX = GX + 2;
        unsigned* raw = (unsigned*)(smem + kHaloBytes + 9 * C * C * 2);
        double inv = 0.0;
        if (in.r) inv = *in.sigma > 0.0 ? 1.0 / *in.sigma : 0.0;
        for (int i = threadIdx.x; i < RX * GY * GZ; i += kConvThreads) {
            const int rx = i % RX, hy = (i / RX) % GY, hz = i / (RX * GY);
            const int x = x0 + rx - 2, y = y0 + hy - 1, z = zl0 + hz - 1;
            unsigned word = 0u;
            if (x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.zs) {
                const long gi = ((sbase + z) * g.ny + y) * g.nx + x;
                if (in.r)
                    word = pack2(__float2bfloat16_rn((float)(__ldg(in.r + gi) * inv)), in.aux[gi]);
                else
                    word = __ldg((const unsigned*)(X + gi * C));
            }
            raw[i] = word;
        }
        __syncthreads();
        // 2) the expanded halo entries
        for (int v = threadIdx.x; v < GX * GY * GZ; v += kConvThreads) {
            const int hx = v % GX, hyz = v / GX;
            const unsigned* rr = raw + hyz * RX + hx;
            asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(sx + swz(v, 0)), "r"(rr[0]), "r"(rr[1]), "r"(rr[2]),
                         "r"(0u));
            asm volatile("st.shared.v4.u32 [%0], {%1,%1,%1,%1};" ::"r"(sx + swz(v, 1)), "r"(0u));
        }
    } else {
        for (int i = threadIdx.x; i < GX * GY * GZ * 2; i += kConvThreads) {
            const int v = i >> 1, half = i & 1;
            const int hx = v % GX, hy = (v / GX) % GY, hz = v / (GX * GY);
            const int x = x0 + hx - 1, y = y0 + hy - 1, z = zl0 + hz - 1;
            const bool inb = x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.zs;
            const long gi = inb ? ((sbase + z) * g.ny + y) * g.nx + x : 0;
            if constexpr (MODE == MASKED) {
                uint4 val = make_uint4(0, 0, 0, 0);
                if (inb) val = apply_mask(__ldg((const uint4*)X + gi * 2 + half), __ldg((const uint4*)in.mask + gi * 2 + half));
                asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(sx + swz(v, half)), "r"(val.x), "r"(val.y),
                             "r"(val.z), "r"(val.w));
            } else {
                cp_async16(sx + swz(v, half), X + gi * C + half * 8, inb ? 16 : 0);
            }
        }
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int zl = zl0 + w;
    if (zl >= g.zs) return;  // no barrier follows
    const int gq = lane >> 2, t = lane & 3;
    // ldmatrix row addresses: lane l gives row (l & 7) of matrix (l >> 3)
    const int lr = lane & 7, lm = lane >> 3;
    const int a_off = lr + (lm & 1) * 8, a_half = lm >> 1;  // A: voxel offset, channel half
    const int b_row = lr + (lm >> 1) * 8, b_half = lm & 1;  // B: output channel, input-channel half

    float acc[FY][2][NT][4];
#pragma unroll
    for (int a = 0; a < FY; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < NT; ++c)
#pragma unroll
                for (int d = 0; d < 4; ++d) acc[a][b][c][d] = 0.f;

#pragma unroll
    for (int dz = 0; dz < 3; ++dz) {
#pragma unroll
        for (int dxi = 0; dxi < (MODE == EXPAND ? 1 : 3); ++dxi) {
            const int dx = MODE == EXPAND ? 1 : dxi;
            unsigned bf[3][NT][2];
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const int tap = MODE == EXPAND ? dz * 3 + dy : (dz * 3 + dy) * 3 + dx;
                const unsigned row = tap * C + b_row;
                if constexpr (NT == 2) {
                    unsigned r[4];
                    ldsm_x4(r, sw + swz(row, b_half));
                    bf[dy][0][0] = r[0];
                    bf[dy][0][1] = r[1];
                    bf[dy][1][0] = r[2];
                    bf[dy][1][1] = r[3];
                } else {
                    ldsm_x2(bf[dy][0][0], bf[dy][0][1], sw + swz(tap * C + lr, lm & 1));
                }
            }
#pragma unroll
            for (int yi = 0; yi < GY; ++yi) {
                unsigned af[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const unsigned v = ((w + dz) * GY + yi) * GX + mt * 16 + dx + a_off;
                    ldsm_x4(af[mt], sx + swz(v, a_half));
                }
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) {
                    const int ly = yi - dy;
                    if (ly < 0 || ly >= FY) continue;
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                        for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[ly][mt][nt], af[mt], bf[dy][nt]);
                }
            }
        }
    }

#pragma unroll
    for (int ly = 0; ly < FY; ++ly) {
        const int y = y0 + ly;
        if (y >= g.ny) break;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int x = x0 + mt * 16 + gq + half * 8;
                if (x >= g.nx) continue;
                const long vox = ((sbase + zl) * g.ny + y) * g.nx + x;
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const int co = nt * 8 + 2 * t;
                    float v0 = acc[ly][mt][nt][half * 2 + 0], v1 = acc[ly][mt][nt][half * 2 + 1];
                    if (bias) {
                        v0 += bias[co];
                        v1 += bias[co + 1];
                    }
                    if (relu) {
                        v0 = fmaxf(v0, 0.f);
                        v1 = fmaxf(v1, 0.f);
                    }
                    if (out.Y) {
                        *(unsigned*)&out.Y[vox * C + co] = pack2(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
                        if (NT == 1) *(unsigned*)&out.Y[vox * C + co + 8] = 0u;
                    }
                    if (co == 0) {
                        if (out.Y0) out.Y0[vox] = v0 * out.y0_scale;
                        if (out.Yd) out.Yd[vox] = *out.yd_scale * (double)(v0 * out.y0_scale);
                    }
                }
            }
        }
    }
}

// ---- the 16 -> 16 (and 16 -> 1) forward convolution on the 5th-generation tensor cores ---------
// Implicit GEMM with tcgen05.mma (kind::f16: BF16 operands, FP32 accumulators in tensor memory),
// streamed along z.  A work item is a strip of output voxels 128 (x) x TCY (y) x up to TCZ (z);
// the CTA walks the item's input planes z0-1 .. z0+zc.  One input plane's slab (its TCY+2 rows of
// 130 voxels, x0-1 .. x0+128, 32 bytes each) is brought into shared memory by one TMA load
// (voxels outside the grid or the sample read as zeros) and multiplied, for every output row y and tap (dy, dx), by the three dz taps at once: one MMA of
// M = 128 voxels, N = 48 = 3 dz x 16 output channels, K = 16 input channels whose three 16-column
// groups land in the accumulators of output planes z_in+1, z_in, z_in-1.  The accumulators of an
// item's planes sit in TMEM in descending z order (per output row), so those three are
// contiguous; at the ends of the chunk N drops to 32 or 16.  Each input voxel row is therefore
// read by 9 MMAs per output row instead of 27.
//   Operand layout (K-major): A's rows are the slab's voxels, 32 bytes (16 channels) each, in the
// 32-byte swizzle the TMA load writes (the two 16-byte halves of a row swapped where bit 7 of its
// shared-memory address is set; 8-row groups 256 bytes apart).  The swizzle follows the absolute
// address, so a tap's shift (dy rows of 130 voxels, dx voxels) is an offset of the start address.
// B for tap (dy, dx), unswizzled: rows dz*16 + co (16 bytes apart), its channel halves 768 bytes
// apart.
//   Warp roles: warp 4 issues the TMA loads into a ring of TC_RING slabs, warp 5 issues the MMAs
// (one thread), warps 0-3 drain finished planes (warp w reads TMEM lanes 32w .. 32w+31, i.e.
// voxels x0 + 32w ..), add the bias, apply the ReLU, round to BF16 and zero the accumulator for
// its next use.  mbarriers link the roles: slab full (TMA bytes) / slab free (MMA commit), plane
// finished (MMA commit) / plane drained (the four epilogue warps).  Every wait is bounded: one
// that runs out sets the kernel's abort flag and the status word, all roles leave their loops,
// the loads and MMAs already issued are waited for (bounded) and the TMEM is freed.
constexpr int TCX = 128, TCY = 2, TCZ = 8, TC_RING = 5;
constexpr int TC_HX = TCX + 2, TC_HY = TCY + 2;
constexpr int TC_WBLK = 3 * C * C * 2;                     // B of one (dy, dx): 48 rows x 16 channels
constexpr int TC_COLS = TCY * TCZ * 16;                    // 256 TMEM columns per CTA
// per variant (EXP = 0: 16 input channels, TMA slabs of 130 voxels per row; EXP = 1: the first
// layer, slabs of 128 x-expanded voxels per row built by four producer warps)
constexpr int tc_slab(int exp) { return TC_HY * (exp ? TCX : TC_HX) * 32; }  // 16,384 / 16,640 bytes
constexpr int tc_sstr(int exp) { return (tc_slab(exp) + 1023) / 1024 * 1024; }  // 1024-byte aligned slabs
constexpr int tc_nblk(int exp) { return exp ? 3 : 9; }                      // B blocks: dy, or (dy, dx)
constexpr int TC_RAWR = 6, TC_RAWX = 132;                 // first layer: raw word rows, 6 planes deep
constexpr int TC_RAWB = TC_HY * TC_RAWX * 4;               // one plane's raw rows: 2,112 bytes
constexpr int tc_smem(int exp) {                           // 99,200 / 100,864 bytes
    return TC_RING * tc_sstr(exp) + tc_nblk(exp) * TC_WBLK + (exp ? TC_RAWR * TC_RAWB : 0);
}
constexpr int tc_pwarps(int exp) { return exp ? 4 : 1; }                    // producer warps
constexpr int tc_threads(int exp) { return 32 * (5 + tc_pwarps(exp)); }     // + 4 epilogue warps + 1 MMA warp
constexpr long long kTcWaitBudget = 2000000000LL;          // clock cycles (about 1 s)

// shared-memory matrix descriptors (version 1, base offset 0).  tc_desc: K-major, no swizzle,
// 8-row groups 128 bytes apart, the two 8-element halves of K `lbo` bytes apart.  tc_desc_sw32:
// K-major, 32-byte swizzle (mode 6), rows of 32 bytes, 8-row groups 256 bytes apart.
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((128u >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ unsigned long long tc_desc_sw32(unsigned addr) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | (1ull << 16) | ((unsigned long long)(256u >> 4) << 32) |
           (1ull << 46) | (6ull << 61);
}
__device__ __forceinline__ bool mbar_try(unsigned mb, unsigned parity) {
    unsigned ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(mb), "r"(parity) : "memory");
    return ok != 0;
}
// wait for the phase of parity `parity`; false when the budget ran out (sets *abort) or another
// role aborted
__device__ __forceinline__ bool mbar_wait(unsigned mb, unsigned parity, volatile int* abort) {
    const long long t0 = clock64();
    for (unsigned it = 0;; ++it) {
        if (mbar_try(mb, parity)) return true;
        if ((it & 63u) == 63u) {
            if (*abort) return false;
            if (clock64() - t0 > kTcWaitBudget) {
                *abort = 1;
                return false;
            }
        }
    }
}
// the same wait on the way out: ignores the abort flag, gives up after the budget
__device__ __forceinline__ void mbar_drain(unsigned mb, unsigned parity) {
    const long long t0 = clock64();
    for (unsigned it = 0; !mbar_try(mb, parity); ++it)
        if ((it & 63u) == 63u && clock64() - t0 > kTcWaitBudget) return;
}
__device__ __forceinline__ void tc_commit(unsigned mb) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
}

struct TcItem {
    int x0, y0, z0, zc, sample;
};
// item i: x tile fastest, then y strip, z chunk (zl planes, zl <= TCZ) and sample
__device__ __forceinline__ TcItem tc_item(int i, int xt, int yt, int zt, int zl, int zs) {
    TcItem t;
    t.x0 = (i % xt) * TCX;
    i /= xt;
    t.y0 = (i % yt) * TCY;
    i /= yt;
    t.z0 = (i % zt) * zl;
    t.sample = i / zt;
    t.zc = min(zl, zs - t.z0);
    return t;
}

template <int NT, int EXP>
__global__ void __launch_bounds__(tc_threads(EXP), 2)
    k_conv_tc(Geom g, int xt, int yt, int zt, int zl, int nitems, const __grid_constant__ CUtensorMap tmap, ConvIn in,
              int wstride,
              const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias, int relu, ConvOut out, int* status) {
    constexpr int SSTR = tc_sstr(EXP), NBLK = tc_nblk(EXP), NTHR = tc_threads(EXP), PW = tc_pwarps(EXP);
    constexpr int MMA_WARP = 4 + PW;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bar_full[TC_RING], bar_free[TC_RING], bar_done[TCZ], bar_drained[TCZ],
        bar_fin;
    __shared__ unsigned tmem_slot;
    __shared__ int abort_flag;
    volatile int* abort = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned sh = (unsigned)__cvta_generic_to_shared(smem);
    const unsigned sw = sh + TC_RING * SSTR;
    auto bar = [](unsigned long long* b) { return (unsigned)__cvta_generic_to_shared(b); };

    // B blocks: j = (dy, dx) (dy for EXP), row n = dz*16 + co, half h -> sw + j*1536 + h*768 + n*16.
    // W is [27 taps][co][ci], or for EXP [9 (dz, dy)][co][slot = 2 dx + ci]
    for (int i = tid; i < NBLK * 48 * 2; i += NTHR) {
        const int h = i & 1, n = (i >> 1) % 48, j = (i >> 1) / 48;
        const int tap = (n >> 4) * NBLK + j, co = n & 15;
        cp_async16(sw + j * TC_WBLK + h * (TC_WBLK / 2) + n * 16, W + ((long)tap * C + co) * C + h * 8, 16);
    }
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < TC_RING; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(&bar_full[s])), "n"(EXP ? 32 * PW : 1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(&bar_free[s])));
        }
        for (int k = 0; k < TCZ; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(&bar_done[k])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(bar(&bar_drained[k])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(&bar_fin)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(&tmem_slot)),
                     "n"(TC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the tensor cores read the B blocks
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_slot;
    if (warp < 4) {
        // all accumulators start at zero; the MMAs always accumulate
        const unsigned z = 0u;
        for (int c = 0; c < TC_COLS; c += 16)
            asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};"
                         ::"r"(tmem + ((unsigned)(warp * 32) << 16) + c), "r"(z) : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (warp >= 4 && warp < 4 + PW) {
        if constexpr (EXP == 0) {
            // ---- TMA producer ----
            if (lane == 0) {
                int it = 0;
                const unsigned long long tm = reinterpret_cast<unsigned long long>(&tmap);
                for (int i = blockIdx.x; i < nitems && !*abort; i += gridDim.x) {
                    const TcItem t = tc_item(i, xt, yt, zt, zl, g.zs);
                    for (int p = 0; p <= t.zc + 1; ++p, ++it) {
                        const int s = it % TC_RING, use = it / TC_RING;
                        if (use > 0 && !mbar_wait(bar(&bar_free[s]), (use - 1) & 1, abort)) break;
                        const unsigned fb = bar(&bar_full[s]);
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "n"(tc_slab(0))
                                     : "memory");
                        asm volatile(
                            "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                            "%3, %4, %5, %6}], [%7];" ::"r"(sh + s * SSTR), "l"(tm), "r"(0), "r"(t.x0 - 1), "r"(t.y0 - 1),
                            "r"(t.z0 - 1 + p), "r"(t.sample), "r"(fb)
                            : "memory");
                    }
                    if (*abort) break;
                }
                // the loads already issued land before the CTA ends (each slab's last fill)
                for (int k = it - 1; k >= 0 && k >= it - TC_RING; --k)
                    mbar_drain(bar(&bar_full[k % TC_RING]), (k / TC_RING) & 1);
            }
        } else {
            // ---- first layer: four warps build the x-expanded slab.  The source is one 32-bit word per
            // voxel holding channels 0-1 (in.X with a stride of wstride words).  Its rows x0-1 ..
            // x0+128 of the next TC_RAWR-1 planes are in flight in a ring of raw rows (cp.async, zeros
            // outside the grid or the sample); row e = hr * 128 + m of the slab then gets, for voxel
            // x0 + m of halo row hr, the words of x-1, x, x+1 in slots 0-5, in the 32-byte swizzle the
            // MMAs read.  The four warps step together (named barrier 1); a stop decided by thread 0
            // from the abort flag is read by all of them after the barrier.
            __shared__ int prod_stop[2];
            const int m = tid - 128;
            const unsigned raw = sw + NBLK * TC_WBLK;
            const unsigned* __restrict__ src = (const unsigned*)in.X;
            int fi = blockIdx.x, fp = 0, nf = 0;  // fetch cursor: item, plane, planes fetched
            TcItem ft{};
            if (fi < nitems) ft = tc_item(fi, xt, yt, zt, zl, g.zs);
            auto fetch = [&]() {
                if (fi < nitems) {
                    const unsigned base = raw + (nf % TC_RAWR) * TC_RAWB;
                    const long sbase = (long)ft.sample * g.zs;
                    const int z = ft.z0 - 1 + fp;
                    for (int e = m; e < TC_HY * (TCX + 2); e += 32 * PW) {
                        const int hr = e / (TCX + 2), j = e % (TCX + 2), x = ft.x0 - 1 + j, y = ft.y0 - 1 + hr;
                        const bool inb = x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.zs;
                        const unsigned* a = inb ? src + (((sbase + z) * g.ny + y) * g.nx + x) * wstride : src;
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(base + (hr * TC_RAWX + j) * 4),
                                     "l"(a), "r"(inb ? 4 : 0)
                                     : "memory");
                    }
                    ++nf;
                    if (++fp > ft.zc + 1) {
                        fp = 0;
                        fi += gridDim.x;
                        if (fi < nitems) ft = tc_item(fi, xt, yt, zt, zl, g.zs);
                    }
                }
                asm volatile("cp.async.commit_group;" ::: "memory");  // one group per call, empty or not
            };
            for (int k = 0; k < TC_RAWR - 1; ++k) fetch();
            int i = blockIdx.x, p = 0, q = 0;  // convert cursor: item, plane, planes converted
            TcItem t{};
            if (i < nitems) t = tc_item(i, xt, yt, zt, zl, g.zs);
            while (i < nitems) {
                if (m == 0) prod_stop[q & 1] = *abort;
                asm volatile("bar.sync 1, %0;" ::"n"(32 * PW) : "memory");  // plane q-1's raw rows are free
                if (prod_stop[q & 1]) break;
                fetch();                                                     // plane q + TC_RAWR - 1
                asm volatile("cp.async.wait_group %0;" ::"n"(TC_RAWR - 1) : "memory");
                asm volatile("bar.sync 1, %0;" ::"n"(32 * PW) : "memory");  // plane q's raw rows landed
                const int s = q % TC_RING, use = q / TC_RING;
                if (use > 0) mbar_wait(bar(&bar_free[s]), (use - 1) & 1, abort);  // a timeout stops us next plane
                const unsigned rb = raw + (q % TC_RAWR) * TC_RAWB;
#pragma unroll
                for (int hr = 0; hr < TC_HY; ++hr) {
                    unsigned w0, w1, w2;
                    const unsigned ra = rb + (hr * TC_RAWX + m) * 4;
                    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(w0) : "r"(ra));
                    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(w1) : "r"(ra + 4));
                    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(w2) : "r"(ra + 8));
                    const int e = hr * TCX + m;
                    const unsigned sa = sh + s * SSTR + e * 32, sw_bit = ((unsigned)e >> 2) & 1u;
                    asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(sa + (sw_bit << 4)), "r"(w0), "r"(w1),
                                 "r"(w2), "r"(0u));
                    asm volatile("st.shared.v4.u32 [%0], {%1,%1,%1,%1};" ::"r"(sa + ((sw_bit ^ 1u) << 4)), "r"(0u));
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(&bar_full[s])) : "memory");
                ++q;
                if (++p > t.zc + 1) {
                    p = 0;
                    i += gridDim.x;
                    if (i < nitems) t = tc_item(i, xt, yt, zt, zl, g.zs);
                }
            }
            asm volatile("cp.async.wait_all;" ::: "memory");  // no copy lands after the CTA ends
        }
    } else if (warp == MMA_WARP) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const unsigned base_idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TCX >> 4) << 24);
            unsigned used = 0, wpar = 0;  // per accumulator plane: used by an earlier item, next drained parity
            int it = 0;
            bool issued = false;
            for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
                const TcItem t = tc_item(i, xt, yt, zt, zl, g.zs);
                bool ok = true;
                for (int p = 0; p <= t.zc + 1 && ok; ++p, ++it) {
                    const int s = it % TC_RING;
                    if (!mbar_wait(bar(&bar_full[s]), (it / TC_RING) & 1, abort)) { ok = false; break; }
                    if (p < t.zc && ((used >> p) & 1u)) {  // plane p is written first now: drained?
                        if (!mbar_wait(bar(&bar_drained[p]), (wpar >> p) & 1u, abort)) { ok = false; break; }
                        wpar ^= 1u << p;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int dz_lo = max(0, p - t.zc + 1), dz_hi = min(2, p);
                    const int nn = (dz_hi - dz_lo + 1) * 16;
                    const unsigned idesc = base_idesc | ((unsigned)(nn >> 3) << 17);
                    const int kcol = (TCZ - 1 - (p - dz_lo)) * 16;  // first column: plane p - dz_lo
                    const unsigned slab = sh + s * SSTR;
#pragma unroll
                    for (int y = 0; y < TCY; ++y)
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                            for (int dx = 0; dx < 3 - 2 * EXP; ++dx) {
                                // EXP: the three dx taps are in K; the A row of voxel x0 + m is row m
                                const unsigned long long ad =
                                    tc_desc_sw32(slab + (EXP ? (y + dy) * TCX : (y + dy) * TC_HX + dx) * 32);
                                const unsigned long long bd =
                                    tc_desc(sw + (EXP ? dy : dy * 3 + dx) * TC_WBLK + dz_lo * 256, TC_WBLK / 2);
                                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, 1, 0;\n"
                                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                             ::"r"(tmem + y * (TCZ * 16) + kcol), "l"(ad), "l"(bd), "r"(idesc));
                            }
                    issued = true;
                    tc_commit(bar(&bar_free[s]));                 // the slab may be refilled once these finish
                    if (p >= 2) tc_commit(bar(&bar_done[p - 2]));  // plane p-2 has all its contributions
                    if (p < t.zc) used |= 1u << p;
                }
                if (!ok) break;
            }
            if (issued) {  // every MMA issued has finished before the TMEM is freed
                tc_commit(bar(&bar_fin));
                mbar_drain(bar(&bar_fin), 0);
            }
        }
    } else {
        // ---- epilogue: warps 0-3 ----
        float bv[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) bv[c] = bias ? bias[c] : 0.f;
        unsigned dpar = 0;
        const unsigned lane_base = tmem + ((unsigned)(warp * 32) << 16);
        bool ok = true;
        for (int i = blockIdx.x; i < nitems && ok; i += gridDim.x) {
            const TcItem t = tc_item(i, xt, yt, zt, zl, g.zs);
            const int x = t.x0 + warp * 32 + lane;
            for (int k = 0; k < t.zc; ++k) {
                ok = __all_sync(0xffffffffu, mbar_wait(bar(&bar_done[k]), (dpar >> k) & 1u, abort));
                if (!ok) break;
                dpar ^= 1u << k;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int z = t.z0 + k;
#pragma unroll
                for (int y = 0; y < TCY; ++y) {
                    const unsigned ta = lane_base + y * (TCZ * 16) + (TCZ - 1 - k) * 16;
                    unsigned r[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                        : "r"(ta));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    const unsigned zr = 0u;
                    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};"
                                 ::"r"(ta), "r"(zr) : "memory");
                    const int yy = t.y0 + y;
                    if (x >= g.nx || yy >= g.ny) continue;
                    const long vox = (((long)t.sample * g.zs + z) * g.ny + yy) * g.nx + x;
                    float v[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        v[c] = __uint_as_float(r[c]) + bv[c];
                        if (relu) v[c] = fmaxf(v[c], 0.f);
                    }
                    if (out.Y) {
                        uint4 lo, hi = make_uint4(0u, 0u, 0u, 0u);  // one output channel: channels 8-15 stored as zeros
                        lo.x = pack2(__float2bfloat16_rn(v[0]), __float2bfloat16_rn(v[1]));
                        lo.y = pack2(__float2bfloat16_rn(v[2]), __float2bfloat16_rn(v[3]));
                        lo.z = pack2(__float2bfloat16_rn(v[4]), __float2bfloat16_rn(v[5]));
                        lo.w = pack2(__float2bfloat16_rn(v[6]), __float2bfloat16_rn(v[7]));
                        if (NT == 2) {
                            hi.x = pack2(__float2bfloat16_rn(v[8]), __float2bfloat16_rn(v[9]));
                            hi.y = pack2(__float2bfloat16_rn(v[10]), __float2bfloat16_rn(v[11]));
                            hi.z = pack2(__float2bfloat16_rn(v[12]), __float2bfloat16_rn(v[13]));
                            hi.w = pack2(__float2bfloat16_rn(v[14]), __float2bfloat16_rn(v[15]));
                        }
                        ((uint4*)(out.Y + vox * C))[0] = lo;
                        ((uint4*)(out.Y + vox * C))[1] = hi;
                    }
                    if (out.Y0) out.Y0[vox] = v[0] * out.y0_scale;
                    if (out.Yd) out.Yd[vox] = *out.yd_scale * (double)(v[0] * out.y0_scale);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(&bar_drained[k])) : "memory");
            }
        }
    }
    if (*abort && tid == 0 && status) atomicCAS(status, 0, HEC_ERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == MMA_WARP) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TC_COLS));
}

// Weight and bias gradients of one layer: partial[block][tap][ci][co] = sum over this tile's voxels
// of Ain[v + off(tap)][ci] * dZ[v][co], partial[block][WSZ + co] = sum of dZ[v][co];
// dZ = dA masked by the layer's ReLU (mask = its output) when mask is given.
__global__ void __launch_bounds__(kConvThreads) k_conv_wgrad(Geom g, const __nv_bfloat16* __restrict__ Ain,
                                                             const __nv_bfloat16* __restrict__ dA,
                                                             const __nv_bfloat16* __restrict__ mask,
                                                             float* __restrict__ partial) {
    __shared__ __align__(16) __nv_bfloat16 sx[HZ][HY][HX][C];
    __shared__ __align__(16) __nv_bfloat16 sd[TY][TX][C];
    __shared__ float sbias[kConvThreads / 32][C];
    const int bx = blockIdx.x * TX, by = blockIdx.y * TY, bz = blockIdx.z;
    load_halo(g, Ain, nullptr, bx, by, bz, sx);
    for (int i = threadIdx.x; i < TY * TX * 2; i += blockDim.x) {
        const int v = i >> 1, half = i & 1;
        const int lx = v % TX, ly = v / TX;
        const int x = bx + lx, y = by + ly;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (x < g.nx && y < g.ny) {
            const long gi = ((long)bz * g.ny + y) * g.nx + x;
            val = __ldg((const uint4*)dA + gi * 2 + half);
            if (mask) val = apply_mask(val, __ldg((const uint4*)mask + gi * 2 + half));
        }
        ((uint4*)&sd[0][0][0])[v * 2 + half] = val;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gq = lane >> 2, t = lane & 3;
    const long pbase = (long)((blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * PSZ;
    // taps w, w + 4, w + 8, ... for this warp
    for (int tap = w; tap < NTAP; tap += 4) {
        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        float acc[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[nt][c] = 0.f;
#pragma unroll
        for (int ks = 0; ks < TX * TY / 16; ++ks) {
            const int vy = (ks * 16) / TX, vx0 = (ks * 16) % TX;
            // A[m = ci][k = voxel]: Ain at the shifted voxel
            const __nv_bfloat16* srow = &sx[dz][vy + dy][0][0];
            unsigned af[4];
            af[0] = pack2(srow[(vx0 + 2 * t + dx) * C + gq], srow[(vx0 + 2 * t + 1 + dx) * C + gq]);
            af[1] = pack2(srow[(vx0 + 2 * t + dx) * C + gq + 8], srow[(vx0 + 2 * t + 1 + dx) * C + gq + 8]);
            af[2] = pack2(srow[(vx0 + 2 * t + 8 + dx) * C + gq], srow[(vx0 + 2 * t + 9 + dx) * C + gq]);
            af[3] = pack2(srow[(vx0 + 2 * t + 8 + dx) * C + gq + 8], srow[(vx0 + 2 * t + 9 + dx) * C + gq + 8]);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int co = nt * 8 + gq;
                unsigned bfr[2];
                bfr[0] = pack2(sd[vy][vx0 + 2 * t][co], sd[vy][vx0 + 2 * t + 1][co]);
                bfr[1] = pack2(sd[vy][vx0 + 2 * t + 8][co], sd[vy][vx0 + 2 * t + 9][co]);
                mma_bf16(acc[nt], af, bfr);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int co = nt * 8 + 2 * t;
            partial[pbase + (long)tap * C * C + gq * C + co] = acc[nt][0];
            partial[pbase + (long)tap * C * C + gq * C + co + 1] = acc[nt][1];
            partial[pbase + (long)tap * C * C + (gq + 8) * C + co] = acc[nt][2];
            partial[pbase + (long)tap * C * C + (gq + 8) * C + co + 1] = acc[nt][3];
        }
    }
    // bias gradient: warp w sums rows y = w of the tile
    if (lane < C) {
        float s = 0.f;
        for (int x = 0; x < TX; ++x) s += __bfloat162float(sd[w][x][lane]);
        sbias[w][lane] = s;
    }
    __syncthreads();
    if (threadIdx.x < C) {
        float s = 0.f;
        for (int i = 0; i < kConvThreads / 32; ++i) s += sbias[i][threadIdx.x];
        partial[pbase + WSZ + threadIdx.x] = s;
    }
}

// grad[j] = sum over blocks of partial[b][j], in block order
__global__ void k_reduce_partials(int nblk, const float* __restrict__ partial, float* __restrict__ grad) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= PSZ) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += partial[(long)b * PSZ + j];
    grad[j] = s;
}

// From FP32 master parameters P[tap][ci][co] (+ bias) to the BF16 forward layout Wf[tap][co][ci]
// and the data-gradient layout Wd[26 - tap][ci][co] (flipped taps, channels transposed).  For the
// first layer, Wx (when given) receives the x-expanded layout of its input channels 0 and 1:
// Wx[dz * 3 + dy][co][2 dx + ci] (slots 6-15 stay zero).
__global__ void k_weights(const float* __restrict__ P, __nv_bfloat16* __restrict__ Wf, __nv_bfloat16* __restrict__ Wd,
                          __nv_bfloat16* __restrict__ Wx) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= WSZ) return;
    const int tap = j / (C * C), ci = (j / C) % C, co = j % C;
    const __nv_bfloat16 v = __float2bfloat16_rn(P[j]);
    Wf[(tap * C + co) * C + ci] = v;
    Wd[((NTAP - 1 - tap) * C + ci) * C + co] = v;
    if (Wx && ci < 2) Wx[((tap / 3) * C + co) * C + 2 * (tap % 3) + ci] = v;
}

__global__ void k_adam(int n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float gj = g[j];
    const float mj = b1 * m[j] + (1.f - b1) * gj;
    const float vj = b2 * v[j] + (1.f - b2) * gj * gj;
    m[j] = mj;
    v[j] = vj;
    p[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + eps);
}

// dOut (16-channel BF16, channel 0 only) = 2 (out - target) / N; partial squared errors per block
__global__ void k_mse(long nvox, const float* __restrict__ out, const float* __restrict__ target, float inv_n,
                      __nv_bfloat16* __restrict__ dout, float* __restrict__ part) {
    __shared__ float red[8];
    float s = 0.f;
    for (long v = (long)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (long)gridDim.x * blockDim.x) {
        const float d = out[v] - target[v];
        s += d * d;
        uint4 z0 = make_uint4(0, 0, 0, 0), z1 = z0;
        z0.x = (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(2.f * d * inv_n));
        ((uint4*)dout)[v * 2] = z0;
        ((uint4*)dout)[v * 2 + 1] = z1;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        part[blockIdx.x] = t;
    }
}

}  // namespace
}  // namespace hec

// ---- the network handle ----------------------------------------------------------------------
struct hec_net {
    float* P = nullptr;                // [NL][PSZ] FP32 master parameters
    float* G = nullptr;                // gradients
    float* M = nullptr;                // Adam first moment
    float* V = nullptr;                // Adam second moment
    __nv_bfloat16* Wf = nullptr;       // [NL][WSZ] forward weights
    __nv_bfloat16* Wd = nullptr;       // [NL][WSZ] data-gradient weights
    __nv_bfloat16* Wx = nullptr;       // [9][16][16] first layer, x-expanded input channels
    int step = 0;
    long cap = 0;                      // voxels the activation buffers hold
    __nv_bfloat16* act[hec::NL + 1] = {};  // act[0] = input, act[l] = output of layer l
    __nv_bfloat16* dA[2] = {};
    float* out = nullptr;              // FP32 channel 0 of the last layer
    float* partial = nullptr;
    long partial_cap = 0;
    float* lpart = nullptr;
    int tensor_cores = 1;              // forward pass on tcgen05 (else mma.sync)
    unsigned* words = nullptr;         // [cap] first-layer input: BF16 channels 0-1 of each voxel
    int* status = nullptr;             // device word: HEC_ERR_TIMEOUT if a tensor-core wait ran out
};

namespace hec {
namespace {

void free_net(hec_net* N) {
    if (!N) return;
    dfree(N->P); dfree(N->G); dfree(N->M); dfree(N->V); dfree(N->Wf); dfree(N->Wd); dfree(N->Wx);
    for (auto& a : N->act) dfree(a);
    for (auto& a : N->dA) dfree(a);
    dfree(N->out); dfree(N->partial); dfree(N->lpart); dfree(N->status); dfree(N->words);
    delete N;
}

hec_status ensure(hec_net* N, long nvox, long nblk) {
    if (nvox > N->cap) {
        for (auto& a : N->act) { dfree(a); a = nullptr; }
        for (auto& a : N->dA) { dfree(a); a = nullptr; }
        dfree(N->out);
        dfree(N->words);
        N->out = nullptr;
        N->words = nullptr;
        N->cap = 0;
        for (auto& a : N->act) HEC_CHECK(dalloc(&a, (size_t)nvox * C));
        for (auto& a : N->dA) HEC_CHECK(dalloc(&a, (size_t)nvox * C));
        HEC_CHECK(dalloc(&N->out, (size_t)nvox));
        HEC_CHECK(dalloc(&N->words, (size_t)nvox));
        N->cap = nvox;
    }
    if (nblk > N->partial_cap) {
        dfree(N->partial);
        N->partial = nullptr;
        HEC_CHECK(dalloc(&N->partial, (size_t)nblk * PSZ));
        N->partial_cap = nblk;
    }
    return HEC_OK;
}

hec_status refresh_weights(hec_net* N, cudaStream_t s) {
    for (int l = 0; l < NL; ++l)
        k_weights<<<(WSZ + 255) / 256, 256, 0, s>>>(N->P + (long)l * PSZ, N->Wf + (long)l * WSZ, N->Wd + (long)l * WSZ,
                                                    l == 0 ? N->Wx : nullptr);
    count_launch(NL);
    HEC_CUDA(cudaGetLastError());
    return HEC_OK;
}

// grid of the weight-gradient kernel (one 32 x 4 x 1 tile per block)
dim3 conv_grid(const Geom& g) { return dim3((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, g.nz); }

hec_status check_geom(const Geom& g) {
    if (g.nx <= 0 || g.ny <= 0 || g.nz <= 0 || g.zs <= 0 || g.nz % g.zs != 0 || (g.ny + TY - 1) / TY > 65535 ||
        g.nz > 65535)
        return set_error(HEC_ERR_INVALID_ARG, "net: bad grid (need nz a multiple of zs, ny/4 and nz <= 65535)");
    return HEC_OK;
}

// one forward-type convolution (see k_conv)
template <int MODE, int NT>
hec_status conv(const Geom& g, const ConvIn& in, const __nv_bfloat16* W, const float* bias, int relu, const ConvOut& out,
                cudaStream_t s) {
    static bool smem_set = false;
    if (!smem_set) {
        HEC_CUDA(cudaFuncSetAttribute(k_conv<MODE, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem));
        smem_set = true;
    }
    const int zt = (g.zs + FZ - 1) / FZ;
    const dim3 grid((g.nx + FX - 1) / FX, (g.ny + FY - 1) / FY, (g.nz / g.zs) * zt);
    k_conv<MODE, NT><<<grid, kConvThreads, kFwdSmem, s>>>(g, zt, in, W, bias, relu, out);
    count_launch();
    return HEC_OK;
}

// first-layer input from the solver's vectors: word v = (BF16(r[v] / sigma), aux[v]), channel 0 = 0
// when sigma is not positive (as the mma.sync path stages it)
__global__ void k_words(long n, const double* __restrict__ r, const double* __restrict__ sigma,
                        const __nv_bfloat16* __restrict__ aux, unsigned* __restrict__ w) {
    const double inv = *sigma > 0.0 ? 1.0 / *sigma : 0.0;
    for (long v = (long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long)gridDim.x * blockDim.x)
        w[v] = pack2(__float2bfloat16_rn((float)(r[v] * inv)), aux[v]);
}

// the 16-input-channel forward convolution on the tensor cores (see k_conv_tc)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

template <int NT, int EXP>
hec_status conv_tc(const Geom& g, const ConvIn& in, const __nv_bfloat16* W, const float* bias, int relu,
                   const ConvOut& out, int* status, cudaStream_t s, int wstride = 0) {
    static bool smem_set = false;
    if (!smem_set) {
        HEC_CUDA(cudaFuncSetAttribute(k_conv_tc<NT, EXP>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(EXP)));
        smem_set = true;
    }
    CUtensorMap tm;
    memset(&tm, 0, sizeof(tm));
    if (!EXP) {
        auto encode = tensor_map_encoder();
        if (!encode) return set_error(HEC_ERR_CUDA, "net: cuTensorMapEncodeTiled is not available");
        // X viewed as [sample][z][y][x][16 channels]; a box is 130 voxels x (TCY+2) rows of one
        // plane, written to shared memory in the 32-byte swizzle
        const cuuint64_t row = 32, nx = (cuuint64_t)g.nx, ny = (cuuint64_t)g.ny, zs = (cuuint64_t)g.zs;
        const cuuint64_t dims[5] = {16, nx, ny, zs, (cuuint64_t)(g.nz / g.zs)};
        const cuuint64_t strides[4] = {row, row * nx, row * nx * ny, row * nx * ny * zs};
        const cuuint32_t box[5] = {16, TC_HX, TC_HY, 1, 1};
        const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        const CUresult r = encode(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)in.X, dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return set_error(HEC_ERR_CUDA, "net: cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    }
    const int xt = (g.nx + TCX - 1) / TCX, yt = (g.ny + TCY - 1) / TCY, ns = g.nz / g.zs;
    const long G = 2L * std::max(1, num_sms());  // two CTAs per SM, persistent
    // z-chunk length: the one that minimises the busiest CTA's plane steps, ceil(items / G) x (zl + 2)
    int zl = TCZ;
    long best = -1;
    for (int L = TCZ; L >= 1; --L) {
        const long zt = (g.zs + L - 1) / L, items = (long)xt * yt * zt * ns;
        const long cost = (items + G - 1) / G * (L + 2);
        if (best < 0 || cost < best) best = cost, zl = L;
    }
    const int zt = (g.zs + zl - 1) / zl;
    const long items = (long)xt * yt * zt * ns;
    if (items > (1L << 30)) return set_error(HEC_ERR_INVALID_ARG, "net: grid too large");
    const int grid = (int)std::min<long>(items, G);
    k_conv_tc<NT, EXP><<<grid, tc_threads(EXP), tc_smem(EXP), s>>>(g, xt, yt, zt, zl, (int)items, tm, in, wstride, W,
                                                                  bias, relu, out, status);
    count_launch();
    return HEC_OK;
}

// forward through all layers from `in` (N->act[0], or the solver's vectors); `last` receives
// the last layer's output
hec_status forward(hec_net* N, const Geom& g, const ConvIn& in, const ConvOut& last, cudaStream_t s) {
    ProfScope ps_(s, PROF_VEC);
    const float* b[NL];
    for (int l = 0; l < NL; ++l) b[l] = N->P + (long)l * PSZ + WSZ;
    const ConvOut none{nullptr, nullptr, 1.f, nullptr, nullptr};
    ConvOut o = none;
    o.Y = N->act[1];
    const bool tc = N->tensor_cores != 0;
    if (tc && in.r) {
        // the solver's vectors: channels 0-1 packed into one word per voxel first
        const long nvox = (long)g.nx * g.ny * g.nz;
        k_words<<<(int)std::min<long>((nvox + 255) / 256, 8L * std::max(1, num_sms())), 256, 0, s>>>(nvox, in.r, in.sigma,
                                                                                                   in.aux, N->words);
        count_launch();
        HEC_CHECK((conv_tc<2, 1>(g, ConvIn{(const __nv_bfloat16*)N->words, nullptr, nullptr, nullptr, nullptr}, N->Wx,
                                 b[0], 1, o, N->status, s, 1)));
    } else if (tc) {
        HEC_CHECK((conv_tc<2, 1>(g, in, N->Wx, b[0], 1, o, N->status, s, C / 2)));  // word 0 of each 16-channel voxel
    } else
        HEC_CHECK((conv<EXPAND, 2>(g, in, N->Wx, b[0], 1, o, s)));
    for (int l = 1; l < NL - 1; ++l) {
        o.Y = N->act[l + 1];
        if (tc)
            HEC_CHECK((conv_tc<2, 0>(g, ConvIn{N->act[l], nullptr, nullptr, nullptr, nullptr}, N->Wf + (long)l * WSZ, b[l],
                                     1, o, N->status, s)));
        else
            HEC_CHECK((conv<PLAIN, 2>(g, ConvIn{N->act[l], nullptr, nullptr, nullptr, nullptr}, N->Wf + (long)l * WSZ,
                                      b[l], 1, o, s)));
    }
    if (tc)
        HEC_CHECK((conv_tc<1, 0>(g, ConvIn{N->act[NL - 1], nullptr, nullptr, nullptr, nullptr},
                                 N->Wf + (long)(NL - 1) * WSZ, b[NL - 1], 0, last, N->status, s)));
    else
        HEC_CHECK((conv<PLAIN, 1>(g, ConvIn{N->act[NL - 1], nullptr, nullptr, nullptr, nullptr},
                                  N->Wf + (long)(NL - 1) * WSZ, b[NL - 1], 0, last, s)));
    HEC_CUDA(cudaGetLastError());
    return HEC_OK;
}

// backward from dA[0] = dLoss/dOutput (16-channel, channel 0); gradients into N->G
hec_status backward(hec_net* N, const Geom& g, cudaStream_t s) {
    const dim3 grid = conv_grid(g);
    const long nblk = (long)grid.x * grid.y * grid.z;
    int cur = 0;
    for (int l = NL - 1; l >= 0; --l) {
        const __nv_bfloat16* mask = l == NL - 1 ? nullptr : N->act[l + 1];  // ReLU of layer l
        k_conv_wgrad<<<grid, kConvThreads, 0, s>>>(g, N->act[l], N->dA[cur], mask, N->partial);
        k_reduce_partials<<<(PSZ + 255) / 256, 256, 0, s>>>((int)nblk, N->partial, N->G + (long)l * PSZ);
        count_launch(2);
        if (l > 0) {
            const ConvIn din{N->dA[cur], mask, nullptr, nullptr, nullptr};
            const ConvOut dout{N->dA[cur ^ 1], nullptr, 1.f, nullptr, nullptr};
            if (mask)
                HEC_CHECK((conv<MASKED, 2>(g, din, N->Wd + (long)l * WSZ, nullptr, 0, dout, s)));
            else
                HEC_CHECK((conv<PLAIN, 2>(g, din, N->Wd + (long)l * WSZ, nullptr, 0, dout, s)));
            cur ^= 1;
        }
    }
    HEC_CUDA(cudaGetLastError());
    return HEC_OK;
}

}  // namespace

// used by the learned FGMRES stage (krylov.cu): c = sigma * Net([r / sigma, aux]) on an
// nx x ny x nz grid, the input channels read straight from r and aux, c written in FP64
hec_status net_apply_field(hec_net* N, int nx, int ny, int nz, const double* r, const double* sigma,
                           const __nv_bfloat16* aux, double* c, cudaStream_t s) {
    Geom g{nx, ny, nz, nz};
    HEC_CHECK(check_geom(g));
    const long nvox = (long)nx * ny * nz;
    const dim3 grid = conv_grid(g);
    HEC_CHECK(ensure(N, nvox, (long)grid.x * grid.y * grid.z));
    return forward(N, g, ConvIn{nullptr, nullptr, r, sigma, aux}, ConvOut{nullptr, nullptr, 1.f, c, sigma}, s);
}

}  // namespace hec

using namespace hec;

namespace hec {
namespace {
// one block: sum of squares of r[0..n) into out[0] (FP64)
__global__ void k_sumsq(long n, const double* __restrict__ r, double* out) {
    __shared__ double red[32];
    double s = 0.0;
    for (long i = threadIdx.x; i < n; i += blockDim.x) s = fma(r[i], r[i], s);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        out[0] = sqrt(t / (double)n);  // sigma = RMS
    }
}
__global__ void k_make_sample(long n, const double* __restrict__ r, const double* __restrict__ e,
                              const double* __restrict__ aux, double aux_scale, const double* __restrict__ sigma,
                              __nv_bfloat16* __restrict__ X, float* __restrict__ T) {
    const double inv = *sigma > 0.0 ? 1.0 / *sigma : 0.0;
    for (long v = (long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long)gridDim.x * blockDim.x) {
        uint4 z0 = make_uint4(0, 0, 0, 0), z1 = z0;
        z0.x = pack2(__float2bfloat16_rn((float)(r[v] * inv)), __float2bfloat16_rn((float)(aux[v] * aux_scale)));
        ((uint4*)X)[v * 2] = z0;
        ((uint4*)X)[v * 2 + 1] = z1;
        if (T) T[v] = (float)(e[v] * inv);
    }
}
}  // namespace
}  // namespace hec

HEC_API int net_param_count(void) { return NL * PSZ; }

HEC_API hec_status net_make_sample(int n, const double* r, const double* e, const double* aux, double aux_scale,
                                   void* x_out, float* target_out, double* sigma_out, void* stream) {
    clear_error();
    if (n <= 0 || !r || !aux || !x_out || !sigma_out || (target_out && !e))
        return set_error(HEC_ERR_INVALID_ARG, "net_make_sample: bad argument");
    cudaStream_t s = S(stream);
    k_sumsq<<<1, 1024, 0, s>>>(n, r, sigma_out);
    k_make_sample<<<(int)std::min<long>(((long)n + 255) / 256, 65536), 256, 0, s>>>(
        n, r, e, aux, aux_scale, sigma_out, (__nv_bfloat16*)x_out, target_out);
    count_launch(2);
    HEC_CUDA(cudaGetLastError());
    return HEC_OK;
}

HEC_API hec_status net_create(const float* params, hec_net** out) {
    clear_error();
    if (!params || !out) return set_error(HEC_ERR_INVALID_ARG, "net_create: NULL");
    *out = nullptr;
    hec_net* N = new hec_net();
    const size_t np = (size_t)NL * PSZ;
    hec_status st = HEC_OK;
    if ((st = dalloc(&N->P, np)) || (st = dalloc(&N->G, np)) || (st = dalloc(&N->M, np)) || (st = dalloc(&N->V, np)) ||
        (st = dalloc(&N->Wf, (size_t)NL * WSZ)) || (st = dalloc(&N->Wd, (size_t)NL * WSZ)) ||
        (st = dalloc(&N->Wx, (size_t)9 * C * C)) || (st = dalloc(&N->lpart, 4096)) || (st = dalloc(&N->status, 1))) {
        free_net(N);
        return st;
    }
    cudaMemcpy(N->P, params, sizeof(float) * np, cudaMemcpyHostToDevice);
    cudaMemset(N->M, 0, sizeof(float) * np);
    cudaMemset(N->V, 0, sizeof(float) * np);
    cudaMemset(N->G, 0, sizeof(float) * np);
    cudaMemset(N->Wx, 0, sizeof(__nv_bfloat16) * 9 * C * C);
    cudaMemset(N->status, 0, sizeof(int));
    st = refresh_weights(N, 0);
    if (st == HEC_OK && cudaDeviceSynchronize() != cudaSuccess) st = cuda_error(cudaGetLastError(), "net_create");
    if (st) { free_net(N); return st; }
    *out = N;
    return HEC_OK;
}

HEC_API hec_status net_set_engine(hec_net* N, int tensor_cores) {
    clear_error();
    if (!N) return set_error(HEC_ERR_INVALID_ARG, "net_set_engine: NULL");
    N->tensor_cores = tensor_cores ? 1 : 0;
    return HEC_OK;
}

HEC_API hec_status net_sync_status(hec_net* N, void* stream) {
    clear_error();
    if (!N) return set_error(HEC_ERR_INVALID_ARG, "net_sync_status: NULL");
    cudaStream_t s = S(stream);
    int h = 0;
    HEC_CUDA(cudaMemcpyAsync(&h, N->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    HEC_CUDA(cudaStreamSynchronize(s));
    if (h == HEC_OK) return HEC_OK;
    HEC_CUDA(cudaMemsetAsync(N->status, 0, sizeof(int), s));
    HEC_CUDA(cudaStreamSynchronize(s));
    return set_error((hec_status)h, "net: a tensor-core convolution's wait for its MMAs timed out");
}

HEC_API hec_status net_destroy(hec_net* N) {
    free_net(N);
    return HEC_OK;
}

HEC_API hec_status net_get_params(const hec_net* N, float* params, float* grads) {
    if (!N) return set_error(HEC_ERR_INVALID_ARG, "net_get_params: NULL");
    const size_t np = (size_t)NL * PSZ;
    if (params) HEC_CUDA(cudaMemcpy(params, N->P, sizeof(float) * np, cudaMemcpyDeviceToHost));
    if (grads) HEC_CUDA(cudaMemcpy(grads, N->G, sizeof(float) * np, cudaMemcpyDeviceToHost));
    return HEC_OK;
}

HEC_API hec_status net_set_params(hec_net* N, const float* params) {
    if (!N || !params) return set_error(HEC_ERR_INVALID_ARG, "net_set_params: NULL");
    HEC_CUDA(cudaMemcpy(N->P, params, sizeof(float) * (size_t)NL * PSZ, cudaMemcpyHostToDevice));
    HEC_CHECK(refresh_weights(N, 0));
    HEC_CUDA(cudaDeviceSynchronize());
    return HEC_OK;
}

HEC_API hec_status net_forward(hec_net* N, int nx, int ny, int nz, int zs, const void* x_in, void* acts_out,
                               float* out, void* stream) {
    clear_error();
    if (!N || !x_in) return set_error(HEC_ERR_INVALID_ARG, "net_forward: NULL");
    Geom g{nx, ny, nz, zs};
    HEC_CHECK(check_geom(g));
    cudaStream_t s = S(stream);
    const long nvox = (long)nx * ny * nz;
    const dim3 grid = conv_grid(g);
    HEC_CHECK(ensure(N, nvox, (long)grid.x * grid.y * grid.z));
    HEC_CUDA(cudaMemcpyAsync(N->act[0], x_in, sizeof(__nv_bfloat16) * C * nvox, cudaMemcpyDeviceToDevice, s));
    HEC_CHECK(forward(N, g, ConvIn{N->act[0], nullptr, nullptr, nullptr, nullptr},
                      ConvOut{N->act[NL], N->out, 1.f, nullptr, nullptr}, s));
    if (acts_out)
        for (int l = 1; l <= NL; ++l)
            HEC_CUDA(cudaMemcpyAsync((__nv_bfloat16*)acts_out + (long)(l - 1) * nvox * C, N->act[l],
                                     sizeof(__nv_bfloat16) * C * nvox, cudaMemcpyDeviceToDevice, s));
    if (out) HEC_CUDA(cudaMemcpyAsync(out, N->out, sizeof(float) * nvox, cudaMemcpyDeviceToDevice, s));
    return HEC_OK;
}

// forward, loss and backward on one minibatch; the gradients stay in N->G
static hec_status net_backward_impl(hec_net* N, int nx, int ny, int nz, int zs, const void* x_in, const float* target,
                                    float* loss_out, cudaStream_t s, const char* who) {
    if (!N || !x_in || !target) return set_error(HEC_ERR_INVALID_ARG, std::string(who) + ": NULL");
    Geom g{nx, ny, nz, zs};
    HEC_CHECK(check_geom(g));
    const long nvox = (long)nx * ny * nz;
    const dim3 grid = conv_grid(g);
    HEC_CHECK(ensure(N, nvox, (long)grid.x * grid.y * grid.z));
    HEC_CUDA(cudaMemcpyAsync(N->act[0], x_in, sizeof(__nv_bfloat16) * C * nvox, cudaMemcpyDeviceToDevice, s));
    HEC_CHECK(forward(N, g, ConvIn{N->act[0], nullptr, nullptr, nullptr, nullptr},
                      ConvOut{N->act[NL], N->out, 1.f, nullptr, nullptr}, s));
    const int lb = 1024;
    k_mse<<<lb, 256, 0, s>>>(nvox, N->out, target, 1.f / (float)nvox, N->dA[0], N->lpart);
    count_launch();
    HEC_CHECK(backward(N, g, s));
    if (loss_out) {
        std::vector<float> h(lb);
        HEC_CUDA(cudaMemcpyAsync(h.data(), N->lpart, sizeof(float) * lb, cudaMemcpyDeviceToHost, s));
        HEC_CUDA(cudaStreamSynchronize(s));
        double t = 0.0;
        for (float v : h) t += v;
        *loss_out = (float)(t / (double)nvox);
    }
    HEC_CUDA(cudaGetLastError());
    return HEC_OK;
}

// one bias-corrected Adam step on the kept gradients, then the BF16 weight copies
static hec_status net_adam_impl(hec_net* N, float lr, cudaStream_t s) {
    if (!N) return set_error(HEC_ERR_INVALID_ARG, "net_adam_step: NULL");
    N->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)N->step), c2 = 1.f - powf(b2, (float)N->step);
    k_adam<<<(NL * PSZ + 255) / 256, 256, 0, s>>>(NL * PSZ, N->P, N->G, N->M, N->V, lr, b1, b2, 1e-8f, c1, c2);
    count_launch();
    HEC_CHECK(refresh_weights(N, s));
    HEC_CUDA(cudaGetLastError());
    return HEC_OK;
}

HEC_API hec_status net_backward(hec_net* N, int nx, int ny, int nz, int zs, const void* x_in, const float* target,
                                float* loss_out, void* stream) {
    clear_error();
    return net_backward_impl(N, nx, ny, nz, zs, x_in, target, loss_out, S(stream), "net_backward");
}

HEC_API hec_status net_adam_step(hec_net* N, float lr, void* stream) {
    clear_error();
    return net_adam_impl(N, lr, S(stream));
}

HEC_API hec_status net_train_step(hec_net* N, int nx, int ny, int nz, int zs, const void* x_in, const float* target,
                                  float lr, int update, float* loss_out, void* stream) {
    clear_error();
    cudaStream_t s = S(stream);
    // the loss is read back after the update, as one call of the two steps would
    HEC_CHECK(net_backward_impl(N, nx, ny, nz, zs, x_in, target, nullptr, s, "net_train_step"));
    if (update) HEC_CHECK(net_adam_impl(N, lr, s));
    if (loss_out) {
        const int lb = 1024;
        std::vector<float> h(lb);
        HEC_CUDA(cudaMemcpyAsync(h.data(), N->lpart, sizeof(float) * lb, cudaMemcpyDeviceToHost, s));
        HEC_CUDA(cudaStreamSynchronize(s));
        double t = 0.0;
        for (float v : h) t += v;
        *loss_out = (float)(t / (double)((long)nx * ny * nz));
    }
    return HEC_OK;
}
