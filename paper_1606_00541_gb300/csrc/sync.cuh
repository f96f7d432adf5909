// Point-to-point dependency waits used by the sync-free level-ordered kernels.
//
// A consumer waits for a producer's value by polling the value itself: the producer's output
// array is filled with a sentinel bit pattern before the kernel and the producer publishes with
// one relaxed GPU-scope store of an aligned 32- or 64-bit word (single-copy atomic), so no
// separate flag and no fence are needed.  Polls are relaxed GPU-scope loads, which read L2 and
// never a stale L1 line.  Every wait is bounded: after `budget` SM cycles (or once another
// thread has recorded a failure) it records DEV_TIMEOUT in the status word and returns 0, so a
// kernel whose producer never publishes still terminates.
#pragma once
#include <stdint.h>

namespace hec {

// Sentinels: NaN payloads that FP arithmetic never produces (results that happen to match are
// replaced by a canonical quiet NaN before they are published).
constexpr unsigned long long kSent64 = 0xFFF7A5A5A5A5A5A5ull;
constexpr unsigned int kSent32 = 0xFFB5A5A5u;
constexpr int kSentI = -1;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const void* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned int ld_relaxed_u32(const void* p) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(void* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u32(void* p, unsigned int v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_i32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_i32(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void record(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// Slow path of a wait: spin with a cycle budget, bail out on any recorded failure.
template <typename Word, typename Load>
__device__ __noinline__ Word spin_until_not(const void* p, Word sentinel, int* status, long long budget, Load load) {
    long long t0 = clock64();
    unsigned failed = 0u;  // the status word as read at the previous check (not waited on)
    for (unsigned it = 1;; ++it) {
        Word v = load(p);
        if (v != sentinel) return v;
        if ((it & 63u) == 0u) {
            if (clock64() - t0 > budget || failed != 0u) {
                record(status, HEC_ERR_TIMEOUT);
                return Word(0);
            }
            if (status) failed = ld_relaxed_u32(status);
        }
    }
}

struct LoadU64 { __device__ unsigned long long operator()(const void* p) const { return ld_relaxed_u64(p); } };
struct LoadU32 { __device__ unsigned int operator()(const void* p) const { return ld_relaxed_u32(p); } };

__device__ __forceinline__ double wait_f64(const double* p, int* status, long long budget) {
    unsigned long long v = ld_relaxed_u64(p);
    if (v == kSent64) v = spin_until_not<unsigned long long>(p, kSent64, status, budget, LoadU64());
    return __longlong_as_double((long long)v);
}
__device__ __forceinline__ float wait_f32(const float* p, int* status, long long budget) {
    unsigned int v = ld_relaxed_u32(p);
    if (v == kSent32) v = spin_until_not<unsigned int>(p, kSent32, status, budget, LoadU32());
    return __uint_as_float(v);
}
__device__ __forceinline__ int wait_i32(const int* p, int* status, long long budget) {
    unsigned int v = ld_relaxed_u32(p);
    if (v == (unsigned)kSentI) v = spin_until_not<unsigned int>(p, (unsigned)kSentI, status, budget, LoadU32());
    return (int)v;
}

__device__ __forceinline__ void publish_f64(double* p, double x) {
    unsigned long long u = (unsigned long long)__double_as_longlong(x);
    if (u == kSent64) u = 0x7FF8000000000000ull;
    st_relaxed_u64(p, u);
}
__device__ __forceinline__ void publish_f32(float* p, float x) {
    unsigned int u = __float_as_uint(x);
    if (u == kSent32) u = 0x7FC00000u;
    st_relaxed_u32(p, u);
}
__device__ __forceinline__ void publish_i32(int* p, int x) { st_relaxed_u32(p, (unsigned)x); }

}  // namespace hec
