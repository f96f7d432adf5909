// Error reporting, allocation helpers, launch accounting and the device exclusive scan.
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <unordered_map>
#include <string>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace hec {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

hec_status set_error(hec_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

hec_status cuda_error(cudaError_t e, const char* what) {
    cudaGetLastError();  // a non-sticky error must not be reported again by the next call
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return set_error(HEC_ERR_OOM, m);
    return set_error(HEC_ERR_CUDA, m);
}

void clear_error() { g_last_error.clear(); }
void count_launch(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---- device memory cache -------------------------------------------------------------------
// Handles and the temporaries of set-up are allocated and released many times with the same sizes
// (a solver built per system, a restart's workspace per solve).  cudaMalloc and cudaFree cost tens
// to hundreds of microseconds each (cudaFree also waits for the device), so released blocks are
// kept per device and handed out again: dfree waits for the device, as cudaFree does, and then
// keeps the block, so a cached block is never in use by queued work.  Sizes are rounded (512 bytes
// below 1 MiB, 1 MiB above) and a cached block is reused for a request of at least 4/5 of its
// size.  The cache holds at most kCacheCap bytes a process; hec_release_cached_memory() and a
// failing cudaMalloc release it.
namespace {
struct Block {
    size_t size;
    int dev;
};
std::mutex g_mem_mu;
std::unordered_map<void*, Block>* g_live = new std::unordered_map<void*, Block>();      // handed out
std::multimap<std::pair<int, size_t>, void*>* g_cache = new std::multimap<std::pair<int, size_t>, void*>();
size_t g_cached_bytes = 0;
constexpr size_t kCacheCap = (size_t)16 << 30;

size_t round_block(size_t b) {
    if (b == 0) b = 16;
    if (b < ((size_t)1 << 20)) return (b + 511) & ~(size_t)511;
    return (b + ((size_t)1 << 20) - 1) & ~(((size_t)1 << 20) - 1);
}

// frees cached blocks (of every device when dev < 0) until at most `keep` bytes stay; lock held
size_t trim_cache_locked(int dev, size_t keep) {
    size_t freed = 0;
    int cur = -1;
    cudaGetDevice(&cur);
    for (auto it = g_cache->end(); it != g_cache->begin() && g_cached_bytes > keep;) {
        --it;
        if (dev >= 0 && it->first.first != dev) continue;
        if (it->first.first != cur) cudaSetDevice(it->first.first);
        cudaFree(it->second);
        if (it->first.first != cur) cudaSetDevice(cur);
        g_cached_bytes -= it->first.second;
        freed += it->first.second;
        it = g_cache->erase(it);
    }
    return freed;
}
}  // namespace

hec_status dmalloc(void** p, size_t bytes) {
    *p = nullptr;
    const size_t sz = round_block(bytes);
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> g(g_mem_mu);
        auto it = g_cache->lower_bound({dev, sz});
        if (it != g_cache->end() && it->first.first == dev && it->first.second - sz <= it->first.second / 5) {
            *p = it->second;
            (*g_live)[*p] = Block{it->first.second, dev};
            g_cached_bytes -= it->first.second;
            g_cache->erase(it);
            return HEC_OK;
        }
    }
    cudaError_t e = cudaMalloc(p, sz);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        {
            std::lock_guard<std::mutex> g(g_mem_mu);
            trim_cache_locked(dev, 0);
        }
        e = cudaMalloc(p, sz);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return cuda_error(e, "cudaMalloc");
    }
    std::lock_guard<std::mutex> g(g_mem_mu);
    (*g_live)[*p] = Block{sz, dev};
    return HEC_OK;
}

void dfree(void* p) {
    if (!p) return;
    Block b{0, -1};
    {
        std::lock_guard<std::mutex> g(g_mem_mu);
        auto it = g_live->find(p);
        if (it != g_live->end()) {
            b = it->second;
            g_live->erase(it);
        }
    }
    int cur = -1;
    cudaGetDevice(&cur);
    if (b.dev < 0 || b.dev != cur) {  // not from dmalloc, or another device: release it outright
        cudaFree(p);
        return;
    }
    // queued work may still use the block: wait for the device, as cudaFree does
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p);
        return;
    }
    std::lock_guard<std::mutex> g(g_mem_mu);
    g_cache->insert({{b.dev, b.size}, p});
    g_cached_bytes += b.size;
    if (g_cached_bytes > kCacheCap) trim_cache_locked(-1, kCacheCap);
}

int num_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

int max_coop_blocks(const void* kernel, int threads, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// ---- exclusive scan ---------------------------------------------------------------------
// Three phases: per-tile sums, a scan of the tile sums (recursively), per-tile scan plus the
// tile's offset.  Tiles are 256 threads x 8 items.
namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int* smem_warp, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < (kScanThreads / 32) ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < (kScanThreads / 32)) smem_warp[lane] = s;
    }
    __syncthreads();
    int warp_off = warp ? smem_warp[warp - 1] : 0;
    total = smem_warp[kScanThreads / 32 - 1];
    __syncthreads();
    return warp_off + x - v;
}

__global__ void k_tile_sums(const int* __restrict__ in, int n, int* __restrict__ sums) {
    __shared__ int sw[kScanThreads / 32];
    long base = (long)blockIdx.x * kScanTile + (long)threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long i = base + k;
        if (i < n) s += in[i];
    }
    int total;
    block_exclusive_scan(s, sw, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_tile_scan(const int* in, int n, int* out, const int* __restrict__ offs, int write_total) {
    __shared__ int sw[kScanThreads / 32];
    long base = (long)blockIdx.x * kScanTile + (long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long i = base + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int total;
    int run = block_exclusive_scan(s, sw, total) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = run;
}

}  // namespace

hec_status exclusive_scan_i32(const int* in, int* out, int n, bool write_total, cudaStream_t s) {
    if (n <= 0) {
        if (write_total) {
            HEC_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
        }
        return HEC_OK;
    }
    int tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_tile_scan<<<1, kScanThreads, 0, s>>>(in, n, out, nullptr, write_total ? 1 : 0);
        HEC_LAUNCHED();
        return HEC_OK;
    }
    int* sums = nullptr;
    HEC_CHECK(dalloc(&sums, (size_t)tiles + 1));
    k_tile_sums<<<tiles, kScanThreads, 0, s>>>(in, n, sums);
    count_launch();
    hec_status st = exclusive_scan_i32(sums, sums, tiles, false, s);
    if (st == HEC_OK) {
        k_tile_scan<<<tiles, kScanThreads, 0, s>>>(in, n, out, sums, write_total ? 1 : 0);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_error(e, "scan");
    }
    // sums must outlive the kernels that read it: free after the stream drains this work
    cudaError_t e = cudaStreamSynchronize(s);
    dfree(sums);
    if (st == HEC_OK && e != cudaSuccess) st = cuda_error(e, "scan sync");
    return st;
}

}  // namespace hec

// ---- kernel timing by category (measurement only) ------------------------------------------
namespace hec {
namespace {
struct ProfEntry {
    cudaEvent_t a, b;
    int cat;
};
std::mutex g_prof_mu;
unsigned int g_prof_mask = 0u;  // bit c: category c is recorded
std::vector<ProfEntry> g_prof_used;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_free;
}  // namespace

bool profiling() { return g_prof_mask != 0u; }

void profile_begin(cudaStream_t s, void** token, int cat) {
    *token = nullptr;
    if (!(g_prof_mask & (1u << cat))) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    std::pair<cudaEvent_t, cudaEvent_t> ev;
    if (!g_prof_free.empty()) {
        ev = g_prof_free.back();
        g_prof_free.pop_back();
    } else {
        if (cudaEventCreate(&ev.first) != cudaSuccess || cudaEventCreate(&ev.second) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
    }
    cudaEventRecord(ev.first, s);
    g_prof_used.push_back({ev.first, ev.second, cat});
    *token = (void*)(g_prof_used.size());
}

void profile_end(cudaStream_t s, void* token) {
    if (!token) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    size_t idx = (size_t)token - 1;
    if (idx < g_prof_used.size()) cudaEventRecord(g_prof_used[idx].b, s);
}

static void prof_sum(int cat, double* ms_out, long long* n_out) {
    double tot = 0.0;
    long long cnt = 0;
    for (auto& ev : g_prof_used) {
        if (ev.cat != cat) continue;
        cudaEventSynchronize(ev.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev.a, ev.b) == cudaSuccess) tot += ms;
        else cudaGetLastError();
        cnt++;
    }
    if (ms_out) *ms_out = tot;
    if (n_out) *n_out = cnt;
}
}  // namespace hec

HEC_API hec_status hec_profile_enable(int on) {
    hec::g_prof_mask = on != 0 ? 0xFFFFFFFFu : 0u;
    return HEC_OK;
}

HEC_API hec_status hec_profile_enable_categories(unsigned int mask) {
    hec::g_prof_mask = mask;
    return HEC_OK;
}

HEC_API hec_status hec_profile_read_category(int category, double* ms, long long* launches) {
    std::lock_guard<std::mutex> g(hec::g_prof_mu);
    hec::prof_sum(category, ms, launches);
    return HEC_OK;
}

HEC_API hec_status hec_profile_read(double* sweep_ms, long long* launches, int reset) {
    std::lock_guard<std::mutex> g(hec::g_prof_mu);
    hec::prof_sum(0, sweep_ms, launches);
    if (reset) {
        for (auto& ev : hec::g_prof_used) hec::g_prof_free.push_back({ev.a, ev.b});
        hec::g_prof_used.clear();
    }
    return HEC_OK;
}

HEC_API const char* hec_last_error(void) { return hec::g_last_error.c_str(); }
HEC_API int hec_version(void) { return 1; }
HEC_API long long hec_launch_count(void) { return hec::g_launches.load(); }

HEC_API size_t hec_release_cached_memory(void) {
    std::lock_guard<std::mutex> g(hec::g_mem_mu);
    return hec::trim_cache_locked(-1, 0);
}
