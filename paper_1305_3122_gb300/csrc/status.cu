// status.cu -- error reporting, allocation helpers, device queries and the scan utility.
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include "internal.cuh"

static thread_local std::string g_last_error;

fe_status fe_fail(fe_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

fe_status fe_cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_CUDA;
}

static thread_local cudaStream_t t_stream = nullptr;

FeStreamScope::FeStreamScope(cudaStream_t s) : prev(t_stream) { t_stream = s; }
FeStreamScope::~FeStreamScope() { t_stream = prev; }

static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64];

static cudaError_t pool_for_device(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = ~0ULL;   // keep freed blocks for reuse
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

// Allocation-failure injection (fe_debug_fail_alloc): the count of allocations still to pass
// before the one that fails; 0: off.
static std::atomic<int64_t> g_fail_alloc{0};

extern "C" void fe_debug_fail_alloc(int64_t n) { g_fail_alloc.store(n > 0 ? n : 0); }

extern "C" fe_status fe_debug_pool_used(int64_t* bytes) {
    if (!bytes) return fe_fail(FE_ERR_INVALID_ARG, "bytes is null");
    cudaMemPool_t pool;
    uint64_t v = 0;
    cudaError_t e = pool_for_device(&pool);
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v);
    if (e != cudaSuccess) return fe_cuda_fail(e, "allocation pool attribute");
    *bytes = (int64_t)v;
    return FE_OK;
}

fe_status fe_alloc(void** p, size_t bytes, const char* what) {
    *p = nullptr;
    int64_t c = g_fail_alloc.load();
    while (c > 0 && !g_fail_alloc.compare_exchange_weak(c, c - 1)) {
    }
    if (c == 1)
        return fe_fail(FE_ERR_OOM, std::string("device allocation of ") + std::to_string(bytes) + " bytes for " + what +
                                       ": injected failure (fe_debug_fail_alloc)");
    cudaMemPool_t pool;
    cudaError_t e = pool_for_device(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, pool, t_stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fe_fail(e == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_CUDA,
                       std::string("device allocation of ") + std::to_string(bytes) + " bytes for " + what +
                           ": " + cudaGetErrorString(e));
    }
    return FE_OK;
}

void fe_free(void* p) {
    if (p) cudaFreeAsync(p, t_stream);
}

int fe_sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// ------------------------------------------------------------------ FP64 rate probe

// Independent fused multiply-add chains: each thread keeps FP64_CHAINS accumulators, so the FP64
// pipe always has independent work and the rate measured is its issue rate. b and c are kernel
// arguments (nothing folds at compile time); the store happens only for a sum the inputs cannot
// produce, so the chains are kept without a store per thread.
constexpr int FP64_CHAINS = 8;

__global__ void __launch_bounds__(256) k_fp64_rate(double* __restrict__ sink, int iters, double b, double c) {
    double a[FP64_CHAINS];
#pragma unroll
    for (int j = 0; j < FP64_CHAINS; j++) a[j] = 1e-3 * (double)(threadIdx.x + j);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < FP64_CHAINS; j++) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < FP64_CHAINS; j++) s += a[j];
    if (s == -1.0) sink[0] = s;
}

extern "C" fe_status fe_measure_fp64_rate(double* instr_per_s, fe_stream stream) {
    FE_RANGE(__func__);
    if (!instr_per_s) return fe_fail(FE_ERR_INVALID_ARG, "instr_per_s is null");
    *instr_per_s = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    double* sink = nullptr;
    fe_status st = fe_alloc_n(&sink, 1, "probe sink");
    if (st) return st;
    const int blocks = fe_sm_count() * 8, threads = 256, iters = 2048;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // two warm-up launches (the clocks ramp up over the first ones), then the fastest of five
    float ms = 0.f;
    for (int r = 0; r < 7 && e == cudaSuccess; r++) {
        if (r >= 2) cudaEventRecord(e0, s);
        k_fp64_rate<<<blocks, threads, 0, s>>>(sink, iters, 0.999999, 1e-7);
        if (r < 2) continue;
        cudaEventRecord(e1, s);
        e = cudaGetLastError();
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && (ms == 0.f || t < ms)) ms = t;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    fe_free(sink);
    if (e != cudaSuccess) return fe_cuda_fail(e, "FP64 rate probe");
    const double n = (double)blocks * threads * FP64_CHAINS * iters;
    *instr_per_s = ms > 0.f ? n / (ms * 1e-3) : 0.0;
    return FE_OK;
}

extern "C" const char* fe_status_string(fe_status st) {
    switch (st) {
        case FE_OK: return "FE_OK";
        case FE_ERR_INVALID_ARG: return "FE_ERR_INVALID_ARG";
        case FE_ERR_INDEX_RANGE: return "FE_ERR_INDEX_RANGE";
        case FE_ERR_DEGENERATE: return "FE_ERR_DEGENERATE";
        case FE_ERR_ORIENTATION: return "FE_ERR_ORIENTATION";
        case FE_ERR_BUFFER_TOO_SMALL: return "FE_ERR_BUFFER_TOO_SMALL";
        case FE_ERR_OOM: return "FE_ERR_OOM";
        case FE_ERR_CUDA: return "FE_ERR_CUDA";
        case FE_ERR_TIMEOUT: return "FE_ERR_TIMEOUT";
        case FE_ERR_LIMIT: return "FE_ERR_LIMIT";
    }
    return "FE_ERR_UNKNOWN";
}

extern "C" const char* fe_last_error(void) { return g_last_error.c_str(); }

fe_status fe_check_pair(fe_mesh mesh, fe_pattern pat, int dofs) {
    if (!mesh || !pat) return fe_fail(FE_ERR_INVALID_ARG, "null mesh or pattern");
    if (pat->topology_id != mesh->topology_id || pat->nq != mesh->nq || pat->nme != mesh->nme)
        return fe_fail(FE_ERR_INVALID_ARG, "pattern was built for another mesh topology");
    if (dofs && pat->dofs != dofs)
        return fe_fail(FE_ERR_INVALID_ARG, dofs == 2 ? "elasticity needs a dofs_per_vertex=2 pattern"
                                                     : "scalar matrices need a dofs_per_vertex=1 pattern");
    return FE_OK;
}

// ------------------------------------------------------------------------ scan
//
// Two passes: per-tile sums, then a per-tile scan whose block first adds up the sums of the
// tiles before its own (its offset). Tiles are SCAN_TILE consecutive elements; the total lands in
// out[n].

static constexpr int SCAN_BLOCK = 512;
static constexpr int SCAN_ITEMS = 8;
static constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

// round: each input is rounded up to a multiple of `round` (a power of two) before summing.
__device__ __forceinline__ long long scan_round(int32_t v, int round) {
    return round > 1 ? (long long)((v + round - 1) & ~(round - 1)) : (long long)v;
}
__device__ __forceinline__ long long scan_in(const int32_t* __restrict__ in, int64_t i, int round) {
    return scan_round(in[i], round);
}

// The SCAN_ITEMS = 8 consecutive inputs of one thread: two 16-byte loads when the arrays are
// 16-byte aligned (vec) and all eight lie below n, else eight scalar loads (zeros past n).
__device__ __forceinline__ void scan_load8(const int32_t* __restrict__ in, int64_t i0, int64_t n, bool vec, int round,
                                           long long v[SCAN_ITEMS]) {
    static_assert(SCAN_ITEMS == 8, "two 16-byte vectors per thread");
    if (vec && i0 + SCAN_ITEMS <= n) {
        const int4 a = *reinterpret_cast<const int4*>(in + i0);
        const int4 b = *reinterpret_cast<const int4*>(in + i0 + 4);
        v[0] = scan_round(a.x, round); v[1] = scan_round(a.y, round);
        v[2] = scan_round(a.z, round); v[3] = scan_round(a.w, round);
        v[4] = scan_round(b.x, round); v[5] = scan_round(b.y, round);
        v[6] = scan_round(b.z, round); v[7] = scan_round(b.w, round);
    } else {
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) v[j] = i0 + j < n ? scan_in(in, i0 + j, round) : 0;
    }
}

// Tiles are read in the same thread-to-element order as k_tile_scan (eight consecutive elements
// per thread), so each warp reads 1 KB of consecutive memory per pair of vector loads.
__global__ void k_tile_sums(const int32_t* __restrict__ in, int64_t n, long long* __restrict__ sums, int round, bool vec) {
    __shared__ long long red[SCAN_BLOCK / 32];
    long long v[SCAN_ITEMS];
    scan_load8(in, (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS, n, vec, round, v);
    long long s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) s += v[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < SCAN_BLOCK / 32 ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = s;
    }
}

// The tile's offset is the sum of the tile sums before it, which each block adds up itself (a few
// KB, in L2; a separate one-block scan of the sums was a launch of pure latency). The last block
// writes the total to sums[ntiles] and to out[n].
__global__ void k_tile_scan(const int32_t* __restrict__ in, int32_t* __restrict__ out, int32_t* __restrict__ out2,
                            int64_t n, long long* __restrict__ sums, int* __restrict__ overflow, int round, bool vec) {
    __shared__ long long warp_tot[SCAN_BLOCK / 32];
    __shared__ long long boff;
    {
        long long a = 0;
        for (int64_t t = threadIdx.x; t < blockIdx.x; t += SCAN_BLOCK) a += sums[t];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = a;
        __syncthreads();
        if (threadIdx.x < 32) {
            a = threadIdx.x < SCAN_BLOCK / 32 ? warp_tot[threadIdx.x] : 0;
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (threadIdx.x == 0) boff = a;
        }
        __syncthreads();
    }
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    long long v[SCAN_ITEMS];
    scan_load8(in, base, n, vec, round, v);
    long long local = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) local += v[j];
    long long x = local;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long t = threadIdx.x < SCAN_BLOCK / 32 ? warp_tot[threadIdx.x] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (threadIdx.x >= o) t += y;
        }
        if (threadIdx.x < SCAN_BLOCK / 32) warp_tot[threadIdx.x] = t;
    }
    __syncthreads();
    long long run = boff + ((threadIdx.x >> 5) ? warp_tot[(threadIdx.x >> 5) - 1] : 0) + x - local;
    if (vec && base + SCAN_ITEMS <= n) {
        int32_t r[SCAN_ITEMS];
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            if (run > INT32_MAX) *overflow = 1;
            r[j] = (int32_t)run;
            run += v[j];
        }
        const int4 a = make_int4(r[0], r[1], r[2], r[3]), b = make_int4(r[4], r[5], r[6], r[7]);
        *reinterpret_cast<int4*>(out + base) = a;
        *reinterpret_cast<int4*>(out + base + 4) = b;
        if (out2) {
            *reinterpret_cast<int4*>(out2 + base) = a;
            *reinterpret_cast<int4*>(out2 + base + 4) = b;
        }
    } else {
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            int64_t i = base + j;
            if (i < n) {
                if (run > INT32_MAX) *overflow = 1;
                out[i] = (int32_t)run;
                if (out2) out2[i] = (int32_t)run;
            }
            run += v[j];
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        long long tot = boff + warp_tot[SCAN_BLOCK / 32 - 1];
        sums[gridDim.x] = tot;
        if (tot > INT32_MAX) *overflow = 1;
        out[n] = (int32_t)tot;
        if (out2) out2[n] = (int32_t)tot;
    }
}

fe_status fe_exclusive_scan(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s,
                            int64_t* total_out, int round, int32_t* out2) {
    int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles < 1) ntiles = 1;
    long long* sums = nullptr;
    int* ovf = nullptr;
    fe_status st = fe_alloc_n(&sums, (size_t)ntiles + 1, "scan tile sums");
    if (st) return st;
    st = fe_alloc_n(&ovf, 1, "scan overflow flag");
    if (st) { fe_free(sums); return st; }
    cudaMemsetAsync(ovf, 0, sizeof(int), s);
    const bool vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out) |
                       reinterpret_cast<uintptr_t>(out2)) & 15u) == 0;
    { FE_PROF("k_tile_sums", s); k_tile_sums<<<(unsigned)ntiles, SCAN_BLOCK, 0, s>>>(in, n, sums, round, vec); }
    { FE_PROF("k_tile_scan", s); k_tile_scan<<<(unsigned)ntiles, SCAN_BLOCK, 0, s>>>(in, out, out2, n, sums, ovf, round, vec); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { fe_free(sums); fe_free(ovf); return fe_cuda_fail(e, "scan kernels"); }
    fe_status ret = FE_OK;
    if (total_out) {
        long long tot = 0;
        int ov = 0;
        e = cudaMemcpyAsync(&tot, sums + ntiles, sizeof(tot), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ov, ovf, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) ret = fe_cuda_fail(e, "scan total read-back");
        else if (ov || tot > INT32_MAX) ret = fe_fail(FE_ERR_LIMIT, "prefix sum exceeds int32 (too many non-zeros)");
        else *total_out = tot;
    }
    fe_free(sums);
    fe_free(ovf);
    return ret;
}

// ------------------------------------------------------------------------ kernel timing
//
// When enabled, every kernel launch of the library is bracketed by two CUDA events recorded
// on its launch stream (skipped while the stream is being captured into a graph). Pending
// event pairs are resolved into per-kernel totals by fe_profile_read.

#include <map>
#include <vector>

namespace {
struct Pending {
    const char* name;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free_events;
std::map<std::string, std::pair<double, long long>> g_totals;

cudaEvent_t take_event() {
    if (!g_free_events.empty()) {
        cudaEvent_t e = g_free_events.back();
        g_free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}
}  // namespace

FeProf::FeProf(const char* name, cudaStream_t s) : name_(name), s_(s) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) { cudaGetLastError(); return; }
    a_ = take_event();
    if (a_ && cudaEventRecord(a_, s) != cudaSuccess) { cudaGetLastError(); g_free_events.push_back(a_); a_ = nullptr; }
}

FeProf::~FeProf() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t b = take_event();
    if (!b || cudaEventRecord(b, s_) != cudaSuccess) {
        cudaGetLastError();
        g_free_events.push_back(a_);
        if (b) g_free_events.push_back(b);
        return;
    }
    g_pending.push_back({name_, a_, b});
}

extern "C" fe_status fe_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return FE_OK;
}

extern "C" fe_status fe_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& p : g_pending) {
        cudaEventSynchronize(p.b);
        g_free_events.push_back(p.a);
        g_free_events.push_back(p.b);
    }
    g_pending.clear();
    g_totals.clear();
    return FE_OK;
}

extern "C" fe_status fe_profile_read(int32_t max_entries, char* names, double* total_ms, int64_t* launches,
                                     int32_t* count) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& p : g_pending) {
        cudaError_t e = cudaEventSynchronize(p.b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e != cudaSuccess) { cudaGetLastError(); continue; }
        auto& t = g_totals[p.name];
        t.first += ms;
        t.second += 1;
        g_free_events.push_back(p.a);
        g_free_events.push_back(p.b);
    }
    g_pending.clear();
    int32_t n = 0;
    for (auto& kv : g_totals) {
        if (n < max_entries) {
            if (names) {
                strncpy(names + 64 * (size_t)n, kv.first.c_str(), 63);
                names[64 * (size_t)n + 63] = 0;
            }
            if (total_ms) total_ms[n] = kv.second.first;
            if (launches) launches[n] = kv.second.second;
        }
        n++;
    }
    if (count) *count = n;
    return FE_OK;
}

// ---------------------------------------------------------------- bounds-checked builds

#include <mutex>
#include <vector>

namespace {
std::mutex g_oob_mu;
std::vector<unsigned long long (*)(int)>& oob_readers() {
    static std::vector<unsigned long long (*)(int)> v;
    return v;
}
}  // namespace

void fe_oob_register(unsigned long long (*reader)(int reset)) {
    std::lock_guard<std::mutex> lk(g_oob_mu);
    oob_readers().push_back(reader);
}

extern "C" fe_status fe_debug_bounds(int32_t* checked, int64_t* violations, int32_t reset) {
    if (checked) {
#ifdef FEASM_BOUNDS_CHECK
        *checked = 1;
#else
        *checked = 0;
#endif
    }
    FE_CUDA(cudaDeviceSynchronize());
    unsigned long long tot = 0;
    {
        std::lock_guard<std::mutex> lk(g_oob_mu);
        for (auto r : oob_readers()) tot += r(reset);
    }
    FE_CUDA(cudaGetLastError());
    if (violations) *violations = (int64_t)tot;
    return FE_OK;
}
