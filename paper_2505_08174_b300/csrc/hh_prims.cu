// hh_prims.cu -- device scan and stable LSD radix sort used by the tree,
// the partition and the work lists.  256-thread CTAs, 2048 items per tile,
// warp-synchronous stable ranking with __match_any_sync.

#include <atomic>
#include <utility>
#include <vector>

#include "hh_internal.h"

unsigned long long g_hh_launches = 0;

// Temporaries of the running call (see AllocScope) and the test hook that
// makes an allocation fail.
namespace {
thread_local std::vector<std::pair<void*, cudaStream_t>>* g_live = nullptr;
std::atomic<long long> g_fail_countdown{0};
}  // namespace

void* dev_alloc(size_t bytes, cudaStream_t s)
{
    long long c = g_fail_countdown.load();
    while (c > 0 && !g_fail_countdown.compare_exchange_weak(c, c - 1)) {
    }
    if (c == 1) throw HHError{HH_ERR_OOM, "device allocation failed (injected by hh_debug_fail_alloc)"};
    void* p = nullptr;
    HH_CUDA(cudaMallocAsync(&p, bytes ? bytes : 16, s));
    if (g_live) g_live->emplace_back(p, s);
    return p;
}

void dev_free(void* p, cudaStream_t s)
{
    if (!p) return;
    if (g_live)
        for (auto it = g_live->rbegin(); it != g_live->rend(); ++it)
            if (it->first == p) {
                g_live->erase(std::next(it).base());
                break;
            }
    HH_CUDA(cudaFreeAsync(p, s));
}

AllocScope::AllocScope() : prev_(g_live) { g_live = &live_; }
AllocScope::~AllocScope() { g_live = prev_; }
void AllocScope::release()
{
    // the failed call may have left kernels running on several streams: wait
    // for all of them, then free newest first
    (void)cudaDeviceSynchronize();
    for (auto it = live_.rbegin(); it != live_.rend(); ++it) (void)cudaFreeAsync(it->first, it->second);
    live_.clear();
}

extern "C" void hh_debug_fail_alloc(int64_t n) { g_fail_countdown.store(n > 0 ? n : 0); }

// ---------------------------------------------------------------------------
// Exclusive scan (int64)
// ---------------------------------------------------------------------------
namespace {
constexpr int SCAN_T = 256, SCAN_I = 8, SCAN_TILE = SCAN_T * SCAN_I;

__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                                       int64_t* __restrict__ tile_sum, int64_t n)
{
    __shared__ int64_t s[SCAN_TILE];
    __shared__ int64_t wsum[SCAN_T / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int j = 0; j < SCAN_I; ++j) {
        int64_t i = base + j * SCAN_T + tid;
        s[j * SCAN_T + tid] = i < n ? in[i] : 0;
    }
    __syncthreads();
    int64_t v[SCAN_I], acc = 0;
#pragma unroll
    for (int j = 0; j < SCAN_I; ++j) { v[j] = s[tid * SCAN_I + j]; acc += v[j]; }
    int64_t x = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < SCAN_T / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SCAN_T / 32) wsum[lane] = w;
    }
    __syncthreads();
    int64_t ex = x - acc + (warp > 0 ? wsum[warp - 1] : 0);
#pragma unroll
    for (int j = 0; j < SCAN_I; ++j) { s[tid * SCAN_I + j] = ex; ex += v[j]; }
    if (tid == SCAN_T - 1) tile_sum[blockIdx.x] = ex;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < SCAN_I; ++j) {
        int64_t i = base + j * SCAN_T + tid;
        if (i < n) out[i] = s[j * SCAN_T + tid];
    }
}

__global__ void k_scan_add(int64_t* __restrict__ out, const int64_t* __restrict__ tile_off, int64_t n)
{
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    const int64_t add = tile_off[blockIdx.x];
    for (int j = threadIdx.x; j < SCAN_TILE; j += blockDim.x) {
        int64_t i = base + j;
        if (i < n) out[i] += add;
    }
}

__global__ void k_scan_total(const int64_t* __restrict__ in, const int64_t* __restrict__ out, int64_t n,
                             int64_t* total)
{
    *total = n > 0 ? out[n - 1] + in[n - 1] : 0;
}
}  // namespace

void dev_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total, cudaStream_t s)
{
    if (n <= 0) {
        if (total) HH_CUDA(cudaMemsetAsync(total, 0, sizeof(int64_t), s));
        return;
    }
    int64_t tiles = ceil_div(n, SCAN_TILE);
    int64_t* ts = dev_alloc_t<int64_t>(tiles, s);
    k_scan_tiles<<<(unsigned)tiles, SCAN_T, 0, s>>>(in, out, ts, n);
    HH_CHECK_LAUNCH();
    if (tiles > 1) {
        int64_t* to = dev_alloc_t<int64_t>(tiles, s);
        dev_scan_i64(ts, to, tiles, nullptr, s);
        k_scan_add<<<(unsigned)tiles, SCAN_T, 0, s>>>(out, to, n);
        HH_CHECK_LAUNCH();
        dev_free(to, s);
    }
    if (total) {
        k_scan_total<<<1, 1, 0, s>>>(in, out, n, total);
        HH_CHECK_LAUNCH();
    }
    dev_free(ts, s);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits.
// Items of a tile are held "striped": item j*256 + tid of the tile belongs to
// thread tid, slot j.  Slots are ranked in order, so tile order (slot-major,
// thread-minor) is the input order and the sort is stable.
// ---------------------------------------------------------------------------
namespace {
constexpr int RS_T = 256, RS_I = 8, RS_TILE = RS_T * RS_I, RS_W = RS_T / 32;

__global__ void __launch_bounds__(RS_T) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                  int64_t n_tiles, int64_t* __restrict__ hist)
{
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int j = 0; j < RS_I; ++j) {
        int64_t i = base + j * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(RS_T) k_rs_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                                                     uint64_t* __restrict__ kout, int32_t* __restrict__ vout,
                                                     int64_t n, int shift, int64_t n_tiles,
                                                     const int64_t* __restrict__ off)
{
    __shared__ int run[256];
    __shared__ int wcnt[RS_W][256];
    __shared__ int64_t goff[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    run[tid] = 0;
    goff[tid] = off[(int64_t)tid * n_tiles + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    for (int j = 0; j < RS_I; ++j) {
        int64_t i = base + j * RS_T + tid;
        bool valid = i < n;
        uint64_t k = valid ? kin[i] : 0;
        int v = (valid && vin) ? vin[i] : 0;
        int d = valid ? (int)((k >> shift) & 255u) : 256;
#pragma unroll
        for (int w = 0; w < RS_W; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = __popc(peers & lt);
        if (valid && before == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int r = run[d] + before;
            for (int w = 0; w < warp; ++w) r += wcnt[w][d];
            int64_t pos = goff[d] + r;
            kout[pos] = k;
            if (vin) vout[pos] = v;
        }
        __syncthreads();
        int tot = 0;
#pragma unroll
        for (int w = 0; w < RS_W; ++w) tot += wcnt[w][tid];
        run[tid] += tot;
        __syncthreads();
    }
}
}  // namespace

void dev_radix_sort(uint64_t* keys, int32_t* vals, int64_t n, int key_bits, cudaStream_t s)
{
    if (n <= 1 || key_bits <= 0) return;
    int passes = (key_bits + 7) / 8;
    int64_t n_tiles = ceil_div(n, RS_TILE);
    uint64_t* k2 = dev_alloc_t<uint64_t>(n, s);
    int32_t* v2 = vals ? dev_alloc_t<int32_t>(n, s) : nullptr;
    int64_t* hist = dev_alloc_t<int64_t>(256 * n_tiles, s);
    int64_t* off = dev_alloc_t<int64_t>(256 * n_tiles, s);
    uint64_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_rs_hist<<<(unsigned)n_tiles, RS_T, 0, s>>>(ka, n, shift, n_tiles, hist);
        HH_CHECK_LAUNCH();
        dev_scan_i64(hist, off, 256 * n_tiles, nullptr, s);
        k_rs_scatter<<<(unsigned)n_tiles, RS_T, 0, s>>>(ka, va, kb, vb, n, shift, n_tiles, off);
        HH_CHECK_LAUNCH();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        HH_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        if (vals) HH_CUDA(cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    dev_free(k2, s);
    dev_free(v2, s);
    dev_free(hist, s);
    dev_free(off, s);
}
