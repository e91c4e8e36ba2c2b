// hh_api.cu -- the C-ABI of libhhignn (declared in include/hhignn.h).
//
// Orchestrates the stages of one H-matrix mobility product:
//   tree (Definition 1) -> partition (Eq. 7, Algorithm 1) -> ACA on P^G
//   (Algorithm 2) -> dense P^H blocks -> FP64 accumulation of Eq. 6.
// Every entry point catches the library's internal errors and turns them
// into an hh_status plus a message for hh_last_error().
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>

#include <algorithm>
#include <vector>

#include "hh_internal.h"

namespace {

constexpr int kMaxTheta = 16384;

__global__ void k_widen(const float* __restrict__ in, double* __restrict__ out, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}

// Packed layout (W [out,in], b per layer) -> the SIMT layout of mlp_f32:
// W1t [4][w], b1, W2t [w][w], b2, W3t [w][w], b3, W4t [w][8] (zero pad), b4 [8].
__global__ void k_transpose_theta(const float* __restrict__ in, float* __restrict__ out, int w)
{
    const int dims[5] = {4, w, w, w, 6};
    int src = 0, dst = 0;
    for (int l = 0; l < 4; ++l) {
        const int ni = dims[l], no = dims[l + 1], nop = (l == 3) ? 8 : no;
        for (int x = threadIdx.x; x < ni * nop; x += blockDim.x) {
            const int i = x / nop, o = x % nop;
            out[dst + x] = o < no ? in[src + o * ni + i] : 0.0f;
        }
        for (int o = threadIdx.x; o < nop; o += blockDim.x) out[dst + ni * nop + o] = o < no ? in[src + ni * no + o] : 0.0f;
        src += ni * no + no;
        dst += ni * nop + nop;
    }
}

double alpha1(const hh_params& p) { return 1.0 / (6.0 * HH_PI * p.viscosity * p.radius); }

void check_params(const hh_ctx* ctx, const hh_params* p)
{
    HH_REQUIRE(p != nullptr, HH_ERR_ARG, "params is NULL");
    HH_REQUIRE(p->leaf_size >= 2 && p->leaf_size <= 129, HH_ERR_ARG, "leaf_size must be in [2, 129]");
    HH_REQUIRE(p->eta > 0.0, HH_ERR_ARG, "eta must be > 0");
    HH_REQUIRE(p->eps >= 0.0, HH_ERR_ARG, "eps must be >= 0");
    HH_REQUIRE(p->max_rank >= 1 && p->max_rank <= 64, HH_ERR_ARG, "max_rank must be in [1, 64]");
    HH_REQUIRE(p->precision == HH_FP64 || p->precision == HH_FP32 || p->precision == HH_BF16, HH_ERR_ARG,
               "unknown precision");
    HH_REQUIRE(p->kernel == HH_MLP || p->kernel == HH_RPY, HH_ERR_ARG, "unknown kernel");
    HH_REQUIRE(p->precision != HH_BF16 || p->kernel == HH_MLP, HH_ERR_ARG,
               "precision HH_BF16 evaluates the MLP on tensor cores; use HH_FP32/HH_FP64 for HH_RPY");
    HH_REQUIRE(p->kernel == HH_RPY || ctx->n_theta > 0, HH_ERR_ARG, "MLP kernel requested but hh_set_mlp not called");
    HH_REQUIRE(p->radius > 0.0 && p->viscosity > 0.0, HH_ERR_ARG, "radius and viscosity must be > 0");
    HH_REQUIRE(p->n_shards >= 1 && p->shard_id >= 0 && p->shard_id < p->n_shards, HH_ERR_ARG, "bad shard");
    HH_REQUIRE(p->j1_rule == 0 || p->j1_rule == 1, HH_ERR_ARG, "j1_rule must be 0 or 1");
    HH_REQUIRE((p->flags & ~(HH_FLAG_SHORT_RANGE | HH_FLAG_PIVOTS_ONLY)) == 0, HH_ERR_ARG, "unknown flags");
    HH_REQUIRE(p->mem_budget >= 0, HH_ERR_ARG, "mem_budget must be >= 0 (0 = default)");
    HH_REQUIRE(!(p->flags & HH_FLAG_SHORT_RANGE) || ctx->sr_width > 0, HH_ERR_ARG,
               "HH_FLAG_SHORT_RANGE needs hh_set_short_range");
}

// gF[perm[m]] = a1 w(m) + near^T w (m) + far^T w (m), sorted inputs.
__global__ void k_gf_out(const double* __restrict__ Ws, const double* __restrict__ y, const double* __restrict__ far,
                         const int32_t* __restrict__ perm, int64_t n, double a1, double* __restrict__ gF)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const int64_t i = perm[m];
    for (int u = 0; u < 3; ++u) gF[3 * i + u] = a1 * Ws[3 * m + u] + y[3 * m + u] + far[3 * m + u];
}

__global__ void k_fill(double* __restrict__ a, int64_t n, double v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// Runs an entry point: its errors become a status and a message, and the
// temporaries it had taken when it failed are freed.
template <typename F>
hh_status guarded(hh_ctx* ctx, F&& f)
{
    AllocScope scope;
    try {
        hh_status st = f();
        if (ctx) ctx->err.clear();
        return st;
    } catch (const HHError& e) {
        scope.release();
        if (ctx) ctx->err = e.msg;
        return e.st;
    } catch (const std::bad_alloc&) {
        scope.release();
        if (ctx) ctx->err = "host allocation failed";
        return HH_ERR_OOM;
    }
}

// The default memory pool's high-water mark (the library's stream-ordered
// temporaries), reset at the start of a call and read at its end.  Failures
// are not errors of the call: the mark is then reported as -1.
void mem_mark_reset(hh_ctx* ctx)
{
    cudaMemPool_t pool;
    uint64_t zero = 0;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) != cudaSuccess ||
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero) != cudaSuccess)
        (void)cudaGetLastError();
}

int64_t mem_mark_read(hh_ctx* ctx)
{
    cudaMemPool_t pool;
    uint64_t high = 0;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    return (int64_t)high;
}

void reset_call(hh_ctx* ctx, cudaStream_t s)
{
    mem_mark_reset(ctx);
    HH_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), s));
    HH_CUDA(cudaMemsetAsync(ctx->d_counters, 0, 8 * sizeof(unsigned long long), s));
    ctx->last_stream = s;
    ctx->kev_aca_used = 0;
    ctx->kev_near_used = 0;
    ctx->launch_base = g_hh_launches;
    ctx->stats.n_aca_rounds = 0;
    ctx->stats.t_aca_tiles = ctx->stats.t_aca_steps = 0.0;
    ctx->stats.n_aca_groups = 0;
}

// Kernel event times and the launch count of the call (after a stream sync).
void finish_stats(hh_ctx* ctx)
{
    float ms = 0.f;
    double aca = 0.0;
    if (ctx->kev_aca_used & 1) { HH_CUDA(cudaEventElapsedTime(&ms, ctx->kev[0], ctx->kev[1])); aca += ms; }
    if (ctx->kev_aca_used & 2) { HH_CUDA(cudaEventElapsedTime(&ms, ctx->kev[2], ctx->kev[3])); aca += ms; }
    ctx->stats.t_kernel_aca = aca;
    ctx->stats.t_kernel_near = 0.0;
    if (ctx->kev_near_used) {
        HH_CUDA(cudaEventElapsedTime(&ms, ctx->kev[4], ctx->kev[5]));
        ctx->stats.t_kernel_near = ms;
    }
    ctx->stats.n_launches = (int64_t)(g_hh_launches - ctx->launch_base);
    ctx->stats.mem_peak_bytes = mem_mark_read(ctx);
}

hh_status read_status(hh_ctx* ctx, cudaStream_t s)
{
    unsigned st = 0;
    HH_CUDA(cudaMemcpyAsync(&st, ctx->d_status, sizeof st, cudaMemcpyDeviceToHost, s));
    HH_CUDA(cudaStreamSynchronize(s));
    HH_CUDA(cudaGetLastError());
    if (st & HH_DEV_TIMEOUT) throw HHError{HH_ERR_TIMEOUT, "a bounded device wait gave up"};
    if (st & HH_DEV_NUMERIC) throw HHError{HH_ERR_NUMERIC, "non-finite input"};
    return (st & HH_DEV_RANK_CAP) ? HH_WARN_RANK_CAP : HH_OK;
}

__global__ void k_rank_hist(const int32_t* __restrict__ rank, int64_t n, unsigned long long* hist)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&hist[min(rank[i], 64)], 1ull);
}

__global__ void k_fac_len(const int32_t* __restrict__ PG, int64_t nG, const int32_t* __restrict__ nbeg,
                          const int32_t* __restrict__ nend, const int32_t* __restrict__ rank, int64_t* __restrict__ len)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nG) {
        int32_t t = PG[2 * b], s = PG[2 * b + 1];
        len[b] = (int64_t)(nend[t] - nbeg[t] + nend[s] - nbeg[s]) * rank[b];
    }
}

}  // namespace

void check_params_public(const hh_ctx* ctx, const hh_params* p) { check_params(ctx, p); }

void free_hmat(hh_hmat* h)
{
    if (!h) return;
    cudaFree(h->rank); cudaFree(h->pivI); cudaFree(h->pivJ); cudaFree(h->fofs); cudaFree(h->factors);
    cudaFree(h->srank); cudaFree(h->sofs); cudaFree(h->sfac);
    delete h;
}

extern "C" {

void hh_default_params(hh_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->leaf_size = 32;
    p->eta = 1.0;
    p->eps = 1e-4;
    p->max_rank = 48;
    p->precision = HH_FP32;
    p->kernel = HH_MLP;
    p->radius = 1.0;
    p->viscosity = 1.0;
    p->j1_rule = 0;
    p->seed = 0;
    p->shard_id = 0;
    p->n_shards = 1;
    p->flags = 0;
}

hh_status hh_create(hh_ctx** out, int device)
{
    if (!out) return HH_ERR_ARG;
    *out = nullptr;
    hh_ctx* ctx = new hh_ctx();
    int prev = 0;
    cudaGetDevice(&prev);
    hh_status st = guarded(ctx, [&]() {
        int n = 0;
        HH_CUDA(cudaGetDeviceCount(&n));
        HH_REQUIRE(device >= 0 && device < n, HH_ERR_ARG, "no such device");
        HH_CUDA(cudaSetDevice(device));
        ctx->device = device;
        HH_CUDA(cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device));
        cudaMemPool_t pool;
        HH_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
        uint64_t thr = UINT64_MAX;
        HH_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        HH_CUDA(cudaMalloc(&ctx->d_status, 2 * sizeof(unsigned)));   // status bits, MMA-wait stall polls (test)
        HH_CUDA(cudaMalloc(&ctx->d_counters, 8 * sizeof(unsigned long long)));
        HH_CUDA(cudaMemset(ctx->d_status, 0, 2 * sizeof(unsigned)));
        HH_CUDA(cudaMemset(ctx->d_counters, 0, 8 * sizeof(unsigned long long)));
        for (auto& e : ctx->ev) HH_CUDA(cudaEventCreate(&e));
        HH_CUDA(cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
        HH_CUDA(cudaStreamCreateWithFlags(&ctx->aux2, cudaStreamNonBlocking));
        HH_CUDA(cudaEventCreateWithFlags(&ctx->join2_ev, cudaEventDisableTiming));
        HH_CUDA(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
        HH_CUDA(cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming));
        for (auto& e : ctx->kev) HH_CUDA(cudaEventCreate(&e));
        HH_CUDA(cudaEventCreateWithFlags(&ctx->poll_ev, cudaEventDisableTiming));
        HH_CUDA(cudaMallocHost(&ctx->h_pinned, sizeof(int) * 4));
        return HH_OK;
    });
    cudaSetDevice(prev);
    if (st != HH_OK) {
        fprintf(stderr, "hh_create: %s\n", ctx->err.c_str());
        hh_destroy(ctx);
        return st;
    }
    *out = ctx;
    return HH_OK;
}

void hh_destroy(hh_ctx* ctx)
{
    if (!ctx) return;
    cudaFree(ctx->theta32);
    cudaFree(ctx->theta32t);
    cudaFree(ctx->theta64);
    cudaFree(ctx->sr_theta_s32);
    cudaFree(ctx->sr_theta_332);
    cudaFree(ctx->sr_theta_s64);
    cudaFree(ctx->sr_theta_364);
    cudaFree(ctx->d_status);
    cudaFree(ctx->d_counters);
    for (auto& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->aux2) cudaStreamDestroy(ctx->aux2);
    if (ctx->join2_ev) cudaEventDestroy(ctx->join2_ev);
    for (auto& e : ctx->kev)
        if (e) cudaEventDestroy(e);
    if (ctx->poll_ev) cudaEventDestroy(ctx->poll_ev);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    delete ctx;
}

const char* hh_last_error(const hh_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

hh_status hh_set_mlp(hh_ctx* ctx, const float* theta_dev, int width, int depth, void* stream)
{
    if (!ctx) return HH_ERR_ARG;
    return guarded(ctx, [&]() {
        HH_REQUIRE(theta_dev != nullptr, HH_ERR_ARG, "theta is NULL");
        HH_REQUIRE(depth == 3, HH_ERR_ARG, "depth must be 3 (4 -> w -> w -> w -> 6)");
        HH_REQUIRE(width == 32 || width == 64, HH_ERR_ARG, "width must be 32 or 64");
        cudaStream_t s = (cudaStream_t)stream;
        const int n = 4 * width + width + 2 * (width * width + width) + 6 * width + 6;
        HH_REQUIRE(n <= kMaxTheta, HH_ERR_ARG, "too many parameters");
        const int nt = width == 32 ? mlp_t_size<32>() : mlp_t_size<64>();
        if (ctx->theta32) {
            HH_CUDA(cudaDeviceSynchronize());
            cudaFree(ctx->theta32);
            cudaFree(ctx->theta32t);
            cudaFree(ctx->theta64);
        }
        ctx->theta32 = nullptr;
        ctx->theta32t = nullptr;
        ctx->theta64 = nullptr;
        HH_CUDA(cudaMalloc(&ctx->theta32, sizeof(float) * n));
        HH_CUDA(cudaMalloc(&ctx->theta32t, sizeof(float) * nt));
        HH_CUDA(cudaMalloc(&ctx->theta64, sizeof(double) * n));
        HH_CUDA(cudaMemcpyAsync(ctx->theta32, theta_dev, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
        k_widen<<<(n + 255) / 256, 256, 0, s>>>(ctx->theta32, ctx->theta64, n);
        HH_CHECK_LAUNCH();
        k_transpose_theta<<<1, 256, 0, s>>>(ctx->theta32, ctx->theta32t, width);
        HH_CHECK_LAUNCH();
        ctx->width = width;
        ctx->n_theta = n;
        ctx->n_theta_t = nt;
        return HH_OK;
    });
}

hh_status hh_build_tree(hh_ctx* ctx, const double* X_dev, const int64_t* offsets, int32_t batch, const hh_params* p,
                        void* stream, hh_tree** out)
{
    if (!ctx || !out) return HH_ERR_ARG;
    return guarded(ctx, [&]() {
        check_params(ctx, p);
        HH_REQUIRE(offsets != nullptr, HH_ERR_ARG, "offsets is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        reset_call(ctx, s);
        hh_tree* t = build_tree_impl(ctx, X_dev, offsets, batch, *p, s);
        try {
            read_status(ctx, s);
        } catch (...) {
            free_tree(t);
            throw;
        }
        *out = t;
        ctx->stats.n_nodes = t->n_nodes;
        return HH_OK;
    });
}

hh_status hh_partition(hh_ctx* ctx, const hh_tree* tree, const hh_params* p, void* stream, hh_blocks** out)
{
    if (!ctx || !out || !tree) return HH_ERR_ARG;
    return guarded(ctx, [&]() {
        check_params(ctx, p);
        cudaStream_t s = (cudaStream_t)stream;
        *out = partition_impl(ctx, tree, *p, s);
        ctx->stats.n_blocks_G = (*out)->nG;
        ctx->stats.n_blocks_H = (*out)->nH;
        return HH_OK;
    });
}

hh_status hh_aca(hh_ctx* ctx, const hh_tree* tree, const hh_blocks* blocks, const hh_params* p, void* stream,
                 hh_hmat** out)
{
    if (!ctx || !out || !tree || !blocks) return HH_ERR_ARG;
    hh_hmat* h = nullptr;
    hh_status st = guarded(ctx, [&]() {
        check_params(ctx, p);
        HH_REQUIRE(blocks->tree == tree, HH_ERR_ARG, "blocks belong to another tree");
        HH_REQUIRE(p->leaf_size == tree->params.leaf_size && p->eta == blocks->params.eta, HH_ERR_ARG,
                   "leaf_size / eta differ from the partition's");
        cudaStream_t s = (cudaStream_t)stream;
        reset_call(ctx, s);
        h = new hh_hmat();
        h->ctx = ctx;
        h->tree = tree;
        h->blocks = blocks;
        h->params = *p;
        h->real_bytes = real_bytes(*p);
        const int64_t nG = blocks->nG;
        const int64_t nGa = nG > 0 ? nG : 1;
        HH_CUDA(cudaMalloc(&h->rank, sizeof(int32_t) * nGa));
        HH_CUDA(cudaMalloc(&h->pivI, sizeof(int32_t) * nGa * p->max_rank));
        HH_CUDA(cudaMalloc(&h->pivJ, sizeof(int32_t) * nGa * p->max_rank));
        HH_CUDA(cudaMalloc(&h->fofs, sizeof(int64_t) * (nG + 1)));
        HH_CUDA(cudaMemsetAsync(h->rank, 0, sizeof(int32_t) * nGa, s));
        HH_CUDA(cudaMemsetAsync(h->pivI, 0xff, sizeof(int32_t) * nGa * p->max_rank, s));
        HH_CUDA(cudaMemsetAsync(h->pivJ, 0xff, sizeof(int32_t) * nGa * p->max_rank, s));
        HH_CUDA(cudaMemsetAsync(h->fofs, 0, sizeof(int64_t) * (nG + 1), s));
        HH_CUDA(cudaEventRecord(ctx->ev[0], s));
        AcaRun r;
        r.rank = h->rank;
        r.pivI = h->pivI;
        r.pivJ = h->pivJ;
        r.mode = 1;
        aca_run(ctx, tree, blocks, *p, r, s);
        if (nG > 0) {
            int64_t* len = dev_alloc_t<int64_t>(nG, s);
            k_fac_len<<<(unsigned)ceil_div(nG, 256), 256, 0, s>>>(blocks->PG, nG, tree->nbeg, tree->nend, h->rank, len);
            HH_CHECK_LAUNCH();
            dev_scan_i64(len, h->fofs, nG, h->fofs + nG, s);
            HH_CUDA(cudaMemcpyAsync(&h->n_factor, h->fofs + nG, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            HH_CUDA(cudaStreamSynchronize(s));
            dev_free(len, s);
        }
        if (!(p->flags & HH_FLAG_PIVOTS_ONLY)) {
            HH_CUDA(cudaMalloc(&h->factors, (size_t)h->real_bytes * 9 * (h->n_factor > 0 ? h->n_factor : 1)));
            r.factors = h->factors;
            r.fofs = h->fofs;
            r.mode = 2;
            aca_run(ctx, tree, blocks, *p, r, s);
        }
        HH_CUDA(cudaEventRecord(ctx->ev[1], s));
        hh_status w = read_status(ctx, s);
        float ms = 0.f;
        HH_CUDA(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
        ctx->stats.t_aca = ms;
        unsigned long long* hist = dev_alloc_t<unsigned long long>(65, s);
        HH_CUDA(cudaMemsetAsync(hist, 0, 65 * sizeof(unsigned long long), s));
        if (nG > 0) {
            k_rank_hist<<<(unsigned)ceil_div(nG, 256), 256, 0, s>>>(h->rank, nG, hist);
            HH_CHECK_LAUNCH();
        }
        unsigned long long hh[65], cnt[8];
        HH_CUDA(cudaMemcpyAsync(hh, hist, sizeof hh, cudaMemcpyDeviceToHost, s));
        HH_CUDA(cudaMemcpyAsync(cnt, ctx->d_counters, sizeof cnt, cudaMemcpyDeviceToHost, s));
        HH_CUDA(cudaStreamSynchronize(s));
        dev_free(hist, s);
        for (int i = 0; i < 65; ++i) ctx->stats.rank_hist[i] = (int64_t)hh[i];
        ctx->stats.n_aca_queries = (int64_t)cnt[4] / 2;  // the rank loop ran twice
        finish_stats(ctx);
        ctx->stats.n_blocks_G = nG;
        ctx->stats.n_blocks_H = blocks->nH;
        *out = h;
        return w;
    });
    if (st != HH_OK && st != HH_WARN_RANK_CAP) {
        free_hmat(h);
        *out = nullptr;
    }
    return st;
}

hh_status hh_matvec(hh_ctx* ctx, const hh_hmat* h, const double* F_dev, double* U_dev, int transpose, void* stream)
{
    if (!ctx || !h) return HH_ERR_ARG;
    return guarded(ctx, [&]() {
        HH_REQUIRE(F_dev && U_dev, HH_ERR_ARG, "F or U is NULL");
        HH_REQUIRE(h->factors != nullptr || h->sfac != nullptr, HH_ERR_ARG,
                   "H-matrix built with HH_FLAG_PIVOTS_ONLY has no factors");
        cudaStream_t s = (cudaStream_t)stream;
        const hh_tree* t = h->tree;
        const hh_blocks* b = h->blocks;
        const hh_params& p = h->params;
        const int rb = real_bytes(p);
        double* Fs = dev_alloc_t<double>(3 * t->n, s);
        gather_rows(F_dev, t->perm, t->n, Fs, s);
        HH_REQUIRE(!(transpose && (p.flags & HH_FLAG_SHORT_RANGE)), HH_ERR_ARG,
                   "the transposed product does not cover the short-range terms");
        void* y = dev_alloc(rb * 3 * (size_t)t->n, s);
        near_field(ctx, t, b, p, Fs, y, transpose, s);
        if ((p.flags & HH_FLAG_SHORT_RANGE) && p.shard_id == 0)
            short_range_add(ctx, t->Xs, Fs, t->n, t->offsets, t->d_offsets, p, y, rb == 8, s);
        int64_t* pofs = dev_alloc_t<int64_t>(b->nG + 1, s);
        int64_t total = partial_offsets(t, b, transpose, pofs, s);
        void* part = dev_alloc(rb * 3 * (size_t)(total > 0 ? total : 1), s);
        HH_CUDA(cudaEventRecord(ctx->kev[6], s));
        if (h->sfac) recompressed_apply(h, Fs, part, pofs, transpose, s);
        else lowrank_apply(ctx, h, Fs, part, pofs, transpose, s);
        HH_CUDA(cudaEventRecord(ctx->kev[7], s));
        ctx->kev_apply_pending = true;
        int32_t* order = nullptr;
        int64_t* col = nullptr;
        if (transpose) {
            order = dev_alloc_t<int32_t>(b->nG, s);
            col = dev_alloc_t<int64_t>(t->n_nodes + 1, s);
            source_index(t, b, order, col, s);
        }
        double a1 = p.shard_id == 0 ? alpha1(p) : 0.0;
        accumulate_impl(ctx, t, p, Fs, y, b->nG > 0 ? part : nullptr, pofs, transpose ? col : b->rowG, order, a1,
                        U_dev, s);
        dev_free(order, s);
        dev_free(col, s);
        dev_free(part, s);
        dev_free(pofs, s);
        dev_free(y, s);
        dev_free(Fs, s);
        return HH_OK;
    });
}

hh_status hh_predict(hh_ctx* ctx, const double* X_dev, const double* F_dev, const int64_t* offsets, int32_t batch,
                     const hh_params* p, void* stream, double* U_dev)
{
    if (!ctx) return HH_ERR_ARG;
    hh_tree* t = nullptr;
    hh_blocks* b = nullptr;
    hh_status st = guarded(ctx, [&]() {
        check_params(ctx, p);
        HH_REQUIRE(offsets != nullptr && F_dev && U_dev && X_dev, HH_ERR_ARG, "NULL argument");
        cudaStream_t s = (cudaStream_t)stream;
        reset_call(ctx, s);
        cudaEvent_t* ev = ctx->ev;
        HH_CUDA(cudaEventRecord(ev[0], s));
        t = build_tree_impl(ctx, X_dev, offsets, batch, *p, s);
        read_status(ctx, s);  // stop early on non-finite positions
        HH_CUDA(cudaEventRecord(ev[1], s));
        b = partition_impl(ctx, t, *p, s);
        HH_CUDA(cudaEventRecord(ev[2], s));
        const int rb = real_bytes(*p);
        double* Fs = dev_alloc_t<double>(3 * t->n, s);
        gather_rows(F_dev, t->perm, t->n, Fs, s);
        void* y = dev_alloc(rb * 3 * (size_t)t->n, s);
        near_field(ctx, t, b, *p, Fs, y, 0, s);
        ctx->stats.t_short = 0.0;
        ctx->stats.n_short_pairs = 0;
        if ((p->flags & HH_FLAG_SHORT_RANGE) && p->shard_id == 0) {
            HH_CUDA(cudaEventRecord(ev[6], s));
            short_range_add(ctx, t->Xs, Fs, t->n, t->offsets, t->d_offsets, *p, y, rb == 8, s);
            HH_CUDA(cudaEventRecord(ev[7], s));
        }
        HH_CUDA(cudaEventRecord(ev[3], s));
        // the admissible blocks in groups whose partial outputs fit their share
        // of the memory budget, each folded into the FP64 sum before the next
        int64_t* pofs = dev_alloc_t<int64_t>(b->nG + 1, s);
        const int64_t total = partial_offsets(t, b, 0, pofs, s);
        double* Us = dev_alloc_t<double>(3 * t->n, s);
        const double a1 = p->shard_id == 0 ? alpha1(*p) : 0.0;
        accumulate_begin(t, *p, Fs, y, a1, Us, s);
        std::vector<int64_t> pofs_at;
        const auto groups = block_groups(b, pofs, total, budget_partials(*p) / (3 * rb), &pofs_at, s);
        double aca_kernel_ms = 0.0;
        for (size_t g = 0; g < groups.size(); ++g) {
            const int64_t len = pofs_at[g + 1] - pofs_at[g];
            void* part = dev_alloc(rb * 3 * (size_t)(len > 0 ? len : 1), s);
            // blocks of other shards are not written by this call
            if (p->n_shards > 1) HH_CUDA(cudaMemsetAsync(part, 0, rb * 3 * (size_t)(len > 0 ? len : 1), s));
            AcaRun r;
            r.Fs = Fs;
            r.part = part;
            r.pofs = pofs;
            r.pofs_base = pofs_at[g];
            r.b0 = groups[g].first;
            r.b1 = groups[g].second;
            r.mode = 0;
            ctx->kev_aca_used = 0;
            aca_run(ctx, t, b, *p, r, s);
            accumulate_group(t, *p, part, pofs, pofs_at[g], b->rowG, groups[g].first, groups[g].second, Us, s);
            dev_free(part, s);
            if (ctx->kev_aca_used & 2) {   // this group's ACA kernels (the events are reused by the next)
                float ms = 0.f;
                HH_CUDA(cudaEventSynchronize(ctx->kev[3]));
                HH_CUDA(cudaEventElapsedTime(&ms, ctx->kev[2], ctx->kev[3]));
                aca_kernel_ms += ms;
            }
        }
        ctx->kev_aca_used = 0;
        HH_CUDA(cudaEventRecord(ev[4], s));
        accumulate_end(t, Us, U_dev, s);
        HH_CUDA(cudaEventRecord(ev[5], s));
        dev_free(Us, s);
        dev_free(pofs, s);
        dev_free(y, s);
        dev_free(Fs, s);
        hh_status w = read_status(ctx, s);
        float ms[5];
        for (int i = 0; i < 5; ++i) HH_CUDA(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
        ctx->stats.t_tree = ms[0];
        ctx->stats.t_part = ms[1];
        ctx->stats.t_near = ms[2];
        if ((p->flags & HH_FLAG_SHORT_RANGE) && p->shard_id == 0) {
            float msr = 0.f;
            HH_CUDA(cudaEventElapsedTime(&msr, ev[6], ev[7]));
            ctx->stats.t_short = msr;
        }
        ctx->stats.t_aca = ms[3];
        ctx->stats.t_apply = 0.0;
        ctx->stats.t_acc = ms[4];
        ctx->stats.n_nodes = t->n_nodes;
        ctx->stats.n_blocks_G = b->nG;
        ctx->stats.n_blocks_H = b->nH;
        unsigned long long cnt[8];
        HH_CUDA(cudaMemcpy(cnt, ctx->d_counters, sizeof cnt, cudaMemcpyDeviceToHost));
        ctx->stats.n_aca_queries = (int64_t)cnt[4];
        ctx->stats.n_near_pairs = (int64_t)cnt[5];
        ctx->stats.n_aca_groups = (int64_t)groups.size();
        finish_stats(ctx);
        ctx->stats.t_kernel_aca = aca_kernel_ms;
        return w;
    });
    free_blocks(b);
    free_tree(t);
    return st;
}

hh_status hh_eval_pairs(hh_ctx* ctx, const double* r_dev, int64_t n, const hh_params* p, void* stream, double* K_dev)
{
    if (!ctx) return HH_ERR_ARG;
    return guarded(ctx, [&]() {
        check_params(ctx, p);
        HH_REQUIRE(n >= 0 && (n == 0 || (r_dev && K_dev)), HH_ERR_ARG, "NULL argument");
        cudaStream_t s = (cudaStream_t)stream;
        if (p->precision == HH_BF16) eval_pairs_tc(ctx, r_dev, n, p->radius, K_dev, s);
        else eval_pairs_simt(ctx, *p, r_dev, n, K_dev, s);
        return HH_OK;
    });
}

hh_status hh_train_loss_grad(hh_ctx* ctx, const float* theta_dev, int width, const double* r_dev, const double* e_dev,
                             const double* U_dev, int64_t batch, double radius, float* grad_dev, void* stream,
                             double* loss)
{
    if (!ctx) return HH_ERR_ARG;
    return guarded(ctx, [&]() {
        HH_REQUIRE(theta_dev && r_dev && e_dev && loss, HH_ERR_ARG, "NULL argument");
        HH_REQUIRE(radius > 0.0, HH_ERR_ARG, "radius must be > 0");
        *loss = train_loss_grad(ctx, theta_dev, width, r_dev, e_dev, U_dev, batch, radius, grad_dev,
                                (cudaStream_t)stream);
        return HH_OK;
    });
}

hh_status hh_train_step(hh_ctx* ctx, float* theta_dev, float* m_dev, float* v_dev, int64_t step, int width,
                        const double* r_dev, const double* e_dev, const double* U_dev, int64_t batch, double radius,
                        double lr, void* stream, double* loss)
{
    if (!ctx) return HH_ERR_ARG;
    return guarded(ctx, [&]() {
        HH_REQUIRE(theta_dev && m_dev && v_dev && r_dev && e_dev && loss, HH_ERR_ARG, "NULL argument");
        HH_REQUIRE(radius > 0.0 && lr > 0.0, HH_ERR_ARG, "radius and lr must be > 0");
        cudaStream_t s = (cudaStream_t)stream;
        HH_REQUIRE(width == 32 || width == 64, HH_ERR_ARG, "width must be 32 or 64");
        const int P = 4 * width + width + 2 * (width * width + width) + 6 * width + 6;
        float* g = dev_alloc_t<float>(P, s);
        *loss = train_loss_grad(ctx, theta_dev, width, r_dev, e_dev, U_dev, batch, radius, g, s);
        adam_step(theta_dev, g, m_dev, v_dev, P, step, lr, 0.9, 0.999, 1e-8, s);
        dev_free(g, s);
        return HH_OK;
    });
}

hh_status hh_matvec_backward(hh_ctx* ctx, const hh_hmat* h, const double* gU_dev, const double* F_dev, double* gF_dev,
                             double* gX_dev, float* gtheta_dev, void* stream)
{
    if (!ctx || !h) return HH_ERR_ARG;
    if (h->params.flags & HH_FLAG_SHORT_RANGE) {
        ctx->err = "the adjoint covers M^(1) + M^(t,2) only: build the H-matrix without HH_FLAG_SHORT_RANGE";
        return HH_ERR_ARG;
    }
    const bool factors = h->factors != nullptr;
    if (gF_dev && factors) {
        // dL/dF = alpha_1 gU + M_H^T gU: the transposed product
        hh_status st = hh_matvec(ctx, h, gU_dev, gF_dev, 1, stream);
        if (st != HH_OK) return st;
    }
    const bool gF_here = gF_dev && !factors;
    if (!gX_dev && !gtheta_dev && !gF_here) return HH_OK;
    // dL/dX and dL/dtheta differentiate the FP64 rank recursion: a narrower
    // H-matrix is re-approximated in FP64 (pivots only) on the same tree and
    // partition
    hh_hmat* h64 = nullptr;
    if (h->real_bytes != 8) {
        hh_params p64 = h->params;
        p64.precision = HH_FP64;
        p64.flags |= HH_FLAG_PIVOTS_ONLY;
        hh_status st = hh_aca(ctx, h->tree, h->blocks, &p64, stream, &h64);
        if (st != HH_OK && st != HH_WARN_RANK_CAP) return st;
    }
    const hh_hmat* hx = h64 ? h64 : h;
    hh_status st = guarded(ctx, [&]() -> hh_status {
        HH_REQUIRE(gU_dev && F_dev, HH_ERR_ARG, "gU or F is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        const hh_tree* t = hx->tree;
        double* Fs = dev_alloc_t<double>(3 * t->n, s);
        double* Ws = dev_alloc_t<double>(3 * t->n, s);
        gather_rows(F_dev, t->perm, t->n, Fs, s);
        gather_rows(gU_dev, t->perm, t->n, Ws, s);
        double* gFs = nullptr;
        if (gF_here) {
            gFs = dev_alloc_t<double>(3 * t->n, s);
            HH_CUDA(cudaMemsetAsync(gFs, 0, sizeof(double) * 3 * t->n, s));
        }
        matvec_backward_xtheta(ctx, hx, h->params.precision != HH_FP64, Fs, Ws, gX_dev, gtheta_dev, gFs, s);
        if (gF_here) {
            // near part (transposed, FP64) and alpha_1 w, then caller order
            const hh_params& px = hx->params;
            double* y = dev_alloc_t<double>(3 * t->n, s);
            near_field(ctx, t, hx->blocks, px, Ws, y, 1, s);
            const double a1 = px.shard_id == 0 ? alpha1(px) : 0.0;
            k_gf_out<<<(unsigned)ceil_div(t->n, 256), 256, 0, s>>>(Ws, y, gFs, t->perm, t->n, a1, gF_dev);
            HH_CHECK_LAUNCH();
            dev_free(y, s);
            dev_free(gFs, s);
        }
        dev_free(Fs, s);
        dev_free(Ws, s);
        return HH_OK;
    });
    if (h64) hh_hmat_free(h64);
    return st;
}

hh_status hh_export_tree(const hh_tree* t, int32_t* perm, uint64_t* codes, int32_t* node_begin, int32_t* node_end,
                         int32_t* node_child, double* node_lo, double* node_hi, int64_t* n_nodes, int64_t* n)
{
    if (!t) return HH_ERR_ARG;
    return guarded(t->ctx, [&]() {
        HH_CUDA(cudaDeviceSynchronize());
        if (perm) HH_CUDA(cudaMemcpy(perm, t->perm, sizeof(int32_t) * t->n, cudaMemcpyDeviceToHost));
        if (codes) HH_CUDA(cudaMemcpy(codes, t->codes, sizeof(uint64_t) * t->n, cudaMemcpyDeviceToHost));
        if (node_begin) HH_CUDA(cudaMemcpy(node_begin, t->nbeg, sizeof(int32_t) * t->n_nodes, cudaMemcpyDeviceToHost));
        if (node_end) HH_CUDA(cudaMemcpy(node_end, t->nend, sizeof(int32_t) * t->n_nodes, cudaMemcpyDeviceToHost));
        if (node_child)
            HH_CUDA(cudaMemcpy(node_child, t->child, sizeof(int32_t) * 2 * t->n_nodes, cudaMemcpyDeviceToHost));
        if (node_lo) HH_CUDA(cudaMemcpy(node_lo, t->lo, sizeof(double) * 3 * t->n_nodes, cudaMemcpyDeviceToHost));
        if (node_hi) HH_CUDA(cudaMemcpy(node_hi, t->hi, sizeof(double) * 3 * t->n_nodes, cudaMemcpyDeviceToHost));
        if (n_nodes) *n_nodes = t->n_nodes;
        if (n) *n = t->n;
        return HH_OK;
    });
}

hh_status hh_export_blocks(const hh_blocks* b, int32_t* PG, int64_t* nG, int32_t* PH, int64_t* nH)
{
    if (!b) return HH_ERR_ARG;
    return guarded(b->tree->ctx, [&]() {
        HH_CUDA(cudaDeviceSynchronize());
        if (PG && b->nG) HH_CUDA(cudaMemcpy(PG, b->PG, sizeof(int32_t) * 2 * b->nG, cudaMemcpyDeviceToHost));
        if (PH && b->nH) HH_CUDA(cudaMemcpy(PH, b->PH, sizeof(int32_t) * 2 * b->nH, cudaMemcpyDeviceToHost));
        if (nG) *nG = b->nG;
        if (nH) *nH = b->nH;
        return HH_OK;
    });
}

hh_status hh_export_aca(const hh_hmat* h, int32_t* ranks, int32_t* piv_rows, int32_t* piv_cols, int64_t* nG,
                        int32_t* max_rank)
{
    if (!h) return HH_ERR_ARG;
    return guarded(h->ctx, [&]() {
        HH_CUDA(cudaDeviceSynchronize());
        const int64_t n = h->blocks->nG;
        if (ranks && n) HH_CUDA(cudaMemcpy(ranks, h->rank, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
        if (piv_rows && n)
            HH_CUDA(cudaMemcpy(piv_rows, h->pivI, sizeof(int32_t) * n * h->params.max_rank, cudaMemcpyDeviceToHost));
        if (piv_cols && n)
            HH_CUDA(cudaMemcpy(piv_cols, h->pivJ, sizeof(int32_t) * n * h->params.max_rank, cudaMemcpyDeviceToHost));
        if (nG) *nG = n;
        if (max_rank) *max_rank = h->params.max_rank;
        return HH_OK;
    });
}

hh_status hh_export_factors(const hh_hmat* h, int64_t* fofs, void* factors, int64_t* n_factor, int32_t* real_bytes)
{
    if (!h) return HH_ERR_ARG;
    return guarded(h->ctx, [&]() {
        HH_REQUIRE(h->factors != nullptr, HH_ERR_ARG, "H-matrix built with HH_FLAG_PIVOTS_ONLY has no factors");
        HH_CUDA(cudaDeviceSynchronize());
        const int64_t n = h->blocks->nG;
        if (fofs) HH_CUDA(cudaMemcpy(fofs, h->fofs, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost));
        if (factors && h->n_factor > 0)
            HH_CUDA(cudaMemcpy(factors, h->factors, (size_t)h->real_bytes * 9 * h->n_factor, cudaMemcpyDeviceToHost));
        if (n_factor) *n_factor = h->n_factor;
        if (real_bytes) *real_bytes = h->real_bytes;
        return HH_OK;
    });
}

hh_status hh_stats(hh_ctx* ctx, hh_stats_t* out)
{
    if (!ctx || !out) return HH_ERR_ARG;
    return guarded(ctx, [&]() {
        if (ctx->kev_apply_pending) {   // the last hh_matvec's low-rank apply
            float ms = 0.f;
            HH_CUDA(cudaEventSynchronize(ctx->kev[7]));
            HH_CUDA(cudaEventElapsedTime(&ms, ctx->kev[6], ctx->kev[7]));
            ctx->stats.t_apply = ms;
            ctx->kev_apply_pending = false;
        }
        *out = ctx->stats;
        return HH_OK;
    });
}

hh_status hh_recompress(hh_ctx* ctx, hh_hmat* h, double eps_rc, void* stream)
{
    if (!ctx || !h) return HH_ERR_ARG;
    return guarded(ctx, [&]() {
        HH_REQUIRE(h->ctx == ctx, HH_ERR_ARG, "the H-matrix belongs to another context");
        recompress_factors(ctx, h, eps_rc, (cudaStream_t)stream);
        return HH_OK;
    });
}

hh_status hh_export_recompressed(const hh_hmat* h, int32_t* srank, int64_t* sofs, void* sfac, int64_t* n_sfac,
                                 int32_t* real_bytes)
{
    if (!h) return HH_ERR_ARG;
    return guarded(h->ctx, [&]() {
        HH_REQUIRE(h->srank != nullptr, HH_ERR_ARG, "the H-matrix has not been recompressed");
        HH_CUDA(cudaDeviceSynchronize());
        const int64_t n = h->blocks->nG;
        if (srank && n) HH_CUDA(cudaMemcpy(srank, h->srank, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
        if (sofs) HH_CUDA(cudaMemcpy(sofs, h->sofs, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost));
        if (sfac && h->n_sfac > 0)
            HH_CUDA(cudaMemcpy(sfac, h->sfac, (size_t)h->real_bytes * h->n_sfac, cudaMemcpyDeviceToHost));
        if (n_sfac) *n_sfac = h->n_sfac;
        if (real_bytes) *real_bytes = h->real_bytes;
        return HH_OK;
    });
}

hh_status hh_set_short_range(hh_ctx* ctx, const float* theta_s_dev, const float* theta_3_dev, int width,
                             double r_cut, void* stream)
{
    if (!ctx) return HH_ERR_ARG;
    return guarded(ctx, [&]() {
        HH_REQUIRE(width == 32 || width == 64, HH_ERR_ARG, "width must be 32 or 64");
        HH_REQUIRE(r_cut > 0.0 && std::isfinite(r_cut), HH_ERR_ARG, "r_cut must be finite and > 0");
        HH_REQUIRE(theta_s_dev || theta_3_dev, HH_ERR_ARG, "both networks are NULL");
        cudaStream_t s = (cudaStream_t)stream;
        const int ns = 4 * width + width + 2 * (width * width + width) + 6 * width + 6;
        const int n3 = 7 * width + width + 2 * (width * width + width) + 12 * width + 12;
        HH_CUDA(cudaStreamSynchronize(s));
        cudaFree(ctx->sr_theta_s32); cudaFree(ctx->sr_theta_332);
        cudaFree(ctx->sr_theta_s64); cudaFree(ctx->sr_theta_364);
        ctx->sr_theta_s32 = ctx->sr_theta_332 = nullptr;
        ctx->sr_theta_s64 = ctx->sr_theta_364 = nullptr;
        ctx->sr_width = 0;
        HH_CUDA(cudaMalloc(&ctx->sr_theta_s32, sizeof(float) * ns));
        HH_CUDA(cudaMalloc(&ctx->sr_theta_332, sizeof(float) * n3));
        HH_CUDA(cudaMalloc(&ctx->sr_theta_s64, sizeof(double) * ns));
        HH_CUDA(cudaMalloc(&ctx->sr_theta_364, sizeof(double) * n3));
        if (theta_s_dev) HH_CUDA(cudaMemcpyAsync(ctx->sr_theta_s32, theta_s_dev, sizeof(float) * ns, cudaMemcpyDeviceToDevice, s));
        else HH_CUDA(cudaMemsetAsync(ctx->sr_theta_s32, 0, sizeof(float) * ns, s));
        if (theta_3_dev) HH_CUDA(cudaMemcpyAsync(ctx->sr_theta_332, theta_3_dev, sizeof(float) * n3, cudaMemcpyDeviceToDevice, s));
        else HH_CUDA(cudaMemsetAsync(ctx->sr_theta_332, 0, sizeof(float) * n3, s));
        k_widen<<<(ns + 255) / 256, 256, 0, s>>>(ctx->sr_theta_s32, ctx->sr_theta_s64, ns);
        HH_CHECK_LAUNCH();
        k_widen<<<(n3 + 255) / 256, 256, 0, s>>>(ctx->sr_theta_332, ctx->sr_theta_364, n3);
        HH_CHECK_LAUNCH();
        HH_CUDA(cudaStreamSynchronize(s));
        ctx->sr_width = width;
        ctx->sr_two_body = theta_s_dev != nullptr;
        ctx->sr_three_body = theta_3_dev != nullptr;
        ctx->sr_rcut = r_cut;
        return HH_OK;
    });
}

hh_status hh_short_range(hh_ctx* ctx, const double* X_dev, const double* F_dev, const int64_t* offsets,
                         int32_t batch, const hh_params* p, void* stream, double* U_dev)
{
    if (!ctx) return HH_ERR_ARG;
    return guarded(ctx, [&]() -> hh_status {
        HH_REQUIRE(p != nullptr && X_dev && F_dev && U_dev && offsets, HH_ERR_ARG, "NULL argument");
        HH_REQUIRE(batch >= 1 && offsets[0] == 0, HH_ERR_ARG, "bad offsets");
        for (int32_t b = 0; b < batch; ++b) HH_REQUIRE(offsets[b + 1] >= offsets[b], HH_ERR_ARG, "bad offsets");
        HH_REQUIRE(ctx->sr_width > 0, HH_ERR_ARG, "hh_set_short_range was not called");
        HH_REQUIRE(p->radius > 0.0, HH_ERR_ARG, "radius must be > 0");
        cudaStream_t s = (cudaStream_t)stream;
        reset_call(ctx, s);
        std::vector<int64_t> off(offsets, offsets + batch + 1);
        int64_t* d_off = dev_alloc_t<int64_t>(batch + 1, s);
        HH_CUDA(cudaMemcpyAsync(d_off, offsets, sizeof(int64_t) * (batch + 1), cudaMemcpyHostToDevice, s));
        short_range_add(ctx, X_dev, F_dev, off[batch], off, d_off, *p, U_dev, 1, s);
        dev_free(d_off, s);
        return read_status(ctx, s);
    });
}

hh_status hh_set_launch(hh_ctx* ctx, const hh_launch_cfg* cfg)
{
    if (!ctx || !cfg) return HH_ERR_ARG;
    return guarded(ctx, [&]() {
        HH_REQUIRE(cfg->small_max == 0 || (cfg->small_max >= 32 && cfg->small_max <= 512), HH_ERR_ARG,
                   "small_max must be 0 or in [32, 512]");
        auto ok = [](int32_t v) { return v >= 0 && v <= 8; };
        HH_REQUIRE(ok(cfg->aca_small_cps) && ok(cfg->aca_large_cps) && ok(cfg->near_cps), HH_ERR_ARG,
                   "CTAs per SM must be 0 or in [1, 8]");
        HH_REQUIRE(cfg->rounds_min_cq == 0 || (cfg->rounds_min_cq >= 513 && cfg->rounds_min_cq <= (1 << 30)),
                   HH_ERR_ARG, "rounds_min_cq must be 0 or in [513, 2^30]");
        for (int i = 0; i < 3; ++i) HH_REQUIRE(cfg->reserved[i] == 0, HH_ERR_ARG, "reserved fields must be 0");
        ctx->launch = *cfg;
        return HH_OK;
    });
}

hh_status hh_get_launch(hh_ctx* ctx, hh_launch_cfg* cfg)
{
    if (!ctx || !cfg) return HH_ERR_ARG;
    *cfg = ctx->launch;
    return HH_OK;
}

hh_status hh_autotune(hh_ctx* ctx, const double* X_dev, const int64_t* offsets, int32_t batch, const hh_params* p,
                      int32_t reps, void* stream, hh_launch_cfg* best)
{
    if (!ctx || !X_dev || !offsets || !p || batch < 1) return HH_ERR_ARG;
    const int64_t n = offsets[batch];
    if (n < 1) return HH_ERR_ARG;
    if (reps < 1) reps = 1;
    cudaStream_t s = (cudaStream_t)stream;
    double* F = nullptr;
    double* U = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    hh_status st = guarded(ctx, [&]() {
        HH_CUDA(cudaMalloc(&F, sizeof(double) * 3 * n));
        HH_CUDA(cudaMalloc(&U, sizeof(double) * 3 * n));
        k_fill<<<(unsigned)ceil_div(3 * n, 256), 256, 0, s>>>(F, 3 * n, 1.0);
        HH_CHECK_LAUNCH();
        HH_CUDA(cudaEventCreate(&e0));
        HH_CUDA(cudaEventCreate(&e1));
        return HH_OK;
    });
    // median time of reps predictions (after one untimed run) under cfg
    auto score = [&](const hh_launch_cfg& cfg, double* ms) -> hh_status {
        ctx->launch = cfg;
        std::vector<double> t;
        for (int r = 0; r <= reps; ++r) {
            if (cudaEventRecord(e0, s) != cudaSuccess) return HH_ERR_CUDA;
            hh_status q = hh_predict(ctx, X_dev, F, offsets, batch, p, stream, U);
            if (q != HH_OK) return q;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return HH_ERR_CUDA;
            float v = 0.f;
            if (cudaEventElapsedTime(&v, e0, e1) != cudaSuccess) return HH_ERR_CUDA;
            if (r > 0) t.push_back(v);
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return HH_OK;
    };
    const hh_launch_cfg start = ctx->launch;
    hh_launch_cfg cur = start;
    double cur_ms = 0.0;
    if (st == HH_OK) st = score(cur, &cur_ms);
    static const int32_t cand_small_max[] = {128, 256, 512};
    static const int32_t cand_small_cps[] = {1, 2, 3, 4};
    static const int32_t cand_large_cps[] = {1, 2, 4};
    static const int32_t cand_near_cps[] = {2, 4, 5, 8};
    static const int32_t cand_rounds[] = {2048, 4096, 16384};
    struct Field { int32_t hh_launch_cfg::*f; const int32_t* v; int nv; };
    const Field fields[] = {{&hh_launch_cfg::small_max, cand_small_max, 3},
                            {&hh_launch_cfg::aca_small_cps, cand_small_cps, 4},
                            {&hh_launch_cfg::aca_large_cps, cand_large_cps, 3},
                            {&hh_launch_cfg::near_cps, cand_near_cps, 4},
                            {&hh_launch_cfg::rounds_min_cq, cand_rounds, 3}};
    for (const Field& fd : fields) {
        for (int i = 0; i < fd.nv && st == HH_OK; ++i) {
            hh_launch_cfg c = cur;
            if (c.*fd.f == fd.v[i]) continue;
            c.*fd.f = fd.v[i];
            double ms = 0.0;
            st = score(c, &ms);
            if (st == HH_OK && ms < cur_ms) { cur = c; cur_ms = ms; }
        }
    }
    ctx->launch = st == HH_OK ? cur : start;
    if (st == HH_OK && best) *best = cur;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (F) cudaFree(F);
    if (U) cudaFree(U);
    return st;
}

void hh_tree_free(hh_tree* t) { free_tree(t); }
void hh_blocks_free(hh_blocks* b) { free_blocks(b); }
void hh_hmat_free(hh_hmat* h) { free_hmat(h); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Filament suspension: bead forces and the explicit Euler step
// ---------------------------------------------------------------------------
namespace {

FilamentArgs filament_args(const hh_filament_params* fp)
{
    HH_REQUIRE(fp != nullptr, HH_ERR_ARG, "NULL filament parameters");
    FilamentArgs a{fp->k_bond, fp->l0, fp->kappa, {fp->g[0], fp->g[1], fp->g[2]}};
    bool fin = std::isfinite(a.k) && std::isfinite(a.l0) && std::isfinite(a.kappa);
    for (double v : a.g) fin = fin && std::isfinite(v);
    HH_REQUIRE(fin, HH_ERR_ARG, "filament parameters must be finite");
    return a;
}

void check_chains(int64_t n_chains, int32_t beads)
{
    HH_REQUIRE(n_chains >= 0 && beads >= 1, HH_ERR_ARG, "need n_chains >= 0 and beads >= 1");
    HH_REQUIRE(n_chains <= (int64_t)INT32_MAX / beads, HH_ERR_ARG, "n_chains * beads exceeds 2^31 - 1");
}

}  // namespace

hh_status hh_filament_forces(hh_ctx* ctx, const double* X_dev, int64_t n_chains, int32_t beads,
                             const hh_filament_params* fp, void* stream, double* F_dev)
{
    if (!ctx) return HH_ERR_ARG;
    return guarded(ctx, [&]() {
        check_chains(n_chains, beads);
        const FilamentArgs a = filament_args(fp);
        HH_REQUIRE(n_chains == 0 || (X_dev && F_dev), HH_ERR_ARG, "NULL argument");
        cudaStream_t s = (cudaStream_t)stream;
        reset_call(ctx, s);
        filament_forces_launch(ctx, X_dev, n_chains, beads, a, F_dev, s);
        return read_status(ctx, s);
    });
}

hh_status hh_filament_step(hh_ctx* ctx, double* X_dev, int64_t n_chains, int32_t beads, const hh_filament_params* fp,
                           const hh_params* p, double dt, void* stream, double* F_dev, double* U_dev)
{
    if (!ctx) return HH_ERR_ARG;
    const unsigned long long base = g_hh_launches;   // the step's launches, forces through update
    hh_status st = guarded(ctx, [&]() {
        check_chains(n_chains, beads);
        const FilamentArgs a = filament_args(fp);
        check_params(ctx, p);
        HH_REQUIRE(std::isfinite(dt), HH_ERR_ARG, "dt must be finite");
        HH_REQUIRE(n_chains >= 1, HH_ERR_ARG, "need at least one chain");
        HH_REQUIRE(X_dev && F_dev && U_dev, HH_ERR_ARG, "NULL argument");
        cudaStream_t s = (cudaStream_t)stream;
        reset_call(ctx, s);
        filament_forces_launch(ctx, X_dev, n_chains, beads, a, F_dev, s);
        return read_status(ctx, s);
    });
    if (st != HH_OK) return st;
    const int64_t offsets[2] = {0, n_chains * beads};
    st = hh_predict(ctx, X_dev, F_dev, offsets, 1, p, stream, U_dev);
    if (st != HH_OK && st != HH_WARN_RANK_CAP) return st;
    const hh_status st2 = guarded(ctx, [&]() {
        euler_launch(X_dev, U_dev, 3 * n_chains * beads, dt, (cudaStream_t)stream);
        return HH_OK;
    });
    ctx->stats.n_launches = (int64_t)(g_hh_launches - base);
    return st2 != HH_OK ? st2 : st;
}

hh_status hh_simulate(hh_ctx* ctx, double* X_dev, int64_t n_chains, int32_t beads, int64_t n_free,
                      const hh_filament_params* fp, const hh_params* p, double dt, int32_t n_steps,
                      int32_t dump_every, double* X_dump_host, double* t_step_ms, void* stream)
{
    if (!ctx) return HH_ERR_ARG;
    double* F = nullptr;
    double* U = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int64_t n = 0;
    cudaStream_t s = (cudaStream_t)stream;
    FilamentArgs a{};
    // checks and the per-run buffers
    hh_status st = guarded(ctx, [&]() {
        check_chains(n_chains, beads);
        HH_REQUIRE(n_free >= 0 && n_free < (1LL << 30), HH_ERR_ARG, "n_free must be in [0, 2^30)");
        n = n_chains * beads + n_free;
        HH_REQUIRE(n >= 1 && n < (1LL << 30), HH_ERR_ARG, "need 1 <= n_chains * beads + n_free < 2^30");
        a = filament_args(fp);
        check_params(ctx, p);
        HH_REQUIRE(std::isfinite(dt), HH_ERR_ARG, "dt must be finite");
        HH_REQUIRE(n_steps >= 0 && dump_every >= 0, HH_ERR_ARG, "n_steps and dump_every must be >= 0");
        HH_REQUIRE(X_dev != nullptr && (dump_every == 0 || X_dump_host != nullptr), HH_ERR_ARG, "NULL argument");
        HH_CUDA(cudaMalloc(&F, sizeof(double) * 3 * n));
        HH_CUDA(cudaMalloc(&U, sizeof(double) * 3 * n));
        HH_CUDA(cudaEventCreate(&ev[0]));
        HH_CUDA(cudaEventCreate(&ev[1]));
        if (dump_every > 0)
            HH_CUDA(cudaMemcpyAsync(X_dump_host, X_dev, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
        return HH_OK;
    });
    const int64_t offsets[2] = {0, n};
    hh_status worst = HH_OK;
    for (int32_t k = 1; st == HH_OK && k <= n_steps; ++k) {
        st = guarded(ctx, [&]() {
            reset_call(ctx, s);
            HH_CUDA(cudaEventRecord(ev[0], s));
            const int64_t nc = n_chains * beads;
            if (n_chains > 0) filament_forces_launch(ctx, X_dev, n_chains, beads, a, F, s);
            if (n_free > 0) filament_forces_launch(ctx, X_dev + 3 * nc, n_free, 1, a, F + 3 * nc, s);   // g only
            return read_status(ctx, s);
        });
        if (st != HH_OK) break;
        hh_status sp = hh_predict(ctx, X_dev, F, offsets, 1, p, stream, U);
        if (sp != HH_OK && sp != HH_WARN_RANK_CAP) { st = sp; break; }
        if (sp == HH_WARN_RANK_CAP) worst = sp;
        st = guarded(ctx, [&]() {
            euler_launch(X_dev, U, 3 * n, dt, s);
            HH_CUDA(cudaEventRecord(ev[1], s));
            if (dump_every > 0 && k % dump_every == 0)
                HH_CUDA(cudaMemcpyAsync(X_dump_host + (int64_t)(k / dump_every) * 3 * n, X_dev,
                                        sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
            HH_CUDA(cudaEventSynchronize(ev[1]));
            if (t_step_ms) {
                float ms = 0.f;
                HH_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
                t_step_ms[k - 1] = ms;
            }
            return HH_OK;
        });
    }
    if (st == HH_OK && stream != nullptr) (void)cudaStreamSynchronize(s);
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    if (F) cudaFree(F);
    if (U) cudaFree(U);
    return st != HH_OK ? st : worst;
}

extern "C" hh_status hh_debug_stall_mma_waits(hh_ctx* ctx, uint32_t polls)
{
    if (!ctx) return HH_ERR_ARG;
    return guarded(ctx, [&]() {
        HH_CUDA(cudaDeviceSynchronize());
        HH_CUDA(cudaMemcpy(ctx->d_status + 1, &polls, sizeof(unsigned), cudaMemcpyHostToDevice));
        return HH_OK;
    });
}
