// hh_tree.cu -- cluster tree (Definition 1, Section 3.1) on the GPU.
//
// Geometry-based bisection by bounding boxes, read as Morton bisection:
//   1. per-instance bounding cube, 2^21 grid per axis, 63-bit codes with the
//      bits interleaved x, y, z from the top (x highest);
//   2. stable LSD radix sort of (code, row) -- ties keep input order;
//   3. breadth-first, level-synchronous bisection: a node with
//      |tau| >= C_leaf splits at the highest bit on which its first and last
//      codes differ (the midpoint plane of its octree cell), or at
//      begin + |tau|/2 when all its codes are equal; |tau| < C_leaf is a leaf;
//   4. bounding boxes bottom-up as exact min/max of the sorted centres.
// Every floating-point step is a single correctly rounded FP64 operation
// (explicit __d*_rn intrinsics, no FMA), so codes, splits and boxes are
// reproducible bit for bit.
#include <algorithm>

#include "hh_internal.h"

namespace {

__global__ void k_inst_bbox(const double* __restrict__ X, const int64_t* __restrict__ off, double* __restrict__ bb)
{
    const int b = blockIdx.x;
    const int64_t i0 = off[b], i1 = off[b + 1];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double v = X[3 * i + a];
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
    __shared__ double s[6][32];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) { s[a][warp] = lo[a]; s[3 + a][warp] = hi[a]; }
    __syncthreads();
    if (threadIdx.x < 6) {
        int q = threadIdx.x;
        double v = s[q][0];
        for (int w = 1; w < nw; ++w) v = q < 3 ? fmin(v, s[q][w]) : fmax(v, s[q][w]);
        bb[6 * b + q] = v;
    }
}

__device__ __forceinline__ int find_instance(const int64_t* off, int B, int64_t i)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_morton(const double* __restrict__ X, const int64_t* __restrict__ off, int B,
                         const double* __restrict__ bb, int64_t n, uint64_t* __restrict__ codes,
                         int32_t* __restrict__ idx, unsigned* status)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = B > 1 ? find_instance(off, B, i) : 0;
    const double* lo = bb + 6 * b;
    double E = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double e = __dsub_rn(lo[3 + a], lo[a]);
        if (e > E) E = e;
    }
    double s = E > 0.0 ? __ddiv_rn(2097152.0, E) : 0.0;
    uint32_t q[3];
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = X[3 * i + a];
        bad |= !isfinite(x);
        double t = floor(__dmul_rn(__dsub_rn(x, lo[a]), s));
        q[a] = !(t >= 0.0) ? 0u : (t > 2097151.0 ? 2097151u : (uint32_t)t);
    }
    if (bad) atomicOr(status, (unsigned)HH_DEV_NUMERIC);
    uint64_t c = 0;
#pragma unroll
    for (int bit = 20; bit >= 0; --bit)
        c = (c << 3) | ((uint64_t)((q[0] >> bit) & 1u) << 2) | ((uint64_t)((q[1] >> bit) & 1u) << 1) |
            (uint64_t)((q[2] >> bit) & 1u);
    codes[i] = c;
    idx[i] = (int32_t)i;
}

__global__ void k_inst_key(const int32_t* __restrict__ idx, const int64_t* __restrict__ off, int B, int64_t n,
                           uint64_t* __restrict__ key)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) key[i] = (uint64_t)find_instance(off, B, idx[i]);
}

__global__ void k_gather_codes(const uint64_t* __restrict__ codes_in, const int32_t* __restrict__ perm, int64_t n,
                               uint64_t* __restrict__ codes_out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) codes_out[i] = codes_in[perm[i]];
}

__global__ void k_gather_rows(const double* __restrict__ in, const int32_t* __restrict__ perm, int64_t n,
                              double* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        int64_t p = perm[i];
        out[3 * i] = in[3 * p];
        out[3 * i + 1] = in[3 * p + 1];
        out[3 * i + 2] = in[3 * p + 2];
    }
}

__global__ void k_roots(const int64_t* __restrict__ off, int B, int32_t* nbeg, int32_t* nend, int32_t* parent)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) {
        nbeg[b] = (int32_t)off[b];
        nend[b] = (int32_t)off[b + 1];
        parent[b] = -1;
    }
}

// Per node of one level: split position and number of children (0 or 2).
__global__ void k_split(const uint64_t* __restrict__ codes, const int32_t* __restrict__ nbeg,
                        const int32_t* __restrict__ nend, int32_t l0, int32_t l1, int leaf,
                        int32_t* __restrict__ split, int64_t* __restrict__ cnt)
{
    int32_t i = l0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= l1) return;
    int32_t b = nbeg[i], e = nend[i], sz = e - b;
    if (sz < leaf) {
        cnt[i - l0] = 0;
        split[i] = -1;
        return;
    }
    uint64_t d = codes[b] ^ codes[e - 1];
    int32_t s;
    if (d == 0) {
        s = b + sz / 2;
    } else {
        int bit = 63 - __clzll((long long)d);
        // first index in [b, e) with the bit set (codes sorted, prefix above the bit equal)
        int32_t lo = b, hi = e - 1;
        while (lo < hi) {
            int32_t mid = lo + ((hi - lo) >> 1);
            if ((codes[mid] >> bit) & 1u) hi = mid; else lo = mid + 1;
        }
        s = lo;
    }
    split[i] = s;
    cnt[i - l0] = 2;
}

__global__ void k_children(const int32_t* __restrict__ split, const int64_t* __restrict__ coff, int32_t l0,
                           int32_t l1, int32_t* nbeg, int32_t* nend, int32_t* child, int32_t* parent)
{
    int32_t i = l0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= l1) return;
    int32_t s = split[i];
    if (s < 0) {
        child[2 * i] = child[2 * i + 1] = -1;
        return;
    }
    int32_t c0 = l1 + (int32_t)coff[i - l0];
    child[2 * i] = c0;
    child[2 * i + 1] = c0 + 1;
    nbeg[c0] = nbeg[i];
    nend[c0] = s;
    parent[c0] = i;
    nbeg[c0 + 1] = s;
    nend[c0 + 1] = nend[i];
    parent[c0 + 1] = i;
}

// Boxes of one level: leaves from their particles, inner nodes from children.
__global__ void k_boxes(const double* __restrict__ Xs, const int32_t* __restrict__ nbeg,
                        const int32_t* __restrict__ nend, const int32_t* __restrict__ child, int32_t l0, int32_t l1,
                        double* lo, double* hi)
{
    int32_t i = l0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= l1) return;
    int32_t c0 = child[2 * i];
    if (c0 < 0) {
        int32_t b = nbeg[i], e = nend[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double l = Xs[3 * (int64_t)b + a], h = l;
            for (int32_t m = b + 1; m < e; ++m) {
                double v = Xs[3 * (int64_t)m + a];
                l = v < l ? v : l;
                h = v > h ? v : h;
            }
            lo[3 * i + a] = l;
            hi[3 * i + a] = h;
        }
    } else {
        int32_t c1 = child[2 * i + 1];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double l0v = lo[3 * c0 + a], l1v = lo[3 * c1 + a];
            double h0v = hi[3 * c0 + a], h1v = hi[3 * c1 + a];
            lo[3 * i + a] = l1v < l0v ? l1v : l0v;
            hi[3 * i + a] = h1v > h0v ? h1v : h0v;
        }
    }
}

// FP32 (hi, lo) copy of the sorted positions (see sep_split).
__global__ void k_split_pos(const double* __restrict__ X, int64_t n, float* __restrict__ P)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int u = 0; u < 3; ++u) {
        const double v = X[3 * i + u];
        const float h = (float)v;
        P[6 * i + u] = h;
        P[6 * i + 3 + u] = (float)(v - (double)h);
    }
}

}  // namespace

void gather_rows(const double* in, const int32_t* perm, int64_t n, double* out, cudaStream_t s)
{
    if (n <= 0) return;
    k_gather_rows<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(in, perm, n, out);
    HH_CHECK_LAUNCH();
}

void free_tree(hh_tree* t)
{
    if (!t) return;
    cudaFree(t->d_offsets); cudaFree(t->perm); cudaFree(t->codes); cudaFree(t->Xs); cudaFree(t->Xp);
    cudaFree(t->nbeg); cudaFree(t->nend); cudaFree(t->child); cudaFree(t->parent);
    cudaFree(t->lo); cudaFree(t->hi);
    delete t;
}

hh_tree* build_tree_impl(hh_ctx* ctx, const double* X, const int64_t* offsets, int32_t batch, const hh_params& p,
                         cudaStream_t s)
{
    HH_REQUIRE(batch >= 1, HH_ERR_ARG, "batch must be >= 1");
    HH_REQUIRE(offsets[0] == 0, HH_ERR_ARG, "offsets[0] must be 0");
    for (int b = 0; b < batch; ++b)
        HH_REQUIRE(offsets[b + 1] > offsets[b], HH_ERR_ARG, "every instance needs >= 1 particle");
    const int64_t n = offsets[batch];
    HH_REQUIRE(n < (1LL << 30), HH_ERR_ARG, "N must be < 2^30");
    HH_REQUIRE(X != nullptr, HH_ERR_ARG, "X is NULL");

    hh_tree* t = new hh_tree();
    try {
        t->ctx = ctx;
        t->params = p;
        t->n = n;
        t->batch = batch;
        t->offsets.assign(offsets, offsets + batch + 1);
        HH_CUDA(cudaMalloc(&t->d_offsets, sizeof(int64_t) * (batch + 1)));
        HH_CUDA(cudaMemcpyAsync(t->d_offsets, offsets, sizeof(int64_t) * (batch + 1), cudaMemcpyHostToDevice, s));
        HH_CUDA(cudaMalloc(&t->perm, sizeof(int32_t) * n));
        HH_CUDA(cudaMalloc(&t->codes, sizeof(uint64_t) * n));
        HH_CUDA(cudaMalloc(&t->Xs, sizeof(double) * 3 * n));
        HH_CUDA(cudaMalloc(&t->Xp, sizeof(float) * 6 * n));

        // 1. Morton codes per instance
        double* bb = dev_alloc_t<double>(6 * batch, s);
        k_inst_bbox<<<batch, 256, 0, s>>>(X, t->d_offsets, bb);
        HH_CHECK_LAUNCH();
        uint64_t* codes0 = dev_alloc_t<uint64_t>(n, s);
        uint64_t* keys = dev_alloc_t<uint64_t>(n, s);
        k_morton<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(X, t->d_offsets, batch, bb, n, codes0, t->perm,
                                                            ctx->d_status);
        HH_CHECK_LAUNCH();
        HH_CUDA(cudaMemcpyAsync(keys, codes0, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        // 2. stable sort by code, then (stable) by instance
        dev_radix_sort(keys, t->perm, n, 63, s);
        if (batch > 1) {
            k_inst_key<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(t->perm, t->d_offsets, batch, n, keys);
            HH_CHECK_LAUNCH();
            int bits = 1;
            while ((1LL << bits) < batch) ++bits;
            dev_radix_sort(keys, t->perm, n, bits, s);
        }
        k_gather_codes<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(codes0, t->perm, n, t->codes);
        HH_CHECK_LAUNCH();
        gather_rows(X, t->perm, n, t->Xs, s);
        k_split_pos<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(t->Xs, n, t->Xp);
        HH_CHECK_LAUNCH();
        dev_free(codes0, s);
        dev_free(keys, s);
        dev_free(bb, s);

        // 3. level-synchronous bisection
        const int64_t cap = 2 * n + batch;
        HH_CUDA(cudaMalloc(&t->nbeg, sizeof(int32_t) * cap));
        HH_CUDA(cudaMalloc(&t->nend, sizeof(int32_t) * cap));
        HH_CUDA(cudaMalloc(&t->child, sizeof(int32_t) * 2 * cap));
        HH_CUDA(cudaMalloc(&t->parent, sizeof(int32_t) * cap));
        int32_t* split = dev_alloc_t<int32_t>(cap, s);
        int64_t* cnt = dev_alloc_t<int64_t>(cap, s);
        int64_t* coff = dev_alloc_t<int64_t>(cap, s);
        int64_t* tot = dev_alloc_t<int64_t>(1, s);
        k_roots<<<(unsigned)ceil_div(batch, 128), 128, 0, s>>>(t->d_offsets, batch, t->nbeg, t->nend, t->parent);
        HH_CHECK_LAUNCH();
        t->level_start = {0, batch};
        int32_t l0 = 0, l1 = batch;
        while (l1 > l0) {
            int32_t m = l1 - l0;
            k_split<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(t->codes, t->nbeg, t->nend, l0, l1, p.leaf_size, split,
                                                               cnt);
            HH_CHECK_LAUNCH();
            dev_scan_i64(cnt, coff, m, tot, s);
            k_children<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(split, coff, l0, l1, t->nbeg, t->nend, t->child,
                                                                  t->parent);
            HH_CHECK_LAUNCH();
            int64_t h_tot = 0;
            HH_CUDA(cudaMemcpyAsync(&h_tot, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            HH_CUDA(cudaStreamSynchronize(s));
            HH_REQUIRE(l1 + h_tot <= cap, HH_ERR_CUDA, "tree capacity exceeded");
            l0 = l1;
            l1 = l1 + (int32_t)h_tot;
            if (l1 > l0) t->level_start.push_back(l1);
        }
        t->n_nodes = l1;
        dev_free(split, s);
        dev_free(cnt, s);
        dev_free(coff, s);
        dev_free(tot, s);

        // 4. bounding boxes, deepest level first
        HH_CUDA(cudaMalloc(&t->lo, sizeof(double) * 3 * t->n_nodes));
        HH_CUDA(cudaMalloc(&t->hi, sizeof(double) * 3 * t->n_nodes));
        for (int L = (int)t->level_start.size() - 2; L >= 0; --L) {
            int32_t a = t->level_start[L], b = t->level_start[L + 1];
            k_boxes<<<(unsigned)ceil_div(b - a, 128), 128, 0, s>>>(t->Xs, t->nbeg, t->nend, t->child, a, b, t->lo,
                                                                   t->hi);
            HH_CHECK_LAUNCH();
        }
    } catch (...) {
        free_tree(t);
        throw;
    }
    return t;
}
