// hh_part.cu -- admissibility partition (Eq. 7, Algorithm 1) on the GPU.
//
// Algorithm 1 is a recursive descent from (root, root).  Its result does not
// depend on the visiting order, so it is run level-synchronously: a frontier
// of candidate pairs is classified in parallel (admissible -> P^G; both
// leaves -> P^H; otherwise the children pairs of Algorithm 1 form the next
// frontier), with prefix sums placing every output.  Both lists are then
// radix-sorted by (target, source) node id.
//
// Admissibility on bounding boxes, squared form, correctly rounded FP64
// operations in a fixed order (bit-identical to a sequential evaluation):
//   diam^2 = sum_a (hi_a - lo_a)^2,
//   dist^2 = sum_a max(0, lo_s,a - hi_t,a, lo_t,a - hi_s,a)^2,
//   admissible iff dist^2 > 0 and max(diam_t^2, diam_s^2) <= (eta*eta) dist^2.
// Touching boxes (dist = 0) are never admissible, which keeps every self
// pair in a dense block.
#include <utility>

#include "hh_internal.h"

namespace {

__device__ __forceinline__ bool admissible(const double* __restrict__ lo, const double* __restrict__ hi, int32_t t,
                                           int32_t s, double eta)
{
    double dt = 0.0, ds = 0.0, g = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double et = __dsub_rn(hi[3 * t + a], lo[3 * t + a]);
        double es = __dsub_rn(hi[3 * s + a], lo[3 * s + a]);
        double g1 = __dsub_rn(lo[3 * s + a], hi[3 * t + a]);
        double g2 = __dsub_rn(lo[3 * t + a], hi[3 * s + a]);
        double gap = 0.0;
        if (g1 > gap) gap = g1;
        if (g2 > gap) gap = g2;
        dt = __dadd_rn(dt, __dmul_rn(et, et));
        ds = __dadd_rn(ds, __dmul_rn(es, es));
        g = __dadd_rn(g, __dmul_rn(gap, gap));
    }
    double dm = dt > ds ? dt : ds;
    return g > 0.0 && dm <= __dmul_rn(__dmul_rn(eta, eta), g);
}

// kind: 0 = admissible, 1 = inadmissible leaf pair, 2 = split target,
// 3 = split source, 4 = split both.
__global__ void k_classify(const int32_t* __restrict__ fr, int64_t nf, const int32_t* __restrict__ nbeg,
                           const int32_t* __restrict__ nend, const double* __restrict__ lo,
                           const double* __restrict__ hi, int leaf, double eta, int8_t* __restrict__ kind,
                           int64_t* __restrict__ cG, int64_t* __restrict__ cH, int64_t* __restrict__ cS)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    int32_t t = fr[2 * i], s = fr[2 * i + 1];
    int32_t zt = nend[t] - nbeg[t], zs = nend[s] - nbeg[s];
    int8_t k;
    if (admissible(lo, hi, t, s, eta)) k = 0;
    else if (zt < leaf && zs < leaf) k = 1;
    else if (zs < leaf) k = 2;
    else if (zt < leaf) k = 3;
    else k = 4;
    kind[i] = k;
    cG[i] = k == 0;
    cH[i] = k == 1;
    cS[i] = k == 2 || k == 3 ? 2 : (k == 4 ? 4 : 0);
}

__global__ void k_emit(const int32_t* __restrict__ fr, int64_t nf, const int8_t* __restrict__ kind,
                       const int64_t* __restrict__ oG, const int64_t* __restrict__ oH, const int64_t* __restrict__ oS,
                       const int32_t* __restrict__ child, int32_t* __restrict__ PG, int32_t* __restrict__ PH,
                       int32_t* __restrict__ nx)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    int32_t t = fr[2 * i], s = fr[2 * i + 1];
    int8_t k = kind[i];
    if (k == 0) {
        PG[2 * oG[i]] = t;
        PG[2 * oG[i] + 1] = s;
    } else if (k == 1) {
        PH[2 * oH[i]] = t;
        PH[2 * oH[i] + 1] = s;
    } else {
        int32_t* o = nx + 2 * oS[i];
        if (k == 2) {
            o[0] = child[2 * t]; o[1] = s;
            o[2] = child[2 * t + 1]; o[3] = s;
        } else if (k == 3) {
            o[0] = t; o[1] = child[2 * s];
            o[2] = t; o[3] = child[2 * s + 1];
        } else {
            o[0] = child[2 * t]; o[1] = child[2 * s];
            o[2] = child[2 * t]; o[3] = child[2 * s + 1];
            o[4] = child[2 * t + 1]; o[5] = child[2 * s];
            o[6] = child[2 * t + 1]; o[7] = child[2 * s + 1];
        }
    }
}

__global__ void k_root_pairs(int B, int32_t* fr)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) { fr[2 * b] = b; fr[2 * b + 1] = b; }
}

__global__ void k_pack(const int32_t* __restrict__ P, int64_t n, int bits, uint64_t* __restrict__ key)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) key[i] = ((uint64_t)(uint32_t)P[2 * i] << bits) | (uint64_t)(uint32_t)P[2 * i + 1];
}

__global__ void k_pack_src(const int32_t* __restrict__ P, int64_t n, int bits, uint64_t* __restrict__ key,
                           int32_t* __restrict__ val)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        key[i] = ((uint64_t)(uint32_t)P[2 * i + 1] << bits) | (uint64_t)(uint32_t)P[2 * i];
        val[i] = (int32_t)i;
    }
}

__global__ void k_unpack(const uint64_t* __restrict__ key, int64_t n, int bits, int32_t* __restrict__ P)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        uint64_t k = key[i];
        P[2 * i] = (int32_t)(k >> bits);
        P[2 * i + 1] = (int32_t)(k & ((1ull << bits) - 1));
    }
}

// row[t] = first key with high part >= t (t in 0..n_nodes).
__global__ void k_rowptr(const uint64_t* __restrict__ key, int64_t n, int bits, int32_t n_nodes, int64_t* row)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > n_nodes) return;
    uint64_t k = (uint64_t)(uint32_t)t << bits;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (key[mid] < k) lo = mid + 1; else hi = mid;
    }
    row[t] = lo;
}

int node_bits(int32_t n_nodes)
{
    int bits = 1;
    while ((1LL << bits) <= n_nodes) ++bits;
    return bits;
}

void sort_blocks(int32_t* P, int64_t n, int32_t n_nodes, int64_t* row, cudaStream_t s)
{
    const int bits = node_bits(n_nodes);
    uint64_t* key = dev_alloc_t<uint64_t>(n, s);
    if (n > 0) {
        k_pack<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(P, n, bits, key);
        HH_CHECK_LAUNCH();
        dev_radix_sort(key, nullptr, n, 2 * bits, s);
        k_unpack<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(key, n, bits, P);
        HH_CHECK_LAUNCH();
    }
    k_rowptr<<<(unsigned)ceil_div(n_nodes + 1, 256), 256, 0, s>>>(key, n, bits, n_nodes, row);
    HH_CHECK_LAUNCH();
    dev_free(key, s);
}

}  // namespace

void free_blocks(hh_blocks* b)
{
    if (!b) return;
    cudaFree(b->PG); cudaFree(b->PH); cudaFree(b->rowG); cudaFree(b->rowH);
    delete b;
}

void source_index(const hh_tree* t, const hh_blocks* b, int32_t* order, int64_t* col, cudaStream_t s)
{
    const int64_t n = b->nG;
    const int bits = node_bits(t->n_nodes);
    uint64_t* key = dev_alloc_t<uint64_t>(n, s);
    if (n > 0) {
        k_pack_src<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(b->PG, n, bits, key, order);
        HH_CHECK_LAUNCH();
        dev_radix_sort(key, order, n, 2 * bits, s);
    }
    k_rowptr<<<(unsigned)ceil_div(t->n_nodes + 1, 256), 256, 0, s>>>(key, n, bits, t->n_nodes, col);
    HH_CHECK_LAUNCH();
    dev_free(key, s);
}

hh_blocks* partition_impl(hh_ctx* ctx, const hh_tree* t, const hh_params& p, cudaStream_t s)
{
    HH_REQUIRE(p.eta > 0.0, HH_ERR_ARG, "eta must be > 0");
    HH_REQUIRE(p.leaf_size == t->params.leaf_size, HH_ERR_ARG, "leaf_size differs from the tree's");
    (void)ctx;
    hh_blocks* B = new hh_blocks();
    try {
        B->tree = t;
        B->params = p;
        int64_t capG = 1 << 12, capH = 1 << 12, capFr = 1 << 12, capNx = 1 << 12;
        while (capFr < t->batch) capFr *= 2;
        int32_t* PG = dev_alloc_t<int32_t>(2 * capG, s);
        int32_t* PH = dev_alloc_t<int32_t>(2 * capH, s);
        int32_t* fr = dev_alloc_t<int32_t>(2 * capFr, s);
        int32_t* nx = dev_alloc_t<int32_t>(2 * capNx, s);
        int64_t nf = t->batch, nG = 0, nH = 0;
        k_root_pairs<<<(unsigned)ceil_div(nf, 128), 128, 0, s>>>(t->batch, fr);
        HH_CHECK_LAUNCH();
        int64_t* tot = dev_alloc_t<int64_t>(3, s);
        auto grow = [&](int32_t*& buf, int64_t& cap, int64_t used, int64_t need) {
            if (need <= cap) return;
            int64_t nc = cap;
            while (nc < need) nc *= 2;
            int32_t* nb = dev_alloc_t<int32_t>(2 * nc, s);
            if (used) HH_CUDA(cudaMemcpyAsync(nb, buf, sizeof(int32_t) * 2 * used, cudaMemcpyDeviceToDevice, s));
            dev_free(buf, s);
            buf = nb;
            cap = nc;
        };
        while (nf > 0) {
            int8_t* kind = dev_alloc_t<int8_t>(nf, s);
            int64_t* c3 = dev_alloc_t<int64_t>(3 * nf, s);
            int64_t* o3 = dev_alloc_t<int64_t>(3 * nf, s);
            k_classify<<<(unsigned)ceil_div(nf, 256), 256, 0, s>>>(fr, nf, t->nbeg, t->nend, t->lo, t->hi,
                                                                   p.leaf_size, p.eta, kind, c3, c3 + nf,
                                                                   c3 + 2 * nf);
            HH_CHECK_LAUNCH();
            for (int j = 0; j < 3; ++j) dev_scan_i64(c3 + j * nf, o3 + j * nf, nf, tot + j, s);
            int64_t h[3];
            HH_CUDA(cudaMemcpyAsync(h, tot, sizeof h, cudaMemcpyDeviceToHost, s));
            HH_CUDA(cudaStreamSynchronize(s));
            grow(PG, capG, nG, nG + h[0]);
            grow(PH, capH, nH, nH + h[1]);
            grow(nx, capNx, 0, h[2]);
            k_emit<<<(unsigned)ceil_div(nf, 256), 256, 0, s>>>(fr, nf, kind, o3, o3 + nf, o3 + 2 * nf, t->child,
                                                               PG + 2 * nG, PH + 2 * nH, nx);
            HH_CHECK_LAUNCH();
            dev_free(kind, s);
            dev_free(c3, s);
            dev_free(o3, s);
            nG += h[0];
            nH += h[1];
            nf = h[2];
            std::swap(fr, nx);
            std::swap(capFr, capNx);
        }
        dev_free(tot, s);
        dev_free(fr, s);
        dev_free(nx, s);
        B->nG = nG;
        B->nH = nH;
        HH_CUDA(cudaMalloc(&B->PG, sizeof(int32_t) * 2 * (nG > 0 ? nG : 1)));
        HH_CUDA(cudaMalloc(&B->PH, sizeof(int32_t) * 2 * (nH > 0 ? nH : 1)));
        if (nG) HH_CUDA(cudaMemcpyAsync(B->PG, PG, sizeof(int32_t) * 2 * nG, cudaMemcpyDeviceToDevice, s));
        if (nH) HH_CUDA(cudaMemcpyAsync(B->PH, PH, sizeof(int32_t) * 2 * nH, cudaMemcpyDeviceToDevice, s));
        dev_free(PG, s);
        dev_free(PH, s);
        HH_CUDA(cudaMalloc(&B->rowG, sizeof(int64_t) * (t->n_nodes + 1)));
        HH_CUDA(cudaMalloc(&B->rowH, sizeof(int64_t) * (t->n_nodes + 1)));
        sort_blocks(B->PG, nG, t->n_nodes, B->rowG, s);
        sort_blocks(B->PH, nH, t->n_nodes, B->rowH, s);
    } catch (...) {
        free_blocks(B);
        throw;
    }
    return B;
}
