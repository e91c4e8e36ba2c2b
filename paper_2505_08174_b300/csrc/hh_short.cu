// hh_short.cu -- the short-range terms of Eq. 6, M^(s,2) + M^(t,3) + M^(s,3)
// (Eq. 2 sums with the normalisations of Eq. 4), over neighbours within R_cut:
//
//   two-body self part, j in N(i), r = x_i - x_j, d = |r|:
//     U_i += (a/d)^4 / d * S(MLP_s([r/d, a/d])) F_i
//   three-body, 3-cliques (j, k, i): i, j in N(k), j != i, i.e. k in N(i)
//   and j in N(k) \ {i}; r_ji = x_j - x_i, r_ki = x_k - x_i, d_jk = |x_j - x_k|:
//     o = MLP_3([r_ji/|r_ji|, r_ki/|r_ki|, a/d_jk])   (12 outputs)
//     U_i += (S(o_0..5) F_i + S(o_6..11) F_j) / (d_jk |r_ki|)
//
// N(i) = { j != i in the same suspension : |x_i - x_j| < R_cut }.
// Neighbour search: a uniform grid of cell size R_cut per suspension (cell
// keys carry the suspension index, so batched suspensions never interact),
// keys radix-sorted with the particle index as a stable tie-break, then for
// each particle the 27 surrounding cells are found by binary search.  The
// neighbour list (CSR) is written in a fixed order (cells dz, dy, dx, then
// particle index), so every sum below has a fixed order and the results are
// bit-reproducible.
//
// Evaluation: one warp per target particle; its lanes take the pair terms
// and then the target's 3-cliques, flattened over (k, j) by a warp prefix sum
// of |N(k)| for 32 neighbours k at a time; each lane evaluates the MLP of its
// pair or clique in the working precision (FP64 for HH_FP64, FP32 otherwise)
// with the parameters in shared memory, and the warp sums the lanes' 3-vectors
// in a fixed order.  The sums are added to the caller's per-particle array.
#include <algorithm>

#include "hh_internal.h"

namespace {

constexpr int SR_WARPS = 4;        // warps (targets in flight) per CTA
constexpr int SR_CELL_BITS = 16;   // grid coordinates per axis < 2^16
constexpr uint64_t SR_CELL_MASK = (1ull << SR_CELL_BITS) - 1;

template <int DIN, int W, int DOUT>
__host__ __device__ constexpr int mlp_size() { return DIN * W + W + 2 * (W * W + W) + W * DOUT + DOUT; }

// MLP DIN -> W -> W -> W -> DOUT (SiLU), parameters packed per layer as
// W[out, in] then b[out], in shared memory.
template <typename R, int DIN, int W, int DOUT>
__device__ void mlp_any(const R* __restrict__ th, const R* f, R* o)
{
    const R* W1 = th;
    const R* b1 = W1 + DIN * W;
    const R* W2 = b1 + W;
    const R* b2 = W2 + W * W;
    const R* W3 = b2 + W;
    const R* b3 = W3 + W * W;
    const R* W4 = b3 + W;
    const R* b4 = W4 + DOUT * W;
    R h[W], g[W];
#pragma unroll 4
    for (int j = 0; j < W; ++j) {
        R t = b1[j];
#pragma unroll
        for (int i = 0; i < DIN; ++i) t += W1[DIN * j + i] * f[i];
        h[j] = silu<R>(t);
    }
#pragma unroll 2
    for (int j = 0; j < W; ++j) {
        R t = b2[j];
#pragma unroll 8
        for (int i = 0; i < W; ++i) t += W2[W * j + i] * h[i];
        g[j] = silu<R>(t);
    }
#pragma unroll 2
    for (int j = 0; j < W; ++j) {
        R t = b3[j];
#pragma unroll 8
        for (int i = 0; i < W; ++i) t += W3[W * j + i] * g[i];
        h[j] = silu<R>(t);
    }
#pragma unroll 1
    for (int j = 0; j < DOUT; ++j) {
        R t = b4[j];
#pragma unroll 8
        for (int i = 0; i < W; ++i) t += W4[W * j + i] * h[i];
        o[j] = t;
    }
}

template <typename R>
__device__ __forceinline__ void sym_apply(const R* o, const double* F, R* u)   // u += S(o) F
{
    const R f0 = (R)F[0], f1 = (R)F[1], f2 = (R)F[2];
    u[0] += o[0] * f0 + o[3] * f1 + o[4] * f2;
    u[1] += o[3] * f0 + o[1] * f1 + o[5] * f2;
    u[2] += o[4] * f0 + o[5] * f1 + o[2] * f2;
}

// ---- neighbour lists -----------------------------------------------------------
__global__ void k_inst_of(const int64_t* __restrict__ off, int B, int64_t n, int32_t* __restrict__ inst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    inst[i] = lo;
}

// lo[b] = per-axis minimum of suspension b (one CTA per suspension).
__global__ void k_inst_lo(const double* __restrict__ X, const int64_t* __restrict__ off, double* __restrict__ lo)
{
    __shared__ double red[3][256];
    const int b = blockIdx.x;
    double m[3] = {1e300, 1e300, 1e300};
    for (int64_t i = off[b] + threadIdx.x; i < off[b + 1]; i += blockDim.x)
        for (int u = 0; u < 3; ++u) m[u] = fmin(m[u], X[3 * i + u]);
    for (int u = 0; u < 3; ++u) red[u][threadIdx.x] = m[u];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int u = 0; u < 3; ++u) red[u][threadIdx.x] = fmin(red[u][threadIdx.x], red[u][threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int u = 0; u < 3; ++u) lo[3 * b + u] = red[u][0];
}

__device__ __forceinline__ bool cell_of(const double* x, const double* lo, double inv_rc, int c[3])
{
    bool ok = true;
    for (int u = 0; u < 3; ++u) {
        const double v = floor((x[u] - lo[u]) * inv_rc);
        ok = ok && v >= 0.0 && v < (double)SR_CELL_MASK;
        c[u] = (int)fmin(fmax(v, 0.0), (double)(SR_CELL_MASK - 1));
    }
    return ok;
}

__device__ __forceinline__ uint64_t cell_key(int inst, int cx, int cy, int cz)
{
    return ((uint64_t)inst << (3 * SR_CELL_BITS)) | ((uint64_t)cz << (2 * SR_CELL_BITS)) |
           ((uint64_t)cy << SR_CELL_BITS) | (uint64_t)cx;
}

__global__ void k_cell_keys(const double* __restrict__ X, const int32_t* __restrict__ inst, const double* __restrict__ lo,
                            int64_t n, double inv_rc, uint64_t* __restrict__ key, int32_t* __restrict__ idx,
                            unsigned* status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3];
    const int b = inst[i];
    if (!cell_of(X + 3 * i, lo + 3 * b, inv_rc, c)) atomicOr(status, (unsigned)HH_DEV_NUMERIC);
    key[i] = cell_key(b, c[0], c[1], c[2]);
    idx[i] = (int32_t)i;
}

__device__ __forceinline__ int64_t lower_key(const uint64_t* __restrict__ k, int64_t n, uint64_t v)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (k[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Pass 0 counts the neighbours of every particle, pass 1 writes them at off[i].
__global__ void k_neighbours(const double* __restrict__ X, const int32_t* __restrict__ inst,
                             const double* __restrict__ lo, int64_t n, double rc, double inv_rc,
                             const uint64_t* __restrict__ skey, const int32_t* __restrict__ sidx,
                             int64_t* __restrict__ cnt, const int64_t* __restrict__ off, int32_t* __restrict__ nbr)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = inst[i];
    int c[3];
    cell_of(X + 3 * i, lo + 3 * b, inv_rc, c);
    const double xi = X[3 * i], yi = X[3 * i + 1], zi = X[3 * i + 2], rc2 = rc * rc;
    int64_t w = off ? off[i] : 0, count = 0;
    for (int dz = -1; dz <= 1; ++dz) {
        const int cz = c[2] + dz;
        if (cz < 0 || cz >= (int)SR_CELL_MASK) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int cy = c[1] + dy;
            if (cy < 0 || cy >= (int)SR_CELL_MASK) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int cx = c[0] + dx;
                if (cx < 0 || cx >= (int)SR_CELL_MASK) continue;
                const uint64_t kk = cell_key(b, cx, cy, cz);
                for (int64_t p = lower_key(skey, n, kk); p < n && skey[p] == kk; ++p) {
                    const int32_t j = sidx[p];
                    if (j == i) continue;
                    const double ex = X[3 * j] - xi, ey = X[3 * j + 1] - yi, ez = X[3 * j + 2] - zi;
                    if (ex * ex + ey * ey + ez * ez < rc2) {
                        if (nbr) nbr[w++] = j;
                        ++count;
                    }
                }
            }
        }
    }
    if (cnt) cnt[i] = count;
}

// ---- the short-range sums --------------------------------------------------------
template <typename R, int W>
struct SrSmem {
    R ths[mlp_size<4, W, 6>()];
    R th3[mlp_size<7, W, 12>()];
    int32_t pre[SR_WARPS][33];
};

template <typename R, int W>
__global__ void __launch_bounds__(32 * SR_WARPS) k_short(const double* __restrict__ X, const double* __restrict__ F,
                                                       int64_t n, const int64_t* __restrict__ off,
                                                       const int32_t* __restrict__ nbr, const R* __restrict__ ths_g,
                                                       const R* __restrict__ th3_g, R a, int two_body, int three_body,
                                                       void* __restrict__ y, int y_double)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SrSmem<R, W>& sm = *reinterpret_cast<SrSmem<R, W>*>(smem_raw);
    for (int x = threadIdx.x; x < mlp_size<4, W, 6>(); x += blockDim.x) sm.ths[x] = ths_g[x];
    for (int x = threadIdx.x; x < mlp_size<7, W, 12>(); x += blockDim.x) sm.th3[x] = th3_g[x];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t* pre = sm.pre[wid];
    for (int64_t i = (int64_t)blockIdx.x * SR_WARPS + wid; i < n; i += (int64_t)gridDim.x * SR_WARPS) {
        const double* xi = X + 3 * i;
        const int64_t b0 = off[i], deg = off[i + 1] - b0;
        R u[3] = {0, 0, 0};
        if (two_body) {
            for (int64_t e = lane; e < deg; e += 32) {
                const int32_t j = nbr[b0 + e];
                const R rx = (R)(xi[0] - X[3 * j]), ry = (R)(xi[1] - X[3 * j + 1]), rz = (R)(xi[2] - X[3 * j + 2]);
                const R id = rsqrt_<R>(rx * rx + ry * ry + rz * rz);
                const R f[4] = {rx * id, ry * id, rz * id, a * id};
                R o[6];
                mlp_any<R, 4, W, 6>(sm.ths, f, o);
                const R q = a * id, c = q * q * q * q * id;
#pragma unroll
                for (int e2 = 0; e2 < 6; ++e2) o[e2] *= c;
                sym_apply(o, F + 3 * i, u);
            }
        }
        if (three_body) {
            for (int64_t k0 = 0; k0 < deg; k0 += 32) {
                // flatten the cliques of up to 32 neighbours k: pre[t] = sum of |N(k_s)| - [i in N(k_s)], s < t
                const int nk = (int)min((int64_t)32, deg - k0);
                int32_t mine = 0;
                if (lane < nk) {
                    const int32_t k = nbr[b0 + k0 + lane];
                    mine = (int32_t)(off[k + 1] - off[k]) - 1;   // i is in N(k) (symmetric relation)
                }
                int32_t incl = mine;
#pragma unroll
                for (int h = 1; h < 32; h <<= 1) {
                    const int32_t v = __shfl_up_sync(0xffffffffu, incl, h);
                    if (lane >= h) incl += v;
                }
                pre[lane + 1] = incl;
                if (lane == 0) pre[0] = 0;
                __syncwarp();
                const int32_t total = pre[nk];
                for (int32_t cidx = lane; cidx < total; cidx += 32) {
                    int s = 0;   // neighbour slot: pre[s] <= cidx < pre[s + 1]
                    while (pre[s + 1] <= cidx) ++s;
                    const int32_t k = nbr[b0 + k0 + s];
                    // the (cidx - pre[s])-th entry of N(k) other than i
                    int64_t pos = off[k] + (cidx - pre[s]);
                    const int64_t ipos = [&] {
                        for (int64_t q = off[k]; q < off[k + 1]; ++q)
                            if (nbr[q] == (int32_t)i) return q;
                        return off[k + 1];
                    }();
                    if (pos >= ipos) ++pos;
                    const int32_t j = nbr[pos];
                    const R rjx = (R)(X[3 * j] - xi[0]), rjy = (R)(X[3 * j + 1] - xi[1]), rjz = (R)(X[3 * j + 2] - xi[2]);
                    const R rkx = (R)(X[3 * k] - xi[0]), rky = (R)(X[3 * k + 1] - xi[1]), rkz = (R)(X[3 * k + 2] - xi[2]);
                    const R dxk = (R)(X[3 * j] - X[3 * k]), dyk = (R)(X[3 * j + 1] - X[3 * k + 1]),
                            dzk = (R)(X[3 * j + 2] - X[3 * k + 2]);
                    const R iji = rsqrt_<R>(rjx * rjx + rjy * rjy + rjz * rjz);
                    const R iki = rsqrt_<R>(rkx * rkx + rky * rky + rkz * rkz);
                    const R ijk = rsqrt_<R>(dxk * dxk + dyk * dyk + dzk * dzk);
                    const R f[7] = {rjx * iji, rjy * iji, rjz * iji, rkx * iki, rky * iki, rkz * iki, a * ijk};
                    R o[12];
                    mlp_any<R, 7, W, 12>(sm.th3, f, o);
                    const R c = ijk * iki;
#pragma unroll
                    for (int e2 = 0; e2 < 12; ++e2) o[e2] *= c;
                    sym_apply(o, F + 3 * i, u);
                    sym_apply(o + 6, F + 3 * j, u);
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) u[e] = warp_sum(u[e]);
        if (lane == 0) {
            if (y_double) {
                double* yd = static_cast<double*>(y) + 3 * i;
                yd[0] += (double)u[0]; yd[1] += (double)u[1]; yd[2] += (double)u[2];
            } else {
                float* yf = static_cast<float*>(y) + 3 * i;
                yf[0] += (float)u[0]; yf[1] += (float)u[1]; yf[2] += (float)u[2];
            }
        }
    }
}

template <typename R, int W>
void launch_short(hh_ctx* ctx, const double* X, const double* F, int64_t n, const int64_t* off,
                  const int32_t* nbr, const hh_params& p, void* y, int y_double, cudaStream_t s)
{
    const R* ths = sizeof(R) == 8 ? (const R*)ctx->sr_theta_s64 : (const R*)ctx->sr_theta_s32;
    const R* th3 = sizeof(R) == 8 ? (const R*)ctx->sr_theta_364 : (const R*)ctx->sr_theta_332;
    const size_t smem = sizeof(SrSmem<R, W>);
    HH_CUDA(cudaFuncSetAttribute(k_short<R, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t grid = std::min<int64_t>(ceil_div(n, SR_WARPS), (int64_t)ctx->n_sm * 8);
    k_short<R, W><<<(unsigned)grid, 32 * SR_WARPS, smem, s>>>(X, F, n, off, nbr, ths, th3, (R)p.radius,
                                                             ctx->sr_two_body, ctx->sr_three_body, y, y_double);
    HH_CHECK_LAUNCH();
}

}  // namespace

void short_range_add(hh_ctx* ctx, const double* X, const double* F, int64_t n, const std::vector<int64_t>& offsets,
                     const int64_t* d_offsets, const hh_params& p, void* y, int y_double, cudaStream_t s)
{
    HH_REQUIRE(ctx->sr_width == 32 || ctx->sr_width == 64, HH_ERR_ARG,
               "short-range terms requested but hh_set_short_range was not called");
    if (n <= 0) return;
    const int B = (int)offsets.size() - 1;
    const double rc = ctx->sr_rcut, inv_rc = 1.0 / rc;
    int32_t* inst = dev_alloc_t<int32_t>(n, s);
    double* lo = dev_alloc_t<double>(3 * B, s);
    uint64_t* key = dev_alloc_t<uint64_t>(n, s);
    int32_t* idx = dev_alloc_t<int32_t>(n, s);
    int64_t* cnt = dev_alloc_t<int64_t>(n + 1, s);
    int64_t* off = dev_alloc_t<int64_t>(n + 1, s);
    k_inst_of<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(d_offsets, B, n, inst);
    HH_CHECK_LAUNCH();
    k_inst_lo<<<(unsigned)B, 256, 0, s>>>(X, d_offsets, lo);
    HH_CHECK_LAUNCH();
    k_cell_keys<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(X, inst, lo, n, inv_rc, key, idx, ctx->d_status);
    HH_CHECK_LAUNCH();
    dev_radix_sort(key, idx, n, 64, s);
    k_neighbours<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(X, inst, lo, n, rc, inv_rc, key, idx, cnt, nullptr,
                                                            nullptr);
    HH_CHECK_LAUNCH();
    HH_CUDA(cudaMemsetAsync(cnt + n, 0, sizeof(int64_t), s));
    dev_scan_i64(cnt, off, n + 1, nullptr, s);
    int64_t total = 0;
    HH_CUDA(cudaMemcpyAsync(&total, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HH_CUDA(cudaStreamSynchronize(s));
    int32_t* nbr = dev_alloc_t<int32_t>(total, s);
    k_neighbours<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(X, inst, lo, n, rc, inv_rc, key, idx, nullptr, off, nbr);
    HH_CHECK_LAUNCH();
    const bool dbl = p.precision == HH_FP64;
    if (ctx->sr_width == 32) {
        if (dbl) launch_short<double, 32>(ctx, X, F, n, off, nbr, p, y, y_double, s);
        else launch_short<float, 32>(ctx, X, F, n, off, nbr, p, y, y_double, s);
    } else {
        if (dbl) launch_short<double, 64>(ctx, X, F, n, off, nbr, p, y, y_double, s);
        else launch_short<float, 64>(ctx, X, F, n, off, nbr, p, y, y_double, s);
    }
    ctx->stats.n_short_pairs = total;
    dev_free(inst, s); dev_free(lo, s); dev_free(key, s); dev_free(idx, s);
    dev_free(cnt, s); dev_free(off, s); dev_free(nbr, s);
}
