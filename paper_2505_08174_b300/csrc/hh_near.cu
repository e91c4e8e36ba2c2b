// hh_near.cu -- inadmissible (dense) blocks, partial offsets and the final
// FP64 accumulation of U (Section 3.3, "Inadmissible blocks"; Eq. 6).
//
// Near field: one warp per target leaf tau walks every inadmissible block
// (tau, sigma) of its row.  Lane l serves target row (l mod c') and source
// subset (l div c'), c' = next power of two >= |tau| (<= 32), so leaves
// smaller than a warp still keep all lanes busy; the subsets are folded with
// xor-shuffles in a fixed order, so the result is bit-reproducible.  The self
// pair (m == n) is skipped: it is the single-body term alpha_1.
//
// Accumulation: for every particle m (sorted order) the FP64 sum
//   U_m = alpha_1 F_m + y_near(m) + sum over the ancestors tau of m, and the
//         admissible blocks (tau, sigma) of each, of the block partial at m,
// taken root to leaf, sources ascending; written to the caller's row perm[m].
#include <algorithm>

#include "hh_internal.h"

namespace {

constexpr int NEAR_WPB = 4;

template <typename R, int KIND>
__global__ void __launch_bounds__(32 * NEAR_WPB) k_near(const double* __restrict__ Xs, const double* __restrict__ Fs,
                                                        const int32_t* __restrict__ PH, const int64_t* __restrict__ rowH,
                                                        const int32_t* __restrict__ work, int64_t n_work,
                                                        const int32_t* __restrict__ nbeg,
                                                        const int32_t* __restrict__ nend, const R* __restrict__ th_g,
                                                        int n_th, PairParams pp, int transpose, R* __restrict__ y,
                                                        unsigned long long* n_pairs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* th = reinterpret_cast<R*>(smem_raw);
    for (int i = threadIdx.x; i < n_th; i += blockDim.x) th[i] = th_g[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    R* hs = th + n_th + (threadIdx.x >> 5) * act_floats_per_warp<R, KIND>() + lane;
    const int64_t wid = (int64_t)blockIdx.x * NEAR_WPB + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * NEAR_WPB;
    for (int64_t w = wid; w < n_work; w += nwarps) {
        const int32_t tau = work[w];
        const int32_t t0 = nbeg[tau], c = nend[tau] - t0;
        int cp = 1;
        while (cp < c && cp < 32) cp <<= 1;
        const int G = 32 / cp;            // source subsets
        const int row = lane % cp, g = lane / cp;
        const int rpl = (c + 31) / 32;    // rows per lane when c > 32 (then G == 1)
        R acc[4][3];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = acc[i][2] = 0;
        int64_t pairs = 0;
        for (int64_t bb = rowH[tau]; bb < rowH[tau + 1]; ++bb) {
            const int32_t sg = PH[2 * bb + 1];
            const int32_t s0 = nbeg[sg], q = nend[sg] - s0;
            for (int n = g; n < q; n += G) {
                const int64_t gn = s0 + n;
                const double* f = Fs + 3 * gn;
                const R f0 = (R)f[0], f1 = (R)f[1], f2 = (R)f[2];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (i >= rpl) break;
                    const int m = row + 32 * i;
                    if (m >= c) break;
                    const int64_t gm = t0 + m;
                    if (gm == gn) continue;
                    R rx, ry, rz, K[9];
                    if (!transpose) sep<R>(Xs, gm, gn, rx, ry, rz);
                    else sep<R>(Xs, gn, gm, rx, ry, rz);
                    pair_block<R, KIND>(th, pp, rx, ry, rz, K, hs);
                    acc[i][0] += K[0] * f0 + K[1] * f1 + K[2] * f2;
                    acc[i][1] += K[3] * f0 + K[4] * f1 + K[5] * f2;
                    acc[i][2] += K[6] * f0 + K[7] * f1 + K[8] * f2;
                    ++pairs;
                }
            }
        }
        for (int o = cp; o < 32; o <<= 1)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int a = 0; a < 3; ++a) acc[i][a] += __shfl_xor_sync(0xffffffffu, acc[i][a], o);
        if (g == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (i >= rpl) break;
                const int m = row + 32 * i;
                if (m >= c) break;
                R* out = y + 3 * (int64_t)(t0 + m);
                out[0] = acc[i][0]; out[1] = acc[i][1]; out[2] = acc[i][2];
            }
        }
        pairs = warp_sum(pairs);
        if (lane == 0) atomicAdd(n_pairs, (unsigned long long)pairs);
    }
}

// Leaves of this shard: flag[t] = 1 for leaf nodes this shard owns (all
// leaves when mine is NULL).
__global__ void k_leaf_flags(const int32_t* __restrict__ child, int32_t n_nodes, const uint8_t* __restrict__ mine,
                             int64_t* __restrict__ flag)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_nodes) flag[t] = child[2 * t] < 0 && (mine == nullptr || mine[t]);
}

__global__ void k_compact32(const int64_t* __restrict__ flag, const int64_t* __restrict__ off, int64_t n,
                            int32_t* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[off[i]] = (int32_t)i;
}

template <typename R, int KIND>
void launch_near(hh_ctx* ctx, const hh_tree* t, const hh_blocks* b, const hh_params& p, const double* Fs, R* y,
                 const int32_t* work, int64_t n_work, int transpose, cudaStream_t s)
{
    int n_th = 0;
    const R* th = theta_for<R>(ctx, p, &n_th);
    const size_t smem = sizeof(R) * ((size_t)n_th + act_floats_per_warp<R, KIND>() * NEAR_WPB);
    HH_CUDA(cudaFuncSetAttribute(k_near<R, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t blocks = std::min<int64_t>(ceil_div(n_work, NEAR_WPB), (int64_t)ctx->n_sm * 16);
    HH_CUDA(cudaEventRecord(ctx->kev[4], s));
    k_near<R, KIND><<<(unsigned)blocks, 32 * NEAR_WPB, smem, s>>>(
        t->Xs, Fs, b->PH, b->rowH, work, n_work, t->nbeg, t->nend, th, n_th, PairParams{p.radius, p.viscosity},
        transpose, y, ctx->d_counters + 5);
    HH_CHECK_LAUNCH();
    HH_CUDA(cudaEventRecord(ctx->kev[5], s));
    ctx->kev_near_used = 1;
}

template <typename R>
__global__ void k_accum(int64_t n, const double* __restrict__ Fs, const R* __restrict__ ynear,
                        const R* __restrict__ part, const int64_t* __restrict__ pofs, const int64_t* __restrict__ rowG,
                        const int32_t* __restrict__ order, const int32_t* __restrict__ child,
                        const int32_t* __restrict__ nbeg, const int32_t* __restrict__ nend,
                        const int64_t* __restrict__ off, int B, const int32_t* __restrict__ perm, double a1,
                        double* __restrict__ U)
{
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= m) lo = mid; else hi = mid - 1;
    }
    double u0 = a1 * Fs[3 * m], u1 = a1 * Fs[3 * m + 1], u2 = a1 * Fs[3 * m + 2];
    if (ynear) {
        u0 += (double)ynear[3 * m];
        u1 += (double)ynear[3 * m + 1];
        u2 += (double)ynear[3 * m + 2];
    }
    int32_t node = lo;
    if (part) {
        for (;;) {
            const int64_t r0 = rowG[node], r1 = rowG[node + 1];
            const int64_t loc = m - nbeg[node];
            for (int64_t k = r0; k < r1; ++k) {
                const int64_t blk = order ? order[k] : k;
                const R* pb = part + 3 * (pofs[blk] + loc);
                u0 += (double)pb[0];
                u1 += (double)pb[1];
                u2 += (double)pb[2];
            }
            const int32_t c0 = child[2 * node];
            if (c0 < 0) break;
            node = m < nend[c0] ? c0 : child[2 * node + 1];
        }
    }
    const int64_t dst = perm[m];
    U[3 * dst] = u0;
    U[3 * dst + 1] = u1;
    U[3 * dst + 2] = u2;
}

__global__ void k_block_len(const int32_t* __restrict__ PG, int64_t nG, const int32_t* __restrict__ nbeg,
                            const int32_t* __restrict__ nend, int side, int64_t* __restrict__ len)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nG) {
        int32_t nd = PG[2 * b + side];
        len[b] = nend[nd] - nbeg[nd];
    }
}

}  // namespace

void near_field(hh_ctx* ctx, const hh_tree* t, const hh_blocks* b, const hh_params& p, const double* Fs, void* y,
                int transpose, cudaStream_t s)
{
    HH_REQUIRE(p.leaf_size <= 129, HH_ERR_ARG, "leaf_size must be <= 129 (a near-field warp holds <= 128 rows)");
    const int32_t nn = t->n_nodes;
    int64_t* flag = dev_alloc_t<int64_t>(nn, s);
    int64_t* off = dev_alloc_t<int64_t>(nn, s);
    int64_t* tot = dev_alloc_t<int64_t>(1, s);
    uint8_t* mine = shard_node_flags(t, b, p, s);
    k_leaf_flags<<<(unsigned)ceil_div(nn, 256), 256, 0, s>>>(t->child, nn, mine, flag);
    HH_CHECK_LAUNCH();
    if (mine) dev_free(mine, s);
    dev_scan_i64(flag, off, nn, tot, s);
    int64_t n_work = 0;
    HH_CUDA(cudaMemcpyAsync(&n_work, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HH_CUDA(cudaStreamSynchronize(s));
    int32_t* work = dev_alloc_t<int32_t>(n_work, s);
    k_compact32<<<(unsigned)ceil_div(nn, 256), 256, 0, s>>>(flag, off, nn, work);
    HH_CHECK_LAUNCH();
    HH_CUDA(cudaMemsetAsync(y, 0, (size_t)real_bytes(p) * 3 * t->n, s));
    if (n_work > 0 && p.precision == HH_BF16) {
        near_field_tc(ctx, t, b, p, Fs, (float*)y, work, n_work, transpose, s);
    } else if (n_work > 0) {
        const int kind = kernel_kind(p, ctx->width);
        if (p.precision == HH_FP64) {
            if (kind == 0) launch_near<double, 0>(ctx, t, b, p, Fs, (double*)y, work, n_work, transpose, s);
            else if (kind == 1) launch_near<double, 1>(ctx, t, b, p, Fs, (double*)y, work, n_work, transpose, s);
            else launch_near<double, 2>(ctx, t, b, p, Fs, (double*)y, work, n_work, transpose, s);
        } else {
            if (kind == 0) launch_near<float, 0>(ctx, t, b, p, Fs, (float*)y, work, n_work, transpose, s);
            else if (kind == 1) launch_near<float, 1>(ctx, t, b, p, Fs, (float*)y, work, n_work, transpose, s);
            else launch_near<float, 2>(ctx, t, b, p, Fs, (float*)y, work, n_work, transpose, s);
        }
    }
    dev_free(flag, s);
    dev_free(off, s);
    dev_free(tot, s);
    dev_free(work, s);
}

namespace {
template <typename R, int KIND>
__global__ void k_eval_pairs(const double* __restrict__ r, int64_t n, const R* __restrict__ th_g, int n_th,
                             PairParams pp, double* __restrict__ K)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* th = reinterpret_cast<R*>(smem_raw);
    for (int i = threadIdx.x; i < n_th; i += blockDim.x) th[i] = th_g[i];
    __syncthreads();
    R* hs = th + n_th + (threadIdx.x >> 5) * act_floats_per_warp<R, KIND>() + (threadIdx.x & 31);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        R k[9];
        pair_block<R, KIND>(th, pp, (R)r[3 * i], (R)r[3 * i + 1], (R)r[3 * i + 2], k, hs);
#pragma unroll
        for (int e = 0; e < 9; ++e) K[9 * i + e] = (double)k[e];
    }
}

template <typename R, int KIND>
void launch_eval(hh_ctx* ctx, const hh_params& p, const double* r, int64_t n, double* K, cudaStream_t s)
{
    int n_th = 0;
    const R* th = theta_for<R>(ctx, p, &n_th);
    const size_t smem = sizeof(R) * ((size_t)n_th + act_floats_per_warp<R, KIND>() * 4);
    HH_CUDA(cudaFuncSetAttribute(k_eval_pairs<R, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t blocks = std::min<int64_t>(ceil_div(n, 128), (int64_t)ctx->n_sm * 8);
    k_eval_pairs<R, KIND><<<(unsigned)blocks, 128, smem, s>>>(r, n, th, n_th, PairParams{p.radius, p.viscosity}, K);
    HH_CHECK_LAUNCH();
}
}  // namespace

void eval_pairs_simt(hh_ctx* ctx, const hh_params& p, const double* r, int64_t n, double* K, cudaStream_t s)
{
    if (n <= 0) return;
    const int kind = kernel_kind(p, ctx->width);
    if (p.precision == HH_FP64) {
        if (kind == 0) launch_eval<double, 0>(ctx, p, r, n, K, s);
        else if (kind == 1) launch_eval<double, 1>(ctx, p, r, n, K, s);
        else launch_eval<double, 2>(ctx, p, r, n, K, s);
    } else {
        if (kind == 0) launch_eval<float, 0>(ctx, p, r, n, K, s);
        else if (kind == 1) launch_eval<float, 1>(ctx, p, r, n, K, s);
        else launch_eval<float, 2>(ctx, p, r, n, K, s);
    }
}

// Us[m] = alpha1 F_m + y_near(m) (sorted order, FP64): the first terms of
// k_accum's sum, to which the partials of the groups of blocks are added.
template <typename R>
__global__ void k_accum_begin(int64_t n, const double* __restrict__ Fs, const R* __restrict__ ynear, double a1,
                              double* __restrict__ Us)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    for (int u = 0; u < 3; ++u) {
        double v = a1 * Fs[3 * m + u];
        if (ynear) v += (double)ynear[3 * m + u];
        Us[3 * m + u] = v;
    }
}

// Us[m] += the partial outputs of the admissible blocks b0 <= b < b1 that
// contain m, in increasing b -- root to leaf, sources ascending: the order of
// k_accum, so a grouped prediction adds the same terms in the same order.
template <typename R>
__global__ void k_accum_group(int64_t n, const R* __restrict__ part, const int64_t* __restrict__ pofs,
                              int64_t pofs_base, const int64_t* __restrict__ rowG, int64_t b0, int64_t b1,
                              const int32_t* __restrict__ child, const int32_t* __restrict__ nbeg,
                              const int32_t* __restrict__ nend, const int64_t* __restrict__ off, int B,
                              double* __restrict__ Us)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= m) lo = mid; else hi = mid - 1;
    }
    double u0 = Us[3 * m], u1 = Us[3 * m + 1], u2 = Us[3 * m + 2];
    int32_t node = lo;
    for (;;) {
        const int64_t r0 = max(rowG[node], b0), r1 = min(rowG[node + 1], b1);
        const int64_t loc = m - nbeg[node];
        for (int64_t k = r0; k < r1; ++k) {
            const R* pb = part + 3 * (pofs[k] - pofs_base + loc);
            u0 += (double)pb[0];
            u1 += (double)pb[1];
            u2 += (double)pb[2];
        }
        const int32_t c0 = child[2 * node];
        if (c0 < 0) break;
        node = m < nend[c0] ? c0 : child[2 * node + 1];
    }
    Us[3 * m] = u0;
    Us[3 * m + 1] = u1;
    Us[3 * m + 2] = u2;
}

__global__ void k_accum_end(int64_t n, const double* __restrict__ Us, const int32_t* __restrict__ perm,
                            double* __restrict__ U)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const int64_t dst = perm[m];
    for (int u = 0; u < 3; ++u) U[3 * dst + u] = Us[3 * m + u];
}

// First blocks of the groups: cut[k] = the first block whose partial output
// starts at or after k * cap (k = 0 .. n_groups), and the partial offsets
// there (pofs_at[k]; the total past the last block).
__global__ void k_group_cuts(const int64_t* __restrict__ pofs, int64_t nG, int64_t total, int64_t cap, int n_groups,
                             int64_t* __restrict__ cut, int64_t* __restrict__ pofs_at)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n_groups) return;
    int64_t lo = 0, hi = nG;   // first b with pofs[b] >= k * cap (nG if none)
    const int64_t thr = (int64_t)k * cap;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (pofs[mid] >= thr) hi = mid; else lo = mid + 1;
    }
    if (k == n_groups) lo = nG;
    cut[k] = lo;
    pofs_at[k] = lo < nG ? pofs[lo] : total;
}

int64_t partial_offsets(const hh_tree* t, const hh_blocks* b, int transpose, int64_t* pofs, cudaStream_t s)
{
    const int64_t nG = b->nG;
    if (nG == 0) return 0;
    int64_t* len = dev_alloc_t<int64_t>(nG, s);
    int64_t* tot = dev_alloc_t<int64_t>(1, s);
    k_block_len<<<(unsigned)ceil_div(nG, 256), 256, 0, s>>>(b->PG, nG, t->nbeg, t->nend, transpose ? 1 : 0, len);
    HH_CHECK_LAUNCH();
    dev_scan_i64(len, pofs, nG, tot, s);
    int64_t h = 0;
    HH_CUDA(cudaMemcpyAsync(&h, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HH_CUDA(cudaStreamSynchronize(s));
    dev_free(len, s);
    dev_free(tot, s);
    return h;
}

void accumulate_impl(hh_ctx* ctx, const hh_tree* t, const hh_params& p, const double* Fs, const void* y_near,
                     const void* part, const int64_t* pofs, const int64_t* rowG, const int32_t* order, double alpha1,
                     double* U, cudaStream_t s)
{
    (void)ctx;
    const int64_t n = t->n;
    const unsigned grid = (unsigned)ceil_div(n, 256);
    if (real_bytes(p) == 8)
        k_accum<double><<<grid, 256, 0, s>>>(n, Fs, (const double*)y_near, (const double*)part, pofs, rowG, order,
                                             t->child, t->nbeg, t->nend, t->d_offsets, t->batch, t->perm, alpha1, U);
    else
        k_accum<float><<<grid, 256, 0, s>>>(n, Fs, (const float*)y_near, (const float*)part, pofs, rowG, order,
                                            t->child, t->nbeg, t->nend, t->d_offsets, t->batch, t->perm, alpha1, U);
    HH_CHECK_LAUNCH();
}

void accumulate_begin(const hh_tree* t, const hh_params& p, const double* Fs, const void* y_near, double alpha1,
                      double* Us, cudaStream_t s)
{
    const unsigned grid = (unsigned)ceil_div(t->n, 256);
    if (real_bytes(p) == 8) k_accum_begin<double><<<grid, 256, 0, s>>>(t->n, Fs, (const double*)y_near, alpha1, Us);
    else k_accum_begin<float><<<grid, 256, 0, s>>>(t->n, Fs, (const float*)y_near, alpha1, Us);
    HH_CHECK_LAUNCH();
}

void accumulate_group(const hh_tree* t, const hh_params& p, const void* part, const int64_t* pofs, int64_t pofs_base,
                      const int64_t* rowG, int64_t b0, int64_t b1, double* Us, cudaStream_t s)
{
    const unsigned grid = (unsigned)ceil_div(t->n, 256);
    if (real_bytes(p) == 8)
        k_accum_group<double><<<grid, 256, 0, s>>>(t->n, (const double*)part, pofs, pofs_base, rowG, b0, b1, t->child,
                                                   t->nbeg, t->nend, t->d_offsets, t->batch, Us);
    else
        k_accum_group<float><<<grid, 256, 0, s>>>(t->n, (const float*)part, pofs, pofs_base, rowG, b0, b1, t->child,
                                                  t->nbeg, t->nend, t->d_offsets, t->batch, Us);
    HH_CHECK_LAUNCH();
}

void accumulate_end(const hh_tree* t, const double* Us, double* U, cudaStream_t s)
{
    k_accum_end<<<(unsigned)ceil_div(t->n, 256), 256, 0, s>>>(t->n, Us, t->perm, U);
    HH_CHECK_LAUNCH();
}

std::vector<std::pair<int64_t, int64_t>> block_groups(const hh_blocks* b, const int64_t* pofs, int64_t total,
                                                      int64_t cap, std::vector<int64_t>* pofs_at, cudaStream_t s)
{
    const int64_t nG = b->nG;
    std::vector<std::pair<int64_t, int64_t>> g;
    pofs_at->clear();
    if (nG == 0) return g;
    cap = std::max<int64_t>(1, cap);
    const int ng = (int)std::min<int64_t>(ceil_div(std::max<int64_t>(total, 1), cap), 1 << 20);
    int64_t* cut = dev_alloc_t<int64_t>(ng + 1, s);
    int64_t* pa = dev_alloc_t<int64_t>(ng + 1, s);
    k_group_cuts<<<(unsigned)ceil_div(ng + 1, 256), 256, 0, s>>>(pofs, nG, total, cap, ng, cut, pa);
    HH_CHECK_LAUNCH();
    std::vector<int64_t> hc(ng + 1), hp(ng + 1);
    HH_CUDA(cudaMemcpyAsync(hc.data(), cut, sizeof(int64_t) * (ng + 1), cudaMemcpyDeviceToHost, s));
    HH_CUDA(cudaMemcpyAsync(hp.data(), pa, sizeof(int64_t) * (ng + 1), cudaMemcpyDeviceToHost, s));
    HH_CUDA(cudaStreamSynchronize(s));
    dev_free(cut, s);
    dev_free(pa, s);
    for (int k = 0; k < ng; ++k)
        if (hc[k + 1] > hc[k]) {
            g.emplace_back(hc[k], hc[k + 1]);
            pofs_at->push_back(hp[k]);
        }
    if (!g.empty()) pofs_at->push_back(hp[ng]);
    return g;
}
