// hh_tcmlp.cu -- tensor-core (tcgen05) pair evaluation and the dense
// inadmissible blocks (Section 3.3) built on the MLP tile of hh_tcmlp.cuh.
#include <algorithm>

#include "hh_tcmlp.cuh"

namespace {

template <int W>
struct alignas(128) NearSmem {
    TcCore<W> tc;
    float contrib[TC_T * 3];
    int32_t seg_s0[256], seg_q[256], seg_pre[257];
    int nseg;
};

// ---- pair evaluation: K(r) for a list of separations --------------------------
template <int W>
__global__ void __launch_bounds__(TC_T, 4) k_eval_pairs_tc(const double* __restrict__ r, int64_t n,
                                                          const float* __restrict__ th, float a,
                                                          double* __restrict__ K, unsigned* status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TcCore<W>& sm = *reinterpret_cast<TcCore<W>*>(smem_raw);
    tc_setup<W>(sm, th, status);
    uint32_t phase = 0;
    const int t = threadIdx.x;
    for (int64_t base = (int64_t)blockIdx.x * TC_T; base < n; base += (int64_t)gridDim.x * TC_T) {
        const int64_t i = base + t;
        float f[4], id = 1.f;
        if (i < n) features((float)r[3 * i], (float)r[3 * i + 1], (float)r[3 * i + 2], a, f, id);
        else { f[0] = 1.f; f[1] = f[2] = 0.f; f[3] = a; }
        tc_write_features<W>(sm, t, f);
        float o[6];
        if (!tc_mlp_tile<W>(sm, phase, status, o)) break;
        if (i < n) {
            double* out = K + 9 * i;
            out[0] = o[0] * id; out[1] = o[3] * id; out[2] = o[4] * id;
            out[3] = o[3] * id; out[4] = o[1] * id; out[5] = o[5] * id;
            out[6] = o[4] * id; out[7] = o[5] * id; out[8] = o[2] * id;
        }
    }
    tc_teardown<W>(sm);
}

// ---- near field on tensor cores ----------------------------------------------
// One CTA per target leaf tau at a time.  The sources of all inadmissible
// blocks of tau form a virtual list of Q particles; pair p = v * c + m (v:
// virtual source, m: target) is tile row p mod 128 of tile p / 128.  After
// the MLP, each row's contribution K F_n goes to shared memory and thread m
// adds the rows of its target in increasing order (bit-reproducible).
template <int W>
__global__ void __launch_bounds__(TC_T, 4) k_near_tc(const float* __restrict__ Xp, const double* __restrict__ Fs,
                                                    const int32_t* __restrict__ PH, const int64_t* __restrict__ rowH,
                                                    const int32_t* __restrict__ work, int64_t n_work,
                                                    const int32_t* __restrict__ nbeg, const int32_t* __restrict__ nend,
                                                    const float* __restrict__ th, float a, int transpose,
                                                    float* __restrict__ y, unsigned long long* n_pairs,
                                                    unsigned* status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    NearSmem<W>& sm = *reinterpret_cast<NearSmem<W>*>(smem_raw);
    tc_setup<W>(sm.tc, th, status);
    uint32_t phase = 0;
    const int t = threadIdx.x;
    unsigned long long pairs = 0;
    for (int64_t w = blockIdx.x; w < n_work && !sm.tc.fail; w += gridDim.x) {
        const int32_t tau = work[w];
        const int32_t t0 = nbeg[tau], c = nend[tau] - t0;
        float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
        for (int64_t b0 = rowH[tau]; b0 < rowH[tau + 1] && !sm.tc.fail; b0 += 256) {
            const int64_t left = rowH[tau + 1] - b0;
            const int nseg = left < 256 ? (int)left : 256;
            __syncthreads();
            if (t == 0) {
                int pre = 0;
                for (int i = 0; i < nseg; ++i) {
                    const int32_t sg = PH[2 * (b0 + i) + 1];
                    sm.seg_s0[i] = nbeg[sg];
                    sm.seg_q[i] = nend[sg] - nbeg[sg];
                    sm.seg_pre[i] = pre;
                    pre += sm.seg_q[i];
                }
                sm.seg_pre[nseg] = pre;
                sm.nseg = nseg;
            }
            __syncthreads();
            const int64_t P = (int64_t)sm.seg_pre[nseg] * c;
            for (int64_t p0 = 0; p0 < P; p0 += TC_T) {
                const int64_t p = p0 + t;
                bool valid = p < P;
                int64_t gm = 0, gn = 0;
                float f[4], id = 1.f;
                if (valid) {
                    const int v = (int)(p / c), m = (int)(p - (int64_t)v * c);
                    int lo = 0, hi = nseg - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (sm.seg_pre[mid] <= v) lo = mid; else hi = mid - 1;
                    }
                    gm = t0 + m;
                    gn = sm.seg_s0[lo] + (v - sm.seg_pre[lo]);
                    valid = gm != gn;
                }
                if (valid) {
                    float rx, ry, rz;
                    if (!transpose) sep_split(Xp, gm, gn, rx, ry, rz);
                    else sep_split(Xp, gn, gm, rx, ry, rz);
                    features(rx, ry, rz, a, f, id);
                } else {
                    f[0] = 1.f; f[1] = f[2] = 0.f; f[3] = a;
                }
                tc_write_features<W>(sm.tc, t, f);
                float o[6];
                if (!tc_mlp_tile<W>(sm.tc, phase, status, o)) break;
                float u0 = 0.f, u1 = 0.f, u2 = 0.f;
                if (valid) {
                    const double* fp = Fs + 3 * gn;
                    const float f0 = (float)fp[0], f1 = (float)fp[1], f2 = (float)fp[2];
                    u0 = (o[0] * f0 + o[3] * f1 + o[4] * f2) * id;
                    u1 = (o[3] * f0 + o[1] * f1 + o[5] * f2) * id;
                    u2 = (o[4] * f0 + o[5] * f1 + o[2] * f2) * id;
                    ++pairs;
                }
                sm.contrib[3 * t] = u0;
                sm.contrib[3 * t + 1] = u1;
                sm.contrib[3 * t + 2] = u2;
                __syncthreads();
                if (t < c) {
                    // rows r with (p0 + r) mod c == t
                    int r = (int)((t - p0 % c + c) % c);
                    for (; r < TC_T; r += c) {
                        acc0 += sm.contrib[3 * r];
                        acc1 += sm.contrib[3 * r + 1];
                        acc2 += sm.contrib[3 * r + 2];
                    }
                }
            }
        }
        if (t < c) {
            float* out = y + 3 * (int64_t)(t0 + t);
            out[0] = acc0; out[1] = acc1; out[2] = acc2;
        }
    }
    pairs = warp_sum(pairs);
    if ((t & 31) == 0 && pairs) atomicAdd(n_pairs, pairs);
    tc_teardown<W>(sm.tc);
}

template <int W>
size_t tc_smem_bytes() { return sizeof(TcCore<W>) + 128; }
template <int W>
size_t near_smem_bytes() { return sizeof(NearSmem<W>) + 128; }

}  // namespace

// Near field on tensor cores (precision HH_BF16): same contract as near_field.
void near_field_tc(hh_ctx* ctx, const hh_tree* t, const hh_blocks* b, const hh_params& p, const double* Fs, float* y,
                   const int32_t* work, int64_t n_work, int transpose, cudaStream_t s)
{
    HH_REQUIRE(p.kernel == HH_MLP, HH_ERR_ARG, "the tensor-core path evaluates the MLP kernel only");
    HH_REQUIRE(p.leaf_size <= 129, HH_ERR_ARG, "leaf_size must be <= 129");
    const int64_t grid = std::min<int64_t>(n_work, (int64_t)ctx->n_sm * resolved_launch(ctx, true).near_cps);
    HH_CUDA(cudaEventRecord(ctx->kev[4], s));
    if (ctx->width == 32) {
        const size_t smem = near_smem_bytes<32>();
        HH_CUDA(cudaFuncSetAttribute(k_near_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_near_tc<32><<<(unsigned)grid, TC_T, smem, s>>>(t->Xp, Fs, b->PH, b->rowH, work, n_work, t->nbeg, t->nend,
                                                         ctx->theta32, (float)p.radius, transpose, y,
                                                         ctx->d_counters + 5, ctx->d_status);
    } else {
        const size_t smem = near_smem_bytes<64>();
        HH_CUDA(cudaFuncSetAttribute(k_near_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_near_tc<64><<<(unsigned)grid, TC_T, smem, s>>>(t->Xp, Fs, b->PH, b->rowH, work, n_work, t->nbeg, t->nend,
                                                         ctx->theta32, (float)p.radius, transpose, y,
                                                         ctx->d_counters + 5, ctx->d_status);
    }
    HH_CHECK_LAUNCH();
    HH_CUDA(cudaEventRecord(ctx->kev[5], s));
    ctx->kev_near_used = 1;
}

// K(r) for n separations on tensor cores ([n, 9] out).
void eval_pairs_tc(hh_ctx* ctx, const double* r, int64_t n, double a, double* K, cudaStream_t s)
{
    if (n <= 0) return;
    const int64_t grid = std::min<int64_t>(ceil_div(n, TC_T), (int64_t)ctx->n_sm * 2);
    if (ctx->width == 32) {
        const size_t smem = tc_smem_bytes<32>();
        HH_CUDA(cudaFuncSetAttribute(k_eval_pairs_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_eval_pairs_tc<32><<<(unsigned)grid, TC_T, smem, s>>>(r, n, ctx->theta32, (float)a, K, ctx->d_status);
    } else {
        const size_t smem = tc_smem_bytes<64>();
        HH_CUDA(cudaFuncSetAttribute(k_eval_pairs_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_eval_pairs_tc<64><<<(unsigned)grid, TC_T, smem, s>>>(r, n, ctx->theta32, (float)a, K, ctx->d_status);
    }
    HH_CHECK_LAUNCH();
}
