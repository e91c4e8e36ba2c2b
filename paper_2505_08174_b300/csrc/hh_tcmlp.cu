// hh_tcmlp.cu -- the pair-kernel MLP of Eq. 4 on the 5th-generation tensor
// cores (tcgen05, BF16 operands, FP32 accumulation in TMEM), and the dense
// inadmissible blocks (Section 3.3) built on it.
//
// One CTA of 128 threads evaluates tiles of 128 pairs; thread t owns tile row
// t (TMEM lane t).  Per tile:
//   A1 [128 x 16]  = [f_hi(4) | f_lo(4) | 1 | 0...]  (f = [r/|r|, a/|r|])
//   L1: D = A1 B1^T,  B1 [W x 16] = [W1 | W1 | b1 | 0]          (1 MMA, N = W)
//   epilogue: h = SiLU(D) -> AH [128 x 2W] = [h_hi | h_lo] (bf16)
//   L2: D = AH B2^T,  B2 [W x 2W] = [W2 | W2]                    (2W/16 MMAs)
//   epilogue: h = SiLU(D + b2) -> AH;   L3 likewise with W3, b3
//   L4: D = AH B4^T,  B4 [16 x 2W] = [W4 | W4] padded to 16 rows; o = D + b4
// Splitting every activation into a bf16 "hi" part and a bf16 remainder keeps
// ~16 significant bits of each activation; the weights are exactly bf16 (the
// canonical network), so the products are exact and only the FP32
// accumulation and SiLU round.  The MMA issue is one elected thread; its
// completion is tracked by tcgen05.commit on an mbarrier that every thread
// waits on with an iteration limit.
#include <algorithm>

#include <cuda_bf16.h>

#include "hh_internal.h"
#include "hh_tc.cuh"

namespace {

constexpr int TC_T = 128;                  // threads per CTA = tile rows
constexpr uint32_t TC_WAIT_LIMIT = 1u << 26;

template <int W>
struct alignas(128) TcSmem {
    __nv_bfloat16 A1[TC_T * 16];
    __nv_bfloat16 AH[TC_T * 2 * W];
    __nv_bfloat16 B1[W * 16];
    __nv_bfloat16 B2[W * 2 * W];
    __nv_bfloat16 B3[W * 2 * W];
    __nv_bfloat16 B4[16 * 2 * W];
    float b2[W], b3[W], b4[16];
    float contrib[TC_T * 3];
    int32_t seg_s0[256], seg_q[256], seg_pre[257];
    uint64_t mbar;
    uint32_t tmem;
    int nseg;
    int fail;
    uint32_t pending;
};

template <int W>
__host__ __device__ constexpr uint32_t tmem_cols() { return W <= 32 ? 32u : 64u; }

__device__ __forceinline__ void st_shared_v4(void* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(p)), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);   // .x = first argument (lower address)
    return *reinterpret_cast<uint32_t*>(&v);
}

// x -> (bf16 hi, bf16 remainder)
__device__ __forceinline__ void split_bf16(float x, float& hi, float& lo)
{
    hi = __bfloat162float(__float2bfloat16_rn(x));
    lo = x - hi;
}

// Weights from the packed FP32 parameters into the K-major core-matrix tiles.
template <int W>
__device__ void tc_load_weights(TcSmem<W>& sm, const float* __restrict__ th)
{
    const float* W1 = th;
    const float* b1 = W1 + 4 * W;
    const float* W2 = b1 + W;
    const float* b2 = W2 + W * W;
    const float* W3 = b2 + W;
    const float* b3 = W3 + W * W;
    const float* W4 = b3 + W;
    const float* b4 = W4 + 6 * W;
    unsigned char* B1 = reinterpret_cast<unsigned char*>(sm.B1);
    unsigned char* B2 = reinterpret_cast<unsigned char*>(sm.B2);
    unsigned char* B3 = reinterpret_cast<unsigned char*>(sm.B3);
    unsigned char* B4 = reinterpret_cast<unsigned char*>(sm.B4);
    for (int x = threadIdx.x; x < W * 16; x += blockDim.x) {
        const int j = x / 16, k = x % 16;
        float v = k < 4 ? W1[4 * j + k] : (k < 8 ? W1[4 * j + k - 4] : (k == 8 ? b1[j] : 0.f));
        *reinterpret_cast<__nv_bfloat16*>(B1 + tc_elem_offset(j, k, 16)) = __float2bfloat16_rn(v);
    }
    for (int x = threadIdx.x; x < W * 2 * W; x += blockDim.x) {
        const int j = x / (2 * W), k = x % (2 * W), kk = k % W;
        *reinterpret_cast<__nv_bfloat16*>(B2 + tc_elem_offset(j, k, 2 * W)) = __float2bfloat16_rn(W2[W * j + kk]);
        *reinterpret_cast<__nv_bfloat16*>(B3 + tc_elem_offset(j, k, 2 * W)) = __float2bfloat16_rn(W3[W * j + kk]);
    }
    for (int x = threadIdx.x; x < 16 * 2 * W; x += blockDim.x) {
        const int j = x / (2 * W), k = x % (2 * W), kk = k % W;
        float v = j < 6 ? W4[W * j + kk] : 0.f;
        *reinterpret_cast<__nv_bfloat16*>(B4 + tc_elem_offset(j, k, 2 * W)) = __float2bfloat16_rn(v);
    }
    for (int j = threadIdx.x; j < W; j += blockDim.x) { sm.b2[j] = b2[j]; sm.b3[j] = b3[j]; }
    for (int j = threadIdx.x; j < 16; j += blockDim.x) sm.b4[j] = j < 6 ? b4[j] : 0.f;
}

// Thread t writes its row of A1 from the features f[4].
template <int W>
__device__ __forceinline__ void tc_write_features(TcSmem<W>& sm, int t, const float f[4])
{
    float h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) split_bf16(f[i], h[i], l[i]);
    unsigned char* A1 = reinterpret_cast<unsigned char*>(sm.A1);
    st_shared_v4(A1 + tc_elem_offset(t, 0, 16), pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(l[0], l[1]),
                 pack_bf16(l[2], l[3]));
    st_shared_v4(A1 + tc_elem_offset(t, 8, 16), pack_bf16(1.f, 0.f), 0u, 0u, 0u);
}

// Wait for the MMA group committed to the mbarrier.  The outcome is made
// uniform over the CTA (a thread that gave up makes every thread stop), so
// no thread is left at a barrier the others skip.  A timeout is recorded in
// the status word and in sm.fail; the pending phase stays in sm.
template <int W>
__device__ __forceinline__ bool tc_wait(TcSmem<W>& sm, uint32_t& phase, unsigned* status)
{
    const bool ok = mbar_wait_bounded(&sm.mbar, phase & 1u, TC_WAIT_LIMIT);
    const int any_fail = __syncthreads_or(!ok);
    if (any_fail) {
        if (threadIdx.x == 0) {
            sm.fail = 1;
            sm.pending = phase & 1u;
            atomicOr(status, (unsigned)HH_DEV_TIMEOUT);
        }
        __syncthreads();
        return false;
    }
    ++phase;
    tc_fence_after();
    return true;
}

// Issue one layer: D[tmem] = A (128 x K) * B (N x K)^T, K = 16 * nk.
__device__ __forceinline__ void tc_issue_layer(uint32_t tmem, const void* A, const void* B, int K, int N,
                                               uint64_t* mbar)
{
    const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    const uint32_t idesc = tc_idesc_bf16(128, N);
    for (int kc = 0; kc < K / 16; ++kc) {
        const uint64_t da = tc_smem_desc(a0 + 256u * kc, 128u, sbo);
        const uint64_t db = tc_smem_desc(b0 + 256u * kc, 128u, sbo);
        tc_mma_bf16(tmem, da, db, idesc, kc > 0 ? 1u : 0u);
    }
    tc_commit(mbar);
}

// SiLU(D + bias) of this thread's row -> AH row as (hi | lo).
template <int W>
__device__ __forceinline__ void tc_hidden_epilogue(TcSmem<W>& sm, uint32_t trow, const float* bias, int t)
{
    unsigned char* AH = reinterpret_cast<unsigned char*>(sm.AH);
#pragma unroll
    for (int c0 = 0; c0 < W; c0 += 16) {
        float v[16];
        tmem_ld16(trow + (uint32_t)c0, v);
        float hi[16], lo[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float x = v[j] + (bias ? bias[c0 + j] : 0.f);
            x = silu_f(x);
            split_bf16(x, hi[j], lo[j]);
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const int k = c0 + 8 * g;
            st_shared_v4(AH + tc_elem_offset(t, k, 2 * W), pack_bf16(hi[8 * g], hi[8 * g + 1]),
                         pack_bf16(hi[8 * g + 2], hi[8 * g + 3]), pack_bf16(hi[8 * g + 4], hi[8 * g + 5]),
                         pack_bf16(hi[8 * g + 6], hi[8 * g + 7]));
            st_shared_v4(AH + tc_elem_offset(t, W + k, 2 * W), pack_bf16(lo[8 * g], lo[8 * g + 1]),
                         pack_bf16(lo[8 * g + 2], lo[8 * g + 3]), pack_bf16(lo[8 * g + 4], lo[8 * g + 5]),
                         pack_bf16(lo[8 * g + 6], lo[8 * g + 7]));
        }
    }
}

// The MLP chain on the current A1 tile; o[6] receives this thread's output.
// Returns false on a timeout (sm.fail set; the caller stops).
template <int W>
__device__ bool tc_mlp_tile(TcSmem<W>& sm, uint32_t& phase, unsigned* status, float o[6])
{
    const int t = threadIdx.x;
    const uint32_t trow = sm.tmem + ((uint32_t)(t & ~31) << 16);
    // layer 1
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
        tc_fence_after();
        tc_issue_layer(sm.tmem, sm.A1, sm.B1, 16, W, &sm.mbar);
    }
    if (!tc_wait(sm, phase, status)) return false;
    tc_hidden_epilogue<W>(sm, trow, nullptr, t);
    // layers 2 and 3
#pragma unroll 1
    for (int l = 0; l < 2; ++l) {
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            tc_issue_layer(sm.tmem, sm.AH, l == 0 ? sm.B2 : sm.B3, 2 * W, W, &sm.mbar);
        }
        if (!tc_wait(sm, phase, status)) return false;
        tc_hidden_epilogue<W>(sm, trow, l == 0 ? sm.b2 : sm.b3, t);
    }
    // layer 4 (N = 16, outputs 0..5)
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
        tc_fence_after();
        tc_issue_layer(sm.tmem, sm.AH, sm.B4, 2 * W, 16, &sm.mbar);
    }
    if (!tc_wait(sm, phase, status)) return false;
    float v[16];
    tmem_ld16(trow, v);
#pragma unroll
    for (int j = 0; j < 6; ++j) o[j] = v[j] + sm.b4[j];
    tc_fence_before();
    return true;
}

template <int W>
__device__ void tc_setup(TcSmem<W>& sm, const float* th)
{
    tc_load_weights<W>(sm, th);
    if (threadIdx.x == 0) {
        sm.fail = 0;
        mbar_init(&sm.mbar, 1);
    }
    if (threadIdx.x < 32) {
        tmem_alloc(&sm.tmem, tmem_cols<W>());
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

template <int W>
__device__ void tc_teardown(TcSmem<W>& sm)
{
    tc_fence_before();
    __syncthreads();
    // after a timeout, give the MMA group still in flight one more bounded
    // wait before the accumulator columns are released
    if (sm.fail && threadIdx.x == 0) mbar_wait_bounded(&sm.mbar, sm.pending, TC_WAIT_LIMIT);
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(sm.tmem, tmem_cols<W>());
}

__device__ __forceinline__ void features(float rx, float ry, float rz, float a, float f[4], float& id)
{
    id = rsqrtf(rx * rx + ry * ry + rz * rz);
    f[0] = rx * id; f[1] = ry * id; f[2] = rz * id; f[3] = a * id;
}

// ---- pair evaluation: K(r) for a list of separations --------------------------
template <int W>
__global__ void __launch_bounds__(TC_T, 1) k_eval_pairs_tc(const double* __restrict__ r, int64_t n,
                                                          const float* __restrict__ th, float a,
                                                          double* __restrict__ K, unsigned* status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TcSmem<W>& sm = *reinterpret_cast<TcSmem<W>*>(smem_raw);
    tc_setup<W>(sm, th);
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
__global__ void __launch_bounds__(TC_T, 1) k_near_tc(const double* __restrict__ Xs, const double* __restrict__ Fs,
                                                    const int32_t* __restrict__ PH, const int64_t* __restrict__ rowH,
                                                    const int32_t* __restrict__ work, int64_t n_work,
                                                    const int32_t* __restrict__ nbeg, const int32_t* __restrict__ nend,
                                                    const float* __restrict__ th, float a, int transpose,
                                                    float* __restrict__ y, unsigned long long* n_pairs,
                                                    unsigned* status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TcSmem<W>& sm = *reinterpret_cast<TcSmem<W>*>(smem_raw);
    tc_setup<W>(sm, th);
    uint32_t phase = 0;
    const int t = threadIdx.x;
    unsigned long long pairs = 0;
    for (int64_t w = blockIdx.x; w < n_work && !sm.fail; w += gridDim.x) {
        const int32_t tau = work[w];
        const int32_t t0 = nbeg[tau], c = nend[tau] - t0;
        float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
        for (int64_t b0 = rowH[tau]; b0 < rowH[tau + 1] && !sm.fail; b0 += 256) {
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
                    if (!transpose) sep<float>(Xs, gm, gn, rx, ry, rz);
                    else sep<float>(Xs, gn, gm, rx, ry, rz);
                    features(rx, ry, rz, a, f, id);
                } else {
                    f[0] = 1.f; f[1] = f[2] = 0.f; f[3] = a;
                }
                tc_write_features<W>(sm, t, f);
                float o[6];
                if (!tc_mlp_tile<W>(sm, phase, status, o)) break;
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
    tc_teardown<W>(sm);
}

template <int W>
size_t tc_smem_bytes() { return sizeof(TcSmem<W>) + 128; }

}  // namespace

// Near field on tensor cores (precision HH_BF16): same contract as near_field.
void near_field_tc(hh_ctx* ctx, const hh_tree* t, const hh_blocks* b, const hh_params& p, const double* Fs, float* y,
                   const int32_t* work, int64_t n_work, int transpose, cudaStream_t s)
{
    HH_REQUIRE(p.kernel == HH_MLP, HH_ERR_ARG, "the tensor-core path evaluates the MLP kernel only");
    HH_REQUIRE(p.leaf_size <= 129, HH_ERR_ARG, "leaf_size must be <= 129");
    const int64_t grid = std::min<int64_t>(n_work, (int64_t)ctx->n_sm * 4);
    HH_CUDA(cudaEventRecord(ctx->kev[4], s));
    if (ctx->width == 32) {
        const size_t smem = tc_smem_bytes<32>();
        HH_CUDA(cudaFuncSetAttribute(k_near_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_near_tc<32><<<(unsigned)grid, TC_T, smem, s>>>(t->Xs, Fs, b->PH, b->rowH, work, n_work, t->nbeg, t->nend,
                                                         ctx->theta32, (float)p.radius, transpose, y,
                                                         ctx->d_counters + 5, ctx->d_status);
    } else {
        const size_t smem = tc_smem_bytes<64>();
        HH_CUDA(cudaFuncSetAttribute(k_near_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_near_tc<64><<<(unsigned)grid, TC_T, smem, s>>>(t->Xs, Fs, b->PH, b->rowH, work, n_work, t->nbeg, t->nend,
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
