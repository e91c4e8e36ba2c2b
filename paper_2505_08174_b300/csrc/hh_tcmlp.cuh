// hh_tcmlp.cuh -- the pair-kernel MLP of Eq. 4 on the 5th-generation tensor
// cores (tcgen05, BF16 operands, FP32 accumulation in TMEM): one 128-row tile
// per call, shared by the near-field, pair-evaluation and ACA kernels.
//
// One CTA of 128 threads evaluates tiles of 128 pairs; thread t owns tile row
// t (TMEM lane t).  Per tile:
//   A1 [128 x 16]  = [f_hi(4) | f_lo(4) | 1 | 0...]  (f = [r/|r|, a/|r|])
//   L1: D = A1 B1^T,  B1 [W x 16] = [W1 | W1 | b1 | 0]          (1 MMA, N = W)
//   epilogue: h = SiLU(D) -> AH [128 x 2W] = [h_hi | h_lo] (bf16)
//   L2: D = AH_hi W2^T + AH_lo W2^T,  B2 [W x W] = W2           (2W/16 MMAs)
//   epilogue: h = SiLU(D + b2) -> AH;   L3 likewise with W3, b3
//   L4: D = AH_hi W4^T + AH_lo W4^T,  B4 [16 x W] = W4 padded to 16 rows; o = D + b4
// Splitting every activation into a bf16 "hi" part and a bf16 remainder keeps
// ~16 significant bits of each activation; the weights are exactly bf16 (the
// canonical network), so the products are exact and only the FP32
// accumulation and SiLU round.  The MMA issue is one elected thread; its
// completion is tracked by tcgen05.commit on an mbarrier that every thread
// waits on with an iteration limit.
#pragma once

#include <cuda_bf16.h>

#include "hh_internal.h"
#include "hh_tc.cuh"

namespace {

constexpr int TC_T = 128;                  // threads per CTA = tile rows
constexpr uint32_t TC_WAIT_LIMIT = 1u << 26;

template <int W>
struct alignas(128) TcCore {
    __nv_bfloat16 A1[TC_T * 16];
    __nv_bfloat16 AH[TC_T * 2 * W];
    __nv_bfloat16 B1[W * 16];
    __nv_bfloat16 B2[W * W];    // applied to both halves of AH (two MMAs per K chunk pair)
    __nv_bfloat16 B3[W * W];
    __nv_bfloat16 B4[16 * W];
    float b2[W], b3[W], b4[16];
    uint64_t mbar;
    uint32_t tmem;
    int fail;
    uint32_t pending;
    // Test mode (status[1] = stall_polls > 0, set by the host): every MMA
    // completion wait watches `stall`, an mbarrier that nothing arrives at,
    // for stall_polls polls instead of the MMA's own barrier, so it runs out
    // and takes the timeout path.  The teardown wait is never redirected.
    uint64_t stall;
    uint32_t stall_polls;
};

__device__ __forceinline__ uint32_t tc_stall_polls(const unsigned* status) { return status ? status[1] : 0u; }

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

// Bit pattern of x rounded to bf16 (to nearest, ties away from zero) in the
// upper half-word, lower half-word zero: the bf16 value read as a float.
// Integer add + mask on the FP32 pattern, no conversion instruction.
__device__ __forceinline__ uint32_t bf16_round_bits(float x) { return (__float_as_uint(x) + 0x8000u) & 0xFFFF0000u; }

// x -> bf16 "hi" (x rounded) and bf16 "lo" (the exact remainder x - hi,
// rounded), as FP32 patterns with zero lower halves.
__device__ __forceinline__ void split_bits(float x, uint32_t& hi, uint32_t& lo)
{
    hi = bf16_round_bits(x);
    lo = bf16_round_bits(x - __uint_as_float(hi));
}

// Two such patterns -> one bf16x2 word (first element at the lower address).
__device__ __forceinline__ uint32_t pack_hi_halves(uint32_t first, uint32_t second)
{
    return __byte_perm(first, second, 0x7632);
}

// Weights from the packed FP32 parameters into the K-major core-matrix tiles.
template <int W>
__device__ void tc_load_weights(TcCore<W>& sm, const float* __restrict__ th)
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
    for (int x = threadIdx.x; x < W * W; x += blockDim.x) {
        const int j = x / W, k = x % W;
        *reinterpret_cast<__nv_bfloat16*>(B2 + tc_elem_offset(j, k, W)) = __float2bfloat16_rn(W2[W * j + k]);
        *reinterpret_cast<__nv_bfloat16*>(B3 + tc_elem_offset(j, k, W)) = __float2bfloat16_rn(W3[W * j + k]);
    }
    for (int x = threadIdx.x; x < 16 * W; x += blockDim.x) {
        const int j = x / W, k = x % W;
        float v = j < 6 ? W4[W * j + k] : 0.f;
        *reinterpret_cast<__nv_bfloat16*>(B4 + tc_elem_offset(j, k, W)) = __float2bfloat16_rn(v);
    }
    for (int j = threadIdx.x; j < W; j += blockDim.x) { sm.b2[j] = b2[j]; sm.b3[j] = b3[j]; }
    for (int j = threadIdx.x; j < 16; j += blockDim.x) sm.b4[j] = j < 6 ? b4[j] : 0.f;
}

// Thread t writes its row of A1 from the features f[4].
template <int W>
__device__ __forceinline__ void tc_write_features(TcCore<W>& sm, int t, const float f[4])
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) split_bits(f[i], h[i], l[i]);
    unsigned char* A1 = reinterpret_cast<unsigned char*>(sm.A1);
    st_shared_v4(A1 + tc_elem_offset(t, 0, 16), pack_hi_halves(h[0], h[1]), pack_hi_halves(h[2], h[3]),
                 pack_hi_halves(l[0], l[1]), pack_hi_halves(l[2], l[3]));
    st_shared_v4(A1 + tc_elem_offset(t, 8, 16), pack_bf16(1.f, 0.f), 0u, 0u, 0u);
}

// Wait for the MMA group committed to the mbarrier.  The outcome is made
// uniform over the CTA (a thread that gave up makes every thread stop), so
// no thread is left at a barrier the others skip.  A timeout is recorded in
// the status word and in sm.fail; the pending phase stays in sm.
template <int W>
__device__ __forceinline__ bool tc_wait(TcCore<W>& sm, uint32_t& phase, unsigned* status)
{
    const bool ok = sm.stall_polls ? mbar_wait_bounded(&sm.stall, 0u, sm.stall_polls)
                                   : mbar_wait_bounded(&sm.mbar, phase & 1u, TC_WAIT_LIMIT);
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

// Issue one layer: D[tmem] = sum over the K/16 chunks kc of A(:, kc) B(:, kc
// mod KB/16)^T -- A is 128 x K, B is N x KB with KB dividing K, so B is
// applied to each KB-wide slice of A (the bf16 hi and lo halves of the
// activations share one copy of the weights).
__device__ __forceinline__ void tc_issue_layer(uint32_t tmem, const void* A, const void* B, int K, int KB, int N,
                                               uint64_t* mbar)
{
    const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
    const uint32_t sbo_a = (uint32_t)(K / 8) * 128u, sbo_b = (uint32_t)(KB / 8) * 128u;
    const uint32_t idesc = tc_idesc_bf16(128, N);
    const int nb = KB / 16;
    for (int kc = 0; kc < K / 16; ++kc) {
        const uint64_t da = tc_smem_desc(a0 + 256u * kc, 128u, sbo_a);
        const uint64_t db = tc_smem_desc(b0 + 256u * (kc % nb), 128u, sbo_b);
        tc_mma_bf16(tmem, da, db, idesc, kc > 0 ? 1u : 0u);
    }
    tc_commit(mbar);
}

// SiLU(D + bias) of this thread's row -> AH row as (hi | lo).
template <int W>
__device__ __forceinline__ void tc_hidden_epilogue(TcCore<W>& sm, uint32_t trow, const float* bias, int t)
{
    unsigned char* AH = reinterpret_cast<unsigned char*>(sm.AH);
#pragma unroll
    for (int c0 = 0; c0 < W; c0 += 16) {
        float v[16];
        tmem_ld16(trow + (uint32_t)c0, v);
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float x = silu_f(v[j] + (bias ? bias[c0 + j] : 0.f));
            split_bits(x, hi[j], lo[j]);
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const int k = c0 + 8 * g;
            const uint32_t* H = hi + 8 * g;
            const uint32_t* L = lo + 8 * g;
            st_shared_v4(AH + tc_elem_offset(t, k, 2 * W), pack_hi_halves(H[0], H[1]), pack_hi_halves(H[2], H[3]),
                         pack_hi_halves(H[4], H[5]), pack_hi_halves(H[6], H[7]));
            st_shared_v4(AH + tc_elem_offset(t, W + k, 2 * W), pack_hi_halves(L[0], L[1]), pack_hi_halves(L[2], L[3]),
                         pack_hi_halves(L[4], L[5]), pack_hi_halves(L[6], L[7]));
        }
    }
}

// The MLP chain on the current A1 tile; o[6] receives this thread's output.
// Returns false on a timeout (sm.fail set; the caller stops).
template <int W>
__device__ bool tc_mlp_tile(TcCore<W>& sm, uint32_t& phase, unsigned* status, float o[6])
{
    const int t = threadIdx.x;
    const uint32_t trow = sm.tmem + ((uint32_t)(t & ~31) << 16);
    // layer 1
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
        tc_fence_after();
        tc_issue_layer(sm.tmem, sm.A1, sm.B1, 16, 16, W, &sm.mbar);
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
            tc_issue_layer(sm.tmem, sm.AH, l == 0 ? sm.B2 : sm.B3, 2 * W, W, W, &sm.mbar);
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
        tc_issue_layer(sm.tmem, sm.AH, sm.B4, 2 * W, W, 16, &sm.mbar);
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
__device__ void tc_setup(TcCore<W>& sm, const float* th, const unsigned* status)
{
    tc_load_weights<W>(sm, th);
    if (threadIdx.x == 0) {
        sm.fail = 0;
        sm.stall_polls = tc_stall_polls(status);
        mbar_init(&sm.mbar, 1);
        mbar_init(&sm.stall, 1);
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
__device__ void tc_teardown(TcCore<W>& sm)
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

// ---- per-warp chains ----------------------------------------------------------
// Warp w (quadrant w & 3 of a 128-thread CTA) evaluates its own 32 tile rows
// 32w..32w+31 without waiting for the other warps: it issues the four layers
// itself (full 128-row MMAs over the shared A1 / AH tiles, accumulator in the
// warp's own TMEM columns tcol .. tcol + W - 1), waits on its own mbarrier and
// reads back only its own lanes.  Rows of other warps may change under these
// MMAs; they only feed accumulator lanes this warp never reads.
struct TcWarp {
    uint32_t tcol;     // TMEM address of this warp's first accumulator column
    uint64_t* mbar;    // this warp's MMA-completion barrier
    uint32_t phase;
    int* fail;         // shared: set on a timeout
    uint32_t* pending; // shared: phase still outstanding after a timeout
    uint64_t* stall;   // the CTA's test-mode barrier (see TcCore::stall)
    uint32_t stall_polls;
};

__device__ __forceinline__ bool tcw_wait(TcWarp& w, unsigned* status)
{
    const bool ok = w.stall_polls ? mbar_wait_bounded(w.stall, 0u, w.stall_polls)
                                  : mbar_wait_bounded(w.mbar, w.phase & 1u, TC_WAIT_LIMIT);
    if (__any_sync(0xffffffffu, !ok)) {
        if ((threadIdx.x & 31) == 0) {
            *w.fail = 1;
            *w.pending = w.phase & 1u;
            atomicOr(status, (unsigned)HH_DEV_TIMEOUT);
        }
        __syncwarp();
        return false;
    }
    ++w.phase;
    tc_fence_after();
    return true;
}

template <int W>
__device__ bool tcw_mlp_rows(TcCore<W>& sm, TcWarp& w, unsigned* status, float o[6])
{
    const int lane = threadIdx.x & 31, quad = (threadIdx.x >> 5) & 3;
    const int t = 32 * quad + lane;
    const uint32_t trow = w.tcol + ((uint32_t)(32 * quad) << 16);
#pragma unroll 1
    for (int l = 0; l < 4; ++l) {
        fence_async_smem();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
            tc_fence_after();
            if (l == 0) tc_issue_layer(w.tcol, sm.A1, sm.B1, 16, 16, W, w.mbar);
            else tc_issue_layer(w.tcol, sm.AH, l == 1 ? sm.B2 : (l == 2 ? sm.B3 : sm.B4), 2 * W, W, l == 3 ? 16 : W,
                                w.mbar);
        }
        if (!tcw_wait(w, status)) return false;
        if (l < 3) tc_hidden_epilogue<W>(sm, trow, l == 0 ? nullptr : (l == 1 ? sm.b2 : sm.b3), t);
    }
    float v[16];
    tmem_ld16(trow, v);
#pragma unroll
    for (int j = 0; j < 6; ++j) o[j] = v[j] + sm.b4[j];
    tc_fence_before();
    return true;
}

__device__ __forceinline__ void features(float rx, float ry, float rz, float a, float f[4], float& id)
{
    id = rsqrtf(rx * rx + ry * ry + rz * rz);
    f[0] = rx * id; f[1] = ry * id; f[2] = rz * id; f[3] = a * id;
}

}  // namespace
