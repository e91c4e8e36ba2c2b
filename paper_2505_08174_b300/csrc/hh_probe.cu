// hh_probe.cu -- throughput probes of the arithmetic units the pair-kernel
// MLP leans on (the roofline of the activation-bound kernels): MUFU ex2, rcp
// and tanh, FP32 FMA, FP64 FMA, and the SiLU of the tensor-core epilogues
// (one ex2 and one rcp per activation).  Each probe runs 8 independent
// dependency chains per thread over a grid of 8 CTAs x 256 threads per SM and
// is timed with CUDA events on the caller's stream.
#include "hh_internal.h"

namespace {

constexpr int PR_CHAINS = 8;
constexpr int PR_THREADS = 256;

__device__ __forceinline__ float mufu_ex2(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_rcp(float x)
{
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_tanh(float x)
{
    float y;
    asm volatile("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// KIND: 0 ex2, 1 rcp, 2 tanh, 3 FP32 FMA, 4 FP64 FMA, 5 SiLU (silu_f of x + b).
// The chains are kept in range (ex2 of a negative argument, rcp of a value
// near 1) so no chain under- or overflows, and no two steps fold into one; the result is stored only if a
// runtime-false condition holds, which keeps the work alive.
template <int KIND>
__global__ void __launch_bounds__(PR_THREADS) k_probe(int64_t iters, float seed, float* sink)
{
    const float t = (float)(threadIdx.x & 7) * 1e-3f;
    if constexpr (KIND == 4) {
        double v[PR_CHAINS];
#pragma unroll
        for (int c = 0; c < PR_CHAINS; ++c) v[c] = (double)seed + c * 1e-3 + t;
        const double a = 0.999999, b = 1e-7;
        for (int64_t i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < PR_CHAINS; ++c) v[c] = fma(v[c], a, b);
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < PR_CHAINS; ++c) s += v[c];
        if (s == -1.2345) sink[0] = (float)s;
    } else {
        float v[PR_CHAINS];
#pragma unroll
        for (int c = 0; c < PR_CHAINS; ++c) v[c] = seed + c * 1e-3f + t;
        for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < PR_CHAINS; ++c) {
                if constexpr (KIND == 0) v[c] = mufu_ex2(-v[c]);          // stays in (0.5, 1)
                else if constexpr (KIND == 1) v[c] = mufu_rcp(v[c] + 1e-7f);   // alternates near 1; the add keeps
                                                                               // rcp(rcp(x)) from being folded
                else if constexpr (KIND == 2) v[c] = mufu_tanh(v[c]);     // contracts towards 0 slowly
                else if constexpr (KIND == 3) v[c] = fmaf(v[c], 0.9999999f, 1e-7f);
                else v[c] = silu_f(v[c] + 0.5f);                         // as the epilogues: bias, SiLU
            }
        }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < PR_CHAINS; ++c) s += v[c];
        if (s == -1.2345f) sink[0] = s;
    }
}

template <int KIND>
float probe_ms(int64_t grid, int64_t iters, float* sink, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1)
{
    k_probe<KIND><<<(unsigned)grid, PR_THREADS, 0, s>>>(iters / 8 + 1, 0.75f, sink);   // warm-up
    HH_CHECK_LAUNCH();
    HH_CUDA(cudaEventRecord(e0, s));
    k_probe<KIND><<<(unsigned)grid, PR_THREADS, 0, s>>>(iters, 0.75f, sink);
    HH_CHECK_LAUNCH();
    HH_CUDA(cudaEventRecord(e1, s));
    HH_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    HH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms;
}

}  // namespace

extern "C" hh_status hh_probe_throughput(hh_ctx* ctx, int32_t kind, int64_t iters, void* stream, double* ops_per_s)
{
    if (!ctx || !ops_per_s) return HH_ERR_ARG;
    AllocScope scope;
    try {
        HH_REQUIRE(kind >= 0 && kind <= 5, HH_ERR_ARG, "probe kind must be in [0, 5]");
        HH_REQUIRE(iters >= 1 && iters <= ((int64_t)1 << 30), HH_ERR_ARG, "iters must be in [1, 2^30]");
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t grid = (int64_t)ctx->n_sm * 8;
        float* sink = dev_alloc_t<float>(1, s);
        cudaEvent_t e0 = ctx->ev[6], e1 = ctx->ev[7];
        float ms = 0.f;
        switch (kind) {
            case 0: ms = probe_ms<0>(grid, iters, sink, s, e0, e1); break;
            case 1: ms = probe_ms<1>(grid, iters, sink, s, e0, e1); break;
            case 2: ms = probe_ms<2>(grid, iters, sink, s, e0, e1); break;
            case 3: ms = probe_ms<3>(grid, iters, sink, s, e0, e1); break;
            case 4: ms = probe_ms<4>(grid, iters, sink, s, e0, e1); break;
            default: ms = probe_ms<5>(grid, iters, sink, s, e0, e1); break;
        }
        dev_free(sink, s);
        HH_CUDA(cudaStreamSynchronize(s));
        const double ops = (double)grid * PR_THREADS * PR_CHAINS * (double)iters;
        *ops_per_s = ms > 0.f ? ops / (ms * 1e-3) : 0.0;
        ctx->err.clear();
        return HH_OK;
    } catch (const HHError& e) {
        scope.release();
        ctx->err = e.msg;
        return e.st;
    }
}
