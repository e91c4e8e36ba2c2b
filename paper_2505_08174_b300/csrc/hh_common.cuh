// hh_common.cuh -- shared device helpers of libhhignn (sm_103a).
//
// Pair kernels (Eq. 4 with the MLP surrogate, or closed-form RPY), 3x3
// element arithmetic used by block ACA (Algorithm 2), warp reductions, and
// the library's error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/hhignn.h"

#define HH_PI 3.14159265358979323846

// ---------------------------------------------------------------------------
// Host error plumbing
// ---------------------------------------------------------------------------
struct HHError {
    hh_status st;
    std::string msg;
};

#define HH_CUDA(call)                                                                             \
    do {                                                                                          \
        cudaError_t _e = (call);                                                                  \
        if (_e != cudaSuccess)                                                                    \
            throw HHError{_e == cudaErrorMemoryAllocation ? HH_ERR_OOM : HH_ERR_CUDA,             \
                          std::string(#call) + ": " + cudaGetErrorString(_e)};                    \
    } while (0)

// Kernels launched by this library (every launch site is followed by
// HH_CHECK_LAUNCH); read per call into hh_stats_t.n_launches.
extern unsigned long long g_hh_launches;
#define HH_CHECK_LAUNCH()       \
    do {                        \
        ++g_hh_launches;        \
        HH_CUDA(cudaGetLastError()); \
    } while (0)

#define HH_REQUIRE(cond, status, text)                \
    do {                                              \
        if (!(cond)) throw HHError{(status), (text)}; \
    } while (0)

// Device-side status word bits (read back by the host after a call).
enum : unsigned {
    HH_DEV_RANK_CAP = 1u,   // an ACA block stopped at max_rank
    HH_DEV_NUMERIC = 2u,    // non-finite value or coincident particles
    HH_DEV_TIMEOUT = 4u,    // a bounded wait gave up
};

// ---------------------------------------------------------------------------
// 3x3 element arithmetic (row-major)
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void mm3(const R* a, const R* b, R* out)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) out[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

template <typename R>
__device__ __forceinline__ R fro2(const R* a)
{
    R s = 0;
#pragma unroll
    for (int e = 0; e < 9; ++e) s += a[e] * a[e];
    return s;
}

__device__ __forceinline__ double det3d(const double* P)
{
    return P[0] * (P[4] * P[8] - P[5] * P[7]) - P[1] * (P[3] * P[8] - P[5] * P[6]) +
           P[2] * (P[3] * P[7] - P[4] * P[6]);
}

// FP64 inverse by adjugate / determinant; returns det.
__device__ __forceinline__ double inv3d(const double* P, double* Pi)
{
    double det = det3d(P);
    double id = 1.0 / det;
    Pi[0] = (P[4] * P[8] - P[5] * P[7]) * id;
    Pi[1] = (P[2] * P[7] - P[1] * P[8]) * id;
    Pi[2] = (P[1] * P[5] - P[2] * P[4]) * id;
    Pi[3] = (P[5] * P[6] - P[3] * P[8]) * id;
    Pi[4] = (P[0] * P[8] - P[2] * P[6]) * id;
    Pi[5] = (P[2] * P[3] - P[0] * P[5]) * id;
    Pi[6] = (P[3] * P[7] - P[4] * P[6]) * id;
    Pi[7] = (P[1] * P[6] - P[0] * P[7]) * id;
    Pi[8] = (P[0] * P[4] - P[1] * P[3]) * id;
    return det;
}

// Pivot element inverse when the residuals are formed in FP32 (the FP32 and
// BF16 block ACA).  Below its noise floor tau -- the rounding noise of the
// residual entries, or the BF16 MLP's entry error -- a singular value of
// the pivot element P is noise, and inverting it would amplify the noise of
// the whole column into the new rank term (such blocks then never meet
// Eq. 10 and run to max_rank).  So:
//  * 1 / ||P^-1||_F (a lower bound of the smallest singular value) above
//    tau: Pi = P^-1 from the adjugate, as in the FP64 path (*det = det P);
//  * ||P||_F (an upper bound of the largest) at or below tau: the pivot is
//    noise (returns 0);
//  * otherwise the damped inverse Pi = (P^T P + tau^2 I)^-1 P^T, which maps
//    a singular value s to s / (s^2 + tau^2): 1/s for s >> tau, ~0 for
//    s << tau (returns 1; *det = 0).
__device__ __forceinline__ int inv3_floor(const double* P, double tau, double* Pi, double* det)
{
    *det = inv3d(P, Pi);
    const double f = fro2(Pi);
    if (*det != 0.0 && f < 1e300 && 1.0 / sqrt(f) > tau) return 3;
    *det = 0.0;
    if (!(fro2(P) > tau * tau)) return 0;
    double A[9], Ai[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            A[3 * i + j] = P[i] * P[j] + P[3 + i] * P[3 + j] + P[6 + i] * P[6 + j] + (i == j ? tau * tau : 0.0);
    inv3d(A, Ai);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)   // (A^-1 P^T)[i][j] = sum_c A^-1[i][c] P[j][c]
            Pi[3 * i + j] = Ai[3 * i] * P[3 * j] + Ai[3 * i + 1] * P[3 * j + 1] + Ai[3 * i + 2] * P[3 * j + 2];
    return 1;
}

// Noise floors of inv3_floor relative to the Frobenius norm of a block's
// first pivot element: FP32 residual entries carry ~ k u |G| rounding noise
// (u = 2^-24, k <= 48 terms: at most 2.9e-6), below 2^-17 = 128 u; the BF16
// hi/lo MLP's entries carry up to ~2^-16 relative error, below 2^-15.
constexpr double PIVOT_FLOOR_FP32 = 1.0 / 131072.0;
constexpr double PIVOT_FLOOR_BF16 = 1.0 / 32768.0;

// ---------------------------------------------------------------------------
// Pair kernels.  r = x_target - x_source (non-zero).  K is row-major 3x3.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float silu_f(float x) { return __fdividef(x, 1.0f + __expf(-x)); }
__device__ __forceinline__ double silu_d(double x) { return x / (1.0 + exp(-x)); }
template <typename R> __device__ __forceinline__ R silu(R x);
template <> __device__ __forceinline__ float silu<float>(float x) { return silu_f(x); }
template <> __device__ __forceinline__ double silu<double>(double x) { return silu_d(x); }

template <typename R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return 1.0 / sqrt(x); }

// MLP 4 -> W -> W -> W -> 6 (SiLU hidden, linear output) on SIMT cores.
//
// FP32 (the fast SIMT path) reads a transposed copy of the parameters kept in
// shared memory: W1t [4][W], b1, W2t [W][W], b2, W3t [W][W], b3, W4t [W][8]
// (6 outputs padded to 8), b4 [8]; every row starts on a 16-byte boundary so
// weights come in as float4.  A layer's W outputs accumulate in registers;
// its input vector sits in this thread's column of a per-warp shared buffer
// (hs[32 * i], one column per lane: conflict-free), so the input loop stays
// rolled and the whole network is ~900 instructions -- small enough for the
// instruction cache of the large ACA kernels.  The empty asm with a memory
// clobber keeps the weight loads inside the caller's pair loop.
template <int W>
__host__ __device__ constexpr int mlp_t_size() { return 4 * W + W + W * W + W + W * W + W + 8 * W + 8; }

template <int W>
__device__ __forceinline__ void mlp_f32(const float* __restrict__ th, const float* f, float* o, float* hs)
{
    asm volatile("" ::: "memory");
    const float* W1 = th;
    const float* b1 = W1 + 4 * W;
    const float* W2 = b1 + W;
    const float* b2 = W2 + W * W;
    const float* W3 = b2 + W;
    const float* b3 = W3 + W * W;
    const float* W4 = b3 + W;
    const float* b4 = W4 + 8 * W;
    float g[W];
#pragma unroll
    for (int j = 0; j < W; ++j) g[j] = b1[j];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float x = f[i];
#pragma unroll
        for (int j = 0; j < W; j += 4) {
            const float4 w4 = *reinterpret_cast<const float4*>(W1 + i * W + j);
            g[j] += w4.x * x; g[j + 1] += w4.y * x; g[j + 2] += w4.z * x; g[j + 3] += w4.w * x;
        }
    }
#pragma unroll
    for (int j = 0; j < W; ++j) hs[32 * j] = silu_f(g[j]);
#pragma unroll 1
    for (int l = 0; l < 2; ++l) {
        const float* Wl = l == 0 ? W2 : W3;
        const float* bl = l == 0 ? b2 : b3;
#pragma unroll
        for (int j = 0; j < W; ++j) g[j] = bl[j];
#pragma unroll 2
        for (int i = 0; i < W; ++i) {
            const float x = hs[32 * i];
#pragma unroll
            for (int j = 0; j < W; j += 4) {
                const float4 w4 = *reinterpret_cast<const float4*>(Wl + i * W + j);
                g[j] += w4.x * x; g[j + 1] += w4.y * x; g[j + 2] += w4.z * x; g[j + 3] += w4.w * x;
            }
        }
#pragma unroll
        for (int j = 0; j < W; ++j) hs[32 * j] = silu_f(g[j]);
    }
    float oo[6] = {b4[0], b4[1], b4[2], b4[3], b4[4], b4[5]};
#pragma unroll 4
    for (int i = 0; i < W; ++i) {
        const float x = hs[32 * i];
        const float4 a = *reinterpret_cast<const float4*>(W4 + i * 8);
        const float2 c = *reinterpret_cast<const float2*>(W4 + i * 8 + 4);
        oo[0] += a.x * x; oo[1] += a.y * x; oo[2] += a.z * x; oo[3] += a.w * x; oo[4] += c.x * x; oo[5] += c.y * x;
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) o[j] = oo[j];
}

// Floats of per-warp activation buffer a SIMT kernel of (R, KIND) needs.
template <typename R, int KIND>
__host__ __device__ constexpr int act_floats_per_warp() { return (sizeof(R) == 4 && KIND < 2) ? (KIND == 1 ? 64 : 32) * 32 : 0; }

// FP64 (the parity mode) reads the packed layout (W [out,in] row-major, then
// b) with compact loops; one out-of-line copy per width.
template <int W>
__device__ __noinline__ void mlp_f64(const double* __restrict__ th, const double* __restrict__ f,
                                     double* __restrict__ o)
{
    const double* W1 = th;
    const double* b1 = W1 + 4 * W;
    const double* W2 = b1 + W;
    const double* b2 = W2 + W * W;
    const double* W3 = b2 + W;
    const double* b3 = W3 + W * W;
    const double* W4 = b3 + W;
    const double* b4 = W4 + 6 * W;
    double h[W], g[W];
#pragma unroll 1
    for (int j = 0; j < W; ++j) {
        double s = b1[j];
        for (int i = 0; i < 4; ++i) s += W1[4 * j + i] * f[i];
        h[j] = silu_d(s);
    }
#pragma unroll 1
    for (int j = 0; j < W; ++j) {
        double s = b2[j];
#pragma unroll 4
        for (int i = 0; i < W; ++i) s += W2[W * j + i] * h[i];
        g[j] = silu_d(s);
    }
#pragma unroll 1
    for (int j = 0; j < W; ++j) {
        double s = b3[j];
#pragma unroll 4
        for (int i = 0; i < W; ++i) s += W3[W * j + i] * g[i];
        h[j] = silu_d(s);
    }
#pragma unroll 1
    for (int j = 0; j < 6; ++j) {
        double s = b4[j];
#pragma unroll 4
        for (int i = 0; i < W; ++i) s += W4[W * j + i] * h[i];
        o[j] = s;
    }
}

template <typename R, int W>
__device__ __forceinline__ void mlp_simt(const R* __restrict__ th, const R* f, R* o, R* hs)
{
    if constexpr (sizeof(R) == 4) mlp_f32<W>(th, f, o, hs);
    else mlp_f64<W>(th, f, o);
}

struct PairParams {
    double a, mu;
};

// KIND 0 = MLP width 32, 1 = MLP width 64, 2 = RPY.  hs: this thread's
// column of the per-warp activation buffer (FP32 MLP only; see mlp_f32).
template <typename R, int KIND>
__device__ __forceinline__ void pair_block(const R* __restrict__ th, const PairParams& pp, R rx, R ry, R rz, R K[9],
                                           R* hs)
{
    R d2 = rx * rx + ry * ry + rz * rz;
    R id = rsqrt_<R>(d2);
    if constexpr (KIND == 2) {
        R d = d2 * id;
        R a = (R)pp.a, A, B;
        if (d >= 2 * a) {
            R c = (R)(1.0 / (8.0 * HH_PI * pp.mu)) * id;
            A = c * (1 + (R)(2.0 / 3.0) * a * a * id * id);
            B = c * (1 - 2 * a * a * id * id);
        } else {
            R c = (R)(1.0 / (6.0 * HH_PI * pp.mu * pp.a));
            A = c * (1 - (R)(9.0 / 32.0) * d / a);
            B = c * ((R)(3.0 / 32.0) * d / a);
        }
        R u[3] = {rx * id, ry * id, rz * id};
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) K[3 * i + j] = (i == j ? A : (R)0) + B * u[i] * u[j];
    } else {
        R f[4] = {rx * id, ry * id, rz * id, (R)pp.a * id};
        R o[6];
        mlp_simt<R, (KIND == 0 ? 32 : 64)>(th, f, o, hs);
        K[0] = o[0] * id; K[1] = o[3] * id; K[2] = o[4] * id;
        K[3] = o[3] * id; K[4] = o[1] * id; K[5] = o[5] * id;
        K[6] = o[4] * id; K[7] = o[5] * id; K[8] = o[2] * id;
    }
}

// Separation r = x_t - x_s from FP64 positions, rounded once to R.
template <typename R>
__device__ __forceinline__ void sep(const double* __restrict__ X, int64_t t, int64_t s, R& rx, R& ry, R& rz)
{
    rx = (R)(X[3 * t] - X[3 * s]);
    ry = (R)(X[3 * t + 1] - X[3 * s + 1]);
    rz = (R)(X[3 * t + 2] - X[3 * s + 2]);
}

// Positions as FP32 pairs, [n][6] = (x_hi, y_hi, z_hi, x_lo, y_lo, z_lo) with
// v_hi = float(v), v_lo = float(v - v_hi): r = (hi_t - hi_s) + (lo_t - lo_s)
// in FP32 is within ~1e-7 relative of the FP64 difference (the hi difference
// of two nearby particles is exact, the lo parts carry the bits the hi parts
// dropped), at FP32 cost.
__device__ __forceinline__ void sep_split(const float* __restrict__ P, int64_t t, int64_t s, float& rx, float& ry,
                                          float& rz)
{
    const float* a = P + 6 * t;
    const float* b = P + 6 * s;
    rx = (a[0] - b[0]) + (a[3] - b[3]);
    ry = (a[1] - b[1]) + (a[4] - b[4]);
    rz = (a[2] - b[2]) + (a[5] - b[5]);
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Arg-max with ties to the lowest index (idx < 0 means "no candidate").  The
// selection is a total order, so every lane ends with the same result.
template <typename T>
__device__ __forceinline__ void warp_argmax(T& v, int& idx)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        bool take = (oi >= 0) && (idx < 0 || ov > v || (ov == v && oi < idx));
        if (take) { v = ov; idx = oi; }
    }
}

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
