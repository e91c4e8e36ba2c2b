// hh_aca.cuh -- device pieces shared by the SIMT (hh_aca.cu) and tensor-core
// (hh_aca_tc.cu) block-ACA kernels: arguments, team types, per-team shared
// state, the 3x3 Gram reductions of the stopping test (Algorithm 2, Eq. 10).
#pragma once

#include "hh_internal.h"

namespace {

constexpr int MAXR = 64;          // hard cap on max_rank
constexpr int WARP_ROWS = 16;     // warp team: up to 512 rows / columns per block
constexpr int CTA_T = 256;        // CTA team size
constexpr int SMALL_MAX = 32 * WARP_ROWS;

template <typename R>
struct AcaArgs {
    const double* Xs;
    const float* Xp;  // FP32 (hi, lo) positions (tensor-core kernels)
    const R* th_g;   // parameters in global memory (copied to shared)
    int n_th;
    PairParams pp;
    const double* Fs;
    const int32_t* PG;
    const int32_t* nbeg;
    const int32_t* nend;
    const int32_t* work;
    int64_t n_work;
    unsigned long long* counter;
    int max_rank;
    double eps2;
    int j1_rule;
    uint64_t seed;
    R* scratch;
    int64_t team_stride;   // reals per team
    int32_t* rank;
    int32_t* pivI;
    int32_t* pivJ;
    R* part;
    const int64_t* pofs;
    int64_t pofs_base;     // block b's partial output at part + 3 * (pofs[b] - pofs_base)
    R* fac;
    const int64_t* fofs;
    int64_t fofs_base;
    unsigned* status;
    unsigned long long* n_queries;
};

// Shared state of one team; MR bounds the rank (max_rank <= MR).
template <typename R, int MR = MAXR>
struct alignas(16) TeamSmem {
    union {
        R qj[MR * 9];      // Q_p(j_k), p < k (rank loop)
        R tv[MR * 3];      // t_p = sum_n Q_p(n) F(n) (fused apply, after the loop)
    };
    R ci[MR * 9];          // C_p(i_k), p < k
    R A[(MR + 1) * 9];     // A_pk, p <= k
    double red[2][8];      // per-warp partials of nu^2 and the cross term
    R Pi[9];
    double rv[8];
    int ri[8];
    int flag, stop;
    double pscale;         // Frobenius norm of the block's first pivot element
};

__device__ __forceinline__ uint64_t splitmix_once(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// j_1 (drawn at random in the paper): rule 0 = first source, rule 1 =
// splitmix64(seed ^ (t << 32) ^ s) mod q.
__device__ __forceinline__ int j1_of(int rule, uint64_t seed, int t, int s, int q)
{
    if (rule == 0 || q <= 1) return 0;
    uint64_t h = splitmix_once(seed ^ ((uint64_t)(uint32_t)t << 32) ^ (uint64_t)(uint32_t)s);
    return (int)(h % (uint64_t)q);
}

// ---- teams -----------------------------------------------------------------
struct WarpTeam {
    static constexpr int SIZE = 32;
    static constexpr int ROWS = WARP_ROWS;   // rows per thread
    static constexpr int NW = 1;
    static constexpr bool REG_FLAGS = true;  // used-row/column flags in registers
    __device__ __forceinline__ int tid() const { return threadIdx.x & 31; }
    __device__ __forceinline__ int warp() const { return 0; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    template <typename T, typename S>
    __device__ __forceinline__ void argmax(T& v, int& i, S&) const { warp_argmax(v, i); }
};

template <int T>
struct CtaTeamT {
    static constexpr int SIZE = T;
    static constexpr int ROWS = 1 << 20;      // unbounded (loops exit at c / q)
    static constexpr int NW = T / 32;
    static constexpr bool REG_FLAGS = false;  // flags as bytes in the team workspace
    __device__ __forceinline__ int tid() const { return threadIdx.x; }
    __device__ __forceinline__ int warp() const { return threadIdx.x >> 5; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    template <typename V, typename S>
    __device__ __forceinline__ void argmax(V& v, int& i, S& sm) const
    {
        warp_argmax(v, i);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) { sm.rv[w] = (double)v; sm.ri[w] = i; }
        __syncthreads();
        double bv = sm.rv[0];
        int bi = sm.ri[0];
        for (int k = 1; k < NW; ++k) {
            double ov = sm.rv[k];
            int oi = sm.ri[k];
            if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
        }
        v = (V)bv;
        i = bi;
        __syncthreads();
    }
};
using CtaTeam = CtaTeamT<CTA_T>;

template <typename R>
__device__ __forceinline__ void ld9(const R* __restrict__ base, int64_t stride, int64_t idx, R* v)
{
#pragma unroll
    for (int e = 0; e < 9; ++e) v[e] = base[e * stride + idx];
}
template <typename R>
__device__ __forceinline__ void st9(R* __restrict__ base, int64_t stride, int64_t idx, const R* v)
{
#pragma unroll
    for (int e = 0; e < 9; ++e) base[e * stride + idx] = v[e];
}

// Sum over the warp's lanes of 32 values at once: after five halving steps
// (each lane keeps the half of its values whose index bit matches its own
// lane bit and receives the partner's partial sums of that half), lane l
// holds the sum of v[l].  31 shuffles for 32 sums instead of 5 per sum.
template <typename R>
__device__ __forceinline__ R warp_transpose_sum32(R (&v)[32])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const bool upper = (lane & h) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const R send = upper ? v[i] : v[i + h];
            const R keep = upper ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
    return v[0];
}

// sm.A[p] = sum_x C_p(x)^T C_k(x) for p = 0..k.  Each warp of the team owns
// groups of three consecutive p and sweeps all rows with its 32 lanes; the 27
// per-lane partial sums of a group are reduced together (warp_transpose_sum32).
template <typename R, class Team, class S>
__device__ void gram_cols(const Team& tm, S& sm, const R* Cs, int c, int k)
{
    constexpr int G = 3;
    const int lane = threadIdx.x & 31;
    const R* Ck = Cs + (int64_t)k * 9 * c;
    for (int p0 = tm.warp() * G; p0 <= k; p0 += G * Team::NW) {
        const int np = min(G, k + 1 - p0);
        R acc[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) acc[e] = 0;
        for (int x = lane; x < c; x += 32) {
            R b[9];
            ld9(Ck, c, x, b);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (g < np) {
                    R a[9];
                    ld9(Cs + (int64_t)(p0 + g) * 9 * c, c, x, a);
#pragma unroll
                    for (int u = 0; u < 3; ++u)
#pragma unroll
                        for (int v = 0; v < 3; ++v)
                            acc[9 * g + 3 * u + v] += a[u] * b[v] + a[3 + u] * b[3 + v] + a[6 + u] * b[6 + v];
                }
            }
        }
        const R s = warp_transpose_sum32<R>(acc);
        if (lane < 9 * np) sm.A[9 * p0 + lane] = s;
    }
}

// Stopping-test terms of Eq. 10 with 3x3 Grams, gathered while the row
// residual is formed: nu^2 = tr(A_kk B_kk) and cross = sum_{p<k} tr(A_pk
// B_kp), B_kp = sum_n q_k(n) q_p(n)^T.  tr(A B) is linear in B and
//   tr(A_pk q_k(n) q_p(n)^T) = <A_pk q_k(n), q_p(n)>_F = <q_k(n), A_pk^T q_p(n)>_F,
// so the thread that forms q_k(n) keeps V(n) = sum_{p<k} A_pk^T Q_p(n) from
// the same loads of Q_p(n) as the residual update, and adds <A_kk q, q> and
// <q, V> to its running sums (no second pass over the factors).
template <typename R>
__device__ __forceinline__ void add_AtB(R* V, const R* A, const R* B)   // V += A^T B
{
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int w = 0; w < 3; ++w) V[3 * u + w] += A[u] * B[w] + A[3 + u] * B[3 + w] + A[6 + u] * B[6 + w];
}

template <typename R>
__device__ __forceinline__ void row_terms(const R* A_kk, const R* q, const R* V, R& snu, R& scr)
{
    R T[9];
    mm3(A_kk, q, T);
    R d = 0, x = 0;
#pragma unroll
    for (int e = 0; e < 9; ++e) { d += T[e] * q[e]; x += q[e] * V[e]; }
    snu += d;
    scr += x;
}

// Team sums (FP64) of the two per-thread terms; thread 0 receives them.
template <typename R, class Team, class S>
__device__ void team_sum2(const Team& tm, S& sm, R snu, R scr, double& nu2, double& cross)
{
    const int tid = tm.tid(), lane = threadIdx.x & 31;
    double a = warp_sum((double)snu), b = warp_sum((double)scr);
    if constexpr (Team::NW > 1) {
        if (lane == 0) { sm.red[0][tm.warp()] = a; sm.red[1][tm.warp()] = b; }
        tm.sync();
        if (tid == 0) {
            a = 0.0; b = 0.0;
            for (int w = 0; w < Team::NW; ++w) { a += sm.red[0][w]; b += sm.red[1][w]; }
        }
        tm.sync();
    }
    nu2 = a;
    cross = b;
}

// Arguments common to every ACA launch of one run.
template <typename R>
AcaArgs<R> make_aca_args(hh_ctx* ctx, const hh_tree* t, const hh_blocks* bl, const hh_params& p, const AcaRun& r)
{
    AcaArgs<R> A{};
    A.Xs = t->Xs;
    A.Xp = t->Xp;
    A.th_g = theta_for<R>(ctx, p, &A.n_th);
    A.pp = PairParams{p.radius, p.viscosity};
    A.Fs = r.Fs;
    A.PG = bl->PG;
    A.nbeg = t->nbeg;
    A.nend = t->nend;
    A.counter = ctx->d_counters;
    A.max_rank = p.max_rank;
    A.eps2 = p.eps * p.eps;
    A.j1_rule = p.j1_rule;
    A.seed = p.seed;
    A.rank = r.rank;
    A.pivI = r.pivI;
    A.pivJ = r.pivJ;
    A.part = (R*)r.part;
    A.pofs = r.pofs;
    A.pofs_base = r.pofs_base;
    A.fac = (R*)r.factors;
    A.fofs = r.fofs;
    A.fofs_base = r.fofs_base;
    A.status = ctx->d_status;
    A.n_queries = ctx->d_counters + 4;
    return A;
}

}  // namespace
