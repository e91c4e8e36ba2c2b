// hh_backward.cu -- adjoint of the H-matrix mobility product (hh_matvec_backward).
//
// L = sum_i w_i . U_i with U = alpha_1 F + M_H F, tree / partition / ACA pivots
// frozen.  dL/dF = alpha_1 w + M_H^T w is the transposed product (hh_matvec).
// dL/dX and dL/dtheta come from every pair-kernel entry the product uses:
//
//  * inadmissible block (tau, sigma), pair (m, n), m != n: the entry
//    K(x_m - x_n) with cotangent w_m F_n^T;
//  * admissible block: reverse-mode differentiation of the rank loop of
//    Algorithm 2 with the pivots frozen (k_far_rev), which yields a cotangent
//    for every entry G(m, j_k) and G(i_k, n) the ACA evaluated.
//
// For one entry K(r) = S(o(f(r))) / |r|, f = [r/|r|, a/|r|], cotangent G:
//   dL/do = [G00, G11, G22, G01+G10, G02+G20, G12+G21] / |r|,
//   reverse pass through the MLP -> dL/df and the layer cotangents,
//   dL/dr = -<G, S> r / |r|^3 + (I - r r^T/|r|^2) dL/df[0:3] / |r|
//           - a r / |r|^3 dL/df[3],
//   dL/dx_target += dL/dr, dL/dx_source -= dL/dr;
//   dL/dtheta: each layer's weights get the sum over entries of (cotangent
//   of the layer output) x (layer input).
// Activations are recomputed, never stored between the forward and adjoint.
//
// Every sum has a fixed order, so the gradients are reproducible bit for bit:
//  * near field: one warp per target leaf, with the pairs of all its
//    inadmissible blocks in a fixed order; each pair (m, n) is evaluated as
//    the entry K(x_m - x_n) (contributing to x_m and to theta) and as its
//    mirror K(x_n - x_m) in block (sigma, tau) (contributing to x_m only;
//    its theta part is counted when sigma is the target), so every particle
//    row of dL/dX is summed by one lane of one warp.  The entries run in
//    FP32 when the product's near field did (FP32 / BF16 H-matrices), in
//    FP64 otherwise: a pair's contributions do not cancel.
//  * admissible blocks, in groups bounded by the memory budget: the rank
//    loop's reverse pass (FP64, one CTA per block) writes each entry's
//    cotangent; the entries' reverse passes (FP64: the cotangents of a rank
//    loop cancel to the size of its pivots' condition) run flat over the
//    group and write each entry's dL/dr; per block and step the row and
//    column sums of those are formed in order; then each particle gathers
//    its terms, root to leaf and block by block.
//  * dL/dtheta: every warp owns a slot of FP64 accumulators (lanes own
//    disjoint parameters, 32 entries at a time, work assigned statically);
//    the slots are summed in order at the end.
#include <algorithm>

#include "hh_internal.h"

namespace {

constexpr int BWD_MAXL = 64;
constexpr size_t SMEM_MAX = 227 * 1024;

template <int W>
__host__ __device__ constexpr int n_params() { return 4 * W + W + 2 * (W * W + W) + 6 * W + 6; }

// One lane's entry record: the inputs of the four layers (F, H1..H3) and the
// cotangents of their outputs (A1..A3, GO).  A_l first holds the layer's
// sigmoid s = sigma(z) (silu'(z) = s + h (1 - s) with h = z s), then its
// cotangent.
template <int W>
struct Rec {
    static constexpr int F = 0, H1 = 4, H2 = 4 + W, H3 = 4 + 2 * W, A1 = 4 + 3 * W, A2 = 4 + 4 * W, A3 = 4 + 5 * W,
                         GO = 4 + 6 * W, SIZE = 4 + 6 * W + 6;
};

template <typename R> __device__ __forceinline__ R sigm(R x);
template <> __device__ __forceinline__ float sigm<float>(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }
template <> __device__ __forceinline__ double sigm<double>(double x) { return 1.0 / (1.0 + exp(-x)); }

// Forward + reverse pass of one entry into this lane's record; dL/dr in gr.
// valid == false writes a zero record (no gradient).
template <typename R, int W>
__device__ void entry_backward(const R* __restrict__ th, R a, R rx, R ry, R rz, const R* Gc, bool valid, R* rec,
                               R gr[3])
{
    using L = Rec<W>;
    const R* W1 = th;
    const R* b1 = W1 + 4 * W;
    const R* W2 = b1 + W;
    const R* b2 = W2 + W * W;
    const R* W3 = b2 + W;
    const R* b3 = W3 + W * W;
    const R* W4 = b3 + W;
    const R* b4 = W4 + 6 * W;
    gr[0] = gr[1] = gr[2] = 0;
    if (!valid) {
        for (int i = 0; i < L::SIZE; ++i) rec[i] = 0;
        return;
    }
    const R id = rsqrt_<R>(rx * rx + ry * ry + rz * rz);
    R* f = rec + L::F;
    f[0] = rx * id; f[1] = ry * id; f[2] = rz * id; f[3] = a * id;
    for (int j = 0; j < W; ++j) {
        R z = b1[j];
        for (int i = 0; i < 4; ++i) z += W1[4 * j + i] * f[i];
        const R s = sigm<R>(z);
        rec[L::A1 + j] = s;
        rec[L::H1 + j] = z * s;
    }
    for (int j = 0; j < W; ++j) {
        R z = b2[j];
        for (int i = 0; i < W; ++i) z += W2[W * j + i] * rec[L::H1 + i];
        const R s = sigm<R>(z);
        rec[L::A2 + j] = s;
        rec[L::H2 + j] = z * s;
    }
    for (int j = 0; j < W; ++j) {
        R z = b3[j];
        for (int i = 0; i < W; ++i) z += W3[W * j + i] * rec[L::H2 + i];
        const R s = sigm<R>(z);
        rec[L::A3 + j] = s;
        rec[L::H3 + j] = z * s;
    }
    R o[6];
    for (int j = 0; j < 6; ++j) {
        R t = b4[j];
        for (int i = 0; i < W; ++i) t += W4[W * j + i] * rec[L::H3 + i];
        o[j] = t;
    }
    // <G, S(o)> and dL/do
    const R gs = Gc[0] * o[0] + Gc[4] * o[1] + Gc[8] * o[2] + (Gc[1] + Gc[3]) * o[3] + (Gc[2] + Gc[6]) * o[4] +
                 (Gc[5] + Gc[7]) * o[5];
    R* go = rec + L::GO;
    go[0] = Gc[0] * id; go[1] = Gc[4] * id; go[2] = Gc[8] * id;
    go[3] = (Gc[1] + Gc[3]) * id; go[4] = (Gc[2] + Gc[6]) * id; go[5] = (Gc[5] + Gc[7]) * id;
    for (int i = 0; i < W; ++i) {
        R t = 0;
        for (int j = 0; j < 6; ++j) t += W4[W * j + i] * go[j];
        const R s = rec[L::A3 + i], h = rec[L::H3 + i];
        rec[L::A3 + i] = t * (s + h * (1 - s));
    }
    for (int i = 0; i < W; ++i) {
        R t = 0;
        for (int j = 0; j < W; ++j) t += W3[W * j + i] * rec[L::A3 + j];
        const R s = rec[L::A2 + i], h = rec[L::H2 + i];
        rec[L::A2 + i] = t * (s + h * (1 - s));
    }
    for (int i = 0; i < W; ++i) {
        R t = 0;
        for (int j = 0; j < W; ++j) t += W2[W * j + i] * rec[L::A2 + j];
        const R s = rec[L::A1 + i], h = rec[L::H1 + i];
        rec[L::A1 + i] = t * (s + h * (1 - s));
    }
    R gf[4];
    for (int i = 0; i < 4; ++i) {
        R t = 0;
        for (int j = 0; j < W; ++j) t += W1[4 * j + i] * rec[L::A1 + j];
        gf[i] = t;
    }
    const R rg = (rx * gf[0] + ry * gf[1] + rz * gf[2]) * id;
    const R r3[3] = {rx, ry, rz};
    for (int q = 0; q < 3; ++q)
        gr[q] = -gs * id * r3[q] * id * id + (gf[q] - rg * r3[q] * id) * id - a * r3[q] * id * id * id * gf[3];
}

// Parameter cotangents of the warp's 32 records added into its slot (packed
// parameter layout; lane owns parameters lane, lane + 32, ...).
template <typename R, int W>
__device__ void accumulate_theta(const R* recs, double* slot)
{
    using L = Rec<W>;
    const int lane = threadIdx.x & 31;
    constexpr int dims[5] = {4, W, W, W, 6};
    constexpr int hin[4] = {L::F, L::H1, L::H2, L::H3};
    constexpr int gout[4] = {L::A1, L::A2, L::A3, L::GO};
    int base = 0;
#pragma unroll 1
    for (int l = 0; l < 4; ++l) {
        const int ni = dims[l], no = dims[l + 1], nl = ni * no + no;
        for (int x = lane; x < nl; x += 32) {
            const int o = x < ni * no ? x / ni : x - ni * no;
            const int i = x < ni * no ? x % ni : -1;
            R s = 0;
            for (int p = 0; p < 32; ++p) {
                const R* rp = recs + p * L::SIZE;
                s += rp[gout[l] + o] * (i >= 0 ? rp[hin[l] + i] : (R)1);
            }
            slot[base + x] += (double)s;
        }
        base += nl;
    }
}

// Shared-memory layout of the entry kernels: the parameters (R), then per
// warp its 32 records (R) and, for the near field, the per-row sums of its
// target leaf and a 32-entry staging area.
template <typename R, int W>
struct EntLayout {
    __host__ __device__ static constexpr size_t al(size_t x) { return (x + 15) & ~(size_t)15; }
    static constexpr size_t th = al(sizeof(R) * n_params<W>());
    static constexpr size_t recs = al(sizeof(R) * 32 * Rec<W>::SIZE);
    __host__ __device__ static size_t near_extra(int leaf)
    {
        return al(sizeof(double) * 3 * leaf) + al(sizeof(double) * 96) + al(sizeof(int) * 32);
    }
    __host__ __device__ static size_t per_warp(int leaf) { return recs + (leaf > 0 ? near_extra(leaf) : 0); }
    static int warps(int leaf)
    {
        const size_t room = SMEM_MAX - th;
        return (int)std::min<size_t>(8, room / per_warp(leaf));
    }
};

template <typename R, int W>
__device__ void load_theta(R* th_s, const R* __restrict__ th_g)
{
    for (int i = threadIdx.x; i < n_params<W>(); i += blockDim.x) th_s[i] = th_g[i];
    __syncthreads();
}

// ---- inadmissible blocks ------------------------------------------------------
template <typename R, int W>
__global__ void __launch_bounds__(256) k_near_rev(const double* __restrict__ Xs, const double* __restrict__ Fs,
                                                  const double* __restrict__ Ws, const int32_t* __restrict__ PH,
                                                  const int64_t* __restrict__ rowH, const int32_t* __restrict__ leaves,
                                                  int64_t n_leaves, const int32_t* __restrict__ nbeg,
                                                  const int32_t* __restrict__ nend, const R* __restrict__ th_g, R a,
                                                  int leaf_cap, double* __restrict__ GXs, double* __restrict__ slots,
                                                  int want_theta)
{
    using Ly = EntLayout<R, W>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* th = reinterpret_cast<R*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    unsigned char* mine_area = smem_raw + Ly::th + (size_t)warp * Ly::per_warp(leaf_cap);
    R* recs = reinterpret_cast<R*>(mine_area);
    double* gxs = reinterpret_cast<double*>(mine_area + Ly::recs);
    double* stg = reinterpret_cast<double*>(mine_area + Ly::recs + Ly::al(sizeof(double) * 3 * leaf_cap));
    int* stm = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(stg) + Ly::al(sizeof(double) * 96));
    load_theta<R, W>(th, th_g);
    double* slot = slots + ((int64_t)blockIdx.x * nw + warp) * n_params<W>();
    R* rec = recs + lane * Rec<W>::SIZE;
    for (int64_t li = (int64_t)blockIdx.x * nw + warp; li < n_leaves; li += (int64_t)gridDim.x * nw) {
        const int32_t tau = leaves[li];
        const int32_t t0 = nbeg[tau], c = nend[tau] - t0;
        for (int i = lane; i < 3 * c; i += 32) gxs[i] = 0.0;
        __syncwarp();
        for (int64_t bb = rowH[tau]; bb < rowH[tau + 1]; ++bb) {
            const int32_t sg = PH[2 * bb + 1];
            const int32_t s0 = nbeg[sg], q = nend[sg] - s0;
            const int64_t P = (int64_t)c * q;
            for (int64_t p0 = 0; p0 < P; p0 += 32) {
                const int64_t p = p0 + lane;
                int m = 0;
                int64_t ti = 0, si = 0;
                bool valid = p < P;
                if (valid) {
                    m = (int)(p / q);
                    ti = t0 + m;
                    si = s0 + p % q;
                    valid = ti != si;
                }
                R rx = 0, ry = 0, rz = 1, Gc[9], gA[3], gB[3];
                if (valid) {
                    sep<R>(Xs, ti, si, rx, ry, rz);
                    for (int u = 0; u < 3; ++u)
                        for (int v = 0; v < 3; ++v) Gc[3 * u + v] = (R)(Ws[3 * ti + u] * Fs[3 * si + v]);
                }
                // the entry K(x_m - x_n): x_m and theta
                entry_backward<R, W>(th, a, rx, ry, rz, Gc, valid, rec, gA);
                __syncwarp();
                if (want_theta) accumulate_theta<R, W>(recs, slot);
                __syncwarp();
                // its mirror K(x_n - x_m), cotangent w_n F_m^T: x_m only
                if (valid)
                    for (int u = 0; u < 3; ++u)
                        for (int v = 0; v < 3; ++v) Gc[3 * u + v] = (R)(Ws[3 * si + u] * Fs[3 * ti + v]);
                entry_backward<R, W>(th, a, -rx, -ry, -rz, Gc, valid, rec, gB);
                stm[lane] = valid ? m : -1;
                for (int u = 0; u < 3; ++u) stg[3 * lane + u] = (double)gA[u] - (double)gB[u];
                __syncwarp();
                // row m is summed by lane m % 32, entries in lane order
                for (int i = 0; i < 32; ++i) {
                    const int mm = stm[i];
                    if (mm >= 0 && (mm & 31) == lane)
                        for (int u = 0; u < 3; ++u) gxs[3 * mm + u] += stg[3 * i + u];
                }
                __syncwarp();
            }
        }
        for (int i = lane; i < 3 * c; i += 32) GXs[3 * (int64_t)t0 + i] = gxs[i];
        __syncwarp();
    }
}

// ---- admissible blocks ----------------------------------------------------------
// Forward pair kernel (FP64) for the pivot blocks.
template <int W>
__device__ void entry_forward(const double* __restrict__ th, double a, double rx, double ry, double rz, double K[9])
{
    const double* W1 = th;
    const double* b1 = W1 + 4 * W;
    const double* W2 = b1 + W;
    const double* b2 = W2 + W * W;
    const double* W3 = b2 + W;
    const double* b3 = W3 + W * W;
    const double* W4 = b3 + W;
    const double* b4 = W4 + 6 * W;
    const double id = 1.0 / sqrt(rx * rx + ry * ry + rz * rz);
    double f[4] = {rx * id, ry * id, rz * id, a * id}, h[W], g[W], o[6];
    for (int j = 0; j < W; ++j) {
        double t = b1[j];
        for (int i = 0; i < 4; ++i) t += W1[4 * j + i] * f[i];
        h[j] = silu_d(t);
    }
    for (int j = 0; j < W; ++j) {
        double t = b2[j];
        for (int i = 0; i < W; ++i) t += W2[W * j + i] * h[i];
        g[j] = silu_d(t);
    }
    for (int j = 0; j < W; ++j) {
        double t = b3[j];
        for (int i = 0; i < W; ++i) t += W3[W * j + i] * g[i];
        h[j] = silu_d(t);
    }
    for (int j = 0; j < 6; ++j) {
        double t = b4[j];
        for (int i = 0; i < W; ++i) t += W4[W * j + i] * h[i];
        o[j] = t;
    }
    K[0] = o[0] * id; K[1] = o[3] * id; K[2] = o[4] * id;
    K[3] = o[3] * id; K[4] = o[1] * id; K[5] = o[5] * id;
    K[6] = o[4] * id; K[7] = o[5] * id; K[8] = o[2] * id;
}

__device__ __forceinline__ void acc_abt(double* acc, const double* A, const double* B)   // acc += A B^T
{
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v)
            acc[3 * u + v] += A[3 * u] * B[3 * v] + A[3 * u + 1] * B[3 * v + 1] + A[3 * u + 2] * B[3 * v + 2];
}
__device__ __forceinline__ void acc_atb(double* acc, const double* A, const double* B)   // acc += A^T B
{
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v) acc[3 * u + v] += A[u] * B[v] + A[3 + u] * B[3 + v] + A[6 + u] * B[6 + v];
}
__device__ __forceinline__ void ld9g(const double* base, int64_t ld, int64_t x, double* v)
{
#pragma unroll
    for (int e = 0; e < 9; ++e) v[e] = base[e * ld + x];
}
__device__ __forceinline__ void st9g(double* base, int64_t ld, int64_t x, const double* v)
{
#pragma unroll
    for (int e = 0; e < 9; ++e) base[e * ld + x] = v[e];
}

constexpr int REV_T = 128;   // threads of one block's rank-loop reverse pass

// Sum of n <= 9 values over the CTA in a fixed order (shuffle tree per warp,
// then the warps in order); every thread receives the sums.
__device__ void cta_sum(double* v, int n, double* red)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = 0; e < n; ++e) v[e] = warp_sum(v[e]);
    if (lane == 0)
        for (int e = 0; e < n; ++e) red[9 * warp + e] = v[e];
    __syncthreads();
    if (threadIdx.x < n) {
        double s = red[threadIdx.x];
        for (int w = 1; w < REV_T / 32; ++w) s += red[9 * w + threadIdx.x];
        red[9 * (REV_T / 32) + threadIdx.x] = s;
    }
    __syncthreads();
    for (int e = 0; e < n; ++e) v[e] = red[9 * (REV_T / 32) + e];
    __syncthreads();
}

struct FarArgs {
    const double* Xs;
    const double* Fs;
    const double* Ws;
    const int32_t* PG;
    const int32_t* nbeg;
    const int32_t* nend;
    const int32_t* rank;
    const int32_t* pivI;
    const int32_t* pivJ;
    int max_rank;
    const uint8_t* mine;
    const double* fac;       // factors: block b at 9 (fofs[b] - fac_base)
    const int64_t* fofs;
    int64_t fac_base;
    int64_t b0, b1;          // the group's blocks
    int64_t ent_base;        // fofs[b0]: the group's entries start here
    double* cot;             // entry cotangents, laid out as the factors
    double* gr;              // entry dL/dr [3 per entry]
    double* sums;            // per block and step: row sum, column sum of gr, s_k (9 doubles)
    const double* th;        // FP64 parameters
    double a;
};

// Reverse pass of the rank loop of Algorithm 2 on one admissible block per
// CTA, pivots frozen.  Forward (per step k, 3x3 elements):
//   chat_k(m) = G(m, j_k) - sum_{p<k} C_p(m) Q_p(j_k),  P_k = chat_k(i_k),
//   C_k(m) = chat_k(m) P_k^-1,  Q_k(n) = G(i_k, n) - sum_{p<k} C_p(i_k) Q_p(n),
//   y(m) = sum_k C_k(m) t_k with t_k = sum_n Q_k(n) F_n;  L = sum_m w_m . y(m).
// Reverse, k = l-1 .. 0 (cotangents Cb, Qb start at w_m t_k^T and s_k F_n^T,
// s_k = sum_m C_k(m)^T w_m):
//   row k:    Cb_p(i_k) -= sum_n Qb_k(n) Q_p(n)^T,  Qb_p(n) -= C_p(i_k)^T Qb_k(n);
//             Qb_k(n) is the cotangent of the entry G(i_k, n);
//   scaling:  chat-bar_k(m) = Cb_k(m) P_k^-T,
//             chat-bar_k(i_k) -= (sum_m C_k(m)^T Cb_k(m)) P_k^-T;
//   column k: Qb_p(j_k) -= sum_m C_p(m)^T chat-bar_k(m),
//             Cb_p(m) -= chat-bar_k(m) Q_p(j_k)^T;
//             chat-bar_k(m) is the cotangent of the entry G(m, j_k).
// Only the 3x3 pivot blocks the forward pass inverted are inverted again
// (from the factors and one pair-kernel entry, FP64), so the adjoint is as
// well conditioned as the forward recursion.
template <int W>
__global__ void __launch_bounds__(REV_T) k_far_rev(FarArgs A)
{
    __shared__ double tv[BWD_MAXL * 3], sv[BWD_MAXL * 3], piT[9], red[9 * (REV_T / 32 + 1)];
    const int tid = threadIdx.x;
    for (int64_t b = A.b0 + blockIdx.x; b < A.b1; b += gridDim.x) {
        const int l = A.rank[b];
        if (l <= 0 || (A.mine && !A.mine[b])) continue;
        const int32_t t = A.PG[2 * b], s = A.PG[2 * b + 1];
        const int32_t t0 = A.nbeg[t], c = A.nend[t] - t0, s0 = A.nbeg[s], q = A.nend[s] - s0;
        const int32_t* I = A.pivI + b * A.max_rank;
        const int32_t* J = A.pivJ + b * A.max_rank;
        const double* C = A.fac + 9 * (A.fofs[b] - A.fac_base);
        const double* Q = C + (int64_t)l * 9 * c;
        double* Cb = A.cot + 9 * (A.fofs[b] - A.ent_base);
        double* Qb = Cb + (int64_t)l * 9 * c;
        double* sums = A.sums + (b - A.b0) * A.max_rank * 9;
        auto Ck = [&](int k) { return C + (int64_t)k * 9 * c; };
        auto Qk = [&](int k) { return Q + (int64_t)k * 9 * q; };
        auto Cbk = [&](int k) { return Cb + (int64_t)k * 9 * c; };
        auto Qbk = [&](int k) { return Qb + (int64_t)k * 9 * q; };
        // t_k = sum_n Q_k(n) F_n,  s_k = sum_m C_k(m)^T w_m
        for (int k = 0; k < l; ++k) {
            double v[6] = {0, 0, 0, 0, 0, 0};
            for (int n = tid; n < q; n += REV_T) {
                double x[9];
                ld9g(Qk(k), q, n, x);
                const double* f = A.Fs + 3 * (int64_t)(s0 + n);
                for (int u = 0; u < 3; ++u) v[u] += x[3 * u] * f[0] + x[3 * u + 1] * f[1] + x[3 * u + 2] * f[2];
            }
            for (int m = tid; m < c; m += REV_T) {
                double x[9];
                ld9g(Ck(k), c, m, x);
                const double* w = A.Ws + 3 * (int64_t)(t0 + m);
                for (int u = 0; u < 3; ++u) v[3 + u] += x[u] * w[0] + x[3 + u] * w[1] + x[6 + u] * w[2];
            }
            cta_sum(v, 6, red);
            if (tid < 3) {
                tv[3 * k + tid] = v[tid];
                sv[3 * k + tid] = v[3 + tid];
                sums[9 * k + 6 + tid] = v[3 + tid];
            }
        }
        __syncthreads();
        for (int k = 0; k < l; ++k) {
            for (int m = tid; m < c; m += REV_T) {
                const double* w = A.Ws + 3 * (int64_t)(t0 + m);
                double v[9];
                for (int u = 0; u < 3; ++u)
                    for (int x = 0; x < 3; ++x) v[3 * u + x] = w[u] * tv[3 * k + x];
                st9g(Cbk(k), c, m, v);
            }
            for (int n = tid; n < q; n += REV_T) {
                const double* f = A.Fs + 3 * (int64_t)(s0 + n);
                double v[9];
                for (int u = 0; u < 3; ++u)
                    for (int x = 0; x < 3; ++x) v[3 * u + x] = sv[3 * k + u] * f[x];
                st9g(Qbk(k), q, n, v);
            }
        }
        __syncthreads();
        for (int k = l - 1; k >= 0; --k) {
            const int ik = I[k], jk = J[k];
            // row k
            for (int p = 0; p < k; ++p) {
                double cpi[9], acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                ld9g(Ck(p), c, ik, cpi);
                for (int n = tid; n < q; n += REV_T) {
                    double qb[9], qp[9], up[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, cur[9];
                    ld9g(Qbk(k), q, n, qb);
                    ld9g(Qk(p), q, n, qp);
                    acc_abt(acc, qb, qp);
                    acc_atb(up, cpi, qb);
                    ld9g(Qbk(p), q, n, cur);
                    for (int e = 0; e < 9; ++e) cur[e] -= up[e];
                    st9g(Qbk(p), q, n, cur);
                }
                cta_sum(acc, 9, red);
                if (tid == 0) {
                    double cur[9];
                    ld9g(Cbk(p), c, ik, cur);
                    for (int e = 0; e < 9; ++e) cur[e] -= acc[e];
                    st9g(Cbk(p), c, ik, cur);
                }
                __syncthreads();
            }
            // pivot block P_k = G(i_k, j_k) - sum_{p<k} C_p(i_k) Q_p(j_k), inverse-transpose in FP64
            if (tid == 0) {
                double rx, ry, rz, K[9];
                sep<double>(A.Xs, t0 + ik, s0 + jk, rx, ry, rz);
                entry_forward<W>(A.th, A.a, rx, ry, rz, K);
                for (int p = 0; p < k; ++p) {
                    double cp[9], qp[9], t9[9];
                    ld9g(Ck(p), c, ik, cp);
                    ld9g(Qk(p), q, jk, qp);
                    mm3(cp, qp, t9);
                    for (int e = 0; e < 9; ++e) K[e] -= t9[e];
                }
                double Pi[9];
                inv3d(K, Pi);
                for (int u = 0; u < 3; ++u)
                    for (int v = 0; v < 3; ++v) piT[3 * u + v] = Pi[3 * v + u];
            }
            __syncthreads();
            // scaling: chat-bar_k = Cb_k P^-T;  r1 = sum_m C_k(m)^T Cb_k(m)
            double r1[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int m = tid; m < c; m += REV_T) {
                double cb[9], ck[9], o[9];
                ld9g(Cbk(k), c, m, cb);
                ld9g(Ck(k), c, m, ck);
                acc_atb(r1, ck, cb);
                mm3(cb, piT, o);
                st9g(Cbk(k), c, m, o);
            }
            cta_sum(r1, 9, red);
            if (tid == 0) {
                double dP[9], cur[9];
                mm3(r1, piT, dP);
                ld9g(Cbk(k), c, ik, cur);
                for (int e = 0; e < 9; ++e) cur[e] -= dP[e];
                st9g(Cbk(k), c, ik, cur);
            }
            __syncthreads();
            // column k
            for (int p = 0; p < k; ++p) {
                double qpj[9], acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                ld9g(Qk(p), q, jk, qpj);
                for (int m = tid; m < c; m += REV_T) {
                    double cb[9], cp[9], up[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, cur[9];
                    ld9g(Cbk(k), c, m, cb);
                    ld9g(Ck(p), c, m, cp);
                    acc_atb(acc, cp, cb);
                    acc_abt(up, cb, qpj);
                    ld9g(Cbk(p), c, m, cur);
                    for (int e = 0; e < 9; ++e) cur[e] -= up[e];
                    st9g(Cbk(p), c, m, cur);
                }
                cta_sum(acc, 9, red);
                if (tid == 0) {
                    double cur[9];
                    ld9g(Qbk(p), q, jk, cur);
                    for (int e = 0; e < 9; ++e) cur[e] -= acc[e];
                    st9g(Qbk(p), q, jk, cur);
                }
                __syncthreads();
            }
        }
    }
}

// The entries of one group of admissible blocks, 32 per warp at a time, in
// entry order (block by block: the column entries G(m, j_k), k-major, then
// the row entries G(i_k, n)): reverse pass, dL/dr stored per entry, theta
// cotangents into the warp's slot.
template <int W>
__global__ void __launch_bounds__(256) k_far_entries(FarArgs A, int64_t n_ent, double* __restrict__ slots,
                                                     int want_theta)
{
    using Ly = EntLayout<double, W>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* th = reinterpret_cast<double*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double* recs = reinterpret_cast<double*>(smem_raw + Ly::th + (size_t)warp * Ly::per_warp(0));
    load_theta<double, W>(th, A.th);
    double* slot = slots + ((int64_t)blockIdx.x * nw + warp) * n_params<W>();
    double* rec = recs + lane * Rec<W>::SIZE;
    for (int64_t e0 = ((int64_t)blockIdx.x * nw + warp) * 32; e0 < n_ent; e0 += (int64_t)gridDim.x * nw * 32) {
        const int64_t e = e0 + lane;
        bool valid = e < n_ent;
        int64_t ti = 0, si = 0;
        double Gc[9];
        if (valid) {
            const int64_t g = A.ent_base + e;
            int64_t lo = A.b0, hi = A.b1 - 1;   // the block holding entry g: last b with fofs[b] <= g
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (A.fofs[mid] <= g) lo = mid; else hi = mid - 1;
            }
            const int64_t b = lo;
            valid = !A.mine || A.mine[b];
            const int l = A.rank[b];
            const int32_t t = A.PG[2 * b], s = A.PG[2 * b + 1];
            const int32_t t0 = A.nbeg[t], c = A.nend[t] - t0, s0 = A.nbeg[s], q = A.nend[s] - s0;
            const int64_t loc = g - A.fofs[b];
            const double* cb = A.cot + 9 * (A.fofs[b] - A.ent_base);
            if (loc < (int64_t)l * c) {
                const int k = (int)(loc / c), m = (int)(loc % c);
                ti = t0 + m;
                si = s0 + A.pivJ[b * A.max_rank + k];
                ld9g(cb + (int64_t)k * 9 * c, c, m, Gc);
            } else {
                const int64_t x = loc - (int64_t)l * c;
                const int k = (int)(x / q), n = (int)(x % q);
                ti = t0 + A.pivI[b * A.max_rank + k];
                si = s0 + n;
                ld9g(cb + (int64_t)l * 9 * c + (int64_t)k * 9 * q, q, n, Gc);
            }
        }
        double rx = 0, ry = 0, rz = 1, gr[3];
        if (valid) sep<double>(A.Xs, ti, si, rx, ry, rz);
        entry_backward<double, W>(th, A.a, rx, ry, rz, Gc, valid, rec, gr);
        if (e < n_ent)
            for (int u = 0; u < 3; ++u) A.gr[3 * e + u] = gr[u];
        __syncwarp();
        if (want_theta) accumulate_theta<double, W>(recs, slot);
        __syncwarp();
    }
}

// Per block of the group and step k (one warp per block): the sums over the
// row entries (i_k, n) and over the column entries (m, j_k) of dL/dr, in
// order.  They reach x_{t0 + i_k} and x_{s0 + j_k}.
__global__ void k_far_sums(FarArgs A)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = A.b0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < A.b1; b += nwarps) {
        const int l = A.rank[b];
        if (l <= 0 || (A.mine && !A.mine[b])) continue;
        const int32_t t = A.PG[2 * b], s = A.PG[2 * b + 1];
        const int32_t c = A.nend[t] - A.nbeg[t], q = A.nend[s] - A.nbeg[s];
        const double* col = A.gr + 3 * (A.fofs[b] - A.ent_base);
        const double* row = col + 3 * (int64_t)l * c;
        double* sums = A.sums + (b - A.b0) * A.max_rank * 9;
        for (int k = 0; k < l; ++k) {
            double rs[3] = {0, 0, 0}, cs[3] = {0, 0, 0};
            for (int n = lane; n < q; n += 32)
                for (int u = 0; u < 3; ++u) rs[u] += row[3 * ((int64_t)k * q + n) + u];
            for (int m = lane; m < c; m += 32)
                for (int u = 0; u < 3; ++u) cs[u] += col[3 * ((int64_t)k * c + m) + u];
            for (int u = 0; u < 3; ++u) {
                rs[u] = warp_sum(rs[u]);
                cs[u] = warp_sum(cs[u]);
            }
            if (lane < 3) {
                sums[9 * k + lane] = rs[lane];
                sums[9 * k + 3 + lane] = cs[lane];
            }
        }
    }
}

// Each particle m (sorted index) gathers the group's terms, root to leaf:
// as a target of block b (tau = node), sum_k gr(m, j_k) plus the row sums of
// the steps whose pivot row it is; as a source (sigma = node, the blocks in
// increasing order), minus sum_k gr(i_k, m) minus the column sums of the
// steps whose pivot column it is; and, when gFs is given, the block's part of
// M_H^T w, sum_k Q_k(m)^T s_k.
__global__ void k_far_gather(FarArgs A, int64_t n, const int64_t* __restrict__ rowG,
                             const int64_t* __restrict__ colG, const int32_t* __restrict__ colorder,
                             const int32_t* __restrict__ child, const int64_t* __restrict__ off, int B,
                             double* __restrict__ GXs, double* __restrict__ GFs)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= m) lo = mid; else hi = mid - 1;
    }
    double gx[3] = {GXs[3 * m], GXs[3 * m + 1], GXs[3 * m + 2]};
    double gf[3] = {0, 0, 0};
    if (GFs)
        for (int u = 0; u < 3; ++u) gf[u] = GFs[3 * m + u];
    int32_t node = lo;
    for (;;) {
        const int32_t nb = A.nbeg[node], size = A.nend[node] - nb;
        const int32_t loc = (int32_t)(m - nb);
        for (int64_t b = max(rowG[node], A.b0); b < min(rowG[node + 1], A.b1); ++b) {
            const int l = A.rank[b];
            if (l <= 0 || (A.mine && !A.mine[b])) continue;
            const double* col = A.gr + 3 * (A.fofs[b] - A.ent_base);
            const double* sums = A.sums + (b - A.b0) * A.max_rank * 9;
            const int32_t* I = A.pivI + b * A.max_rank;
            for (int k = 0; k < l; ++k)
                for (int u = 0; u < 3; ++u) gx[u] += col[3 * ((int64_t)k * size + loc) + u];
            for (int k = 0; k < l; ++k)
                if (I[k] == loc)
                    for (int u = 0; u < 3; ++u) gx[u] += sums[9 * k + u];
        }
        // the blocks with sigma = node, in increasing order: from the first >= b0
        int64_t a0 = colG[node], a1 = colG[node + 1];
        while (a0 < a1) {
            const int64_t mid = (a0 + a1) >> 1;
            if (colorder[mid] < A.b0) a0 = mid + 1; else a1 = mid;
        }
        for (int64_t x = a0; x < colG[node + 1]; ++x) {
            const int64_t b = colorder[x];
            if (b >= A.b1) break;
            const int l = A.rank[b];
            if (l <= 0 || (A.mine && !A.mine[b])) continue;
            const int32_t t = A.PG[2 * b];
            const int32_t c = A.nend[t] - A.nbeg[t];
            const double* row = A.gr + 3 * (A.fofs[b] - A.ent_base) + 3 * (int64_t)l * c;
            const double* sums = A.sums + (b - A.b0) * A.max_rank * 9;
            const int32_t* J = A.pivJ + b * A.max_rank;
            for (int k = 0; k < l; ++k)
                for (int u = 0; u < 3; ++u) gx[u] -= row[3 * ((int64_t)k * size + loc) + u];
            for (int k = 0; k < l; ++k)
                if (J[k] == loc)
                    for (int u = 0; u < 3; ++u) gx[u] -= sums[9 * k + 3 + u];
            if (GFs) {
                const double* Q = A.fac + 9 * (A.fofs[b] - A.fac_base) + (int64_t)l * 9 * c;
                for (int k = 0; k < l; ++k) {
                    double v[9];
                    ld9g(Q + (int64_t)k * 9 * size, size, loc, v);
                    const double* sk = sums + 9 * k + 6;
                    for (int u = 0; u < 3; ++u) gf[u] += v[u] * sk[0] + v[3 + u] * sk[1] + v[6 + u] * sk[2];
                }
            }
        }
        const int32_t c0 = child[2 * node];
        if (c0 < 0) break;
        node = m < A.nend[c0] ? c0 : child[2 * node + 1];
    }
    for (int u = 0; u < 3; ++u) GXs[3 * m + u] = gx[u];
    if (GFs)
        for (int u = 0; u < 3; ++u) GFs[3 * m + u] = gf[u];
}

__global__ void k_leafs(const int32_t* __restrict__ child, int32_t n, const uint8_t* __restrict__ mine,
                        uint8_t* __restrict__ flag)
{
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) flag[t] = child[2 * t] < 0 && (mine == nullptr || mine[t]);
}

__global__ void k_compact(const uint8_t* __restrict__ flag, const int64_t* __restrict__ pos, int32_t n,
                          int32_t* __restrict__ out)
{
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n && flag[t]) out[pos[t]] = t;
}

__global__ void k_u8_to_i64(const uint8_t* __restrict__ in, int64_t n, int64_t* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

__global__ void k_src_keys(const int32_t* __restrict__ PG, int64_t nG, uint64_t* __restrict__ key,
                           int32_t* __restrict__ val)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nG) {
        key[b] = (uint64_t)PG[2 * b + 1];
        val[b] = (int32_t)b;
    }
}

// colG[node] = first position of the sorted source keys >= node.
__global__ void k_src_offsets(const uint64_t* __restrict__ key, int64_t nG, int32_t n_nodes, int64_t* __restrict__ colG)
{
    const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v > n_nodes) return;
    int64_t lo = 0, hi = nG;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (key[mid] < (uint64_t)v) lo = mid + 1; else hi = mid;
    }
    colG[v] = lo;
}

__global__ void k_theta_reduce(const double* __restrict__ slots, int64_t n_slots, int n, float* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int64_t k = 0; k < n_slots; ++k) s += slots[k * n + i];
    out[i] += (float)s;
}

__global__ void k_gx_out(const double* __restrict__ GXs, const int32_t* __restrict__ perm, int64_t n,
                         double* __restrict__ gX)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const int64_t d = perm[m];
    for (int u = 0; u < 3; ++u) gX[3 * d + u] += GXs[3 * m + u];
}

// The parameters in their packed layout (as hh_set_mlp received them).
template <typename R>
const R* packed_theta(const hh_ctx* ctx)
{
    if constexpr (sizeof(R) == 8) return (const R*)ctx->theta64;
    else return (const R*)ctx->theta32;
}

int64_t entry_grid(hh_ctx* ctx, size_t smem)
{
    const int per_sm = std::max<int>(1, (int)(228 * 1024 / (smem + 1024)));
    return (int64_t)ctx->n_sm * per_sm;
}

template <typename R, int W>
void near_rev(hh_ctx* ctx, const hh_tree* t, const hh_blocks* b, const hh_params& p, const double* Fs,
              const double* Ws, double* GXs, double* slots, int64_t slot_cap, int64_t* n_slots, bool want_theta,
              cudaStream_t s)
{
    using Ly = EntLayout<R, W>;
    // the leaves of this shard, in node order
    uint8_t* node_mine = shard_node_flags(t, b, p, s);
    uint8_t* flag = dev_alloc_t<uint8_t>(t->n_nodes, s);
    k_leafs<<<(unsigned)ceil_div(t->n_nodes, 256), 256, 0, s>>>(t->child, t->n_nodes, node_mine, flag);
    HH_CHECK_LAUNCH();
    if (node_mine) dev_free(node_mine, s);
    int64_t* f64 = dev_alloc_t<int64_t>(t->n_nodes, s);
    int64_t* pos = dev_alloc_t<int64_t>(t->n_nodes, s);
    int64_t* tot = dev_alloc_t<int64_t>(1, s);
    k_u8_to_i64<<<(unsigned)ceil_div(t->n_nodes, 256), 256, 0, s>>>(flag, t->n_nodes, f64);
    HH_CHECK_LAUNCH();
    dev_scan_i64(f64, pos, t->n_nodes, tot, s);
    int32_t* leaves = dev_alloc_t<int32_t>(t->n_nodes, s);
    k_compact<<<(unsigned)ceil_div(t->n_nodes, 256), 256, 0, s>>>(flag, pos, t->n_nodes, leaves);
    HH_CHECK_LAUNCH();
    int64_t n_leaves = 0;
    HH_CUDA(cudaMemcpyAsync(&n_leaves, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HH_CUDA(cudaStreamSynchronize(s));
    dev_free(tot, s);
    dev_free(pos, s);
    dev_free(f64, s);
    dev_free(flag, s);
    const int leaf_cap = p.leaf_size;
    const int warps = Ly::warps(leaf_cap);
    HH_REQUIRE(warps >= 1, HH_ERR_ARG, "adjoint: leaf_size too large for the near-field kernel's shared memory");
    const size_t smem = Ly::th + (size_t)warps * Ly::per_warp(leaf_cap);
    int64_t grid = std::min<int64_t>(entry_grid(ctx, smem), ceil_div(std::max<int64_t>(n_leaves, 1), warps));
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, slot_cap / warps));
    if (n_leaves > 0) {
        HH_CUDA(cudaFuncSetAttribute(k_near_rev<R, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_near_rev<R, W><<<(unsigned)grid, 32 * warps, smem, s>>>(t->Xs, Fs, Ws, b->PH, b->rowH, leaves, n_leaves,
                                                                 t->nbeg, t->nend, packed_theta<R>(ctx),
                                                                 (R)p.radius, leaf_cap, GXs, slots, want_theta);
        HH_CHECK_LAUNCH();
        *n_slots = grid * warps;
    } else {
        *n_slots = 0;
    }
    dev_free(leaves, s);
}

// The admissible blocks in groups of at most about `cap` entries.
template <int W>
void far_rev(hh_ctx* ctx, const hh_hmat* h, const double* Fs, const double* Ws, double* GXs, double* GFs,
             double* slots, int64_t slot_cap, int64_t* n_slots, bool want_theta, cudaStream_t s)
{
    const hh_tree* t = h->tree;
    const hh_blocks* bl = h->blocks;
    const hh_params& p = h->params;
    const int64_t nG = bl->nG;
    *n_slots = 0;
    if (nG == 0 || h->n_factor == 0) return;
    const bool rebuild = h->factors == nullptr;   // pivots only: rebuild the FP64 factors group by group
    const int64_t per_entry = 72 + 24 + (rebuild ? 72 : 0);
    const int64_t cap = std::max<int64_t>(1, aca_budget_bytes(p) / 2 / per_entry);
    std::vector<int64_t> at;
    const auto groups = block_groups(bl, h->fofs, h->n_factor, cap, &at, s);
    int64_t max_ent = 0, max_blocks = 0;
    for (size_t g = 0; g < groups.size(); ++g) {
        max_ent = std::max(max_ent, at[g + 1] - at[g]);
        max_blocks = std::max(max_blocks, groups[g].second - groups[g].first);
    }
    double* cot = dev_alloc_t<double>(9 * max_ent, s);
    double* gr = dev_alloc_t<double>(3 * max_ent, s);
    double* sums = dev_alloc_t<double>(9 * max_blocks * p.max_rank, s);
    double* fac = rebuild ? dev_alloc_t<double>(9 * max_ent, s) : nullptr;
    int32_t* rk = rebuild ? dev_alloc_t<int32_t>(nG, s) : nullptr;
    int32_t* pI = rebuild ? dev_alloc_t<int32_t>(nG * p.max_rank, s) : nullptr;
    int32_t* pJ = rebuild ? dev_alloc_t<int32_t>(nG * p.max_rank, s) : nullptr;
    // the blocks by source node (stable: increasing block within a node)
    uint64_t* key = dev_alloc_t<uint64_t>(nG, s);
    int32_t* colorder = dev_alloc_t<int32_t>(nG, s);
    int64_t* colG = dev_alloc_t<int64_t>(t->n_nodes + 1, s);
    k_src_keys<<<(unsigned)ceil_div(nG, 256), 256, 0, s>>>(bl->PG, nG, key, colorder);
    HH_CHECK_LAUNCH();
    int bits = 1;
    while ((1LL << bits) < t->n_nodes) ++bits;
    dev_radix_sort(key, colorder, nG, bits, s);
    k_src_offsets<<<(unsigned)ceil_div(t->n_nodes + 1, 256), 256, 0, s>>>(key, nG, t->n_nodes, colG);
    HH_CHECK_LAUNCH();
    dev_free(key, s);
    uint8_t* mine = shard_block_flags(t, bl, p, s);

    using Ly = EntLayout<double, W>;
    const int warps = Ly::warps(0);
    const size_t smem = Ly::th + (size_t)warps * Ly::per_warp(0);
    HH_CUDA(cudaFuncSetAttribute(k_far_entries<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t grid_e = std::max<int64_t>(1, std::min<int64_t>(entry_grid(ctx, smem), slot_cap / warps));

    FarArgs A{};
    A.Xs = t->Xs;
    A.Fs = Fs;
    A.Ws = Ws;
    A.PG = bl->PG;
    A.nbeg = t->nbeg;
    A.nend = t->nend;
    A.rank = h->rank;
    A.pivI = h->pivI;
    A.pivJ = h->pivJ;
    A.max_rank = p.max_rank;
    A.mine = mine;
    A.fofs = h->fofs;
    A.cot = cot;
    A.gr = gr;
    A.sums = sums;
    A.th = ctx->theta64;
    A.a = p.radius;
    for (size_t g = 0; g < groups.size(); ++g) {
        A.b0 = groups[g].first;
        A.b1 = groups[g].second;
        A.ent_base = at[g];
        const int64_t n_ent = at[g + 1] - at[g];
        if (rebuild) {
            // the FP64 factors of the group's blocks along the same pivots (the
            // same deterministic rank loop that chose them)
            AcaRun r;
            r.rank = rk;
            r.pivI = pI;
            r.pivJ = pJ;
            r.factors = fac;
            r.fofs = h->fofs;
            r.fofs_base = at[g];
            r.b0 = A.b0;
            r.b1 = A.b1;
            r.mode = 2;
            aca_run(ctx, t, bl, p, r, s);
            A.fac = fac;
            A.fac_base = at[g];
        } else {
            A.fac = (const double*)h->factors;
            A.fac_base = 0;
        }
        const int64_t nb = A.b1 - A.b0;
        k_far_rev<W><<<(unsigned)std::min<int64_t>(nb, (int64_t)ctx->n_sm * 16), REV_T, 0, s>>>(A);
        HH_CHECK_LAUNCH();
        if (n_ent > 0) {
            const int64_t ge = std::max<int64_t>(1, std::min<int64_t>(grid_e, ceil_div(n_ent, 32 * warps)));
            k_far_entries<W><<<(unsigned)ge, 32 * warps, smem, s>>>(A, n_ent, slots, want_theta);
            HH_CHECK_LAUNCH();
            *n_slots = std::max<int64_t>(*n_slots, ge * warps);
        }
        k_far_sums<<<(unsigned)std::min<int64_t>(ceil_div(nb, 8), (int64_t)ctx->n_sm * 8), 256, 0, s>>>(A);
        HH_CHECK_LAUNCH();
        k_far_gather<<<(unsigned)ceil_div(t->n, 256), 256, 0, s>>>(A, t->n, bl->rowG, colG, colorder, t->child,
                                                                  t->d_offsets, t->batch, GXs, GFs);
        HH_CHECK_LAUNCH();
    }
    if (mine) dev_free(mine, s);
    dev_free(colG, s);
    dev_free(colorder, s);
    if (rebuild) {
        dev_free(pJ, s);
        dev_free(pI, s);
        dev_free(rk, s);
        dev_free(fac, s);
    }
    dev_free(sums, s);
    dev_free(gr, s);
    dev_free(cot, s);
}

template <int W>
void backward_all(hh_ctx* ctx, const hh_hmat* h, bool near_fp32, const double* Fs, const double* Ws, double* gX,
                  float* gtheta, double* gFs, cudaStream_t s)
{
    const hh_tree* t = h->tree;
    const hh_params& p = h->params;
    const bool want_theta = gtheta != nullptr;
    const int np = n_params<W>();
    double* GXs = dev_alloc_t<double>(3 * t->n, s);
    HH_CUDA(cudaMemsetAsync(GXs, 0, sizeof(double) * 3 * t->n, s));
    // theta slots: the near kernel's warps, then the far entry kernel's
    const int64_t slot_cap = (int64_t)ctx->n_sm * 8;
    double* slots = nullptr;
    if (want_theta) {
        slots = dev_alloc_t<double>(2 * slot_cap * np, s);
        HH_CUDA(cudaMemsetAsync(slots, 0, sizeof(double) * 2 * slot_cap * np, s));
    }
    double* dummy = slots ? slots : GXs;   // never written when want_theta is false
    int64_t n_near = 0, n_far = 0;
    if (near_fp32) near_rev<float, W>(ctx, t, h->blocks, p, Fs, Ws, GXs, dummy, slot_cap, &n_near, want_theta, s);
    else near_rev<double, W>(ctx, t, h->blocks, p, Fs, Ws, GXs, dummy, slot_cap, &n_near, want_theta, s);
    far_rev<W>(ctx, h, Fs, Ws, GXs, gFs, slots ? slots + slot_cap * np : dummy, slot_cap, &n_far, want_theta, s);
    if (gX) {
        k_gx_out<<<(unsigned)ceil_div(t->n, 256), 256, 0, s>>>(GXs, t->perm, t->n, gX);
        HH_CHECK_LAUNCH();
    }
    if (want_theta) {
        // near slots 0 .. n_near-1 and far slots slot_cap .. slot_cap+n_far-1; the unused ones are zero
        k_theta_reduce<<<(unsigned)ceil_div(np, 256), 256, 0, s>>>(slots, 2 * slot_cap, np, gtheta);
        HH_CHECK_LAUNCH();
        dev_free(slots, s);
    }
    (void)n_near;
    (void)n_far;
    dev_free(GXs, s);
}

}  // namespace

void matvec_backward_xtheta(hh_ctx* ctx, const hh_hmat* h, bool near_fp32, const double* Fs, const double* Ws,
                            double* gX, float* gtheta, double* gFs, cudaStream_t s)
{
    const hh_params& p = h->params;
    HH_REQUIRE(p.kernel == HH_MLP, HH_ERR_ARG, "dL/dX and dL/dtheta need the MLP kernel");
    HH_REQUIRE(p.max_rank <= BWD_MAXL, HH_ERR_ARG, "max_rank too large for the adjoint");
    HH_REQUIRE(h->real_bytes == 8, HH_ERR_ARG, "the adjoint needs FP64 factors");
    if (ctx->width == 32) backward_all<32>(ctx, h, near_fp32, Fs, Ws, gX, gtheta, gFs, s);
    else backward_all<64>(ctx, h, near_fp32, Fs, Ws, gX, gtheta, gFs, s);
}
