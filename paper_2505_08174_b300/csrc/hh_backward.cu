// hh_backward.cu -- adjoint of the H-matrix mobility product (hh_matvec_backward).
//
// L = sum_i w_i . U_i with U = alpha_1 F + M_H F, tree / partition / ACA pivots
// frozen.  dL/dF = alpha_1 w + M_H^T w is the transposed product (hh_matvec).
// dL/dX and dL/dtheta come from every pair-kernel entry the product uses:
//
//  * inadmissible block (tau, sigma), pair (m, n), m != n: the entry
//    K(x_m - x_n) with cotangent w_m F_n^T;
//  * admissible block: reverse-mode differentiation of the rank loop of
//    Algorithm 2 with the pivots frozen (see k_far_bwd), which yields a
//    cotangent for every entry G(m, j_k) and G(i_k, n) the ACA evaluated.
//
// For one entry K(r) = S(o(f(r))) / |r|, f = [r/|r|, a/|r|], cotangent G:
//   dL/do = [G00, G11, G22, G01+G10, G02+G20, G12+G21] / |r|,
//   reverse pass through the MLP -> dL/df and the layer cotangents,
//   dL/dr = -<G, S> r / |r|^3 + (I - r r^T/|r|^2) dL/df[0:3] / |r|
//           - a r / |r|^3 dL/df[3],
//   dL/dx_target += dL/dr, dL/dx_source -= dL/dr (FP64 atomics);
//   dL/dtheta: layer weights get sum over entries of (cotangent of the layer
//   output) x (layer input), accumulated per warp from 32 staged entries at a
//   time (each lane owns a disjoint set of parameters), then added to the
//   global gradient.
// Activations are recomputed, never stored between the forward and adjoint.
#include <algorithm>

#include "hh_internal.h"

namespace {

constexpr int BWD_MAXL = 64;

template <typename R, int W>
struct Rec {  // per-entry record of one lane
    static constexpr int F = 0, Z1 = 4, Z2 = 4 + W, Z3 = 4 + 2 * W, H1 = 4 + 3 * W, H2 = 4 + 4 * W, H3 = 4 + 5 * W,
                         G1 = 4 + 6 * W, G2 = 4 + 7 * W, G3 = 4 + 8 * W, GO = 4 + 9 * W, SIZE = 4 + 9 * W + 6;
};

template <typename R> __device__ __forceinline__ R sig_(R x);
template <> __device__ __forceinline__ double sig_<double>(double x) { return 1.0 / (1.0 + exp(-x)); }

template <int W>
__host__ __device__ constexpr int n_params() { return 4 * W + W + 2 * (W * W + W) + 6 * W + 6; }

// Forward + reverse pass of one entry.  rec: this lane's record (shared).
// Returns dL/dr in gr.  valid == false writes a zero record (no gradient).
template <typename R, int W>
__device__ void entry_backward(const R* __restrict__ th, R a, R rx, R ry, R rz, const R* Gc, bool valid, R* rec, R gr[3])
{
    using L = Rec<R, W>;
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
        R t = b1[j];
        for (int i = 0; i < 4; ++i) t += W1[4 * j + i] * f[i];
        rec[L::Z1 + j] = t;
        rec[L::H1 + j] = silu<R>(t);
    }
    for (int j = 0; j < W; ++j) {
        R t = b2[j];
        for (int i = 0; i < W; ++i) t += W2[W * j + i] * rec[L::H1 + i];
        rec[L::Z2 + j] = t;
        rec[L::H2 + j] = silu<R>(t);
    }
    for (int j = 0; j < W; ++j) {
        R t = b3[j];
        for (int i = 0; i < W; ++i) t += W3[W * j + i] * rec[L::H2 + i];
        rec[L::Z3 + j] = t;
        rec[L::H3 + j] = silu<R>(t);
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
        const R z = rec[L::Z3 + i], sg = sig_<R>(z);
        rec[L::G3 + i] = t * sg * (1 + z * (1 - sg));
    }
    for (int i = 0; i < W; ++i) {
        R t = 0;
        for (int j = 0; j < W; ++j) t += W3[W * j + i] * rec[L::G3 + j];
        const R z = rec[L::Z2 + i], sg = sig_<R>(z);
        rec[L::G2 + i] = t * sg * (1 + z * (1 - sg));
    }
    for (int i = 0; i < W; ++i) {
        R t = 0;
        for (int j = 0; j < W; ++j) t += W2[W * j + i] * rec[L::G2 + j];
        const R z = rec[L::Z1 + i], sg = sig_<R>(z);
        rec[L::G1 + i] = t * sg * (1 + z * (1 - sg));
    }
    R gf[4];
    for (int i = 0; i < 4; ++i) {
        R t = 0;
        for (int j = 0; j < W; ++j) t += W1[4 * j + i] * rec[L::G1 + j];
        gf[i] = t;
    }
    const R rg = (rx * gf[0] + ry * gf[1] + rz * gf[2]) * id;
    const R r3[3] = {rx, ry, rz};
    for (int q = 0; q < 3; ++q)
        gr[q] = -gs * id * r3[q] * id * id + (gf[q] - rg * r3[q] * id) * id - a * r3[q] * id * id * id * gf[3];
}

// Parameter cotangents of the 32 staged records added into acc (shared,
// packed parameter layout).  Each lane owns parameters x = lane, lane+32, ...
template <typename R, int W>
__device__ void accumulate_theta(const R* recs, R* acc)
{
    using L = Rec<R, W>;
    const int lane = threadIdx.x & 31;
    constexpr int dims[5] = {4, W, W, W, 6};
    constexpr int hin[4] = {L::F, L::H1, L::H2, L::H3};
    constexpr int gout[4] = {L::G1, L::G2, L::G3, L::GO};
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
            acc[base + x] += s;
        }
        base += nl;
    }
}

// The parameter-gradient accumulator of a CTA lives in shared memory when it
// fits beside the parameters and the 32 records (W = 32), else in a per-CTA
// slice of global scratch (W = 64 in FP64); lanes own disjoint parameters, so
// either form is updated without atomics.
template <typename R, int W>
__host__ __device__ constexpr bool acc_in_smem()
{
    return sizeof(R) * (2 * n_params<W>() + 32 * Rec<R, W>::SIZE) + 4096 <= 227 * 1024;
}

template <typename R, int W>
struct BwdSmem {
    R th[n_params<W>()];
    R recs[32 * Rec<R, W>::SIZE];
    R acc_s[acc_in_smem<R, W>() ? n_params<W>() : 1];
    R* acc;
};

// One batch of up to 32 entries (one per lane): records, dL/dX atomics, theta staging.
template <typename R, int W>
__device__ void entry_batch(BwdSmem<R, W>& sm, R a, const double* __restrict__ Xs, int64_t ti, int64_t si,
                            const R* Gc, bool valid, const int32_t* __restrict__ perm, double* gX, bool want_theta)
{
    const int lane = threadIdx.x & 31;
    R rx = 0, ry = 0, rz = 1, gr[3];
    if (valid) sep<R>(Xs, ti, si, rx, ry, rz);
    entry_backward<R, W>(sm.th, a, rx, ry, rz, Gc, valid, sm.recs + lane * Rec<R, W>::SIZE, gr);
    if (valid && gX) {
        const int64_t pt = perm[ti], ps = perm[si];
        for (int q = 0; q < 3; ++q) {
            atomicAdd(&gX[3 * pt + q], (double)gr[q]);
            atomicAdd(&gX[3 * ps + q], -(double)gr[q]);
        }
    }
    __syncwarp();
    if (want_theta) accumulate_theta<R, W>(sm.recs, sm.acc);
    __syncwarp();
}

template <typename R, int W>
__device__ void bwd_setup(BwdSmem<R, W>& sm, const R* th_g, R* gacc)
{
    if (threadIdx.x == 0) sm.acc = acc_in_smem<R, W>() ? sm.acc_s : gacc + (int64_t)blockIdx.x * n_params<W>();
    __syncwarp();
    for (int i = threadIdx.x; i < n_params<W>(); i += blockDim.x) { sm.th[i] = th_g[i]; sm.acc[i] = 0; }
    __syncwarp();
}

template <typename R, int W>
__device__ void bwd_flush_theta(BwdSmem<R, W>& sm, double* gth)
{
    __syncwarp();
    if (gth)
        for (int i = threadIdx.x; i < n_params<W>(); i += blockDim.x)
            if (sm.acc[i] != (R)0) atomicAdd(&gth[i], (double)sm.acc[i]);
}

// ---- inadmissible blocks ------------------------------------------------------
template <typename R, int W>
__global__ void __launch_bounds__(32) k_near_bwd(const double* __restrict__ Xs, const double* __restrict__ Fs,
                                                 const double* __restrict__ Ws, const int32_t* __restrict__ PH,
                                                 const int64_t* __restrict__ rowH, const int32_t* __restrict__ work,
                                                 int64_t n_work, const int32_t* __restrict__ nbeg,
                                                 const int32_t* __restrict__ nend, const R* __restrict__ th_g, R a,
                                                 const int32_t* __restrict__ perm, double* gX, double* gth, R* gacc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem<R, W>& sm = *reinterpret_cast<BwdSmem<R, W>*>(smem_raw);
    bwd_setup<R, W>(sm, th_g, gacc);
    const int lane = threadIdx.x & 31;
    for (int64_t w = blockIdx.x; w < n_work; w += gridDim.x) {
        const int32_t tau = work[w];
        const int32_t t0 = nbeg[tau], c = nend[tau] - t0;
        for (int64_t bb = rowH[tau]; bb < rowH[tau + 1]; ++bb) {
            const int32_t sg = PH[2 * bb + 1];
            const int32_t s0 = nbeg[sg], q = nend[sg] - s0;
            const int64_t P = (int64_t)c * q;
            for (int64_t p0 = 0; p0 < P; p0 += 32) {
                const int64_t p = p0 + lane;
                bool valid = p < P;
                int64_t ti = 0, si = 0;
                R Gc[9];
                if (valid) {
                    ti = t0 + p / q;
                    si = s0 + p % q;
                    valid = ti != si;
                }
                if (valid) {
                    const double* wm = Ws + 3 * ti;
                    const double* fn = Fs + 3 * si;
                    for (int u = 0; u < 3; ++u)
                        for (int v = 0; v < 3; ++v) Gc[3 * u + v] = (R)(wm[u] * fn[v]);
                }
                entry_batch<R, W>(sm, a, Xs, ti, si, Gc, valid, perm, gX, gth != nullptr);
            }
        }
    }
    bwd_flush_theta<R, W>(sm, gth);
}

// ---- admissible blocks ----------------------------------------------------------
// Forward pair kernel with the packed parameters (shared) for the y / z sweeps.
template <typename R, int W>
__device__ void entry_forward(const R* __restrict__ th, R a, R rx, R ry, R rz, R K[9])
{
    const R* W1 = th;
    const R* b1 = W1 + 4 * W;
    const R* W2 = b1 + W;
    const R* b2 = W2 + W * W;
    const R* W3 = b2 + W;
    const R* b3 = W3 + W * W;
    const R* W4 = b3 + W;
    const R* b4 = W4 + 6 * W;
    const R id = rsqrt_<R>(rx * rx + ry * ry + rz * rz);
    R f[4] = {rx * id, ry * id, rz * id, a * id}, h[W], g[W], o[6];
    for (int j = 0; j < W; ++j) {
        R t = b1[j];
        for (int i = 0; i < 4; ++i) t += W1[4 * j + i] * f[i];
        h[j] = silu<R>(t);
    }
    for (int j = 0; j < W; ++j) {
        R t = b2[j];
        for (int i = 0; i < W; ++i) t += W2[W * j + i] * h[i];
        g[j] = silu<R>(t);
    }
    for (int j = 0; j < W; ++j) {
        R t = b3[j];
        for (int i = 0; i < W; ++i) t += W3[W * j + i] * g[i];
        h[j] = silu<R>(t);
    }
    for (int j = 0; j < 6; ++j) {
        R t = b4[j];
        for (int i = 0; i < W; ++i) t += W4[W * j + i] * h[i];
        o[j] = t;
    }
    K[0] = o[0] * id; K[1] = o[3] * id; K[2] = o[4] * id;
    K[3] = o[3] * id; K[4] = o[1] * id; K[5] = o[5] * id;
    K[6] = o[4] * id; K[7] = o[5] * id; K[8] = o[2] * id;
}

// Reverse-mode differentiation of Algorithm 2 on one admissible block, with
// the pivots frozen.  Forward (per step k, 3x3 elements):
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
// (recomputed from the stored factors and one pair-kernel entry, FP64), so
// the adjoint is as well conditioned as the forward recursion.
template <typename R>
__device__ __forceinline__ void acc_abt(R* acc, const R* A, const R* B)   // acc += A B^T
{
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v) acc[3 * u + v] += A[3 * u] * B[3 * v] + A[3 * u + 1] * B[3 * v + 1] + A[3 * u + 2] * B[3 * v + 2];
}
template <typename R>
__device__ __forceinline__ void acc_atb(R* acc, const R* A, const R* B)   // acc += A^T B
{
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v) acc[3 * u + v] += A[u] * B[v] + A[3 + u] * B[3 + v] + A[6 + u] * B[6 + v];
}

template <typename R>
__device__ __forceinline__ void ld9g(const R* base, int64_t ld, int64_t x, R* v)
{
#pragma unroll
    for (int e = 0; e < 9; ++e) v[e] = base[e * ld + x];
}
template <typename R>
__device__ __forceinline__ void st9g(R* base, int64_t ld, int64_t x, const R* v)
{
#pragma unroll
    for (int e = 0; e < 9; ++e) base[e * ld + x] = v[e];
}

// Factors of one admissible block rebuilt along its frozen pivots (the
// H-matrix was built with HH_FLAG_PIVOTS_ONLY): the recursion of Algorithm 2
// without the pivot search.  C [l][9][c], then Q [l][9][q].
template <typename R, int W>
__device__ void refactor(const R* th, R a, const double* __restrict__ Xs, int32_t t0, int32_t c, int32_t s0,
                         int32_t q, const int32_t* I, const int32_t* J, int l, R* C, R* Pi)
{
    const int lane = threadIdx.x & 31;
    R* Q = C + (int64_t)l * 9 * c;
    for (int k = 0; k < l; ++k) {
        const int ik = I[k], jk = J[k];
        R* Ck = C + (int64_t)k * 9 * c;
        R* Qk = Q + (int64_t)k * 9 * q;
        for (int m = lane; m < c; m += 32) {
            R rx, ry, rz, K[9];
            sep<R>(Xs, t0 + m, s0 + jk, rx, ry, rz);
            entry_forward<R, W>(th, a, rx, ry, rz, K);
            for (int p = 0; p < k; ++p) {
                R cp[9], qp[9], t9[9];
                ld9g(C + (int64_t)p * 9 * c, c, m, cp);
                ld9g(Q + (int64_t)p * 9 * q, q, jk, qp);
                mm3(cp, qp, t9);
                for (int e = 0; e < 9; ++e) K[e] -= t9[e];
            }
            st9g(Ck, c, m, K);
        }
        __syncwarp();
        if (lane == 0) {
            double P[9], Pd[9];
            for (int e = 0; e < 9; ++e) P[e] = (double)Ck[(int64_t)e * c + ik];
            inv3d(P, Pd);
            for (int e = 0; e < 9; ++e) Pi[e] = (R)Pd[e];
        }
        __syncwarp();
        for (int m = lane; m < c; m += 32) {
            R v[9], o[9];
            ld9g(Ck, c, m, v);
            mm3(v, Pi, o);
            st9g(Ck, c, m, o);
        }
        __syncwarp();
        for (int n = lane; n < q; n += 32) {
            R rx, ry, rz, K[9];
            sep<R>(Xs, t0 + ik, s0 + n, rx, ry, rz);
            entry_forward<R, W>(th, a, rx, ry, rz, K);
            for (int p = 0; p < k; ++p) {
                R cp[9], qp[9], t9[9];
                ld9g(C + (int64_t)p * 9 * c, c, ik, cp);
                ld9g(Q + (int64_t)p * 9 * q, q, n, qp);
                mm3(cp, qp, t9);
                for (int e = 0; e < 9; ++e) K[e] -= t9[e];
            }
            st9g(Qk, q, n, K);
        }
        __syncwarp();
    }
}

template <typename R, int W>
__global__ void __launch_bounds__(32) k_far_bwd(const double* __restrict__ Xs, const double* __restrict__ Fs,
                                                const double* __restrict__ Ws, const int32_t* __restrict__ PG,
                                                int64_t nG, const int32_t* __restrict__ nbeg,
                                                const int32_t* __restrict__ nend, const int32_t* __restrict__ rank,
                                                const int32_t* __restrict__ pivI, const int32_t* __restrict__ pivJ,
                                                int max_rank, const uint8_t* __restrict__ mine, const R* __restrict__ fac,
                                                const int64_t* __restrict__ fofs, const R* __restrict__ th_g, R a,
                                                R* __restrict__ scratch, int64_t ws_stride,
                                                const int32_t* __restrict__ perm, double* gX, double* gth, R* gacc,
                                                double* gFs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem<R, W>& sm = *reinterpret_cast<BwdSmem<R, W>*>(smem_raw);
    __shared__ R tv[BWD_MAXL * 3], sv[BWD_MAXL * 3], piT[9];
    bwd_setup<R, W>(sm, th_g, gacc);
    const int lane = threadIdx.x & 31;
    R* Cb = scratch + (int64_t)blockIdx.x * ws_stride;
    R* Cw = Cb + ws_stride / 2;   // rebuilt factors when the H-matrix holds pivots only
    for (int64_t b = blockIdx.x; b < nG; b += gridDim.x) {
        if (mine && !mine[b]) continue;
        const int l = rank[b];
        if (l <= 0) continue;
        const int32_t t = PG[2 * b], s = PG[2 * b + 1];
        const int32_t t0 = nbeg[t], c = nend[t] - t0, s0 = nbeg[s], q = nend[s] - s0;
        const int32_t* I = pivI + b * max_rank;
        const int32_t* J = pivJ + b * max_rank;
        if (!fac) refactor<R, W>(sm.th, a, Xs, t0, c, s0, q, I, J, l, Cw, piT);
        const R* C = fac ? fac + 9 * fofs[b] : Cw;
        const R* Q = C + (int64_t)l * 9 * c;
        R* Qb = Cb + (int64_t)l * 9 * c;
        auto Ck = [&](int k) { return C + (int64_t)k * 9 * c; };
        auto Qk = [&](int k) { return Q + (int64_t)k * 9 * q; };
        auto Cbk = [&](int k) { return Cb + (int64_t)k * 9 * c; };
        auto Qbk = [&](int k) { return Qb + (int64_t)k * 9 * q; };
        // t_k = sum_n Q_k(n) F_n,  s_k = sum_m C_k(m)^T w_m
        for (int k = 0; k < l; ++k) {
            R at[3] = {0, 0, 0}, as[3] = {0, 0, 0};
            for (int n = lane; n < q; n += 32) {
                R v[9];
                ld9g(Qk(k), q, n, v);
                const double* f = Fs + 3 * (int64_t)(s0 + n);
                for (int u = 0; u < 3; ++u) at[u] += v[3 * u] * (R)f[0] + v[3 * u + 1] * (R)f[1] + v[3 * u + 2] * (R)f[2];
            }
            for (int m = lane; m < c; m += 32) {
                R v[9];
                ld9g(Ck(k), c, m, v);
                const double* w = Ws + 3 * (int64_t)(t0 + m);
                for (int u = 0; u < 3; ++u) as[u] += v[u] * (R)w[0] + v[3 + u] * (R)w[1] + v[6 + u] * (R)w[2];
            }
            for (int u = 0; u < 3; ++u) {
                const R x = warp_sum(at[u]), y = warp_sum(as[u]);
                if (lane == 0) { tv[3 * k + u] = x; sv[3 * k + u] = y; }
            }
        }
        __syncwarp();
        if (gFs) {
            // far part of dL/dF: (C Q)^T w restricted to this block's sources
            for (int n = lane; n < q; n += 32) {
                R g[3] = {0, 0, 0};
                for (int k = 0; k < l; ++k) {
                    R v[9];
                    ld9g(Qk(k), q, n, v);
                    const R* sk = sv + 3 * k;
                    for (int u = 0; u < 3; ++u) g[u] += v[u] * sk[0] + v[3 + u] * sk[1] + v[6 + u] * sk[2];
                }
                double* out = gFs + 3 * (int64_t)(s0 + n);
                for (int u = 0; u < 3; ++u) atomicAdd(&out[u], (double)g[u]);
            }
        }
        for (int k = 0; k < l; ++k) {
            for (int m = lane; m < c; m += 32) {
                const double* w = Ws + 3 * (int64_t)(t0 + m);
                R v[9];
                for (int u = 0; u < 3; ++u)
                    for (int x = 0; x < 3; ++x) v[3 * u + x] = (R)w[u] * tv[3 * k + x];
                st9g(Cbk(k), c, m, v);
            }
            for (int n = lane; n < q; n += 32) {
                const double* f = Fs + 3 * (int64_t)(s0 + n);
                R v[9];
                for (int u = 0; u < 3; ++u)
                    for (int x = 0; x < 3; ++x) v[3 * u + x] = sv[3 * k + u] * (R)f[x];
                st9g(Qbk(k), q, n, v);
            }
        }
        __syncwarp();
        for (int k = l - 1; k >= 0; --k) {
            const int ik = I[k], jk = J[k];
            // row k
            for (int p = 0; p < k; ++p) {
                R cpi[9], acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                ld9g(Ck(p), c, ik, cpi);
                for (int n = lane; n < q; n += 32) {
                    R qb[9], qp[9], up[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, cur[9];
                    ld9g(Qbk(k), q, n, qb);
                    ld9g(Qk(p), q, n, qp);
                    acc_abt(acc, qb, qp);
                    acc_atb(up, cpi, qb);
                    ld9g(Qbk(p), q, n, cur);
                    for (int e = 0; e < 9; ++e) cur[e] -= up[e];
                    st9g(Qbk(p), q, n, cur);
                }
                for (int e = 0; e < 9; ++e) acc[e] = warp_sum(acc[e]);
                if (lane == 0) {
                    R cur[9];
                    ld9g(Cbk(p), c, ik, cur);
                    for (int e = 0; e < 9; ++e) cur[e] -= acc[e];
                    st9g(Cbk(p), c, ik, cur);
                }
                __syncwarp();
            }
            // pivot block P_k = G(i_k, j_k) - sum_{p<k} C_p(i_k) Q_p(j_k), inverse-transpose in FP64
            if (lane == 0) {
                R rx, ry, rz, K[9];
                sep<R>(Xs, t0 + ik, s0 + jk, rx, ry, rz);
                entry_forward<R, W>(sm.th, a, rx, ry, rz, K);
                double P[9], Pi[9];
                for (int e = 0; e < 9; ++e) P[e] = (double)K[e];
                for (int p = 0; p < k; ++p) {
                    R cp[9], qp[9], t9[9];
                    ld9g(Ck(p), c, ik, cp);
                    ld9g(Qk(p), q, jk, qp);
                    mm3(cp, qp, t9);
                    for (int e = 0; e < 9; ++e) P[e] -= (double)t9[e];
                }
                inv3d(P, Pi);
                for (int u = 0; u < 3; ++u)
                    for (int v = 0; v < 3; ++v) piT[3 * u + v] = (R)Pi[3 * v + u];
            }
            __syncwarp();
            // scaling: chat-bar_k = Cb_k P^-T;  r1 = sum_m C_k(m)^T Cb_k(m)
            R r1[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int m = lane; m < c; m += 32) {
                R cb[9], ck[9], o[9];
                ld9g(Cbk(k), c, m, cb);
                ld9g(Ck(k), c, m, ck);
                acc_atb(r1, ck, cb);
                mm3(cb, piT, o);
                st9g(Cbk(k), c, m, o);
            }
            for (int e = 0; e < 9; ++e) r1[e] = warp_sum(r1[e]);
            __syncwarp();
            if (lane == 0) {
                R dP[9], cur[9];
                mm3(r1, piT, dP);
                ld9g(Cbk(k), c, ik, cur);
                for (int e = 0; e < 9; ++e) cur[e] -= dP[e];
                st9g(Cbk(k), c, ik, cur);
            }
            __syncwarp();
            // column k
            for (int p = 0; p < k; ++p) {
                R qpj[9], acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                ld9g(Qk(p), q, jk, qpj);
                for (int m = lane; m < c; m += 32) {
                    R cb[9], cp[9], up[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, cur[9];
                    ld9g(Cbk(k), c, m, cb);
                    ld9g(Ck(p), c, m, cp);
                    acc_atb(acc, cp, cb);
                    acc_abt(up, cb, qpj);
                    ld9g(Cbk(p), c, m, cur);
                    for (int e = 0; e < 9; ++e) cur[e] -= up[e];
                    st9g(Cbk(p), c, m, cur);
                }
                for (int e = 0; e < 9; ++e) acc[e] = warp_sum(acc[e]);
                if (lane == 0) {
                    R cur[9];
                    ld9g(Qbk(p), q, jk, cur);
                    for (int e = 0; e < 9; ++e) cur[e] -= acc[e];
                    st9g(Qbk(p), q, jk, cur);
                }
                __syncwarp();
            }
        }
        // entry cotangents -> pair-kernel reverse passes
        const int64_t nCol = (int64_t)c * l, nAll = (int64_t)(c + q) * l;
        for (int64_t e0 = 0; e0 < nAll; e0 += 32) {
            const int64_t e = e0 + lane;
            const bool valid = e < nAll;
            int64_t ti = 0, si = 0;
            R Gc[9];
            if (valid) {
                if (e < nCol) {
                    const int k = (int)(e / c), m = (int)(e % c);
                    ti = t0 + m; si = s0 + J[k];
                    ld9g(Cbk(k), c, m, Gc);
                } else {
                    const int64_t x = e - nCol;
                    const int k = (int)(x / q), n = (int)(x % q);
                    ti = t0 + I[k]; si = s0 + n;
                    ld9g(Qbk(k), q, n, Gc);
                }
            }
            entry_batch<R, W>(sm, a, Xs, ti, si, Gc, valid, perm, gX, gth != nullptr);
        }
        __syncwarp();
    }
    bwd_flush_theta<R, W>(sm, gth);
}

__global__ void k_max_cq(const int32_t* __restrict__ PG, int64_t nG, const int32_t* __restrict__ nbeg,
                         const int32_t* __restrict__ nend, int* out)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nG) atomicMax(out, nend[PG[2 * b]] - nbeg[PG[2 * b]] + nend[PG[2 * b + 1]] - nbeg[PG[2 * b + 1]]);
}

__global__ void k_theta_out(const double* __restrict__ in, float* __restrict__ out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += (float)in[i];
}

__global__ void k_leafs(const int32_t* __restrict__ child, int32_t n, const uint8_t* __restrict__ mine, int32_t* out,
                        int* count)
{
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n && child[2 * t] < 0 && (mine == nullptr || mine[t])) out[atomicAdd(count, 1)] = t;
}

template <typename R, int W>
void launch_bwd(hh_ctx* ctx, const hh_hmat* h, const double* Fs, const double* Ws, double* gX, double* gth,
                double* gFs, cudaStream_t s)
{
    const hh_tree* t = h->tree;
    const hh_blocks* b = h->blocks;
    const hh_params& p = h->params;
    static_assert(sizeof(R) == 8, "the adjoint runs in FP64");
    const R* th = ctx->theta64;
    const int64_t max_grid = (int64_t)ctx->n_sm * 8;
    const size_t smem = sizeof(BwdSmem<R, W>);
    HH_REQUIRE(smem <= 227 * 1024, HH_ERR_ARG, "adjoint: shared memory per warp exceeds the limit");
    R* gacc = acc_in_smem<R, W>() ? nullptr : dev_alloc_t<R>(max_grid * n_params<W>(), s);
    // near field: all leaves of this shard (order irrelevant: FP64 atomics)
    int32_t* leaves = dev_alloc_t<int32_t>(t->n_nodes, s);
    int* cnt = dev_alloc_t<int>(1, s);
    HH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), s));
    uint8_t* node_mine = shard_node_flags(t, b, p, s);
    k_leafs<<<(unsigned)ceil_div(t->n_nodes, 256), 256, 0, s>>>(t->child, t->n_nodes, node_mine, leaves, cnt);
    HH_CHECK_LAUNCH();
    if (node_mine) dev_free(node_mine, s);
    int n_leaves = 0;
    HH_CUDA(cudaMemcpyAsync(&n_leaves, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
    HH_CUDA(cudaStreamSynchronize(s));
    HH_CUDA(cudaFuncSetAttribute(k_near_bwd<R, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    HH_CUDA(cudaFuncSetAttribute(k_far_bwd<R, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (n_leaves > 0) {
        const int grid = (int)std::min<int64_t>(n_leaves, max_grid);
        k_near_bwd<R, W><<<grid, 32, smem, s>>>(t->Xs, Fs, Ws, b->PH, b->rowH, leaves, n_leaves, t->nbeg, t->nend, th,
                                                (R)p.radius, t->perm, gX, gth, gacc);
        HH_CHECK_LAUNCH();
    }
    if (b->nG > 0) {
        int* dmax = dev_alloc_t<int>(1, s);
        HH_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), s));
        k_max_cq<<<(unsigned)ceil_div(b->nG, 256), 256, 0, s>>>(b->PG, b->nG, t->nbeg, t->nend, dmax);
        HH_CHECK_LAUNCH();
        int max_cq = 0;
        HH_CUDA(cudaMemcpyAsync(&max_cq, dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
        HH_CUDA(cudaStreamSynchronize(s));
        dev_free(dmax, s);
        // Cb and Qb of one block, and the rebuilt factors when h holds pivots only
        const int64_t stride = (int64_t)max_cq * 9 * p.max_rank * (h->factors ? 1 : 2);
        const int64_t budget = (int64_t)16 << 30;
        int64_t grid = std::min<int64_t>(b->nG, max_grid);
        grid = std::max<int64_t>(1, std::min<int64_t>(grid, budget / (stride * (int64_t)sizeof(R))));
        R* scratch = dev_alloc_t<R>(grid * stride, s);
        uint8_t* mine = shard_block_flags(t, b, p, s);
        k_far_bwd<R, W><<<(unsigned)grid, 32, smem, s>>>(t->Xs, Fs, Ws, b->PG, b->nG, t->nbeg, t->nend, h->rank,
                                                        h->pivI, h->pivJ, p.max_rank, mine,
                                                        (const R*)h->factors, h->fofs, th, (R)p.radius, scratch,
                                                        stride, t->perm, gX, gth, gacc, gFs);
        HH_CHECK_LAUNCH();
        if (mine) dev_free(mine, s);
        dev_free(scratch, s);
    }
    dev_free(leaves, s);
    dev_free(cnt, s);
    if (gacc) dev_free(gacc, s);
}

}  // namespace

// dL/dX (accumulated into gX, caller order) and dL/dtheta (accumulated into
// gtheta, float32) for L = sum w . (M_H F); Fs and Ws in sorted order.
void matvec_backward_xtheta(hh_ctx* ctx, const hh_hmat* h, const double* Fs, const double* Ws, double* gX,
                            float* gtheta, double* gFs, cudaStream_t s)
{
    const hh_params& p = h->params;
    HH_REQUIRE(p.kernel == HH_MLP, HH_ERR_ARG, "dL/dX and dL/dtheta need the MLP kernel");
    HH_REQUIRE(p.max_rank <= BWD_MAXL, HH_ERR_ARG, "max_rank too large for the adjoint");
    HH_REQUIRE(h->real_bytes == 8, HH_ERR_ARG, "the adjoint needs FP64 factors");
    double* gth = nullptr;
    if (gtheta) {
        gth = dev_alloc_t<double>(ctx->n_theta, s);
        HH_CUDA(cudaMemsetAsync(gth, 0, sizeof(double) * ctx->n_theta, s));
    }
    // The adjoint runs in FP64 on FP64 factors (the caller re-approximates a
    // narrower H-matrix in FP64): the cotangents of the rank loop cancel only
    // to the working rounding times the squared condition number of the 3x3
    // pivot blocks.
    if (ctx->width == 32) launch_bwd<double, 32>(ctx, h, Fs, Ws, gX, gth, gFs, s);
    else launch_bwd<double, 64>(ctx, h, Fs, Ws, gX, gth, gFs, s);
    if (gtheta) {
        k_theta_out<<<(unsigned)ceil_div(ctx->n_theta, 256), 256, 0, s>>>(gth, gtheta, ctx->n_theta);
        HH_CHECK_LAUNCH();
        dev_free(gth, s);
    }
}
