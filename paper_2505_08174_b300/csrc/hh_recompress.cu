// hh_recompress.cu -- recompression of the stored ACA factors of every
// admissible block by a truncated singular value decomposition, and the
// low-rank apply from the recompressed factors.
//
// A block's ACA approximant in scalar form is M = C Q with C = [C_0 .. C_{l-1}]
// (3c x 3l; column 3k + v of C holds the entries C_k(m)[u][v] at row 3m + u)
// and Q (3l x 3q; row 3k + v holds Q_k(n)[v][w] at column 3n + w).  Its
// scalar rank is at most 3l; the ACA's 3x3 steps usually overshoot it.  The
// columns of C and rows of Q are first scaled to unit norm, C = C^ D_a,
// Q = D_b Q^ (the terms' sizes decay over the rank loop; scaled, the Grams'
// conditioning reflects only the angles between terms).  With the Gram
// matrices C^T^ C^ = V_C L_C V_C^T and Q^ Q^^T = V_Q L_Q V_Q^T (symmetric
// eigendecompositions, cyclic Jacobi with the round-robin pair order, FP64),
// C^ = U_C L_C^(1/2) V_C^T and Q^ = V_Q L_Q^(1/2) U_Q^T with orthonormal
// U_C, U_Q, so M = U_C K U_Q^T for the small core
//   K = L_C^(1/2) V_C^T D_a D_b V_Q L_Q^(1/2)  (3l x 3l),
// whose singular values are M's.  K^T K = Y S^2 Y^T (Jacobi again) gives them
// in decreasing order; the kept rank r is the smallest with
//   sum_{i >= r} s_i^2 <= eps_rc^2 sum_i s_i^2,
// i.e. ||M - M_r||_F <= eps_rc ||M||_F (Eckart-Young), and
//   U = C D_a^-1 V_C L_C^(-1/2) K Y_r   (3c x r, column i = s_i u_i),
//   V = Y_r^T L_Q^(-1/2) V_Q^T D_b^-1 Q (r x 3q, orthonormal rows),
// so U V = M_r.  Gram eigenvalues below 1e-15 of the largest (singular
// values below ~3e-8 of the largest, the Gram's resolution in FP64) are
// treated as zero.  Stored: per block U as [r][3c], then V as [r][3q], in the
// H-matrix's real type.
#include <algorithm>

#include "hh_internal.h"

namespace {

constexpr int RC_T = 256;            // threads of one block's recompression
constexpr int RC_NMAX = 3 * 64;      // 3 x the largest supported rank

struct RcArgs {
    const int32_t* PG;
    const int32_t* nbeg;
    const int32_t* nend;
    const int32_t* rank;
    const int64_t* fofs;
    const void* fac;       // C [l][9][c] then Q [l][9][q] at 9 fofs[b]
    int real_bytes;
    int64_t nG;
    double eps2;
    double* scratch;       // per CTA: 6 matrices of RC_NMAX^2
    int32_t* srank;        // out: kept rank
    const int64_t* sofs;   // pass 2: offsets of the recompressed factors (reals)
    void* sfac;            // pass 2: U [r][3c] then V [r][3q]
};

template <typename R>
__device__ __forceinline__ double ldf(const void* p, int64_t i) { return (double)((const R*)p)[i]; }

__device__ __forceinline__ double fac_at(const RcArgs& A, int64_t i)
{
    return A.real_bytes == 8 ? ldf<double>(A.fac, i) : ldf<float>(A.fac, i);
}

// Sum of v over the CTA in a fixed order; every thread receives it.
__device__ double cta_sum1(double v, double* red)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    v = warp_sum(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < RC_T / 32; ++w) s += red[w];
        red[RC_T / 32] = s;
    }
    __syncthreads();
    const double r = red[RC_T / 32];
    __syncthreads();
    return r;
}

// Eigendecomposition of the symmetric n x n matrix A (row-major, modified in
// place: its diagonal ends as the eigenvalues) by cyclic Jacobi rotations,
// n/2 disjoint pairs at a time in the round-robin (circle) order; V (n x n)
// receives the eigenvectors as columns.  Stops when the off-diagonal part is
// below 1e-15 of the matrix's Frobenius norm, or after 40 sweeps.
__device__ void cta_jacobi(double* A, double* V, int n, int* pp, int* pq, double* pc, double* ps, double* red)
{
    const int tid = threadIdx.x;
    for (int i = tid; i < n * n; i += RC_T) V[i] = (i / n == i % n) ? 1.0 : 0.0;
    const int m = n + (n & 1);   // an even number of players: index n is a dummy when n is odd
    const int np = m / 2;
    __syncthreads();
    for (int sweep = 0; sweep < 40; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = tid; i < n * n; i += RC_T) {
            const double a = A[i];
            tot += a * a;
            if (i / n != i % n) off += a * a;
        }
        off = cta_sum1(off, red);
        tot = cta_sum1(tot, red);
        if (!(off > 1e-30 * tot)) break;
        for (int r = 0; r < m - 1; ++r) {
            for (int i = tid; i < np; i += RC_T) {
                int p, q;
                if (i == 0) { p = m - 1; q = r; }
                else { p = (r + i) % (m - 1); q = (r - i + (m - 1)) % (m - 1); }
                if (p > q) { const int x = p; p = q; q = x; }
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double apq = A[p * n + q];
                    if (apq != 0.0) {
                        const double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                pp[i] = p; pq[i] = q; pc[i] = c; ps[i] = s;
            }
            __syncthreads();
            for (int x = tid; x < np * n; x += RC_T) {   // rows p, q <- J^T A
                const int i = x / n, j = x % n, p = pp[i], q = pq[i];
                if (q >= n) continue;
                const double c = pc[i], s = ps[i], ap = A[p * n + j], aq = A[q * n + j];
                A[p * n + j] = c * ap - s * aq;
                A[q * n + j] = s * ap + c * aq;
            }
            __syncthreads();
            for (int x = tid; x < np * n; x += RC_T) {   // columns p, q <- A J, and V J
                const int i = x / n, j = x % n, p = pp[i], q = pq[i];
                if (q >= n) continue;
                const double c = pc[i], s = ps[i];
                const double ap = A[j * n + p], aq = A[j * n + q];
                A[j * n + p] = c * ap - s * aq;
                A[j * n + q] = s * ap + c * aq;
                const double vp = V[j * n + p], vq = V[j * n + q];
                V[j * n + p] = c * vp - s * vq;
                V[j * n + q] = s * vp + c * vq;
            }
            __syncthreads();
        }
    }
}

// pass 1 (A.sofs == NULL): kept ranks; pass 2: the recompressed factors.
__global__ void __launch_bounds__(RC_T) k_recompress(RcArgs A)
{
    __shared__ int pp[RC_NMAX / 2], pq[RC_NMAX / 2], order[RC_NMAX];
    __shared__ double pc[RC_NMAX / 2], ps[RC_NMAX / 2], red[RC_T / 32 + 1];
    __shared__ double lamC[RC_NMAX], lamQ[RC_NMAX], sig2[RC_NMAX], ia[RC_NMAX], ib[RC_NMAX], ab[RC_NMAX];
    __shared__ int keep_r;
    const int tid = threadIdx.x;
    const int64_t NN = (int64_t)RC_NMAX * RC_NMAX;
    double* M0 = A.scratch + (int64_t)blockIdx.x * 6 * NN;
    double *M1 = M0 + NN, *M2 = M1 + NN, *M3 = M2 + NN, *M4 = M3 + NN, *M5 = M4 + NN;
    for (int64_t b = blockIdx.x; b < A.nG; b += gridDim.x) {
        const int l = A.rank[b];
        if (l <= 0) {
            if (tid == 0 && !A.sofs) A.srank[b] = 0;
            continue;
        }
        const int32_t t = A.PG[2 * b], s = A.PG[2 * b + 1];
        const int c = A.nend[t] - A.nbeg[t], q = A.nend[s] - A.nbeg[s];
        const int n = 3 * l;
        const int64_t C0 = 9 * A.fofs[b];                   // C_k(m)[u][v] at C0 + 9kc + (3u+v)c + m
        const int64_t Q0 = C0 + 9 * (int64_t)l * c;         // Q_k(j)[v][w] at Q0 + 9kq + (3v+w)q + j
        auto Cel = [&](int k, int m, int u, int v) { return fac_at(A, C0 + 9 * (int64_t)k * c + (3 * u + v) * c + m); };
        auto Qel = [&](int k, int j, int v, int w) { return fac_at(A, Q0 + 9 * (int64_t)k * q + (3 * v + w) * q + j); };
        // Grams: M0 = C^T C, M1 = Q Q^T
        for (int x = tid; x < n * n; x += RC_T) {
            const int i = x / n, j = x % n;
            if (j < i) continue;
            const int ki = i / 3, vi = i % 3, kj = j / 3, vj = j % 3;
            double g = 0.0, h = 0.0;
            for (int mm = 0; mm < c; ++mm)
                for (int u = 0; u < 3; ++u) g += Cel(ki, mm, u, vi) * Cel(kj, mm, u, vj);
            for (int jj = 0; jj < q; ++jj)
                for (int w = 0; w < 3; ++w) h += Qel(ki, jj, vi, w) * Qel(kj, jj, vj, w);
            M0[i * n + j] = M0[j * n + i] = g;
            M1[i * n + j] = M1[j * n + i] = h;
        }
        __syncthreads();
        // scale to unit diagonals: C = C^ D_a, Q = D_b Q^ with a_i, b_i the
        // scalar column / row norms, so the Grams' conditioning reflects the
        // angles between the terms, not their decaying sizes
        for (int i = tid; i < n; i += RC_T) {
            const double a = sqrt(M0[i * n + i]), bq = sqrt(M1[i * n + i]);
            ia[i] = a > 0.0 ? 1.0 / a : 0.0;
            ib[i] = bq > 0.0 ? 1.0 / bq : 0.0;
            ab[i] = a * bq;
        }
        __syncthreads();
        for (int x = tid; x < n * n; x += RC_T) {
            const int i = x / n, j = x % n;
            M0[x] *= ia[i] * ia[j];
            M1[x] *= ib[i] * ib[j];
        }
        __syncthreads();
        cta_jacobi(M0, M2, n, pp, pq, pc, ps, red);      // V_C in M2
        cta_jacobi(M1, M3, n, pp, pq, pc, ps, red);      // V_Q in M3
        // eigenvalues, the negligible ones zeroed
        double mc = 0.0, mq = 0.0;
        for (int i = 0; i < n; ++i) { mc = fmax(mc, M0[i * n + i]); mq = fmax(mq, M1[i * n + i]); }
        for (int i = tid; i < n; i += RC_T) {
            const double a = M0[i * n + i], bq = M1[i * n + i];
            lamC[i] = a > 1e-15 * mc ? a : 0.0;
            lamQ[i] = bq > 1e-15 * mq ? bq : 0.0;
        }
        __syncthreads();
        // K = L_C^(1/2) V_C^T V_Q L_Q^(1/2) in M4; then K^T K in M0
        for (int x = tid; x < n * n; x += RC_T) {
            const int i = x / n, j = x % n;
            double v = 0.0;
            if (lamC[i] > 0.0 && lamQ[j] > 0.0) {
                for (int k = 0; k < n; ++k) v += M2[k * n + i] * ab[k] * M3[k * n + j];
                v *= sqrt(lamC[i]) * sqrt(lamQ[j]);
            }
            M4[i * n + j] = v;
        }
        __syncthreads();
        for (int x = tid; x < n * n; x += RC_T) {
            const int i = x / n, j = x % n;
            if (j < i) continue;
            double v = 0.0;
            for (int k = 0; k < n; ++k) v += M4[k * n + i] * M4[k * n + j];
            M0[i * n + j] = M0[j * n + i] = v;
        }
        __syncthreads();
        cta_jacobi(M0, M1, n, pp, pq, pc, ps, red);      // Y in M1, s^2 on M0's diagonal
        // decreasing order of s^2 (ties by index), and the kept rank
        for (int i = tid; i < n; i += RC_T) sig2[i] = fmax(M0[i * n + i], 0.0);
        __syncthreads();
        for (int i = tid; i < n; i += RC_T) {
            int pos = 0;
            for (int j = 0; j < n; ++j) pos += sig2[j] > sig2[i] || (sig2[j] == sig2[i] && j < i);
            order[pos] = i;
        }
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int i = 0; i < n; ++i) tot += sig2[order[i]];
            int r = n;
            double tail = 0.0;
            while (r > 0 && tail + sig2[order[r - 1]] <= A.eps2 * tot) {
                tail += sig2[order[r - 1]];
                --r;
            }
            keep_r = r;
            if (!A.sofs) A.srank[b] = r;
        }
        __syncthreads();
        const int r = keep_r;
        if (!A.sofs || r == 0) continue;
        // T_C = V_C L_C^(-1/2) (K Y_r) in M5 [n][r];  T_Q = V_Q L_Q^(-1/2) Y_r in M0 [n][r]
        for (int x = tid; x < n * r; x += RC_T) {       // Z = K Y_r in M4's spare rows? use M0 as Z first
            const int i = x / r, rho = x % r, col = order[rho];
            double v = 0.0;
            for (int j = 0; j < n; ++j) v += M4[i * n + j] * M1[j * n + col];
            M0[i * r + rho] = v;
        }
        __syncthreads();
        for (int x = tid; x < n * r; x += RC_T) {
            const int k = x / r, rho = x % r, col = order[rho];
            double tc = 0.0, tq = 0.0;
            for (int i = 0; i < n; ++i) {
                if (lamC[i] > 0.0) tc += M2[k * n + i] * M0[i * r + rho] / sqrt(lamC[i]);
                if (lamQ[i] > 0.0) tq += M3[k * n + i] * M1[i * n + col] / sqrt(lamQ[i]);
            }
            M5[k * r + rho] = tc * ia[k];
            M4[k * r + rho] = tq * ib[k];    // K no longer needed
        }
        __syncthreads();
        // U = C T_C [r][3c], V^T = Q^T T_Q stored as V [r][3q]
        const int64_t o = A.sofs[b];
        const int nc = 3 * c, nq = 3 * q;
        for (int64_t x = tid; x < (int64_t)r * nc; x += RC_T) {
            const int rho = (int)(x / nc), i = (int)(x % nc), mm = i / 3, u = i % 3;
            double v = 0.0;
            for (int k = 0; k < l; ++k)
                for (int w = 0; w < 3; ++w) v += Cel(k, mm, u, w) * M5[(3 * k + w) * r + rho];
            if (A.real_bytes == 8) ((double*)A.sfac)[o + x] = v;
            else ((float*)A.sfac)[o + x] = (float)v;
        }
        for (int64_t x = tid; x < (int64_t)r * nq; x += RC_T) {
            const int rho = (int)(x / nq), i = (int)(x % nq), jj = i / 3, w = i % 3;
            double v = 0.0;
            for (int k = 0; k < l; ++k)
                for (int vv = 0; vv < 3; ++vv) v += Qel(k, jj, vv, w) * M4[(3 * k + vv) * r + rho];
            const int64_t d = o + (int64_t)r * nc + x;
            if (A.real_bytes == 8) ((double*)A.sfac)[d] = v;
            else ((float*)A.sfac)[d] = (float)v;
        }
        __syncthreads();
    }
}

__global__ void k_srank_len(const int32_t* __restrict__ PG, int64_t nG, const int32_t* __restrict__ nbeg,
                            const int32_t* __restrict__ nend, const int32_t* __restrict__ srank, int64_t* __restrict__ len)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nG) {
        const int32_t t = PG[2 * b], s = PG[2 * b + 1];
        len[b] = 3 * (int64_t)(nend[t] - nbeg[t] + nend[s] - nbeg[s]) * srank[b];
    }
}

// y_tau = U (V F_sigma) (transpose: y_sigma = V^T (U^T W_tau)), one warp per
// block, into the block's partial output.
template <typename R>
__global__ void __launch_bounds__(128) k_apply_rc(const R* __restrict__ fac, const int64_t* __restrict__ sofs,
                                                  const int32_t* __restrict__ srank, const int32_t* __restrict__ PG,
                                                  int64_t nG, const int32_t* __restrict__ nbeg,
                                                  const int32_t* __restrict__ nend, const double* __restrict__ Fs,
                                                  R* __restrict__ part, const int64_t* __restrict__ pofs,
                                                  int transpose)
{
    __shared__ R tv[4][RC_NMAX];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * 4 + w;
    if (b >= nG) return;
    const int32_t t = PG[2 * b], s = PG[2 * b + 1];
    const int32_t t0 = nbeg[t], c = nend[t] - t0, s0 = nbeg[s], q = nend[s] - s0;
    const int r = srank[b];
    const R* U = fac + sofs[b];
    const R* V = U + (int64_t)r * 3 * c;
    const int nin = transpose ? 3 * c : 3 * q, nout = transpose ? 3 * q : 3 * c;
    const R* Min = transpose ? U : V;
    const R* Mout = transpose ? V : U;
    const double* fin = Fs + 3 * (int64_t)(transpose ? t0 : s0);
    for (int rho = 0; rho < r; ++rho) {
        const R* row = Min + (int64_t)rho * nin;
        R a = 0;
        for (int x = lane; x < nin; x += 32) a += row[x] * (R)fin[x];
        a = warp_sum(a);
        if (lane == 0) tv[w][rho] = a;
    }
    __syncwarp();
    R* out = part + 3 * pofs[b];
    for (int x = lane; x < nout; x += 32) {
        R y = 0;
        for (int rho = 0; rho < r; ++rho) y += Mout[(int64_t)rho * nout + x] * tv[w][rho];
        out[x] = y;
    }
}

}  // namespace

void recompress_factors(hh_ctx* ctx, hh_hmat* h, double eps_rc, cudaStream_t s)
{
    const hh_blocks* bl = h->blocks;
    const hh_tree* t = h->tree;
    const int64_t nG = bl->nG;
    HH_REQUIRE(h->factors != nullptr, HH_ERR_ARG, "recompression needs the stored factors");
    HH_REQUIRE(h->params.max_rank <= RC_NMAX / 3, HH_ERR_ARG, "max_rank too large for the recompression");
    HH_REQUIRE(eps_rc >= 0.0 && eps_rc < 1.0, HH_ERR_ARG, "eps_rc must be in [0, 1)");
    int32_t* srank = nullptr;
    int64_t* sofs = nullptr;
    HH_CUDA(cudaMalloc(&srank, sizeof(int32_t) * (nG > 0 ? nG : 1)));
    HH_CUDA(cudaMalloc(&sofs, sizeof(int64_t) * (nG + 1)));
    HH_CUDA(cudaMemsetAsync(sofs, 0, sizeof(int64_t) * (nG + 1), s));
    void* sfac = nullptr;
    int64_t n_sfac = 0;
    try {
        if (nG > 0) {
            const int64_t grid = std::min<int64_t>(nG, (int64_t)ctx->n_sm * 4);
            double* scratch = dev_alloc_t<double>(grid * 6 * (int64_t)RC_NMAX * RC_NMAX, s);
            RcArgs A{};
            A.PG = bl->PG;
            A.nbeg = t->nbeg;
            A.nend = t->nend;
            A.rank = h->rank;
            A.fofs = h->fofs;
            A.fac = h->factors;
            A.real_bytes = h->real_bytes;
            A.nG = nG;
            A.eps2 = eps_rc * eps_rc;
            A.scratch = scratch;
            A.srank = srank;
            k_recompress<<<(unsigned)grid, RC_T, 0, s>>>(A);
            HH_CHECK_LAUNCH();
            int64_t* len = dev_alloc_t<int64_t>(nG, s);
            k_srank_len<<<(unsigned)ceil_div(nG, 256), 256, 0, s>>>(bl->PG, nG, t->nbeg, t->nend, srank, len);
            HH_CHECK_LAUNCH();
            dev_scan_i64(len, sofs, nG, sofs + nG, s);
            HH_CUDA(cudaMemcpyAsync(&n_sfac, sofs + nG, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            HH_CUDA(cudaStreamSynchronize(s));
            dev_free(len, s);
            HH_CUDA(cudaMalloc(&sfac, (size_t)h->real_bytes * (n_sfac > 0 ? n_sfac : 1)));
            A.sofs = sofs;
            A.sfac = sfac;
            k_recompress<<<(unsigned)grid, RC_T, 0, s>>>(A);
            HH_CHECK_LAUNCH();
            dev_free(scratch, s);
        }
        HH_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        cudaFree(srank);
        cudaFree(sofs);
        if (sfac) cudaFree(sfac);
        throw;
    }
    // the recompressed factors replace the ACA factors
    cudaFree(h->factors);
    h->factors = nullptr;
    cudaFree(h->srank);
    cudaFree(h->sofs);
    cudaFree(h->sfac);
    h->srank = srank;
    h->sofs = sofs;
    h->sfac = sfac;
    h->n_sfac = n_sfac;
}

void recompressed_apply(const hh_hmat* h, const double* Fs, void* part, const int64_t* pofs, int transpose,
                        cudaStream_t s)
{
    const int64_t nG = h->blocks->nG;
    if (nG == 0) return;
    const unsigned grid = (unsigned)ceil_div(nG, 4);
    if (h->real_bytes == 8)
        k_apply_rc<double><<<grid, 128, 0, s>>>((const double*)h->sfac, h->sofs, h->srank, h->blocks->PG, nG,
                                                h->tree->nbeg, h->tree->nend, Fs, (double*)part, pofs, transpose);
    else
        k_apply_rc<float><<<grid, 128, 0, s>>>((const float*)h->sfac, h->sofs, h->srank, h->blocks->PG, nG,
                                               h->tree->nbeg, h->tree->nend, Fs, (float*)part, pofs, transpose);
    HH_CHECK_LAUNCH();
}
