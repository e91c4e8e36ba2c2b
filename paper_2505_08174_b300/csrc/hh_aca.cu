// hh_aca.cu -- batched block adaptive cross approximation (Algorithm 2,
// Eqs. 8-10) and the low-rank product C (Q F) (Eq. 8) on the GPU.
//
// Design: persistent "team" kernels.  A team is one warp (blocks whose
// clusters have <= 128 particles) or one 256-thread CTA (larger blocks).  A
// team pulls the next admissible block from a work list (atomic counter,
// largest blocks first), runs the whole rank loop of Algorithm 2 on it, and
// -- in the fused mode used by hh_predict -- applies the block to F right
// away, so C and Q only ever live in the team's private workspace (bounded,
// independent of N).  Results are written per block, so the output does not
// depend on which team ran which block.
//
// Per rank step k (element = 3x3 block, row-major):
//   column  c_k(m) = G(m, j_k) - sum_{p<k} C_p(m) Q_p(j_k)
//   i_k     = argmax over unused rows of |c_k(m)|_F, ties -> lowest index
//   c_k    <- c_k [c_k(i_k)]^-1, inverse in FP64 (adjugate)
//   row     q_k(n) = G(i_k, n) - sum_{p<k} C_p(i_k) Q_p(n)
//   j_{k+1} = argmax over unused columns of |q_k(n)|_F
//   A_pk = sum_m c_p(m)^T c_k(m),  B_kp = sum_n q_k(n) q_p(n)^T (3x3 Grams)
//   nu^2 = tr(A_kk B_kk), lambda^2 += nu^2 + 2 sum_{p<k} tr(A_pk B_kp)
//   stop if nu^2 <= zeta^2 lambda^2, or k = min(c, q), or k = max_rank
// Pivot guard: a pivot element with det = 0 or 1/(|P|_F |P^-1|_F) < 1e-10
// is replaced by the unused row of largest |det|; a zero column residual (or
// no usable pivot) ends the block with the pairs found so far.
// The 3x3 Gram sums are formed and reduced in the working precision; nu^2,
// the cross term and the lambda^2 recurrence are reduced and kept in FP64.
#include <algorithm>
#include <vector>

#include "hh_aca.cuh"

namespace {

// ---- the per-block ACA -----------------------------------------------------
template <typename R, int KIND, class Team, class S>
__device__ void aca_block(const AcaArgs<R>& A, const Team& tm, S& sm, const R* th, R* hs, R* Cs_base,
                          int64_t b, int mode)
{
    constexpr int ROWS = Team::ROWS, SIZE = Team::SIZE;
    constexpr int NB = Team::REG_FLAGS ? (ROWS + 31) / 32 : 1;
    const int tid = tm.tid();
    const int32_t t = A.PG[2 * b], s = A.PG[2 * b + 1];
    const int32_t t0 = A.nbeg[t], c = A.nend[t] - t0, s0 = A.nbeg[s], q = A.nend[s] - s0;
    const int kmax = min(min(c, q), A.max_rank);
    R* Cs = Cs_base;
    R* Qs = Cs_base + (int64_t)kmax * 9 * c;
    // used-row / used-column flags: register bitmasks (warp team, bit i of the
    // thread's i-th row) or bytes after the factors (CTA team)
    uint32_t usedR[NB], usedC[NB];
    uint8_t* fR = reinterpret_cast<uint8_t*>(Qs + (int64_t)kmax * 9 * q);
    uint8_t* fC = fR + c;
#pragma unroll
    for (int i = 0; i < NB; ++i) usedR[i] = usedC[i] = 0u;
    if constexpr (!Team::REG_FLAGS) {
        for (int x = tid; x < c + q; x += SIZE) fR[x] = 0;
        tm.sync();
    }
    auto is_used = [&](const uint32_t* u, const uint8_t* f, int i, int x) -> bool {
        if constexpr (Team::REG_FLAGS) return (u[i >> 5] >> (i & 31)) & 1u;
        else return f[x] != 0;
    };
    auto set_used = [&](uint32_t* u, uint8_t* f, int x) {
        if constexpr (Team::REG_FLAGS) {
            if (x % SIZE == tid) u[(x / SIZE) >> 5] |= 1u << ((x / SIZE) & 31);
        } else {
            if (tid == 0) f[x] = 1;
        }
    };
    int j = j1_of(A.j1_rule, A.seed, t, s, q);
    set_used(usedC, fC, j);
    double lam2 = 0.0;
    int k = 0;
    bool capped = false;
    int bi = -1, bj = -1;
    while (k < kmax) {
        bool done = false;  // uniform over the team
        // pass 0 generates the column residual c_k over the rows m (line 4) and
        // picks i_k (line 5), pivots and scales it (line 6); pass 1 generates the
        // row residual q_k over the columns n (line 7), picks j_{k+1} (line 8)
        // and updates the norms (lines 9-10).  Both passes share one pair-kernel
        // call site, which keeps the kernel's instruction footprint small.
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            const int nx = pass == 0 ? c : q;
            R* fac = pass == 0 ? Cs : Qs;       // factor being extended (rows x)
            R* line = fac + (int64_t)k * 9 * nx;
            R* piv = pass == 0 ? sm.qj : sm.ci;  // Q_p(j_k) or C_p(i_k), p < k
            for (int idx = tid; idx < k * 9; idx += SIZE)
                piv[idx] = pass == 0 ? Qs[(int64_t)idx * q + j] : Cs[(int64_t)idx * c + bi];
            tm.sync();
            R best = (R)-1;
            int barg = -1;
            R snu = 0, scr = 0;   // stopping-test terms of the row pass
#pragma unroll 1
            for (int i = 0; i < ROWS; ++i) {
                const int x = tid + SIZE * i;
                if (x >= nx) break;
                R rx, ry, rz, K[9];
                sep<R>(A.Xs, pass == 0 ? t0 + x : t0 + bi, pass == 0 ? s0 + j : s0 + x, rx, ry, rz);
                pair_block<R, KIND>(th, A.pp, rx, ry, rz, K, hs);
                R V[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                for (int p = 0; p < k; ++p) {
                    R v[9], t9[9];
                    ld9(fac + (int64_t)p * 9 * nx, nx, x, v);
                    if (pass == 0) {
                        mm3(v, piv + 9 * p, t9);   // C_p(m) Q_p(j_k)
                    } else {
                        mm3(piv + 9 * p, v, t9);   // C_p(i_k) Q_p(n)
                        add_AtB(V, sm.A + 9 * p, v);
                    }
#pragma unroll
                    for (int e = 0; e < 9; ++e) K[e] -= t9[e];
                }
                if (pass == 1) row_terms(sm.A + 9 * k, K, V, snu, scr);
                st9(line, nx, x, K);
                const bool used = pass == 0 ? is_used(usedR, fR, i, x) : is_used(usedC, fC, i, x);
                if (!used) {
                    R v = fro2(K);
                    if (v > best) { best = v; barg = x; }
                }
            }
            tm.argmax(best, barg, sm);
            if (pass == 1) {
                bj = barg;
                tm.sync();
                double nu2, cross;
                team_sum2(tm, sm, snu, scr, nu2, cross);
                if (tid == 0) {
                    lam2 = lam2 + nu2 + 2.0 * cross;
                    sm.stop = (nu2 <= A.eps2 * lam2) || (bj < 0);
                }
                tm.sync();
                break;
            }
            if (barg < 0 || !(best > (R)0)) { done = true; break; }
            bi = barg;
            tm.sync();
            if (tid == 0) {
                double P[9], Pi[9];
#pragma unroll
                for (int e = 0; e < 9; ++e) P[e] = (double)Cs[((int64_t)k * 9 + e) * c + bi];
                int bad;
                if constexpr (sizeof(R) == 4) {   // FP32 residuals: noise floor (inv3_floor)
                    if (k == 0) sm.pscale = sqrt(fro2(P));
                    double det;
                    const int kept = inv3_floor(P, PIVOT_FLOOR_FP32 * sm.pscale, Pi, &det);
                    const double rc = kept == 3 ? 1.0 / sqrt(fro2(P) * fro2(Pi)) : 1.0;
                    bad = kept == 0 ? 2 : (!(rc >= 1e-10) ? 1 : 0);
                } else {
                    double det = inv3d(P, Pi);
                    double rc = det != 0.0 ? 1.0 / sqrt(fro2(P) * fro2(Pi)) : 0.0;
                    bad = !(det != 0.0) || !(rc >= 1e-10);
                }
                sm.flag = bad;
                if (!bad)
#pragma unroll
                    for (int e = 0; e < 9; ++e) sm.Pi[e] = (R)Pi[e];
            }
            tm.sync();
            if (sm.flag == 2) { done = true; break; }   // the pivot element is rounding noise
            if (sm.flag) {
                double bd = 0.0;
                int bdi = -1;
                for (int i = 0; i < ROWS; ++i) {
                    const int m = tid + SIZE * i;
                    if (m >= c) break;
                    if (is_used(usedR, fR, i, m)) continue;
                    double P[9];
#pragma unroll
                    for (int e = 0; e < 9; ++e) P[e] = (double)Cs[((int64_t)k * 9 + e) * c + m];
                    double dv = fabs(det3d(P));
                    if (dv > bd) { bd = dv; bdi = m; }
                }
                tm.argmax(bd, bdi, sm);
                if (bdi < 0) { done = true; break; }
                bi = bdi;
                if (tid == 0) {
                    double P[9], Pi[9];
#pragma unroll
                    for (int e = 0; e < 9; ++e) P[e] = (double)Cs[((int64_t)k * 9 + e) * c + bi];
                    inv3d(P, Pi);
#pragma unroll
                    for (int e = 0; e < 9; ++e) sm.Pi[e] = (R)Pi[e];
                }
                tm.sync();
            }
            set_used(usedR, fR, bi);
            if (tid == 0 && A.pivI) {
                A.pivI[b * A.max_rank + k] = bi;
                A.pivJ[b * A.max_rank + k] = j;
            }
            // c_k <- c_k [c_k(i_k)]^-1
            R Pi[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) Pi[e] = sm.Pi[e];
            for (int i = 0; i < ROWS; ++i) {
                const int m = tid + SIZE * i;
                if (m >= c) break;
                R r[9], o[9];
                ld9(line, c, m, r);
                mm3(r, Pi, o);
                st9(line, c, m, o);
            }
            tm.sync();
            gram_cols<R>(tm, sm, Cs, c, k);
        }
        if (done) break;
        ++k;
        const bool stop = sm.stop;
        tm.sync();
        if (stop) break;
        if (k == kmax) {
            capped = (k == A.max_rank) && (k < min(c, q));
            break;
        }
        j = bj;
        set_used(usedC, fC, j);
    }
    const int l = k;
    if (tid == 0) {
        if (A.rank) A.rank[b] = l;
        if (A.pivI)
            for (int p = l; p < A.max_rank; ++p) { A.pivI[b * A.max_rank + p] = -1; A.pivJ[b * A.max_rank + p] = -1; }
        if (capped) atomicOr(A.status, (unsigned)HH_DEV_RANK_CAP);
        atomicAdd(A.n_queries, (unsigned long long)(c + q) * (unsigned long long)l);
    }
    if (mode == 0) {
        // fused apply: t_p = sum_n Q_p(n) F(s0+n); y(m) = sum_p C_p(m) t_p
        const int lane = threadIdx.x & 31;
        for (int p = tm.warp(); p < l; p += Team::NW) {
            const R* Qp = Qs + (int64_t)p * 9 * q;
            R a0 = 0, a1 = 0, a2 = 0;
            for (int n = lane; n < q; n += 32) {
                R qv[9];
                ld9(Qp, q, n, qv);
                const double* f = A.Fs + 3 * (int64_t)(s0 + n);
                R f0 = (R)f[0], f1 = (R)f[1], f2 = (R)f[2];
                a0 += qv[0] * f0 + qv[1] * f1 + qv[2] * f2;
                a1 += qv[3] * f0 + qv[4] * f1 + qv[5] * f2;
                a2 += qv[6] * f0 + qv[7] * f1 + qv[8] * f2;
            }
            a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2);
            if (lane == 0) { sm.tv[3 * p] = a0; sm.tv[3 * p + 1] = a1; sm.tv[3 * p + 2] = a2; }
        }
        tm.sync();
        R* out = A.part + 3 * (A.pofs[b] - A.pofs_base);
        for (int i = 0; i < ROWS; ++i) {
            const int m = tid + SIZE * i;
            if (m >= c) break;
            R y0 = 0, y1 = 0, y2 = 0;
            for (int p = 0; p < l; ++p) {
                R cv[9];
                ld9(Cs + (int64_t)p * 9 * c, c, m, cv);
                const R* tp = sm.tv + 3 * p;
                y0 += cv[0] * tp[0] + cv[1] * tp[1] + cv[2] * tp[2];
                y1 += cv[3] * tp[0] + cv[4] * tp[1] + cv[5] * tp[2];
                y2 += cv[6] * tp[0] + cv[7] * tp[1] + cv[8] * tp[2];
            }
            out[3 * m] = y0; out[3 * m + 1] = y1; out[3 * m + 2] = y2;
        }
    } else if (mode == 2) {
        R* dst = A.fac + 9 * (A.fofs[b] - A.fofs_base);
        const int64_t nc = (int64_t)l * 9 * c, nq = (int64_t)l * 9 * q;
        for (int64_t x = tid; x < nc; x += SIZE) dst[x] = Cs[x];
        for (int64_t x = tid; x < nq; x += SIZE) dst[nc + x] = Qs[x];
    }
    tm.sync();
}

template <typename R>
__device__ void load_theta(const AcaArgs<R>& A, R* th)
{
    for (int i = threadIdx.x; i < A.n_th; i += blockDim.x) th[i] = A.th_g[i];
    __syncthreads();
}

constexpr int WPB = 4;  // warp teams per CTA

template <typename R, int KIND>
__global__ void __launch_bounds__(32 * WPB) k_aca_warp(AcaArgs<R> A, int mode)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TeamSmem<R>* sms = reinterpret_cast<TeamSmem<R>*>(smem_raw);
    R* th = reinterpret_cast<R*>(smem_raw + sizeof(TeamSmem<R>) * WPB);
    constexpr int ACT = act_floats_per_warp<R, KIND>();
    R* hs = th + A.n_th + (threadIdx.x >> 5) * ACT + (threadIdx.x & 31);
    load_theta(A, th);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    TeamSmem<R>& sm = sms[w];
    const int64_t team = (int64_t)blockIdx.x * WPB + w;
    R* Cs = A.scratch + team * A.team_stride;
    WarpTeam tm;
    for (;;) {
        unsigned long long wi = 0;
        if (lane == 0) wi = atomicAdd(A.counter, 1ull);
        wi = __shfl_sync(0xffffffffu, wi, 0);
        if ((int64_t)wi >= A.n_work) break;
        aca_block<R, KIND>(A, tm, sm, th, hs, Cs, A.work[wi], mode);
    }
}

template <typename R, int KIND>
__global__ void __launch_bounds__(CTA_T) k_aca_cta(AcaArgs<R> A, int mode)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TeamSmem<R>& sm = *reinterpret_cast<TeamSmem<R>*>(smem_raw);
    R* th = reinterpret_cast<R*>(smem_raw + sizeof(TeamSmem<R>));
    constexpr int ACT = act_floats_per_warp<R, KIND>();
    R* hs = th + A.n_th + (threadIdx.x >> 5) * ACT + (threadIdx.x & 31);
    __shared__ unsigned long long wi_s;
    load_theta(A, th);
    R* Cs = A.scratch + (int64_t)blockIdx.x * A.team_stride;
    CtaTeam tm;
    for (;;) {
        if (threadIdx.x == 0) wi_s = atomicAdd(A.counter, 1ull);
        __syncthreads();
        unsigned long long wi = wi_s;
        __syncthreads();
        if ((int64_t)wi >= A.n_work) break;
        aca_block<R, KIND>(A, tm, sm, th, hs, Cs, A.work[wi], mode);
    }
}

// ---- work lists --------------------------------------------------------------
__global__ void k_classify_blocks(const int32_t* __restrict__ PG, int64_t nG, const int32_t* __restrict__ nbeg,
                                  const int32_t* __restrict__ nend, const uint8_t* __restrict__ shard_mine,
                                  int64_t b0, int64_t b1, int small_max, int64_t* __restrict__ small_flag, int64_t* __restrict__ large_flag,
                                  uint64_t* __restrict__ large_key)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nG) return;
    int32_t c = nend[PG[2 * b]] - nbeg[PG[2 * b]], q = nend[PG[2 * b + 1]] - nbeg[PG[2 * b + 1]];
    bool mine = (shard_mine == nullptr || shard_mine[b]) && b >= b0 && b < b1;
    bool small = c <= small_max && q <= small_max;
    small_flag[b] = mine && small;
    large_flag[b] = mine && !small;
    // larger blocks first: key = (2^31 - 1 - (c + q)) << 32 | b
    large_key[b] = ((uint64_t)(0x7fffffffu - (uint32_t)(c + q)) << 32) | (uint64_t)b;
}

__global__ void k_compact(const int64_t* __restrict__ flag, const int64_t* __restrict__ off, int64_t n,
                          int32_t* __restrict__ out)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n && flag[b]) out[off[b]] = (int32_t)b;
}

__global__ void k_compact_keys(const int64_t* __restrict__ flag, const int64_t* __restrict__ off,
                               const uint64_t* __restrict__ key, int64_t n, uint64_t* __restrict__ out)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n && flag[b]) out[off[b]] = key[b];
}

__global__ void k_keys_to_work(const uint64_t* __restrict__ key, int64_t n, int32_t* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int32_t)(key[i] & 0xffffffffu);
}

__global__ void k_max_dim(const int32_t* __restrict__ work, int64_t n, const int32_t* __restrict__ PG,
                          const int32_t* __restrict__ nbeg, const int32_t* __restrict__ nend, int* out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t b = work[i];
    int32_t c = nend[PG[2 * b]] - nbeg[PG[2 * b]], q = nend[PG[2 * b + 1]] - nbeg[PG[2 * b + 1]];
    atomicMax(out, c + q);
}

// Size classes of the sorted large list (keys: (2^31 - 1 - (c + q)) << 32 | b,
// ascending = decreasing c + q): pos[i] = first item with c + q <= lim[i],
// mx[i] = c + q of item pos[i - 1] (class i's largest), mx[0] = the first item's.
constexpr int N_CLASS_LIMITS = 5;
__constant__ int32_t c_class_lim[N_CLASS_LIMITS] = {262144, 65536, 16384, 4096, 1536};

__global__ void k_class_bounds(const uint64_t* __restrict__ key, int64_t n, int64_t* __restrict__ pos,
                               int32_t* __restrict__ mx)
{
    const int i = threadIdx.x;
    auto cq = [&](int64_t x) { return (int32_t)(0x7fffffffu - (uint32_t)(key[x] >> 32)); };
    if (i < N_CLASS_LIMITS) {
        int64_t lo = 0, hi = n;   // first x with cq(x) <= lim
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cq(mid) <= c_class_lim[i]) hi = mid; else lo = mid + 1;
        }
        pos[i] = lo;
        mx[i + 1] = lo < n ? cq(lo) : 0;
    }
    if (i == 0) mx[0] = n > 0 ? cq(0) : 0;
}

template <typename R, int KIND>
void launch_aca(hh_ctx* ctx, const hh_params& p, AcaArgs<R> A, const int32_t* work_small, int64_t n_small,
                const int32_t* work_large, const std::vector<AcaClass>& cls, int max_small_cq, const hh_launch_cfg& lc,
                int mode, cudaStream_t s)
{
    const int th_bytes = A.n_th * (int)sizeof(R);
    const int mr = std::min(A.max_rank, MAXR);
    // large blocks first (CTA teams), then small blocks (warp teams)
    if (!cls.empty()) {
        size_t smem = sizeof(TeamSmem<R>) + th_bytes + sizeof(R) * act_floats_per_warp<R, KIND>() * (CTA_T / 32);
        HH_CUDA(cudaFuncSetAttribute(k_aca_cta<R, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        HH_CUDA(cudaEventRecord(ctx->kev[0], s));
        for (const AcaClass& k : cls) {
            // factors (max_rank x 9 x (c+q) reals) + c+q flag bytes, rounded to 256 B
            int64_t stride = (int64_t)k.max_cq * 9 * mr + ceil_div(k.max_cq, (int64_t)sizeof(R));
            stride = ceil_div(stride * (int64_t)sizeof(R), 256) * 256 / (int64_t)sizeof(R);
            const int64_t budget = budget_cta_teams(p);  // bytes of large-team workspace
            int64_t teams = std::min<int64_t>(k.end - k.begin, (int64_t)lc.aca_large_cps * ctx->n_sm);
            teams = std::max<int64_t>(1, std::min<int64_t>(teams, budget / (stride * (int64_t)sizeof(R))));
            R* scratch = dev_alloc_t<R>(stride * teams, s);
            HH_CUDA(cudaMemsetAsync(A.counter, 0, sizeof(unsigned long long), s));
            AcaArgs<R> B = A;
            B.work = work_large + k.begin;
            B.n_work = k.end - k.begin;
            B.scratch = scratch;
            B.team_stride = stride;
            k_aca_cta<R, KIND><<<(unsigned)teams, CTA_T, smem, s>>>(B, mode);
            HH_CHECK_LAUNCH();
            dev_free(scratch, s);
        }
        HH_CUDA(cudaEventRecord(ctx->kev[1], s));
        ctx->kev_aca_used |= 1;
    }
    if (n_small > 0) {
        // factors (max_rank x 9 x (c+q) reals), rounded to 256 B; as many teams as the budget holds
        int64_t stride = (int64_t)std::min(max_small_cq, 2 * SMALL_MAX) * 9 * mr;
        stride = ceil_div(stride * (int64_t)sizeof(R), 256) * 256 / (int64_t)sizeof(R);
        int64_t blocks = std::min<int64_t>(ceil_div(n_small, WPB), (int64_t)lc.aca_small_cps * ctx->n_sm);
        blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, budget_warp_teams(p) / (stride * WPB * (int64_t)sizeof(R))));
        int64_t teams = blocks * WPB;
        R* scratch = dev_alloc_t<R>(stride * teams, s);
        HH_CUDA(cudaMemsetAsync(A.counter + 1, 0, sizeof(unsigned long long), s));
        AcaArgs<R> B = A;
        B.work = work_small;
        B.n_work = n_small;
        B.counter = A.counter + 1;
        B.scratch = scratch;
        B.team_stride = stride;
        size_t smem = WPB * sizeof(TeamSmem<R>) + th_bytes + sizeof(R) * act_floats_per_warp<R, KIND>() * WPB;
        HH_CUDA(cudaFuncSetAttribute(k_aca_warp<R, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        HH_CUDA(cudaEventRecord(ctx->kev[2], s));
        k_aca_warp<R, KIND><<<(unsigned)blocks, 32 * WPB, smem, s>>>(B, mode);
        HH_CHECK_LAUNCH();
        HH_CUDA(cudaEventRecord(ctx->kev[3], s));
        ctx->kev_aca_used |= 2;
        dev_free(scratch, s);
    }
}

// ---- low-rank apply from stored factors ------------------------------------
// transpose = 0: y_tau(m) = sum_p C_p(m) (sum_n Q_p(n) F(n))
// transpose = 1: y_sigma(n) = sum_p Q_p(n)^T (sum_m C_p(m)^T W(m))
template <typename R>
__global__ void __launch_bounds__(128) k_apply(const R* __restrict__ fac, const int64_t* __restrict__ fofs,
                                               const int32_t* __restrict__ rank, const int32_t* __restrict__ PG,
                                               int64_t nG, const int32_t* __restrict__ nbeg,
                                               const int32_t* __restrict__ nend, const double* __restrict__ Fs,
                                               R* __restrict__ part, const int64_t* __restrict__ pofs, int transpose)
{
    __shared__ R tv[4][MAXR * 3];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * 4 + w;
    if (b >= nG) return;
    const int32_t t = PG[2 * b], s = PG[2 * b + 1];
    const int32_t t0 = nbeg[t], c = nend[t] - t0, s0 = nbeg[s], q = nend[s] - s0;
    const int l = rank[b];
    const R* Cs = fac + 9 * fofs[b];
    const R* Qs = Cs + (int64_t)l * 9 * c;
    const int nin = transpose ? c : q, nout = transpose ? q : c;
    const int in0 = transpose ? t0 : s0;
    const R* Fin = transpose ? Cs : Qs;
    const R* Fout = transpose ? Qs : Cs;
    for (int p = 0; p < l; ++p) {
        const R* Mp = Fin + (int64_t)p * 9 * nin;
        R a0 = 0, a1 = 0, a2 = 0;
        for (int x = lane; x < nin; x += 32) {
            R v[9];
            ld9(Mp, nin, x, v);
            const double* f = Fs + 3 * (int64_t)(in0 + x);
            R f0 = (R)f[0], f1 = (R)f[1], f2 = (R)f[2];
            if (!transpose) {
                a0 += v[0] * f0 + v[1] * f1 + v[2] * f2;
                a1 += v[3] * f0 + v[4] * f1 + v[5] * f2;
                a2 += v[6] * f0 + v[7] * f1 + v[8] * f2;
            } else {  // C_p(m)^T w(m)
                a0 += v[0] * f0 + v[3] * f1 + v[6] * f2;
                a1 += v[1] * f0 + v[4] * f1 + v[7] * f2;
                a2 += v[2] * f0 + v[5] * f1 + v[8] * f2;
            }
        }
        a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2);
        if (lane == 0) { tv[w][3 * p] = a0; tv[w][3 * p + 1] = a1; tv[w][3 * p + 2] = a2; }
    }
    __syncwarp();
    R* out = part + 3 * pofs[b];
    for (int x = lane; x < nout; x += 32) {
        R y0 = 0, y1 = 0, y2 = 0;
        for (int p = 0; p < l; ++p) {
            R v[9];
            ld9(Fout + (int64_t)p * 9 * nout, nout, x, v);
            const R* tp = tv[w] + 3 * p;
            if (!transpose) {
                y0 += v[0] * tp[0] + v[1] * tp[1] + v[2] * tp[2];
                y1 += v[3] * tp[0] + v[4] * tp[1] + v[5] * tp[2];
                y2 += v[6] * tp[0] + v[7] * tp[1] + v[8] * tp[2];
            } else {  // Q_p(n)^T s_p
                y0 += v[0] * tp[0] + v[3] * tp[1] + v[6] * tp[2];
                y1 += v[1] * tp[0] + v[4] * tp[1] + v[7] * tp[2];
                y2 += v[2] * tp[0] + v[5] * tp[1] + v[8] * tp[2];
            }
        }
        out[3 * x] = y0; out[3 * x + 1] = y1; out[3 * x + 2] = y2;
    }
}

// Size classes of the BF16 rounds: c + q in (2^e, 2^(e+1)], largest first;
// pos[i] = first item of the sorted list with c + q <= 2^(RC_TOP - i).
constexpr int RC_TOP = 30, RC_N = RC_TOP - 7 + 1;   // the last class is c + q <= 128

__global__ void k_round_classes(const uint64_t* __restrict__ key, int64_t n, int64_t* __restrict__ pos,
                                int32_t* __restrict__ mx, int32_t min_cq)
{
    const int i = threadIdx.x;
    auto cq = [&](int64_t x) { return (int32_t)(0x7fffffffu - (uint32_t)(key[x] >> 32)); };
    if (i <= RC_N) {   // pos[RC_N]: the items with c + q > min_cq
        const int32_t lim = i < RC_N ? 1 << (RC_TOP - i) : min_cq;
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cq(mid) <= lim) hi = mid; else lo = mid + 1;
        }
        pos[i] = lo;
        if (i < RC_N) mx[i + 1] = lo < n ? cq(lo) : 0;   // largest c + q of the class starting at lo
    }
    if (i == 0) mx[0] = n > 0 ? cq(0) : 0;
}

template <typename R>
void aca_run_t(hh_ctx* ctx, const hh_tree* t, const hh_blocks* bl, const hh_params& p, const AcaRun& r,
               cudaStream_t s)
{
    const int64_t nG = bl->nG;
    if (nG == 0) return;
    HH_REQUIRE(p.max_rank >= 1 && p.max_rank <= MAXR, HH_ERR_ARG, "max_rank must be in [1, 64]");
    AcaArgs<R> A = make_aca_args<R>(ctx, t, bl, p, r);

    // work lists: small blocks in block order, large blocks by decreasing c + q
    int64_t* fs = dev_alloc_t<int64_t>(nG, s);
    int64_t* fl = dev_alloc_t<int64_t>(nG, s);
    int64_t* os = dev_alloc_t<int64_t>(nG, s);
    int64_t* ol = dev_alloc_t<int64_t>(nG, s);
    uint64_t* key = dev_alloc_t<uint64_t>(nG, s);
    int64_t* tot = dev_alloc_t<int64_t>(2, s);
    const bool use_tc = p.precision == HH_BF16 && kernel_kind(p, ctx->width) < 2;
    const hh_launch_cfg lc = resolved_launch(ctx, use_tc);
    uint8_t* mine = shard_block_flags(t, bl, p, s);   // this shard's blocks (NULL: all)
    k_classify_blocks<<<(unsigned)ceil_div(nG, 256), 256, 0, s>>>(bl->PG, nG, t->nbeg, t->nend, mine, r.b0,
                                                                  r.b1 < 0 ? nG : r.b1, std::min(lc.small_max, SMALL_MAX),
                                                                  fs, fl, key);
    HH_CHECK_LAUNCH();
    if (mine) dev_free(mine, s);
    dev_scan_i64(fs, os, nG, tot, s);
    dev_scan_i64(fl, ol, nG, tot + 1, s);
    int64_t h[2];
    HH_CUDA(cudaMemcpyAsync(h, tot, sizeof h, cudaMemcpyDeviceToHost, s));
    HH_CUDA(cudaStreamSynchronize(s));
    int32_t* ws = dev_alloc_t<int32_t>(h[0], s);
    int32_t* wl = dev_alloc_t<int32_t>(h[1], s);
    k_compact<<<(unsigned)ceil_div(nG, 256), 256, 0, s>>>(fs, os, nG, ws);
    HH_CHECK_LAUNCH();
    std::vector<AcaClass> cls;   // size classes of the large list
    // the round engine's classes of the large list (BF16): c + q in (2^e, 2^(e+1)]
    std::vector<int64_t> rb;
    int32_t rm[RC_N + 1] = {};
    int64_t n_rounds = 0;
    if (h[1] > 0) {
        uint64_t* lk = dev_alloc_t<uint64_t>(h[1], s);
        k_compact_keys<<<(unsigned)ceil_div(nG, 256), 256, 0, s>>>(fl, ol, key, nG, lk);
        HH_CHECK_LAUNCH();
        dev_radix_sort(lk, nullptr, h[1], 64, s);
        k_keys_to_work<<<(unsigned)ceil_div(h[1], 256), 256, 0, s>>>(lk, h[1], wl);
        HH_CHECK_LAUNCH();
        int64_t* cpos = dev_alloc_t<int64_t>(N_CLASS_LIMITS, s);
        int32_t* cmx = dev_alloc_t<int32_t>(N_CLASS_LIMITS + 1, s);
        k_class_bounds<<<1, 32, 0, s>>>(lk, h[1], cpos, cmx);
        HH_CHECK_LAUNCH();
        int64_t hp[N_CLASS_LIMITS];
        int32_t hm[N_CLASS_LIMITS + 1];
        HH_CUDA(cudaMemcpyAsync(hp, cpos, sizeof hp, cudaMemcpyDeviceToHost, s));
        HH_CUDA(cudaMemcpyAsync(hm, cmx, sizeof hm, cudaMemcpyDeviceToHost, s));
        HH_CUDA(cudaStreamSynchronize(s));
        if (use_tc) {
            // the prefix of blocks with c + q > rounds_min_cq goes to the round engine
            int64_t* rpos = dev_alloc_t<int64_t>(RC_N + 1, s);
            int32_t* rmx = dev_alloc_t<int32_t>(RC_N + 1, s);
            k_round_classes<<<1, 32, 0, s>>>(lk, h[1], rpos, rmx, lc.rounds_min_cq);
            HH_CHECK_LAUNCH();
            int64_t hp2[RC_N + 1];
            HH_CUDA(cudaMemcpyAsync(hp2, rpos, sizeof hp2, cudaMemcpyDeviceToHost, s));
            HH_CUDA(cudaMemcpyAsync(rm, rmx, sizeof rm, cudaMemcpyDeviceToHost, s));
            HH_CUDA(cudaStreamSynchronize(s));
            n_rounds = hp2[RC_N];
            rb.assign(RC_N + 2, 0);
            for (int i = 0; i < RC_N; ++i) rb[i + 1] = std::min(hp2[i], n_rounds);
            rb[RC_N + 1] = n_rounds;
            dev_free(rpos, s);
            dev_free(rmx, s);
        }
        int64_t b0 = n_rounds;
        for (int i = 0; i <= N_CLASS_LIMITS; ++i) {
            const int64_t e = i < N_CLASS_LIMITS ? hp[i] : h[1];
            if (e > b0) cls.push_back(AcaClass{b0, e, std::min(hm[i == 0 ? 0 : i], b0 == n_rounds && n_rounds > 0
                                                                                        ? (int32_t)lc.rounds_min_cq
                                                                                        : hm[i == 0 ? 0 : i])});
            b0 = std::max(b0, e);
        }
        dev_free(cpos, s);
        dev_free(cmx, s);
        dev_free(lk, s);
    }
    // largest c + q of the small list: sizes the warp teams' factor workspaces
    int dims[1] = {0};
    if (h[0] > 0) {
        int* dmax = dev_alloc_t<int>(1, s);
        HH_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), s));
        k_max_dim<<<(unsigned)ceil_div(h[0], 256), 256, 0, s>>>(ws, h[0], bl->PG, t->nbeg, t->nend, dmax);
        HH_CHECK_LAUNCH();
        HH_CUDA(cudaMemcpyAsync(dims, dmax, sizeof dims, cudaMemcpyDeviceToHost, s));
        HH_CUDA(cudaStreamSynchronize(s));
        dev_free(dmax, s);
    }
    const int max_small_cq = dims[0];
    const int kind = kernel_kind(p, ctx->width);
    if constexpr (sizeof(R) == 4) {
        if (use_tc) {
            aca_tc_run(ctx, t, bl, p, r, ws, h[0], wl, cls.data(), (int)cls.size(), wl,
                       n_rounds > 0 ? rb.data() : nullptr, rm, n_rounds > 0 ? RC_N + 1 : 0, max_small_cq, s);
            dev_free(fs, s); dev_free(fl, s); dev_free(os, s); dev_free(ol, s); dev_free(key, s); dev_free(tot, s);
            dev_free(ws, s); dev_free(wl, s);
            return;
        }
    }
    if (kind == 0) launch_aca<R, 0>(ctx, p, A, ws, h[0], wl, cls, max_small_cq, lc, r.mode, s);
    else if (kind == 1) launch_aca<R, 1>(ctx, p, A, ws, h[0], wl, cls, max_small_cq, lc, r.mode, s);
    else launch_aca<R, 2>(ctx, p, A, ws, h[0], wl, cls, max_small_cq, lc, r.mode, s);
    dev_free(fs, s); dev_free(fl, s); dev_free(os, s); dev_free(ol, s); dev_free(key, s); dev_free(tot, s);
    dev_free(ws, s); dev_free(wl, s);
}

}  // namespace

void aca_run(hh_ctx* ctx, const hh_tree* t, const hh_blocks* b, const hh_params& p, const AcaRun& r, cudaStream_t s)
{
    if (p.precision == HH_FP64) aca_run_t<double>(ctx, t, b, p, r, s);
    else aca_run_t<float>(ctx, t, b, p, r, s);
}

void lowrank_apply(hh_ctx* ctx, const hh_hmat* h, const double* Fs, void* part, const int64_t* pofs, int transpose,
                   cudaStream_t s)
{
    (void)ctx;
    const int64_t nG = h->blocks->nG;
    if (nG == 0) return;
    const unsigned grid = (unsigned)ceil_div(nG, 4);
    if (h->real_bytes == 8)
        k_apply<double><<<grid, 128, 0, s>>>((const double*)h->factors, h->fofs, h->rank, h->blocks->PG, nG,
                                             h->tree->nbeg, h->tree->nend, Fs, (double*)part, pofs, transpose);
    else
        k_apply<float><<<grid, 128, 0, s>>>((const float*)h->factors, h->fofs, h->rank, h->blocks->PG, nG,
                                            h->tree->nbeg, h->tree->nend, Fs, (float*)part, pofs, transpose);
    HH_CHECK_LAUNCH();
}

// One admissible block, ACA fused with the low-rank apply, on caller-provided
// device memory (used by the allocation-free entry point): positions Xs
// [c+q, 3] (targets first), forces Fs [c+q, 3], the one-block lists PG / nbeg
// / nend / work / pofs, a zeroed work counter, the team workspace ws (one
// warp team; every warp of the launch shares it, only the one that takes the
// block touches it), the partial output part [c, 3] and rank[0].
void aca_single_block_ws(hh_ctx* ctx, const hh_params& p, int32_t c, int32_t q, const double* Xs, const double* Fs,
                         const int32_t* PG, const int32_t* nbeg, const int32_t* nend, const int32_t* work,
                         unsigned long long* counter, void* ws, void* part, const int64_t* pofs, int32_t* rank,
                         cudaStream_t s)
{
    HH_REQUIRE(c >= 1 && q >= 1 && c <= SMALL_MAX && q <= SMALL_MAX, HH_ERR_ARG, "block sides must be in [1, 512]");
    auto go = [&](auto tag) {
        using R = decltype(tag);
        AcaArgs<R> A{};
        A.Xs = Xs;
        A.th_g = theta_for<R>(ctx, p, &A.n_th);
        A.pp = PairParams{p.radius, p.viscosity};
        A.Fs = Fs;
        A.PG = PG;
        A.nbeg = nbeg;
        A.nend = nend;
        A.work = work;
        A.n_work = 1;
        A.counter = counter;
        A.max_rank = p.max_rank;
        A.eps2 = p.eps * p.eps;
        A.j1_rule = p.j1_rule;
        A.seed = p.seed;
        A.scratch = (R*)ws;
        A.team_stride = 0;
        A.rank = rank;
        A.part = (R*)part;
        A.pofs = pofs;
        A.status = ctx->d_status;
        A.n_queries = ctx->d_counters + 4;
        const size_t smem0 = WPB * sizeof(TeamSmem<R>) + (size_t)A.n_th * sizeof(R);
        const int kind = kernel_kind(p, ctx->width);
        const size_t act = kind == 2 ? 0 : (kind == 1 ? act_floats_per_warp<R, 1>() : act_floats_per_warp<R, 0>());
        const size_t smem = smem0 + sizeof(R) * act * WPB;
        auto launch = [&](auto kern) {
            HH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<1, 32 * WPB, smem, s>>>(A, 0);
            HH_CHECK_LAUNCH();
        };
        if (kind == 0) launch(k_aca_warp<R, 0>);
        else if (kind == 1) launch(k_aca_warp<R, 1>);
        else launch(k_aca_warp<R, 2>);
    };
    if (p.precision == HH_FP64) go(double{});
    else go(float{});
}
