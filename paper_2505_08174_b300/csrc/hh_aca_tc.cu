// hh_aca_tc.cu -- block ACA (Algorithm 2) with the on-demand rows and columns
// of G evaluated on the tensor cores (precision HH_BF16: MLP with BF16
// operands and FP32 accumulation, ACA arithmetic in FP32, pivot inverses and
// the norm recurrence in FP64).
//
// The rank loop is the one of hh_aca.cu (same pivot rules, stopping test and
// outputs); what changes is who evaluates the pair kernel.  A CTA has 128
// threads and one shared 128-row MLP tile (hh_tcmlp.cuh); every warp owns
// the tile rows of its TMEM quadrant (32w..32w+31) and runs the four MLP
// layers for them on its own: it writes one query per lane (a separation
// x_m - x_n of the column or row being generated), issues the MMAs into its
// own TMEM columns, waits on its own mbarrier and reads back its lanes.  No
// warp waits for another while queries are evaluated.  Teams:
//   * warp teams (blocks with c, q <= small_max): 4 teams per CTA, each takes
//     32 consecutive rows or columns of its current block per round;
//   * one CTA team (larger blocks): the 4 warps share one block, 128 rows or
//     columns per round, and meet only at the end of each pass.
// A team whose pass is complete does its pivot / Gram / stopping work before
// its next round.
//
// Launches: one warp-team launch over the small blocks on the caller's
// stream, and one CTA-team launch per size class of the large blocks on the
// context's second stream, forked from and joined back to the caller's
// stream by events.  The two run concurrently, so the serial tails of the
// few largest blocks overlap with the bulk of the small ones.  Each block
// writes its own outputs, and each launch has its own work counter.
#include <algorithm>

#include "hh_aca.cuh"
#include "hh_tcmlp.cuh"

namespace {

template <int W, class Team, int MR>
struct alignas(128) AcaTcSmem {
    TcCore<W> tc;
    TeamSmem<float, MR> team[TC_T / Team::SIZE];
    int blk[TC_T / Team::SIZE];
    uint64_t mbw[4];      // warp teams: one MMA barrier per warp
    uint32_t pend[4];
    int failw[4];
};

// TMEM columns of a CTA: one W-column accumulator per warp.
template <int W>
__host__ __device__ constexpr uint32_t aca_tmem_cols() { return W <= 32 ? 128u : 256u; }

template <int W, class S>
__device__ void aca_tc_setup(S& sm, const float* th, const unsigned* status)
{
    tc_load_weights<W>(sm.tc, th);
    if (threadIdx.x == 0) {
        for (int w = 0; w < 4; ++w) { mbar_init(&sm.mbw[w], 1); sm.failw[w] = 0; }
        sm.tc.stall_polls = tc_stall_polls(status);
        mbar_init(&sm.tc.stall, 1);
    }
    if (threadIdx.x < 32) {
        tmem_alloc(&sm.tc.tmem, aca_tmem_cols<W>());
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

template <int W, class S>
__device__ void aca_tc_teardown(S& sm)
{
    tc_fence_before();
    __syncthreads();
    // a warp that timed out gives its MMA group one more bounded wait before
    // the accumulator columns are released
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0 && sm.failw[w]) mbar_wait_bounded(&sm.mbw[w], sm.pend[w], TC_WAIT_LIMIT);
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(sm.tc.tmem, aca_tmem_cols<W>());
}

template <int W, class Team, int MR>
__global__ void __launch_bounds__(TC_T, 4) k_aca_tc(AcaArgs<float> A, const float* __restrict__ th_packed, int mode)
{
    constexpr int NT = TC_T / Team::SIZE;
    constexpr int SIZE = Team::SIZE, ROWS = Team::ROWS;
    constexpr bool REG = Team::REG_FLAGS;
    constexpr bool CTA = NT == 1;   // one 128-thread team per CTA, else 4 warp teams
    extern __shared__ __align__(128) unsigned char smem_raw[];
    AcaTcSmem<W, Team, MR>& S = *reinterpret_cast<AcaTcSmem<W, Team, MR>*>(smem_raw);
    aca_tc_setup<W>(S, th_packed, A.status);
    const Team tm;
    const int team = threadIdx.x / SIZE;
    const int tid = tm.tid();
    TeamSmem<float, MR>& sm = S.team[team];
    float* const ws = A.scratch + ((int64_t)blockIdx.x * NT + team) * A.team_stride;
    const float a = (float)A.pp.a;
    const int warp = threadIdx.x >> 5;   // TMEM quadrant, accumulator columns and mbarrier of this warp
    TcWarp tw{S.tc.tmem + (uint32_t)(W * warp), &S.mbw[warp], 0u, &S.failw[warp], &S.pend[warp],
              &S.tc.stall, S.tc.stall_polls};

    // state of the team's current block (uniform over the team; lam2 is
    // maintained by thread 0 only)
    int64_t b = -1;
    bool exhausted = false;
    bool failed = false;
    int32_t t0 = 0, c = 0, s0 = 0, q = 0;
    int kmax = 0, k = 0, pass = 0, x0 = 0, j = 0, bi = -1;
    double lam2 = 0.0;
    float best = -1.f;
    int barg = -1;
    float snu = 0.f, scr = 0.f;      // stopping-test terms of the current row pass
    uint32_t usedR = 0, usedC = 0;   // warp team: bit i <-> row / column tid + 32 i
    float* Cs = ws;
    float* Qs = ws;
    uint8_t* fR = nullptr;           // CTA team: flag bytes after the factors
    uint8_t* fC = nullptr;

    auto is_used = [&](uint32_t u, const uint8_t* f, int i, int x) -> bool {
        if constexpr (REG) return (u >> i) & 1u;
        else return f[x] != 0;
    };
    auto set_used = [&](uint32_t& u, uint8_t* f, int x) {
        if constexpr (REG) {
            if (x % SIZE == tid) u |= 1u << (x / SIZE);
        } else {
            if (tid == 0) f[x] = 1;
        }
    };
    // rank, pivots, counters and the block's output (fused apply or factors)
    auto finish = [&](int l, bool capped) {
        if (tid == 0) {
            if (A.rank) A.rank[b] = l;
            if (A.pivI)
                for (int p = l; p < A.max_rank; ++p) { A.pivI[b * A.max_rank + p] = -1; A.pivJ[b * A.max_rank + p] = -1; }
            if (capped) atomicOr(A.status, (unsigned)HH_DEV_RANK_CAP);
            atomicAdd(A.n_queries, (unsigned long long)(c + q) * (unsigned long long)l);
        }
        if (mode == 0) {
            const int lane = threadIdx.x & 31;
            for (int p = tm.warp(); p < l; p += Team::NW) {
                const float* Qp = Qs + (int64_t)p * 9 * q;
                float a0 = 0.f, a1 = 0.f, a2 = 0.f;
                for (int n = lane; n < q; n += 32) {
                    float qv[9];
                    ld9(Qp, q, n, qv);
                    const double* f = A.Fs + 3 * (int64_t)(s0 + n);
                    const float f0 = (float)f[0], f1 = (float)f[1], f2 = (float)f[2];
                    a0 += qv[0] * f0 + qv[1] * f1 + qv[2] * f2;
                    a1 += qv[3] * f0 + qv[4] * f1 + qv[5] * f2;
                    a2 += qv[6] * f0 + qv[7] * f1 + qv[8] * f2;
                }
                a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2);
                if (lane == 0) { sm.tv[3 * p] = a0; sm.tv[3 * p + 1] = a1; sm.tv[3 * p + 2] = a2; }
            }
            tm.sync();
            float* out = A.part + 3 * (A.pofs[b] - A.pofs_base);
            for (int m = tid; m < c; m += SIZE) {
                float y0 = 0.f, y1 = 0.f, y2 = 0.f;
                for (int p = 0; p < l; ++p) {
                    float cv[9];
                    ld9(Cs + (int64_t)p * 9 * c, c, m, cv);
                    const float* tp = sm.tv + 3 * p;
                    y0 += cv[0] * tp[0] + cv[1] * tp[1] + cv[2] * tp[2];
                    y1 += cv[3] * tp[0] + cv[4] * tp[1] + cv[5] * tp[2];
                    y2 += cv[6] * tp[0] + cv[7] * tp[1] + cv[8] * tp[2];
                }
                out[3 * m] = y0; out[3 * m + 1] = y1; out[3 * m + 2] = y2;
            }
        } else if (mode == 2) {
            float* dst = A.fac + 9 * (A.fofs[b] - A.fofs_base);
            const int64_t nc = (int64_t)l * 9 * c, nq = (int64_t)l * 9 * q;
            for (int64_t x = tid; x < nc; x += SIZE) dst[x] = Cs[x];
            for (int64_t x = tid; x < nq; x += SIZE) dst[nc + x] = Qs[x];
        }
        tm.sync();
        b = -1;
    };

    for (;;) {
        // ---- take the next block when idle
        if (b < 0 && !exhausted) {
            if (tid == 0) {
                const unsigned long long w = atomicAdd(A.counter, 1ull);
                S.blk[team] = w < (unsigned long long)A.n_work ? A.work[w] : -1;
            }
            tm.sync();
            const int nb = S.blk[team];
            tm.sync();
            if (nb < 0) {
                exhausted = true;
            } else {
                b = nb;
                const int32_t tt = A.PG[2 * b], ss = A.PG[2 * b + 1];
                t0 = A.nbeg[tt]; c = A.nend[tt] - t0;
                s0 = A.nbeg[ss]; q = A.nend[ss] - s0;
                kmax = min(min(c, q), A.max_rank);
                Cs = ws;
                Qs = ws + (int64_t)kmax * 9 * c;
                usedR = usedC = 0;
                if constexpr (!REG) {
                    fR = reinterpret_cast<uint8_t*>(Qs + (int64_t)kmax * 9 * q);
                    fC = fR + c;
                    for (int x = tid; x < c + q; x += SIZE) fR[x] = 0;
                    tm.sync();
                }
                j = j1_of(A.j1_rule, A.seed, tt, ss, q);
                set_used(usedC, fC, j);
                k = 0; pass = 0; x0 = 0; bi = -1;
                lam2 = 0.0;
                best = -1.f; barg = -1;
                tm.sync();
            }
        }
        // ---- this thread's query: row x of the column residual (pass 0) or
        // column x of the row residual (pass 1)
        const int nx = pass == 0 ? c : q;
        const int x = x0 + tid;
        const bool valid = b >= 0 && x < nx;
        float f[4], id = 1.f;
        if (valid) {
            float rx, ry, rz;
            sep_split(A.Xp, pass == 0 ? t0 + x : t0 + bi, pass == 0 ? s0 + j : s0 + x, rx, ry, rz);
            features(rx, ry, rz, a, f, id);
        } else {
            f[0] = 1.f; f[1] = f[2] = 0.f; f[3] = a;
        }
        // the residual update below reads element e of C_p (Q_p) for the team's
        // rows x0 .. x0 + SIZE - 1 and every p < k: request those lines into
        // L2 now, so the loads find them there after the MLP chain
        if (b >= 0 && k > 0) {
            const int lane = threadIdx.x & 31;
            const float* fac0 = pass == 0 ? Cs : Qs;
            const int x1 = min(x0 + SIZE, nx) - 1;
            const int wbase = x0 + (tid & ~31);            // this warp's first row
            if (wbase <= x1) {
                const int wlast = min(wbase + 31, x1);
                for (int idx = lane; idx < 18 * k; idx += 32) {
                    const int pe = idx >> 1;
                    const float* a = fac0 + (int64_t)pe * nx + ((idx & 1) ? wlast : wbase);
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                }
            }
        }
        float o[6];
        if (exhausted) break;   // uniform over the team
        // warps without a valid row skip the chain; a warp whose chain timed
        // out stops issuing MMAs (a CTA team leaves at the end of the pass)
        if (!failed && __any_sync(0xffffffffu, valid)) {
            tc_write_features<W>(S.tc, threadIdx.x, f);
            if (!tcw_mlp_rows<W>(S.tc, tw, A.status, o)) failed = true;
        }
        if constexpr (!CTA) {
            if (failed) break;
        }
        // ---- residual entry, stored in the factor being extended
        if (valid) {
            float K[9];
            K[0] = o[0] * id; K[1] = o[3] * id; K[2] = o[4] * id;
            K[3] = o[3] * id; K[4] = o[1] * id; K[5] = o[5] * id;
            K[6] = o[4] * id; K[7] = o[5] * id; K[8] = o[2] * id;
            float* fac = pass == 0 ? Cs : Qs;
            const float* piv = pass == 0 ? sm.qj : sm.ci;
            float V[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int p = 0; p < k; ++p) {
                float v[9], t9[9];
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
            st9(fac + (int64_t)k * 9 * nx, nx, x, K);
            const int i = x0 / SIZE;
            const bool used = pass == 0 ? is_used(usedR, fR, i, x) : is_used(usedC, fC, i, x);
            if (!used) {
                const float v = fro2(K);
                if (v > best) { best = v; barg = x; }
            }
        }
        x0 += SIZE;
        if (b < 0 || x0 < nx) continue;

        // ---- end of a pass (team-uniform)
        if constexpr (CTA) {
            if (__syncthreads_or(failed)) break;
        } else {
            tm.sync();
        }
        if (pass == 0) {
            tm.argmax(best, barg, sm);
            if (barg < 0 || !(best > 0.f)) { finish(k, false); continue; }
            bi = barg;
            tm.sync();
            if (tid == 0) {
                double P[9], Pi[9];
#pragma unroll
                for (int e = 0; e < 9; ++e) P[e] = (double)Cs[((int64_t)k * 9 + e) * c + bi];
                if (k == 0) sm.pscale = sqrt(fro2(P));
                double det;
                const int kept = inv3_floor(P, PIVOT_FLOOR_BF16 * sm.pscale, Pi, &det);
                const double rc = kept == 3 ? 1.0 / sqrt(fro2(P) * fro2(Pi)) : 1.0;
                const int bad = kept == 0 ? 2 : (!(rc >= 1e-10) ? 1 : 0);
                sm.flag = bad;
                if (!bad)
#pragma unroll
                    for (int e = 0; e < 9; ++e) sm.Pi[e] = (float)Pi[e];
            }
            tm.sync();
            if (sm.flag == 2) { finish(k, false); continue; }   // the pivot element is rounding noise
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
                    const double dv = fabs(det3d(P));
                    if (dv > bd) { bd = dv; bdi = m; }
                }
                tm.argmax(bd, bdi, sm);
                if (bdi < 0) { finish(k, false); continue; }
                bi = bdi;
                if (tid == 0) {
                    double P[9], Pi[9];
#pragma unroll
                    for (int e = 0; e < 9; ++e) P[e] = (double)Cs[((int64_t)k * 9 + e) * c + bi];
                    inv3d(P, Pi);
#pragma unroll
                    for (int e = 0; e < 9; ++e) sm.Pi[e] = (float)Pi[e];
                }
                tm.sync();
            }
            set_used(usedR, fR, bi);
            if (tid == 0 && A.pivI) {
                A.pivI[b * A.max_rank + k] = bi;
                A.pivJ[b * A.max_rank + k] = j;
            }
            // c_k <- c_k [c_k(i_k)]^-1
            float Pi[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) Pi[e] = sm.Pi[e];
            float* line = Cs + (int64_t)k * 9 * c;
            for (int m = tid; m < c; m += SIZE) {
                float r[9], o9[9];
                ld9(line, c, m, r);
                mm3(r, Pi, o9);
                st9(line, c, m, o9);
            }
            tm.sync();
            gram_cols<float>(tm, sm, Cs, c, k);
            pass = 1; x0 = 0; best = -1.f; barg = -1; snu = 0.f; scr = 0.f;
            for (int idx = tid; idx < k * 9; idx += SIZE) sm.ci[idx] = Cs[(int64_t)idx * c + bi];
            tm.sync();
        } else {
            tm.argmax(best, barg, sm);
            const int bj = barg;
            tm.sync();
            double nu2, cross;
            team_sum2(tm, sm, snu, scr, nu2, cross);
            if (tid == 0) {
                lam2 = lam2 + nu2 + 2.0 * cross;
                sm.stop = (nu2 <= A.eps2 * lam2) || (bj < 0);
            }
            tm.sync();
            ++k;
            const bool stop = sm.stop;
            tm.sync();
            if (stop) { finish(k, false); continue; }
            if (k == kmax) { finish(k, (k == A.max_rank) && (k < min(c, q))); continue; }
            j = bj;
            set_used(usedC, fC, j);
            pass = 0; x0 = 0; best = -1.f; barg = -1;
            for (int idx = tid; idx < k * 9; idx += SIZE) sm.qj[idx] = Qs[(int64_t)idx * q + j];
            tm.sync();
        }
    }
    aca_tc_teardown<W>(S);
}

template <int W, class Team, int MR>
void launch_tc_mr(hh_ctx* ctx, const AcaArgs<float>& A, int64_t grid, int mode, cudaStream_t s)
{
    const size_t smem = sizeof(AcaTcSmem<W, Team, MR>) + 128;
    HH_CUDA(cudaFuncSetAttribute(k_aca_tc<W, Team, MR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_aca_tc<W, Team, MR><<<(unsigned)grid, TC_T, smem, s>>>(A, ctx->theta32, mode);
    HH_CHECK_LAUNCH();
}

// Shared state sized for max_rank <= 48 (the default) when possible: it
// keeps a CTA under 56 KB, so four CTAs share an SM.
template <int W, class Team>
void launch_tc(hh_ctx* ctx, const AcaArgs<float>& A, int64_t grid, int mode, cudaStream_t s)
{
    if (A.max_rank <= 48) launch_tc_mr<W, Team, 48>(ctx, A, grid, mode, s);
    else launch_tc_mr<W, Team, MAXR>(ctx, A, grid, mode, s);
}

}  // namespace

// Tensor-core ACA over the classified work lists, on three streams at once:
// small blocks on warp teams (caller's stream), mid-size blocks on CTA teams
// by size class (second stream), and the largest blocks through the round
// engine of hh_aca_rounds.cu (third stream; its host loop runs last, so the
// other two lists are already queued).  Both extra streams are forked from
// and joined back to the caller's stream by events.
void aca_tc_run(hh_ctx* ctx, const hh_tree* t, const hh_blocks* bl, const hh_params& p, const AcaRun& r,
                const int32_t* work_small, int64_t n_small, const int32_t* work_large, const AcaClass* cls,
                int n_cls, const int32_t* work_rounds, const int64_t* rcls_begin, const int32_t* rcls_max_cq,
                int n_rcls, int max_small_cq, cudaStream_t s)
{
    HH_REQUIRE(p.kernel == HH_MLP && p.precision == HH_BF16, HH_ERR_ARG, "tensor-core ACA needs the BF16 MLP kernel");
    const int mr = std::min(p.max_rank, MAXR);
    const hh_launch_cfg lc = resolved_launch(ctx, true);
    AcaArgs<float> A = make_aca_args<float>(ctx, t, bl, p, r);
    const int64_t n_rounds = n_rcls > 0 ? rcls_begin[n_rcls] : 0;
    HH_CUDA(cudaEventRecord(ctx->kev[2], s));
    HH_CUDA(cudaEventRecord(ctx->fork_ev, s));
    const cudaStream_t sl = n_cls > 0 ? ctx->aux : s;
    const cudaStream_t sr = n_rounds > 0 ? ctx->aux2 : s;
    if (n_cls > 0) HH_CUDA(cudaStreamWaitEvent(sl, ctx->fork_ev, 0));
    if (n_rounds > 0) HH_CUDA(cudaStreamWaitEvent(sr, ctx->fork_ev, 0));
    // joins the extra streams back even when an error unwinds from here, so
    // the caller's stream-ordered frees never overtake a launch still in flight
    struct Join {
        cudaStream_t from, into;
        cudaEvent_t ev;
        bool on;
        void now()
        {
            if (!on) return;
            on = false;
            HH_CUDA(cudaEventRecord(ev, from));
            HH_CUDA(cudaStreamWaitEvent(into, ev, 0));
        }
        ~Join()
        {
            if (on && cudaEventRecord(ev, from) == cudaSuccess) (void)cudaStreamWaitEvent(into, ev, 0);
        }
    } join_l{sl, s, ctx->join_ev, n_cls > 0}, join_r{sr, s, ctx->join2_ev, n_rounds > 0};
    if (n_small > 0) {
        constexpr int NT = TC_T / 32;
        int64_t stride = (int64_t)std::min(max_small_cq, 2 * SMALL_MAX) * 9 * mr;
        stride = ceil_div(stride * (int64_t)sizeof(float), 256) * 256 / (int64_t)sizeof(float);
        int64_t blocks = std::min<int64_t>(ceil_div(n_small, NT), (int64_t)lc.aca_small_cps * ctx->n_sm);
        blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, budget_warp_teams(p) / (stride * NT * (int64_t)sizeof(float))));
        float* scratch = dev_alloc_t<float>(stride * blocks * NT, s);
        HH_CUDA(cudaMemsetAsync(A.counter + 1, 0, sizeof(unsigned long long), s));
        AcaArgs<float> B = A;
        B.work = work_small;
        B.n_work = n_small;
        B.counter = A.counter + 1;
        B.scratch = scratch;
        B.team_stride = stride;
        if (ctx->width == 32) launch_tc<32, WarpTeam>(ctx, B, blocks, r.mode, s);
        else launch_tc<64, WarpTeam>(ctx, B, blocks, r.mode, s);
        dev_free(scratch, s);
    }
    for (int i = 0; i < n_cls; ++i) {
        const AcaClass& k = cls[i];
        int64_t stride = (int64_t)k.max_cq * 9 * mr + ceil_div(k.max_cq, (int64_t)sizeof(float));
        stride = ceil_div(stride * (int64_t)sizeof(float), 256) * 256 / (int64_t)sizeof(float);
        const int64_t budget = budget_cta_teams(p);
        int64_t teams = std::min<int64_t>(k.end - k.begin, (int64_t)lc.aca_large_cps * ctx->n_sm);
        teams = std::max<int64_t>(1, std::min<int64_t>(teams, budget / (stride * (int64_t)sizeof(float))));
        float* scratch = dev_alloc_t<float>(stride * teams, sl);
        HH_CUDA(cudaMemsetAsync(A.counter, 0, sizeof(unsigned long long), sl));
        AcaArgs<float> B = A;
        B.work = work_large + k.begin;
        B.n_work = k.end - k.begin;
        B.scratch = scratch;
        B.team_stride = stride;
        if (ctx->width == 32) launch_tc<32, CtaTeamT<TC_T>>(ctx, B, teams, r.mode, sl);
        else launch_tc<64, CtaTeamT<TC_T>>(ctx, B, teams, r.mode, sl);
        dev_free(scratch, sl);
    }
    if (n_rounds > 0) aca_rounds_run(ctx, t, bl, p, r, work_rounds, rcls_begin, rcls_max_cq, n_rcls, sr, false);
    join_l.now();
    join_r.now();
    HH_CUDA(cudaEventRecord(ctx->kev[3], s));
    ctx->kev_aca_used |= 2;
}
