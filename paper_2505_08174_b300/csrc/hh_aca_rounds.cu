// hh_aca_rounds.cu -- block ACA (Algorithm 2) for precision HH_BF16 as a
// sequence of rounds over many blocks at once, the pair kernel of every
// generated row and column evaluated on the tensor cores (hh_tcmlp.cuh: MLP
// with BF16 hi/lo operands and FP32 accumulation), ACA arithmetic in FP32,
// pivot inverses and the norm recurrence in FP64.
//
// The paper runs each line of Algorithm 2 as one parallel loop over all
// blocks of a query group (Section 3.3).  Here a bounded set of active
// blocks ("slots", sized by a memory budget) advances one phase per round.
// A block's phase is cut into 32-row segments:
//   COL   rows m of tau: column residual c_k(m) = G(m, j_k) -
//         sum_{p<k} C_p(m) Q_p(j_k) (one pair-kernel query per row), and the
//         Frobenius argmax over unused rows (packed-key atomicMax);
//   GRAM  rows of tau: c_k <- c_k [c_k(i_k)]^-1 and the segment's Gram sums
//         A_pk = sum_m C_p(m)^T C_k(m), p <= k;
//   ROW   columns n of sigma: row residual q_k(n) = G(i_k, n) -
//         sum_{p<k} C_p(i_k) Q_p(n), the segment's Gram sums B_kp =
//         sum_n q_k(n) Q_p(n)^T, p <= k, the apply sums t_k = sum_n q_k(n)
//         F(n), and the argmax over unused columns;
//   OUT   (fused apply) y(m) = sum_p C_p(m) t_p into the block's partial
//         output, or (stored factors) the copy of C and Q;
// a block's GRAM and ROW segments run in the same round.  A round is three
// launches:
//   * the tile kernel.  COL and ROW segments (they need the pair kernel) are
//     packed four to a 128-row tensor-core tile -- segments of different
//     blocks share one MMA chain, so small blocks do not leave most tile
//     rows idle -- and each warp then finishes its own segment; GRAM and OUT
//     segments run warp by warp;
//   * the pivot kernel, one thread per slot: the pivot row and its FP64
//     inverse after a column pass (FP64 work 32 slots to a warp instruction);
//   * the step kernel, one warp per slot (a CTA per slot for classes of large
//     blocks): the largest-|det| guard when the pivot is singular or
//     ill-conditioned, the stopping test nu^2 = tr(A_kk B_kk), lambda^2 +=
//     nu^2 + 2 sum_{p<k} tr(A_pk B_kp) (Eq. 10; segment sums added in segment
//     order, the traces in FP32, the lambda^2 recurrence in FP64) and the next
//     column, admission of the next block into a freed slot; the slots of a
//     CTA append the segments of their next phase with one atomic per list.
// Blocks are admitted largest first in size classes (c + q in (2^e,
// 2^(e+1)]), each class with the number of slots its largest block allows
// within the budget.  Every reduction runs in a fixed order and the argmaxes
// are exact, so results do not depend on which slot, round, tile or warp ran
// a block.
#include <algorithm>
#include <vector>

#include "hh_aca.cuh"
#include "hh_tcmlp.cuh"

namespace {

enum : int32_t { PH_FREE = 0, PH_COL = 1, PH_GR = 2, PH_OUT = 3 };
enum : int32_t { TK_COL = 0, TK_GRAM = 1, TK_ROW = 2, TK_OUT = 3 };
enum : int32_t { LIST_MLP = 0, LIST_PLAIN = 1 };
constexpr int RT = 32;                  // rows per segment = one warp
constexpr int SLOTS_MAX = 65536;
constexpr int STEP_WARPS = 8;           // slots per step CTA

// Per-slot state, structure of arrays.
struct Slots {
    int32_t* blk;
    int32_t* t0;
    int32_t* c;
    int32_t* s0;
    int32_t* q;
    int32_t* kmax;
    int32_t* k;
    int32_t* phase;
    int32_t* ib;       // i_k
    int32_t* jb;       // j_k
    int32_t* pivst;    // pivot status after a column pass (k_round_pivots)
    double* lam2;
    double* pscale;    // Frobenius norm of the block's first pivot element
    unsigned long long* key;   // argmax of the running pass: (value bits << 32) | ~index
    float* Pi;         // [S][9] pivot inverse of the current column
    float* piv;        // [S][9 MR]: Q_p(j_k) (for COL) or C_p(i_k) (for ROW), p < k
    float* tv;         // [S][3 MR]: t_p = sum_n Q_p(n) F(n)
};

// One segment of a round: the slot's fields at the time it was listed.
struct alignas(16) Seg {
    int32_t s, kind_ti, t0, c, s0, q, k, kmax, ib, jb, blk, pad;
};

struct RoundArgs {
    const float* Xp;
    const double* Fs;
    float a;
    const int32_t* PG;
    const int32_t* nbeg;
    const int32_t* nend;
    const int32_t* work;       // this class's blocks
    int64_t n_work;
    unsigned long long* next;  // admission counter
    int S;
    int MR;                    // rank bound of the staging arrays (= max_rank)
    int64_t stride;            // floats per slot workspace
    float* ws;
    Slots st;
    Seg* list[2][2];           // segments of round r: list[r & 1][LIST_MLP / LIST_PLAIN]
    unsigned* cnt;             // [3][2]: segments of round r in cnt[2 (r % 3) + list]
    int round;
    int max_rank;
    double eps2;
    int j1_rule;
    uint64_t seed;
    int mode;                  // 0 fused apply, 1 pivots only, 2 store factors
    int32_t* rank;
    int32_t* pivI;
    int32_t* pivJ;
    float* part;
    const int64_t* pofs;
    int64_t pofs_base;         // block b's partial output at part + 3 * (pofs[b] - pofs_base)
    float* fac;
    const int64_t* fofs;
    int64_t fofs_base;
    unsigned* status;
    unsigned long long* n_queries;
};

__host__ __device__ inline int tiles_of(int n) { return (n + RT - 1) / RT; }

// Layout of one slot's workspace (floats): C lines [kmax][9][c], Q lines
// [kmax][9][q], used flags (c + q bytes), GRAM partials [ntc][9 kmax], ROW
// partials [ntq][9 kmax + 4] (B_kp, then t_k), one entry per 32-row segment.
struct SlotLayout {
    int64_t offQ, offF, offG, offR, rstride, total;
};
__host__ __device__ inline SlotLayout slot_layout(int64_t c, int64_t q, int64_t kmax)
{
    SlotLayout L;
    L.offQ = kmax * 9 * c;
    L.offF = L.offQ + kmax * 9 * q;
    const int64_t ntc = (c + RT - 1) / RT, ntq = (q + RT - 1) / RT;
    L.offG = L.offF + (c + q + 15) / 16 * 4;
    L.offR = L.offG + ntc * 9 * kmax;
    L.rstride = (9 * kmax + 4 + 3) / 4 * 4;
    L.total = (L.offR + ntq * L.rstride + 63) / 64 * 64;   // 256-byte slots
    return L;
}

__device__ __forceinline__ unsigned long long pack_key(float v, int idx)
{
    return ((unsigned long long)__float_as_uint(v) << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)idx);
}
__device__ __forceinline__ void unpack_key(unsigned long long key, float& v, int& idx)
{
    if (key == 0ull) { v = -1.f; idx = -1; return; }
    v = __uint_as_float((uint32_t)(key >> 32));
    idx = (int)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// L2 prefetch of lines 0 .. np-1 of a component-major factor ([np][9][n]) for
// the segment rows x0 .. x0 + 31 (the loads after the MLP chain then hit L2).
__device__ __forceinline__ void prefetch_seg_lines(const float* fac, int n, int x0, int np, int lane)
{
    const int last = min(RT, n - x0) - 1;
    for (int i = lane; i < 18 * np; i += 32) {
        const int pe = i >> 1;
        prefetch_l2(fac + (int64_t)pe * n + x0 + ((i & 1) ? last : 0));
    }
}

// Sum over the warp's 32 rows of up to 27 per-lane values (acc[0..26]); lanes
// 0 .. n_out - 1 store them to out.
__device__ __forceinline__ void warp_sum27_store(float (&acc)[32], float* out, int n_out, int lane)
{
    const float w = warp_transpose_sum32<float>(acc);
    if (lane < n_out) out[lane] = w;
}

// The segment's fields, read by lanes 0..11 and broadcast.
struct SegView {
    int s, kind, ti, t0, c, s0, q, k, kmax, bi, bj;
    int64_t b;
};
__device__ __forceinline__ SegView load_seg(const Seg* e, int lane)
{
    int f = 0;
    if (lane < 12) f = reinterpret_cast<const int32_t*>(e)[lane];
    SegView v;
    v.s = __shfl_sync(0xffffffffu, f, 0);
    const int kt = __shfl_sync(0xffffffffu, f, 1);
    v.kind = kt >> 28;
    v.ti = kt & 0x0FFFFFFF;
    v.t0 = __shfl_sync(0xffffffffu, f, 2);
    v.c = __shfl_sync(0xffffffffu, f, 3);
    v.s0 = __shfl_sync(0xffffffffu, f, 4);
    v.q = __shfl_sync(0xffffffffu, f, 5);
    v.k = __shfl_sync(0xffffffffu, f, 6);
    v.kmax = __shfl_sync(0xffffffffu, f, 7);
    v.bi = __shfl_sync(0xffffffffu, f, 8);
    v.bj = __shfl_sync(0xffffffffu, f, 9);
    v.b = __shfl_sync(0xffffffffu, f, 10);
    return v;
}

// ---- the tile kernel ---------------------------------------------------------------
template <int W>
struct alignas(128) TileSmem {
    TcCore<W> tc;             // A1 / AH tiles (warp w owns rows 32w .. 32w + 31) and weights
    float piv[4][9 * MAXR];   // per warp: Q_p(j_k), C_p(i_k) or t_p of its segment
};

// The rest of a COL or ROW segment after the pair kernel: residual, factor
// line, argmax key, and (ROW) the B_kp and t_k sums of the segment.
__device__ __forceinline__ void finish_query_seg(const RoundArgs& R, const SegView& g, const float* pv,
                                                 const float o[6], float id, bool valid, int lane)
{
    const Slots& S = R.st;
    const bool col = g.kind == TK_COL;
    const SlotLayout L = slot_layout(g.c, g.q, g.kmax);
    float* const ws = R.ws + (int64_t)g.s * R.stride;
    float* const Qs = ws + L.offQ;
    float* const fac = col ? ws : Qs;
    const int nx = col ? g.c : g.q;
    const int x = g.ti * RT + lane;
    const int k = g.k;
    float K[9];
    unsigned long long key = 0ull;
    if (valid) {
        K[0] = o[0] * id; K[1] = o[3] * id; K[2] = o[4] * id;
        K[3] = o[3] * id; K[4] = o[1] * id; K[5] = o[5] * id;
        K[6] = o[4] * id; K[7] = o[5] * id; K[8] = o[2] * id;
        // residual: four earlier factor lines in flight at a time
        for (int p0 = 0; p0 < k; p0 += 4) {
            float v[4][9];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (p0 + u < k) ld9(fac + (int64_t)(p0 + u) * 9 * nx, nx, x, v[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (p0 + u < k) {
                    float t9[9];
                    if (col) mm3(v[u], pv + 9 * (p0 + u), t9);   // C_p(m) Q_p(j_k)
                    else mm3(pv + 9 * (p0 + u), v[u], t9);       // C_p(i_k) Q_p(n)
#pragma unroll
                    for (int e9 = 0; e9 < 9; ++e9) K[e9] -= t9[e9];
                }
            }
        }
        st9(fac + (int64_t)k * 9 * nx, nx, x, K);
        const uint8_t* used = reinterpret_cast<const uint8_t*>(ws + L.offF) + (col ? 0 : g.c);
        if (!used[x]) {
            const float v = fro2(K);
            if (v == v) key = pack_key(v, x);
        }
    } else {
#pragma unroll
        for (int e9 = 0; e9 < 9; ++e9) K[e9] = 0.f;
    }
    key = warp_max_u64(key);
    if (lane == 0 && key) atomicMax(&S.key[g.s], key);
    if (col) return;
    // B_kp = sum_n q_k(n) Q_p(n)^T (p <= k), then t_k
    float* rp = ws + L.offR + (int64_t)g.ti * L.rstride;
    for (int p0 = 0; p0 <= k; p0 += 3) {
        float acc[32];
#pragma unroll
        for (int e9 = 0; e9 < 32; ++e9) acc[e9] = 0.f;
        if (valid) {
#pragma unroll
            for (int gg = 0; gg < 3; ++gg) {
                const int p = p0 + gg;
                if (p <= k) {
                    float qp[9];
                    if (p == k) {
#pragma unroll
                        for (int e9 = 0; e9 < 9; ++e9) qp[e9] = K[e9];
                    } else {
                        ld9(Qs + (int64_t)p * 9 * g.q, g.q, x, qp);
                    }
#pragma unroll
                    for (int u = 0; u < 3; ++u)
#pragma unroll
                        for (int v = 0; v < 3; ++v)
                            acc[9 * gg + 3 * u + v] =
                                K[3 * u] * qp[3 * v] + K[3 * u + 1] * qp[3 * v + 1] + K[3 * u + 2] * qp[3 * v + 2];
                }
            }
        }
        warp_sum27_store(acc, rp + 9 * p0, min(27, 9 * (k + 1 - p0)), lane);
    }
    float u0 = 0.f, u1 = 0.f, u2 = 0.f;
    if (valid && R.mode == 0) {   // apply sums (the other modes have no forces)
        const double* fp = R.Fs + 3 * (int64_t)(g.s0 + x);
        const float f0 = (float)fp[0], f1 = (float)fp[1], f2 = (float)fp[2];
        u0 = K[0] * f0 + K[1] * f1 + K[2] * f2;
        u1 = K[3] * f0 + K[4] * f1 + K[5] * f2;
        u2 = K[6] * f0 + K[7] * f1 + K[8] * f2;
    }
    u0 = warp_sum(u0); u1 = warp_sum(u1); u2 = warp_sum(u2);
    if (lane == 0) { rp[9 * g.kmax] = u0; rp[9 * g.kmax + 1] = u1; rp[9 * g.kmax + 2] = u2; }
}

// A GRAM or OUT segment (no pair kernel), one warp.
__device__ __forceinline__ void plain_seg(const RoundArgs& R, const SegView& g, float* pv, int lane)
{
    const Slots& S = R.st;
    const SlotLayout L = slot_layout(g.c, g.q, g.kmax);
    float* const ws = R.ws + (int64_t)g.s * R.stride;
    float* const Cs = ws;
    float* const Qs = ws + L.offQ;
    const int c = g.c, q = g.q, k = g.k;
    const int x0 = g.ti * RT, x = x0 + lane;
    if (g.kind == TK_GRAM) {
        // c_k <- c_k Pi, then A_pk = sum over the segment's rows of C_p(m)^T C_k(m), p <= k
        const float pi = lane < 9 ? S.Pi[(int64_t)g.s * 9 + lane] : 0.f;
        float Pi[9];
#pragma unroll
        for (int e9 = 0; e9 < 9; ++e9) Pi[e9] = __shfl_sync(0xffffffffu, pi, e9);
        prefetch_seg_lines(Cs, c, x0, k, lane);
        const bool valid = x < c;
        float ck[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float* line = Cs + (int64_t)k * 9 * c;
        if (valid) {
            float rr[9];
            ld9(line, c, x, rr);
            mm3(rr, Pi, ck);
            st9(line, c, x, ck);
        }
        float* gp = ws + L.offG + (int64_t)g.ti * 9 * g.kmax;
        for (int p0 = 0; p0 <= k; p0 += 3) {
            float acc[32];
#pragma unroll
            for (int e9 = 0; e9 < 32; ++e9) acc[e9] = 0.f;
            if (valid) {
#pragma unroll
                for (int gg = 0; gg < 3; ++gg) {
                    const int p = p0 + gg;
                    if (p <= k) {
                        float a9[9];
                        if (p == k) {
#pragma unroll
                            for (int e9 = 0; e9 < 9; ++e9) a9[e9] = ck[e9];
                        } else {
                            ld9(Cs + (int64_t)p * 9 * c, c, x, a9);
                        }
#pragma unroll
                        for (int u = 0; u < 3; ++u)
#pragma unroll
                            for (int v = 0; v < 3; ++v)
                                acc[9 * gg + 3 * u + v] = a9[u] * ck[v] + a9[3 + u] * ck[3 + v] + a9[6 + u] * ck[6 + v];
                    }
                }
            }
            warp_sum27_store(acc, gp + 9 * p0, min(27, 9 * (k + 1 - p0)), lane);
        }
        return;
    }
    // TK_OUT
    const int l = k;
    if (R.mode == 0) {
        __syncwarp();
        for (int i = lane; i < 3 * l; i += 32) pv[i] = S.tv[(int64_t)g.s * 3 * R.MR + i];
        __syncwarp();
        if (x < c) {
            float y0 = 0.f, y1 = 0.f, y2 = 0.f;
            for (int p = 0; p < l; ++p) {
                float cv[9];
                ld9(Cs + (int64_t)p * 9 * c, c, x, cv);
                const float* tp = pv + 3 * p;
                y0 += cv[0] * tp[0] + cv[1] * tp[1] + cv[2] * tp[2];
                y1 += cv[3] * tp[0] + cv[4] * tp[1] + cv[5] * tp[2];
                y2 += cv[6] * tp[0] + cv[7] * tp[1] + cv[8] * tp[2];
            }
            float* out = R.part + 3 * (R.pofs[g.b] - R.pofs_base + x);
            out[0] = y0; out[1] = y1; out[2] = y2;
        }
    } else {   // mode 2: C [l][9][c] then Q [l][9][q] at fofs[b]
        // the room the first (pivots-only) pass sized for this block
        const int64_t cap = (R.fofs[g.b + 1] - R.fofs[g.b]) / (int64_t)(c + q);
        if (l <= cap) {
            float* dst = R.fac + 9 * (R.fofs[g.b] - R.fofs_base);
            if (x < c)
                for (int pe = 0; pe < 9 * l; ++pe) dst[(int64_t)pe * c + x] = Cs[(int64_t)pe * c + x];
            if (x < q)
                for (int pe = 0; pe < 9 * l; ++pe) dst[(int64_t)l * 9 * c + (int64_t)pe * q + x] = Qs[(int64_t)pe * q + x];
        } else if (lane == 0) {
            atomicOr(R.status, (unsigned)HH_DEV_NUMERIC);
        }
    }
}

template <int W>
__global__ void __launch_bounds__(128, 4) k_round_tiles(RoundArgs R, const float* __restrict__ th)
{
    const int r = R.round;
    if (blockIdx.x == 0 && threadIdx.x < 2) R.cnt[2 * ((r + 2) % 3) + threadIdx.x] = 0u;   // round r + 2 starts empty
    const unsigned n_mlp = R.cnt[2 * (r % 3) + LIST_MLP], n_plain = R.cnt[2 * (r % 3) + LIST_PLAIN];
    const unsigned n_groups = (n_mlp + 3) / 4;
    if (blockIdx.x >= n_groups && blockIdx.x * 4u >= n_plain) return;   // nothing for this CTA
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TileSmem<W>& sm = *reinterpret_cast<TileSmem<W>*>(smem_raw);
    tc_setup<W>(sm.tc, th, R.status);
    uint32_t phase_bits = 0;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float* const pv = sm.piv[warp];
    const Slots& S = R.st;
    const Seg* listM = R.list[r & 1][LIST_MLP];
    const Seg* listP = R.list[r & 1][LIST_PLAIN];
    // COL / ROW segments, four to a 128-row MLP tile
    for (unsigned grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
        const unsigned e = 4 * grp + warp;
        const bool seg = e < n_mlp;
        SegView g{};
        bool valid = false;
        float fe[4], id = 1.f;
        fe[0] = 1.f; fe[1] = fe[2] = 0.f; fe[3] = R.a;
        __syncwarp();   // the previous segment's readers of pv are done
        if (seg) {
            g = load_seg(listM + e, lane);
            const bool col = g.kind == TK_COL;
            const int nx = col ? g.c : g.q;
            for (int i = lane; i < 9 * g.k; i += 32) pv[i] = S.piv[(int64_t)g.s * 9 * R.MR + i];
            const SlotLayout L = slot_layout(g.c, g.q, g.kmax);
            const float* fac = R.ws + (int64_t)g.s * R.stride + (col ? 0 : L.offQ);
            prefetch_seg_lines(fac, nx, g.ti * RT, g.k, lane);
            const int x = g.ti * RT + lane;
            valid = x < nx;
            if (valid) {
                float rx, ry, rz;
                sep_split(R.Xp, col ? g.t0 + x : g.t0 + g.bi, col ? g.s0 + g.bj : g.s0 + x, rx, ry, rz);
                features(rx, ry, rz, R.a, fe, id);
            }
        }
        tc_write_features<W>(sm.tc, t, fe);
        float o[6];
        if (!tc_mlp_tile<W>(sm.tc, phase_bits, R.status, o)) break;   // uniform: sm.tc.fail set
        if (seg) finish_query_seg(R, g, pv, o, id, valid, lane);
    }
    // GRAM / OUT segments, one warp each
    if (!sm.tc.fail)
        for (unsigned e = blockIdx.x * 4u + warp; e < n_plain; e += gridDim.x * 4u) {
            __syncwarp();
            const SegView g = load_seg(listP + e, lane);
            plain_seg(R, g, pv, lane);
        }
    tc_teardown<W>(sm.tc);
}

// ---- pivots: one thread per slot --------------------------------------------------
// After a column pass, the pivot row of the argmax and its FP64 inverse (line
// 6 of Algorithm 2), one slot per thread so that B300's scarce FP64 units do
// 32 slots' work per warp instruction.  pivst[s]: 0 no pivot (the block
// ends), 1 inverse in S.Pi, 2 the guard must choose (singular, or reciprocal
// condition number below 1e-10).
__global__ void __launch_bounds__(128) k_round_pivots(RoundArgs R)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= R.S) return;
    const Slots& S = R.st;
    if (S.phase[s] != PH_COL) return;
    float best;
    int bi;
    unpack_key(S.key[s], best, bi);
    if (bi < 0 || !(best > 0.f)) { S.pivst[s] = 0; return; }
    const int c = S.c[s], k = S.k[s];
    const float* Cs = R.ws + (int64_t)s * R.stride;
    double P[9], Pi[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) P[e] = (double)Cs[((int64_t)k * 9 + e) * c + bi];
    if (k == 0) S.pscale[s] = sqrt(fro2(P));
    double det;
    const int kept = inv3_floor(P, PIVOT_FLOOR_BF16 * S.pscale[s], Pi, &det);
    if (kept == 0) { S.pivst[s] = 0; return; }   // the pivot element is rounding noise: the block ends
    const double rc = kept == 3 ? 1.0 / sqrt(fro2(P) * fro2(Pi)) : 1.0;
    if (!(rc >= 1e-10)) { S.pivst[s] = 2; return; }
#pragma unroll
    for (int e = 0; e < 9; ++e) S.Pi[(int64_t)s * 9 + e] = (float)Pi[e];
    S.ib[s] = bi;
    S.pivst[s] = 1;
}

// ---- the step kernel: one warp per slot ---------------------------------------------
// The segments a slot's next phase needs: n_m on the MLP list (kind k_m),
// n_p on the plain list (kind k_p).
struct Req {
    int n_m, k_m, n_p, k_p;
};

__device__ Req phase_req(const RoundArgs& R, int ph, int c, int q)
{
    Req rq{0, TK_COL, 0, TK_GRAM};
    if (ph == PH_COL) { rq.n_m = tiles_of(c); rq.k_m = TK_COL; }
    else if (ph == PH_GR) { rq.n_m = tiles_of(q); rq.k_m = TK_ROW; rq.n_p = tiles_of(c); rq.k_p = TK_GRAM; }
    else if (ph == PH_OUT) { rq.n_p = R.mode == 2 ? tiles_of(max(c, q)) : tiles_of(c); rq.k_p = TK_OUT; }
    return rq;
}

// New phase of slot s (its fields already written): phase word, key.
__device__ Req start_phase(const RoundArgs& R, int s, int ph, int c, int q, int lane)
{
    const Slots& S = R.st;
    if (lane == 0) {
        S.phase[s] = ph;
        S.key[s] = 0ull;
    }
    return phase_req(R, ph, c, q);
}

// Admission of the next block of the class into slot s (or the slot stays free).
__device__ Req admit(const RoundArgs& R, float* ws, int s, int lane)
{
    const Slots& S = R.st;
    unsigned long long w = 0;
    if (lane == 0) w = atomicAdd(R.next, 1ull);
    w = __shfl_sync(0xffffffffu, w, 0);
    if ((int64_t)w >= R.n_work) {
        if (lane == 0) S.phase[s] = PH_FREE;
        return Req{0, TK_COL, 0, TK_GRAM};
    }
    const int32_t nb = R.work[w], tt = R.PG[2 * nb], ss = R.PG[2 * nb + 1];
    const int32_t t0 = R.nbeg[tt], c = R.nend[tt] - t0, s0 = R.nbeg[ss], q = R.nend[ss] - s0;
    const int kmax = min(min(c, q), R.max_rank);
    const int j1 = j1_of(R.j1_rule, R.seed, tt, ss, q);
    const SlotLayout L = slot_layout(c, q, kmax);
    uint8_t* f = reinterpret_cast<uint8_t*>(ws + L.offF);
    for (int m = lane; m < c + q; m += 32) f[m] = (m == c + j1) ? 1 : 0;
    if (lane == 0) {
        S.blk[s] = nb;
        S.t0[s] = t0; S.c[s] = c; S.s0[s] = s0; S.q[s] = q;
        S.kmax[s] = kmax;
        S.k[s] = 0;
        S.jb[s] = j1;
        S.ib[s] = -1;
        S.lam2[s] = 0.0;
    }
    return start_phase(R, s, PH_COL, c, q, lane);
}

// The block of slot s ends with l pairs: rank, pivots past l, counters; then
// its output phase (modes 0 and 2) or the next block.
__device__ Req finish_block(const RoundArgs& R, float* ws, int s, int64_t b, int c, int q, int l, bool capped,
                            int lane)
{
    const Slots& S = R.st;
    if (lane == 0) {
        if (R.rank) R.rank[b] = l;
        if (capped) atomicOr(R.status, (unsigned)HH_DEV_RANK_CAP);
        atomicAdd(R.n_queries, (unsigned long long)(c + q) * (unsigned long long)l);
        S.k[s] = l;
    }
    if (R.pivI)
        for (int p = l + lane; p < R.max_rank; p += 32) {
            R.pivI[b * R.max_rank + p] = -1;
            R.pivJ[b * R.max_rank + p] = -1;
        }
    if (R.mode == 1 || (R.mode == 2 && l == 0)) return admit(R, ws, s, lane);
    return start_phase(R, s, PH_OUT, c, q, lane);   // mode 0 writes zeros when l == 0
}

__device__ Req slot_step(const RoundArgs& R, int s, int lane, float* A, float* B, bool sums_ready)
{
    const Slots& S = R.st;
    float* const ws = R.ws + (int64_t)s * R.stride;
    const int ph = S.phase[s];
    if (ph == PH_FREE || ph == PH_OUT) return admit(R, ws, s, lane);
    const int64_t b = S.blk[s];
    const int c = S.c[s], q = S.q[s], kmax = S.kmax[s], k = S.k[s];
    const SlotLayout L = slot_layout(c, q, kmax);
    const float* const Cs = ws;
    const float* const Qs = ws + L.offQ;
    uint8_t* const usedR = reinterpret_cast<uint8_t*>(ws + L.offF);
    uint8_t* const usedC = usedR + c;
    if (ph == PH_COL) {
        // line 5: pivot row; line 6: its FP64 inverse (k_round_pivots), or the
        // guard of the largest |det| among unused rows for a singular or
        // ill-conditioned one
        const int pst = S.pivst[s];
        if (pst == 0) return finish_block(R, ws, s, b, c, q, k, false, lane);
        int bi = S.ib[s];
        if (pst == 2) {
            double bd = 0.0;
            int bdi = -1;
            for (int m = lane; m < c; m += 32) {
                if (usedR[m]) continue;
                double Pm[9];
#pragma unroll
                for (int e = 0; e < 9; ++e) Pm[e] = (double)Cs[((int64_t)k * 9 + e) * c + m];
                const double dv = fabs(det3d(Pm));
                if (dv > bd) { bd = dv; bdi = m; }
            }
            warp_argmax(bd, bdi);
            if (bdi < 0) return finish_block(R, ws, s, b, c, q, k, false, lane);
            bi = bdi;
            if (lane == 0) {
                double P[9], Pi[9];
#pragma unroll
                for (int e = 0; e < 9; ++e) P[e] = (double)Cs[((int64_t)k * 9 + e) * c + bi];
                inv3d(P, Pi);
#pragma unroll
                for (int e = 0; e < 9; ++e) S.Pi[(int64_t)s * 9 + e] = (float)Pi[e];
            }
        }
        if (lane == 0) {
            usedR[bi] = 1;
            S.ib[s] = bi;
            if (R.pivI) {
                R.pivI[b * R.max_rank + k] = bi;
                R.pivJ[b * R.max_rank + k] = S.jb[s];
            }
        }
        // C_p(i_k), p < k (already scaled), for the row pass
        for (int i = lane; i < 9 * k; i += 32) S.piv[(int64_t)s * 9 * R.MR + i] = Cs[(int64_t)i * c + bi];
        return start_phase(R, s, PH_GR, c, q, lane);
    }
    // PH_GR: lines 9-10 with the 3x3 Gram sums (segment partials added in
    // segment order), then line 8's column pivot
    if (!sums_ready) {
        const int ntc = tiles_of(c), ntq = tiles_of(q);
        const float* gp = ws + L.offG;
        const float* rp = ws + L.offR;
        for (int i = lane; i < 9 * (k + 1); i += 32) {
            float a = 0.f, bsum = 0.f;
            for (int u = 0; u < ntc; ++u) a += gp[(int64_t)u * 9 * kmax + i];
            for (int u = 0; u < ntq; ++u) bsum += rp[(int64_t)u * L.rstride + i];
            A[i] = a;
            B[i] = bsum;
        }
        if (lane < 3) {
            float a = 0.f;
            for (int u = 0; u < ntq; ++u) a += rp[(int64_t)u * L.rstride + 9 * kmax + lane];
            S.tv[(int64_t)s * 3 * R.MR + 3 * k + lane] = a;
        }
    }
    __syncwarp();
    // nu^2 = tr(A_kk B_kk), cross = sum_{p<k} tr(A_pk B_kp): FP32 products
    // and a fixed shuffle tree; the lambda^2 recurrence itself in FP64
    float nu2f = 0.f, crossf = 0.f;
    for (int i = lane; i < 9 * (k + 1); i += 32) {
        const int pp = i / 9, x = (i % 9) / 3, y = i % 3;
        const float term = A[9 * pp + 3 * x + y] * B[9 * pp + 3 * y + x];
        if (pp == k) nu2f += term;
        else crossf += term;
    }
    const double nu2 = (double)warp_sum(nu2f);
    const double cross = (double)warp_sum(crossf);
    const double lam2 = S.lam2[s] + nu2 + 2.0 * cross;
    float best;
    int bj;
    unpack_key(S.key[s], best, bj);
    const int k1 = k + 1;
    __syncwarp();
    if (lane == 0) S.lam2[s] = lam2;
    if ((nu2 <= R.eps2 * lam2) || (bj < 0)) return finish_block(R, ws, s, b, c, q, k1, false, lane);
    if (k1 == kmax) return finish_block(R, ws, s, b, c, q, k1, (k1 == R.max_rank) && (k1 < min(c, q)), lane);
    if (lane == 0) {
        usedC[bj] = 1;
        S.k[s] = k1;
        S.jb[s] = bj;
    }
    // Q_p(j_{k+1}), p <= k, for the next column pass
    for (int i = lane; i < 9 * k1; i += 32) S.piv[(int64_t)s * 9 * R.MR + i] = Qs[(int64_t)i * q + bj];
    return start_phase(R, s, PH_COL, c, q, lane);
}

struct StepSmem {
    float A[STEP_WARPS][9 * MAXR];
    float B[STEP_WARPS][9 * MAXR];
    int n[STEP_WARPS][2];
    unsigned base[STEP_WARPS][2];
};

// Step of slot s = blockIdx.x * STEP_WARPS + warp; the CTA's slots append the
// segments of their next phases with one atomic per list.
__global__ void __launch_bounds__(32 * STEP_WARPS) k_round_step(RoundArgs R)
{
    __shared__ StepSmem sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = blockIdx.x * STEP_WARPS + warp;
    Req rq{0, TK_COL, 0, TK_GRAM};
    if (s < R.S) rq = slot_step(R, s, lane, sh.A[warp], sh.B[warp], false);
    if (lane == 0) { sh.n[warp][0] = rq.n_m; sh.n[warp][1] = rq.n_p; }
    __syncthreads();
    const int nxt = R.round + 1;
    if (threadIdx.x < 2) {
        const int li = threadIdx.x;
        unsigned tot = 0;
        for (int w = 0; w < STEP_WARPS; ++w) { sh.base[w][li] = tot; tot += (unsigned)sh.n[w][li]; }
        const unsigned b0 = tot ? atomicAdd(R.cnt + 2 * (nxt % 3) + li, tot) : 0u;
        for (int w = 0; w < STEP_WARPS; ++w) sh.base[w][li] += b0;
    }
    __syncthreads();
    if (s >= R.S || rq.n_m + rq.n_p == 0) return;
    const Slots& S = R.st;
    Seg tl;
    tl.s = s; tl.t0 = S.t0[s]; tl.c = S.c[s]; tl.s0 = S.s0[s]; tl.q = S.q[s]; tl.k = S.k[s];
    tl.kmax = S.kmax[s]; tl.ib = S.ib[s]; tl.jb = S.jb[s]; tl.blk = S.blk[s]; tl.pad = 0;
    Seg* LM = R.list[nxt & 1][LIST_MLP] + sh.base[warp][0];
    Seg* LP = R.list[nxt & 1][LIST_PLAIN] + sh.base[warp][1];
    for (int u = lane; u < rq.n_m; u += 32) {
        Seg e = tl;
        e.kind_ti = (rq.k_m << 28) | u;
        LM[u] = e;
    }
    for (int u = lane; u < rq.n_p; u += 32) {
        Seg e = tl;
        e.kind_ti = (rq.k_p << 28) | u;
        LP[u] = e;
    }
}

// Step of slot blockIdx.x with the whole CTA, for classes of large blocks:
// the 256 threads add the segment partials of the Gram and apply sums
// (value i by warp i mod 8, its lanes over the segments, then a fixed
// shuffle tree), and warp 0 runs the rest of the step.
__global__ void __launch_bounds__(32 * STEP_WARPS) k_round_step_large(RoundArgs R)
{
    __shared__ float A[9 * MAXR], B[9 * MAXR];
    __shared__ int ph_k[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = blockIdx.x;
    const Slots& S = R.st;
    if (threadIdx.x == 0) { ph_k[0] = S.phase[s]; ph_k[1] = S.k[s]; }
    __syncthreads();
    const bool gr = ph_k[0] == PH_GR;
    if (gr) {
        const int c = S.c[s], q = S.q[s], kmax = S.kmax[s], k = ph_k[1];
        const SlotLayout L = slot_layout(c, q, kmax);
        const float* ws = R.ws + (int64_t)s * R.stride;
        const float* gp = ws + L.offG;
        const float* rp = ws + L.offR;
        const int ntc = tiles_of(c), ntq = tiles_of(q);
        for (int i = warp; i < 9 * (k + 1) + 3; i += STEP_WARPS) {
            float a = 0.f, bsum = 0.f;
            if (i < 9 * (k + 1)) {
                for (int u = lane; u < ntc; u += 32) a += gp[(int64_t)u * 9 * kmax + i];
                for (int u = lane; u < ntq; u += 32) bsum += rp[(int64_t)u * L.rstride + i];
            } else {
                for (int u = lane; u < ntq; u += 32) bsum += rp[(int64_t)u * L.rstride + 9 * kmax + (i - 9 * (k + 1))];
            }
            a = warp_sum(a);
            bsum = warp_sum(bsum);
            if (lane == 0) {
                if (i < 9 * (k + 1)) { A[i] = a; B[i] = bsum; }
                else S.tv[(int64_t)s * 3 * R.MR + 3 * k + (i - 9 * (k + 1))] = bsum;
            }
        }
    }
    __syncthreads();
    if (warp != 0) return;
    const Req rq = slot_step(R, s, lane, A, B, gr);
    const int n = rq.n_m + rq.n_p;
    if (n == 0) return;
    const int nxt = R.round + 1;
    unsigned bm = 0, bp = 0;
    if (lane == 0) {
        if (rq.n_m) bm = atomicAdd(R.cnt + 2 * (nxt % 3) + LIST_MLP, (unsigned)rq.n_m);
        if (rq.n_p) bp = atomicAdd(R.cnt + 2 * (nxt % 3) + LIST_PLAIN, (unsigned)rq.n_p);
    }
    bm = __shfl_sync(0xffffffffu, bm, 0);
    bp = __shfl_sync(0xffffffffu, bp, 0);
    Seg tl;
    tl.s = s; tl.t0 = S.t0[s]; tl.c = S.c[s]; tl.s0 = S.s0[s]; tl.q = S.q[s]; tl.k = S.k[s];
    tl.kmax = S.kmax[s]; tl.ib = S.ib[s]; tl.jb = S.jb[s]; tl.blk = S.blk[s]; tl.pad = 0;
    Seg* LM = R.list[nxt & 1][LIST_MLP] + bm;
    Seg* LP = R.list[nxt & 1][LIST_PLAIN] + bp;
    for (int u = lane; u < rq.n_m; u += 32) {
        Seg e = tl;
        e.kind_ti = (rq.k_m << 28) | u;
        LM[u] = e;
    }
    for (int u = lane; u < rq.n_p; u += 32) {
        Seg e = tl;
        e.kind_ti = (rq.k_p << 28) | u;
        LP[u] = e;
    }
}

template <int W>
size_t tile_smem_bytes() { return sizeof(TileSmem<W>) + 128; }

// Floats of a slot workspace that holds any block with c + q <= M at rank <= MR
// (slot_layout is linear in c + q up to the segment roundings bounded here).
int64_t slot_stride_bound(int64_t M, int64_t MR)
{
    const int64_t tiles = ceil_div(M, RT) + 1;   // ceil(c / RT) + ceil(q / RT)
    const int64_t rstride = (9 * MR + 4 + 3) / 4 * 4;
    const int64_t raw = MR * 9 * M + (M + 15) / 16 * 4 + tiles * 9 * MR + tiles * rstride;
    return (raw + 63) / 64 * 64 + 64;
}

// Bytes of the slot-state arrays for S slots (the carve-up in aca_rounds_run).
size_t slot_state_bytes(int64_t S, int MR)
{
    auto r = [](int64_t b) { return (size_t)((b + 255) / 256 * 256); };
    return 11 * r(4 * S) + 3 * r(8 * S) + r(4 * 9 * S) + r(4 * 9 * MR * S) + r(4 * 3 * MR * S);
}

}  // namespace

// Size classes of the admissible blocks by c + q, processed largest first;
// each class's slots advance round by round until no segment is left.
void aca_rounds_run(hh_ctx* ctx, const hh_tree* t, const hh_blocks* bl, const hh_params& p, const AcaRun& r,
                    const int32_t* work_sorted, const int64_t* cls_begin, const int32_t* cls_max_cq, int n_cls,
                    cudaStream_t s, bool own_events)
{
    HH_REQUIRE(p.kernel == HH_MLP && p.precision == HH_BF16, HH_ERR_ARG, "tensor-core ACA needs the BF16 MLP kernel");
    const int MR = std::min(p.max_rank, MAXR);
    const int64_t budget = budget_rounds(p);
    const int W = ctx->width;
    const size_t smem = W == 32 ? tile_smem_bytes<32>() : tile_smem_bytes<64>();
    if (W == 32) HH_CUDA(cudaFuncSetAttribute(k_round_tiles<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    else HH_CUDA(cudaFuncSetAttribute(k_round_tiles<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));

    // per class: slots within the budget; the largest class sizes the shared arrays
    int64_t S_alloc = 1, ws_floats = 1, list_alloc = 1;
    std::vector<int> S_of(n_cls, 0);
    std::vector<int64_t> stride_of(n_cls, 0);
    for (int i = 0; i < n_cls; ++i) {
        const int64_t n = cls_begin[i + 1] - cls_begin[i];
        if (n <= 0) continue;
        const int64_t M = cls_max_cq[i];
        const int64_t stride = slot_stride_bound(M, MR);
        const int64_t Sc = std::min<int64_t>({n, (int64_t)SLOTS_MAX, std::max<int64_t>(1, budget / (stride * 4))});
        S_of[i] = (int)Sc;
        stride_of[i] = stride;
        S_alloc = std::max(S_alloc, Sc);
        ws_floats = std::max(ws_floats, Sc * stride);
        list_alloc = std::max(list_alloc, Sc * (ceil_div(M, RT) + 1));
    }
    AcaArgs<float> base = make_aca_args<float>(ctx, t, bl, p, r);
    RoundArgs R{};
    R.Xp = t->Xp;
    R.Fs = r.Fs;
    R.a = (float)p.radius;
    R.PG = bl->PG;
    R.nbeg = t->nbeg;
    R.nend = t->nend;
    R.MR = MR;
    R.max_rank = p.max_rank;
    R.eps2 = p.eps * p.eps;
    R.j1_rule = p.j1_rule;
    R.seed = p.seed;
    R.mode = r.mode;
    R.rank = r.rank;
    R.pivI = r.pivI;
    R.pivJ = r.pivJ;
    R.part = (float*)r.part;
    R.pofs = r.pofs;
    R.pofs_base = r.pofs_base;
    R.fac = (float*)r.factors;
    R.fofs = r.fofs;
    R.fofs_base = r.fofs_base;
    R.status = base.status;
    R.n_queries = base.n_queries;

    // device memory of the run: workspaces, slot state, segment lists, counters
    float* ws = dev_alloc_t<float>(ws_floats, s);
    const int64_t Sa = S_alloc;
    const size_t st_bytes = slot_state_bytes(Sa, MR);
    char* st = (char*)dev_alloc(st_bytes, s);
    HH_CUDA(cudaMemsetAsync(st, 0, st_bytes, s));
    Seg* lists = dev_alloc_t<Seg>(4 * list_alloc, s);
    unsigned* cnt = dev_alloc_t<unsigned>(8, s);
    unsigned long long* next = dev_alloc_t<unsigned long long>(1, s);
    {
        char* pp = st;
        auto take = [&](size_t bytes) { char* q = pp; pp += (bytes + 255) / 256 * 256; return q; };
        Slots& S = R.st;
        S.blk = (int32_t*)take(4 * Sa); S.t0 = (int32_t*)take(4 * Sa); S.c = (int32_t*)take(4 * Sa);
        S.s0 = (int32_t*)take(4 * Sa); S.q = (int32_t*)take(4 * Sa); S.kmax = (int32_t*)take(4 * Sa);
        S.k = (int32_t*)take(4 * Sa); S.phase = (int32_t*)take(4 * Sa); S.ib = (int32_t*)take(4 * Sa);
        S.jb = (int32_t*)take(4 * Sa); S.pivst = (int32_t*)take(4 * Sa);
        S.lam2 = (double*)take(8 * Sa);
        S.pscale = (double*)take(8 * Sa);
        S.key = (unsigned long long*)take(8 * Sa);
        S.Pi = (float*)take(4 * 9 * Sa);
        S.piv = (float*)take(4 * 9 * MR * Sa);
        S.tv = (float*)take(4 * 3 * MR * Sa);
    }
    R.ws = ws;
    for (int b2 = 0; b2 < 2; ++b2)
        for (int li = 0; li < 2; ++li) R.list[b2][li] = lists + (2 * b2 + li) * list_alloc;
    R.cnt = cnt;
    R.next = next;
    int* h_cnt = ctx_pinned_int(ctx);

    // events around every round's kernels (double-buffered by batch): the
    // split of the ACA time between tiles and pivots + steps, read at the polls
    constexpr int CHECK = 8;
    struct RoundEvents {
        cudaEvent_t e[2][CHECK][3] = {};
        ~RoundEvents()
        {
            for (auto& a : e)
                for (auto& b : a)
                    for (auto& x : b)
                        if (x) cudaEventDestroy(x);
        }
    } rev;
    for (auto& a : rev.e)
        for (auto& b : a)
            for (auto& x : b) HH_CUDA(cudaEventCreate(&x));
    double t_tiles = 0.0, t_steps = 0.0;
    auto read_batch = [&](int set) {
        for (int u = 0; u < CHECK; ++u) {
            float a = 0.f, c2 = 0.f;
            HH_CUDA(cudaEventElapsedTime(&a, rev.e[set][u][0], rev.e[set][u][1]));
            HH_CUDA(cudaEventElapsedTime(&c2, rev.e[set][u][1], rev.e[set][u][2]));
            t_tiles += a;
            t_steps += c2;
        }
    };
    if (own_events) HH_CUDA(cudaEventRecord(ctx->kev[2], s));
    const unsigned grid = (unsigned)(ctx->n_sm * resolved_launch(ctx, true).aca_small_cps);
    int64_t rounds_total = 0;
    for (int i = 0; i < n_cls; ++i) {
        if (S_of[i] == 0) continue;
        const int64_t n = cls_begin[i + 1] - cls_begin[i];
        R.work = work_sorted + cls_begin[i];
        R.n_work = n;
        R.S = S_of[i];
        R.stride = stride_of[i];
        HH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * 8, s));
        HH_CUDA(cudaMemsetAsync(next, 0, sizeof(unsigned long long), s));
        HH_CUDA(cudaMemsetAsync(R.st.phase, 0, sizeof(int32_t) * R.S, s));
        const unsigned grid_piv = (unsigned)ceil_div(R.S, 128);          // thread per slot
        // a warp per slot, or a CTA per slot where blocks have many segments
        const bool large = ceil_div(cls_max_cq[i], RT) > 16;
        auto step = [&]() {
            if (large) k_round_step_large<<<(unsigned)R.S, 32 * STEP_WARPS, 0, s>>>(R);
            else k_round_step<<<(unsigned)ceil_div(R.S, STEP_WARPS), 32 * STEP_WARPS, 0, s>>>(R);
            HH_CHECK_LAUNCH();
        };
        R.round = -1;   // the first admissions fill round 0's lists
        step();
        // a block takes at most 2 rounds per rank step plus its output round
        const int64_t limit = (ceil_div(n, R.S) + 2) * (2 * (int64_t)p.max_rank + 3) + 64;
        int64_t rr = 0;
        int batch = 0;
        bool pending = false;
        for (;; ++batch) {
            const int set = batch & 1;
            for (int u = 0; u < CHECK; ++u, ++rr) {
                R.round = (int)rr;
                HH_CUDA(cudaEventRecord(rev.e[set][u][0], s));
                if (W == 32) k_round_tiles<32><<<grid, 128, smem, s>>>(R, ctx->theta32);
                else k_round_tiles<64><<<grid, 128, smem, s>>>(R, ctx->theta32);
                HH_CHECK_LAUNCH();
                HH_CUDA(cudaEventRecord(rev.e[set][u][1], s));
                k_round_pivots<<<grid_piv, 128, 0, s>>>(R);
                HH_CHECK_LAUNCH();
                step();
                HH_CUDA(cudaEventRecord(rev.e[set][u][2], s));
            }
            // the segment counts of the next round, read while the next batch runs
            if (pending) {
                HH_CUDA(cudaEventSynchronize(ctx->poll_ev));
                read_batch(set ^ 1);
                // done, or a bounded wait gave up (the caller reads the status)
                if ((h_cnt[0] == 0 && h_cnt[1] == 0) || (h_cnt[2] & HH_DEV_TIMEOUT)) {
                    HH_CUDA(cudaEventSynchronize(rev.e[set][CHECK - 1][2]));
                    read_batch(set);
                    break;
                }
            }
            HH_CUDA(cudaMemcpyAsync(h_cnt, cnt + 2 * (rr % 3), 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
            HH_CUDA(cudaMemcpyAsync(h_cnt + 2, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
            HH_CUDA(cudaEventRecord(ctx->poll_ev, s));
            pending = true;
            if (rr > limit) {
                HH_CUDA(cudaEventSynchronize(ctx->poll_ev));
                read_batch(set);
                if ((h_cnt[0] == 0 && h_cnt[1] == 0) || (h_cnt[2] & HH_DEV_TIMEOUT)) break;
                throw HHError{HH_ERR_CUDA, "ACA rounds did not finish within their bound"};
            }
        }
        rounds_total += rr;
    }
    if (own_events) {
        HH_CUDA(cudaEventRecord(ctx->kev[3], s));
        ctx->kev_aca_used |= 2;
    }
    ctx->stats.n_aca_rounds += rounds_total;
    ctx->stats.t_aca_tiles += t_tiles;
    ctx->stats.t_aca_steps += t_steps;
    dev_free(next, s);
    dev_free(cnt, s);
    dev_free(lists, s);
    dev_free(st, s);
    dev_free(ws, s);
}
