// hh_internal.h -- host-side object layout and cross-file entry points of
// libhhignn.  Not part of the public C-ABI (include/hhignn.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/hhignn.h"
#include "hh_common.cuh"

struct hh_ctx {
    int device = 0;
    int n_sm = 148;
    std::string err;
    float* theta32 = nullptr;   // device copy of the MLP parameters (float32, packed layout)
    float* theta32t = nullptr;  // transposed, padded FP32 layout read by the SIMT kernels
    double* theta64 = nullptr;  // packed layout widened to FP64 (FP64 mode)
    int width = 0, n_theta = 0, n_theta_t = 0;
    unsigned* d_status = nullptr;              // device status word (HH_DEV_* bits)
    unsigned long long* d_counters = nullptr;  // [8]: 0,1 work counters; 4 ACA queries; 5 near pairs
    hh_stats_t stats{};
    cudaStream_t last_stream = nullptr;
    cudaEvent_t ev[8] = {};
    cudaEvent_t kev[8] = {};             // around the ACA (0..3) and near (4,5) kernels
    int kev_aca_used = 0;                // ACA kernel event pairs recorded this call
    int kev_near_used = 0;
    bool kev_apply_pending = false;      // hh_matvec recorded kev[6], kev[7] around its low-rank apply
    unsigned long long launch_base = 0;  // g_hh_launches at the start of the call
    hh_launch_cfg launch{};              // 0 fields: defaults (see resolved_launch)
    cudaStream_t aux = nullptr;          // second stream: CTA-team ACA classes beside the warp teams
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    cudaStream_t aux2 = nullptr;         // third stream: the round-based ACA of the largest blocks
    cudaEvent_t join2_ev = nullptr;
    cudaEvent_t poll_ev = nullptr;       // the ACA rounds' progress reads
    int* h_pinned = nullptr;             // pinned host word those reads land in
    // short-range networks (hh_set_short_range): FP32 and FP64 copies
    float* sr_theta_s32 = nullptr;
    float* sr_theta_332 = nullptr;
    double* sr_theta_s64 = nullptr;
    double* sr_theta_364 = nullptr;
    int sr_width = 0;
    int sr_two_body = 0, sr_three_body = 0;
    double sr_rcut = 0.0;
};

// Launch shape with defaults filled in; tc selects the tensor-core defaults.
inline hh_launch_cfg resolved_launch(const hh_ctx* ctx, bool tc)
{
    hh_launch_cfg c = ctx->launch;
    if (c.small_max <= 0) c.small_max = 512;
    if (c.aca_small_cps <= 0) c.aca_small_cps = 4;
    if (c.aca_large_cps <= 0) c.aca_large_cps = tc ? 4 : 2;
    if (c.near_cps <= 0) c.near_cps = 5;
    if (c.rounds_min_cq <= 0) c.rounds_min_cq = 4096;
    return c;
}

struct hh_tree {
    hh_ctx* ctx = nullptr;
    hh_params params{};
    int64_t n = 0;
    int32_t batch = 0;
    std::vector<int64_t> offsets;    // host copy [batch+1]
    int64_t* d_offsets = nullptr;    // [batch+1]
    int32_t* perm = nullptr;         // [n] sorted position -> caller row
    uint64_t* codes = nullptr;       // [n] sorted Morton codes
    double* Xs = nullptr;            // [n,3] positions in sorted order
    float* Xp = nullptr;             // [n,6] the same as FP32 (hi, lo) pairs (sep_split)
    int32_t n_nodes = 0;
    int32_t* nbeg = nullptr;         // [n_nodes]
    int32_t* nend = nullptr;
    int32_t* child = nullptr;        // [n_nodes,2], -1 for leaves
    int32_t* parent = nullptr;
    double* lo = nullptr;            // [n_nodes,3]
    double* hi = nullptr;
    std::vector<int32_t> level_start;  // BFS level boundaries (host)
};

struct hh_blocks {
    const hh_tree* tree = nullptr;
    hh_params params{};
    int64_t nG = 0, nH = 0;
    int32_t* PG = nullptr;     // [nG,2] (target, source)
    int32_t* PH = nullptr;     // [nH,2]
    int64_t* rowG = nullptr;   // [n_nodes+1]: blocks of target t are rowG[t] .. rowG[t+1]
    int64_t* rowH = nullptr;
};

struct hh_hmat {
    hh_ctx* ctx = nullptr;
    const hh_tree* tree = nullptr;
    const hh_blocks* blocks = nullptr;
    hh_params params{};
    int32_t* rank = nullptr;   // [nG]
    int32_t* pivI = nullptr;   // [nG, max_rank]
    int32_t* pivJ = nullptr;
    int64_t* fofs = nullptr;   // [nG+1] factor offsets in elements of 9 reals ((c+q) * rank)
    void* factors = nullptr;   // per block: C [rank][9][c] then Q [rank][9][q]
    int64_t n_factor = 0;      // total elements
    int real_bytes = 4;
    // after hh_recompress (the ACA factors are then freed): per block the kept
    // scalar rank, the offsets (reals) and U [r][3c] then V [r][3q]
    int32_t* srank = nullptr;
    int64_t* sofs = nullptr;
    void* sfac = nullptr;
    int64_t n_sfac = 0;
};

// --- primitives (hh_prims.cu) ------------------------------------------------
// Exclusive prefix sum of n int64 values; total (optional) receives the sum
// on the device.  in and out must not alias.
void dev_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total, cudaStream_t s);
// Stable LSD radix sort of (keys, vals) by the low key_bits bits of keys;
// vals may be NULL.  Sorted data is returned in keys/vals.
void dev_radix_sort(uint64_t* keys, int32_t* vals, int64_t n, int key_bits, cudaStream_t s);
// Stream-ordered allocation helpers.
void* dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);
// The temporaries (dev_alloc) an entry point takes while it runs: release()
// frees those not freed yet, so a call that fails half-way leaks nothing.
class AllocScope {
public:
    AllocScope();
    ~AllocScope();
    void release();
    AllocScope(const AllocScope&) = delete;
    AllocScope& operator=(const AllocScope&) = delete;

private:
    std::vector<std::pair<void*, cudaStream_t>> live_;
    std::vector<std::pair<void*, cudaStream_t>>* prev_;
};
template <typename T>
T* dev_alloc_t(int64_t n, cudaStream_t s) { return (T*)dev_alloc(sizeof(T) * (size_t)(n > 0 ? n : 1), s); }

// --- stages ----------------------------------------------------------------
hh_tree* build_tree_impl(hh_ctx* ctx, const double* X, const int64_t* offsets, int32_t batch, const hh_params& p,
                         cudaStream_t s);
hh_blocks* partition_impl(hh_ctx* ctx, const hh_tree* t, const hh_params& p, cudaStream_t s);
void free_tree(hh_tree* t);
void free_blocks(hh_blocks* b);
void free_hmat(hh_hmat* h);
// order[k]: admissible blocks sorted by (source, target); col[s]: first entry
// of source node s in order.
void source_index(const hh_tree* t, const hh_blocks* b, int32_t* order, int64_t* col, cudaStream_t s);

// This shard's share of the work (hh_shard.cu; NULL when n_shards == 1):
// flags[nG] over the admissible blocks, flags[n_nodes] over the target nodes
// of the near field.  Stream-ordered allocations the caller frees.
uint8_t* shard_block_flags(const hh_tree* t, const hh_blocks* b, const hh_params& p, cudaStream_t s);
uint8_t* shard_node_flags(const hh_tree* t, const hh_blocks* b, const hh_params& p, cudaStream_t s);

// Gather rows of an [n,3] FP64 array into sorted order: out[m] = in[perm[m]].
void gather_rows(const double* in, const int32_t* perm, int64_t n, double* out, cudaStream_t s);

// Near field (inadmissible blocks, self pair skipped): y[m] (sorted order,
// real type of the precision) = sum over P^H of K(x_m - x_n) F_n
// (transpose: K(x_n - x_m) F_n; the kernels' 3x3 blocks are symmetric).
void near_field(hh_ctx* ctx, const hh_tree* t, const hh_blocks* b, const hh_params& p, const double* Fs,
                void* y, int transpose, cudaStream_t s);

// ACA over admissible blocks.  mode 0: fused apply into per-block partials
// (part, at 3*pofs[b]); mode 1: ranks + pivots only; mode 2: also write
// factors at fofs.
struct AcaRun {
    const double* Fs = nullptr;   // sorted forces (mode 0)
    void* part = nullptr;         // per-block partial outputs (mode 0), block b at 3 * (pofs[b] - pofs_base)
    const int64_t* pofs = nullptr;
    int64_t pofs_base = 0;
    int64_t b0 = 0, b1 = -1;      // the admissible blocks of this run: [b0, b1) (b1 < 0: to the end)
    int32_t* rank = nullptr;
    int32_t* pivI = nullptr;
    int32_t* pivJ = nullptr;
    void* factors = nullptr;       // mode 2: block b at 9 * (fofs[b] - fofs_base)
    const int64_t* fofs = nullptr;
    int64_t fofs_base = 0;
    int mode = 0;
};
void aca_run(hh_ctx* ctx, const hh_tree* t, const hh_blocks* b, const hh_params& p, const AcaRun& r,
             cudaStream_t s);

// A size class of the large-block work list (sorted by decreasing c + q):
// items begin .. end - 1, the largest with c + q = max_cq.  Each class gets
// its own workspace stride, so the many mid-size blocks are not held to the
// team count the few largest blocks allow.
struct AcaClass {
    int64_t begin, end;
    int32_t max_cq;
};

// The device memory a prediction's admissible blocks may hold beyond the
// inputs, the tree and the partition (hh_params.mem_budget, default 32 GB),
// and its shares: the per-block partial outputs of one group of blocks (1/2),
// the warp teams' and the CTA teams' factor workspaces (1/8 each), the round
// engine's active blocks (1/4).
inline int64_t aca_budget_bytes(const hh_params& p) { return p.mem_budget > 0 ? p.mem_budget : (int64_t)32 << 30; }
inline int64_t budget_partials(const hh_params& p) { return aca_budget_bytes(p) / 2; }
inline int64_t budget_warp_teams(const hh_params& p) { return aca_budget_bytes(p) / 8; }
inline int64_t budget_cta_teams(const hh_params& p) { return aca_budget_bytes(p) / 8; }
inline int64_t budget_rounds(const hh_params& p) { return aca_budget_bytes(p) / 4; }

inline int* ctx_pinned_int(hh_ctx* ctx) { return ctx->h_pinned; }

// Round-based tensor-core ACA (hh_aca_rounds.cu, precision HH_BF16): the
// admissible blocks of this shard sorted by decreasing c + q (work_sorted),
// cut into size classes [cls_begin[i], cls_begin[i+1]) whose largest block
// has c + q = cls_max_cq[i].
// own_events: record the ACA kernel events (kev[2], kev[3]) around the run.
void aca_rounds_run(hh_ctx* ctx, const hh_tree* t, const hh_blocks* bl, const hh_params& p, const AcaRun& r,
                    const int32_t* work_sorted, const int64_t* cls_begin, const int32_t* cls_max_cq, int n_cls,
                    cudaStream_t s, bool own_events);

// Tensor-core ACA (hh_aca_tc.cu, precision HH_BF16 with the MLP kernel),
// three lists run concurrently: the small blocks (c, q <= small_max) on warp
// teams on stream s; the mid-size blocks (work_large, size classes cls) on
// CTA teams on the context's second stream; the largest blocks (c + q above
// rounds_min_cq; work_rounds, sorted by decreasing c + q, in the size classes
// rcls_begin / rcls_max_cq of aca_rounds_run) through the round engine on the
// third stream.
void aca_tc_run(hh_ctx* ctx, const hh_tree* t, const hh_blocks* bl, const hh_params& p, const AcaRun& r,
                const int32_t* work_small, int64_t n_small, const int32_t* work_large, const AcaClass* cls,
                int n_cls, const int32_t* work_rounds, const int64_t* rcls_begin, const int32_t* rcls_max_cq,
                int n_rcls, int max_small_cq, cudaStream_t s);

// Tensor-core (tcgen05) MLP paths (hh_tcmlp.cu): near field in HH_BF16 mode
// (work = target leaves) and K(r) for a list of separations.
void near_field_tc(hh_ctx* ctx, const hh_tree* t, const hh_blocks* b, const hh_params& p, const double* Fs, float* y,
                   const int32_t* work, int64_t n_work, int transpose, cudaStream_t s);
void eval_pairs_tc(hh_ctx* ctx, const double* r, int64_t n, double a, double* K, cudaStream_t s);
// SIMT K(r) for a list of separations (hh_near.cu), FP32 or FP64 per p.
void eval_pairs_simt(hh_ctx* ctx, const hh_params& p, const double* r, int64_t n, double* K, cudaStream_t s);

// Short-range terms of Eq. 6 (hh_short.cu): y[i] (FP64 if y_double, else
// float; same order as X and F) += the two- and three-body sums over
// neighbours within R_cut; offsets / d_offsets delimit the suspensions.
void short_range_add(hh_ctx* ctx, const double* X, const double* F, int64_t n, const std::vector<int64_t>& offsets,
                     const int64_t* d_offsets, const hh_params& p, void* y, int y_double, cudaStream_t s);

// Adjoint: dL/dX (added to gX, caller order) and dL/dtheta (added to gtheta)
// of L = sum w . (M_H F) with frozen pivots (hh_backward.cu); Fs, Ws sorted;
// h holds FP64 factors or pivots only.  The near-field entries run in FP32
// when near_fp32 (the product's near field was FP32 or BF16), else FP64.
// gFs (sorted order, may be NULL) += the admissible blocks' part of M_H^T w,
// from the same pass.  Every sum has a fixed order (reproducible bit for bit).
void matvec_backward_xtheta(hh_ctx* ctx, const hh_hmat* h, bool near_fp32, const double* Fs, const double* Ws,
                            double* gX, float* gtheta, double* gFs, cudaStream_t s);

// Training of the pair MLP (hh_train.cu).
double train_loss_grad(hh_ctx* ctx, const float* theta, int width, const double* r, const double* e, const double* U,
                       int64_t B, double a, float* grad_dev, cudaStream_t s);
void adam_step(float* theta, const float* g, float* m, float* v, int n, int64_t t, double lr, double b1, double b2,
               double eps, cudaStream_t s);

// Fused ACA + apply of one block on caller-provided workspace (no allocation).
void aca_single_block_ws(hh_ctx* ctx, const hh_params& p, int32_t c, int32_t q, const double* Xs, const double* Fs,
                         const int32_t* PG, const int32_t* nbeg, const int32_t* nend, const int32_t* work,
                         unsigned long long* counter, void* ws, void* part, const int64_t* pofs, int32_t* rank,
                         cudaStream_t s);
// Parameter checks shared by the entry points (hh_api.cu).
void check_params_public(const hh_ctx* ctx, const hh_params* p);

// Low-rank apply from stored factors into per-block partials.
void lowrank_apply(hh_ctx* ctx, const hh_hmat* h, const double* Fs, void* part, const int64_t* pofs, int transpose,
                   cudaStream_t s);

// Final FP64 accumulation: U[perm[m]] = alpha1 F_m + y_near(m) + the block
// partials of every admissible block containing m (rowG / order index the
// blocks by the accumulated side: targets, or sources when transposed).
void accumulate_impl(hh_ctx* ctx, const hh_tree* t, const hh_params& p, const double* Fs, const void* y_near,
                     const void* part, const int64_t* pofs, const int64_t* rowG, const int32_t* order, double alpha1,
                     double* U, cudaStream_t s);

// The same sum in steps, for a prediction whose admissible blocks run in
// groups (bounded partial-output memory): Us (sorted, FP64 [n,3]) =
// alpha1 F + y_near; then, per group [b0, b1), the group's partials (block b
// at part + 3 (pofs[b] - pofs_base)); finally U[perm[m]] = Us[m].  Each
// particle's terms are added in k_accum's order, so the grouping changes no
// bit of U.
void accumulate_begin(const hh_tree* t, const hh_params& p, const double* Fs, const void* y_near, double alpha1,
                      double* Us, cudaStream_t s);
void accumulate_group(const hh_tree* t, const hh_params& p, const void* part, const int64_t* pofs, int64_t pofs_base,
                      const int64_t* rowG, int64_t b0, int64_t b1, double* Us, cudaStream_t s);
void accumulate_end(const hh_tree* t, const double* Us, double* U, cudaStream_t s);
// Contiguous groups of admissible blocks whose partial outputs hold at most
// about cap entries each (a group starts at each multiple of cap); pofs_at
// receives each group's first offset and, last, the total.  Synchronises.
std::vector<std::pair<int64_t, int64_t>> block_groups(const hh_blocks* b, const int64_t* pofs, int64_t total,
                                                      int64_t cap, std::vector<int64_t>* pofs_at, cudaStream_t s);

// SVD recompression of the stored factors (hh_recompress.cu): replaces
// h->factors by the recompressed U, V (synchronises); and their apply.
void recompress_factors(hh_ctx* ctx, hh_hmat* h, double eps_rc, cudaStream_t s);
void recompressed_apply(const hh_hmat* h, const double* Fs, void* part, const int64_t* pofs, int transpose,
                        cudaStream_t s);

// Partial-output offsets: pofs[b] = sum_{b' < b} |target(b')| (or source if
// transpose); returns the total (synchronises).
int64_t partial_offsets(const hh_tree* t, const hh_blocks* b, int transpose, int64_t* pofs, cudaStream_t s);

// Parameters a kernel of real type R copies to shared memory.
template <typename R>
inline const R* theta_for(const hh_ctx* ctx, const hh_params& p, int* n)
{
    if (p.kernel == HH_RPY) { *n = 0; return nullptr; }
    if constexpr (sizeof(R) == 8) { *n = ctx->n_theta; return (const R*)ctx->theta64; }
    else { *n = ctx->n_theta_t; return (const R*)ctx->theta32t; }
}

inline int real_bytes(const hh_params& p) { return p.precision == HH_FP64 ? 8 : 4; }
inline int kernel_kind(const hh_params& p, int width) { return p.kernel == HH_RPY ? 2 : (width == 64 ? 1 : 0); }

// Filament suspension (hh_step.cu): bead forces of the chain potentials and
// the Euler update X += dt U.
struct FilamentArgs {
    double k, l0, kappa, g[3];
};
void filament_forces_launch(hh_ctx* ctx, const double* X, int64_t n_chains, int32_t beads, const FilamentArgs& a,
                            double* F, cudaStream_t s);
void euler_launch(double* X, const double* U, int64_t n3, double dt, cudaStream_t s);
