/*
 * hhignn.h -- C-ABI of libhhignn.so: the H-matrix mobility product of
 * H-HIGNN (arXiv 2505.08174) on one NVIDIA B300 (sm_103a).
 *
 * The library computes particle velocities
 *
 *     U = alpha_1 F + M_H F                                   (Eq. 6)
 *
 * where alpha_1 = I / (6 pi mu a) is the single-body mobility (Section 2.2,
 * Eq. 2) and M_H is the hierarchical-matrix approximation (Section 3) of the
 * dense two-body matrix M^(t,2) whose 3x3 entries are
 *
 *     M_ij = S(MLP([r/|r|, a/|r|])) / |r|,   r = x_i - x_j     (Eq. 4)
 *
 * with S(o) = [[o0,o3,o4],[o3,o1,o5],[o4,o5,o2]] (or the closed-form
 * Rotne-Prager-Yamakawa tensor when kernel = HH_RPY).  M_H is built from a
 * cluster tree (Definition 1), the admissibility partition (Eq. 7,
 * Algorithm 1), and block adaptive cross approximation on admissible blocks
 * (Algorithm 2, Eqs. 8-10); inadmissible blocks are evaluated densely.
 *
 * Conventions shared by every entry point:
 *  - Pointers named *_dev are device pointers owned by the caller; the
 *    library never frees them.  Opaque objects (hh_ctx, hh_tree, hh_blocks,
 *    hh_hmat) are owned by the library and released with the matching
 *    *_free / hh_destroy call.  An hh_blocks must not outlive its hh_tree,
 *    nor an hh_hmat its hh_blocks.
 *  - X, F, U, gU, gF, gX are [N, 3] row-major FP64.  theta is float32,
 *    packed per layer as W [out, in] row-major followed by b [out], layers
 *    4 -> w -> w -> w -> 6.
 *  - stream is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued asynchronously; calls that must read a size back from the
 *    GPU synchronise the stream internally (stated per call).  The BF16
 *    ACA (inside hh_aca and hh_predict) forks part of its work onto a
 *    second stream owned by the context and joins it back with events
 *    before the call returns, also on an error: everything the call does
 *    stays ordered on the caller's stream.  A context must therefore not
 *    be used from two host threads at once.
 *  - Every call returns hh_status.  On an error the outputs are unspecified
 *    and hh_last_error() returns a message.  HH_WARN_RANK_CAP is a warning:
 *    the outputs are valid.
 *  - The library is single-device: every object belongs to the device the
 *    context was created on; calls must be made with that device current.
 *  - The library allocates its temporaries with cudaMallocAsync on the
 *    call's stream (or the context's second stream, for work forked there)
 *    from the device's default memory pool.
 */
#ifndef HHIGNN_H
#define HHIGNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hh_ctx hh_ctx;
typedef struct hh_tree hh_tree;
typedef struct hh_blocks hh_blocks;
typedef struct hh_hmat hh_hmat;

typedef enum {
    HH_OK = 0,
    HH_ERR_ARG = 1,       /* invalid argument or unsupported combination     */
    HH_ERR_CUDA = 2,      /* a CUDA runtime call or kernel launch failed      */
    HH_ERR_OOM = 3,       /* device allocation failed                         */
    HH_ERR_TIMEOUT = 4,   /* a bounded device wait gave up                    */
    HH_ERR_NUMERIC = 5,   /* NaN/Inf input or coincident particles            */
    HH_WARN_RANK_CAP = 6  /* >= 1 admissible block stopped at max_rank        */
} hh_status;

enum { HH_FP64 = 0, HH_FP32 = 1, HH_BF16 = 2 };   /* hh_params.precision */
enum { HH_MLP = 0, HH_RPY = 1 };                  /* hh_params.kernel    */

/* Parameters of one H-matrix build (Section 3 and Section 4 notation). */
/* hh_params.flags: add the short-range terms M^(s,2) + M^(t,3) + M^(s,3) of
 * Eq. 6 (networks and R_cut from hh_set_short_range) in hh_predict and in
 * hh_matvec (forward only; the transposed product and the adjoint refuse
 * the flag with HH_ERR_ARG). */
#define HH_FLAG_SHORT_RANGE 1
/* hh_params.flags for hh_aca: keep ranks and pivots only, no factors (memory
 * O(blocks x max_rank) instead of O(sum (c+q) rank)).  Such an H-matrix
 * serves hh_matvec_backward, which rebuilds each block's factors in FP64
 * along the stored pivots; hh_matvec refuses it (HH_ERR_ARG). */
#define HH_FLAG_PIVOTS_ONLY 2

typedef struct {
    int32_t leaf_size;   /* C_leaf: a cluster is a leaf iff |tau| < C_leaf (Def. 1); 2..129 */
    double eta;          /* admissibility parameter of Eq. 7 (> 0)                          */
    double eps;          /* zeta, the ACA tolerance of Eq. 10                               */
    int32_t max_rank;    /* N_max^ite: cap on the ACA rank per block (Section 3.3), 1..64   */
    int32_t precision;   /* HH_FP64 | HH_FP32 | HH_BF16                                     */
    int32_t kernel;      /* HH_MLP | HH_RPY                                                 */
    double radius;       /* a                                                               */
    double viscosity;    /* mu                                                              */
    int32_t j1_rule;     /* 0: j_1 = first source; 1: splitmix64 hash of (seed, block)      */
    uint64_t seed;       /* seed of the j_1 hash                                            */
    int32_t shard_id;    /* this shard's share of the block work lists                      */
    int32_t n_shards;    /* number of shards (1 = everything)                               */
    int32_t flags;       /* HH_FLAG_* bits, 0 = none                                        */
    int64_t mem_budget;  /* bytes the admissible blocks of a call may hold beyond inputs,
                            tree and partition (the bounded query groups of Section 3.3):
                            half for one group's partial outputs, an eighth each for the
                            warp- and CTA-team factor workspaces, a quarter for the round
                            engine's active blocks; 0 = 32 GB                               */
} hh_params;

/* Fills *p with the defaults: leaf 32, eta 1, eps 1e-4, max_rank 48, FP32,
 * MLP, a = mu = 1, j1_rule 0, seed 0, one shard, no flags, default ACA
 * memory budget. */
void hh_default_params(hh_params *p);

/* Context: owns the MLP weights copy, a device status word and counters.
 * device: CUDA ordinal.  Leaves the caller's current device unchanged. */
hh_status hh_create(hh_ctx **ctx, int device);
void hh_destroy(hh_ctx *ctx);
/* Message of the last failing call on ctx (never NULL; "" if none). */
const char *hh_last_error(const hh_ctx *ctx);

/* Loads the pair MLP h-hat of Eq. 4: theta_dev is a device float32 vector of
 * the packed parameters of 4 -> width -> width -> width -> 6 (depth must be
 * 3, width 32 or 64).  The library copies it; the caller keeps ownership. */
hh_status hh_set_mlp(hh_ctx *ctx, const float *theta_dev, int width, int depth, void *stream);

/* Cluster tree (Definition 1, Section 3.1).  X_dev: [N, 3] FP64 device.
 * offsets: host array of batch+1 particle offsets (instance b owns rows
 * offsets[b] .. offsets[b+1]-1); batch = 1 with offsets = {0, N} for a
 * single suspension.  Per instance: Morton codes on a 2^21 grid of the
 * instance's bounding cube, a stable radix sort, breadth-first bisection at
 * the highest differing code bit, bounding boxes.  Synchronises the stream
 * once per tree level.  N < 2^30. */
hh_status hh_build_tree(hh_ctx *ctx, const double *X_dev, const int64_t *offsets, int32_t batch,
                        const hh_params *p, void *stream, hh_tree **out);

/* Admissibility partition (Eq. 7, Algorithm 1) of every instance of the tree
 * into admissible blocks P^G and inadmissible leaf blocks P^H, each sorted by
 * (target, source) node id.  Blocks whose boxes touch (dist = 0) are never
 * admissible.  Synchronises once per frontier level. */
hh_status hh_partition(hh_ctx *ctx, const hh_tree *tree, const hh_params *p, void *stream, hh_blocks **out);

/* Block ACA (Algorithm 2) on every admissible block; stores the factors C, Q
 * and the pivots resident in device memory (sum_b (|tau_b| + |sigma_b|) *
 * rank_b * 9 reals).  Runs the rank loop twice (sizes, then factors) and
 * synchronises between.  Returns HH_WARN_RANK_CAP if a block stopped at
 * max_rank before meeting Eq. 10. */
hh_status hh_aca(hh_ctx *ctx, const hh_tree *tree, const hh_blocks *blocks, const hh_params *p, void *stream,
                 hh_hmat **out);

/* U_dev = alpha_1 F + M_H F (transpose = 0) or alpha_1 F + M_H^T F
 * (transpose = 1), FP64 [N, 3] in the caller's particle order.  Inadmissible
 * blocks are recomputed from the pair kernel on every call; admissible
 * blocks use the stored factors (the recompressed ones after hh_recompress).
 * Synchronises once (work-list sizes).  hh_stats' t_apply then holds the
 * low-rank apply's device time (CUDA events, read when hh_stats is called). */
hh_status hh_matvec(hh_ctx *ctx, const hh_hmat *h, const double *F_dev, double *U_dev, int transpose,
                    void *stream);

/* One prediction U = M(X) F end to end (tree, partition, ACA fused with the
 * low-rank apply, inadmissible blocks, FP64 accumulation) without keeping
 * the factors: each admissible block's C and Q live only in a bounded
 * per-team workspace.  This is the per-time-step call of Section 2.5.
 * X_dev, F_dev, U_dev: [N, 3] FP64 device, N = offsets[batch].  Synchronises
 * as hh_build_tree and hh_partition do. */
hh_status hh_predict(hh_ctx *ctx, const double *X_dev, const double *F_dev, const int64_t *offsets,
                     int32_t batch, const hh_params *p, void *stream, double *U_dev);

/* The pair kernel of Eq. 4 (or RPY) for n separations: K_dev [n, 9] FP64
 * (row-major 3x3 per pair) = K(r_i), r_dev [n, 3] FP64 (r = x_target -
 * x_source, non-zero), in the arithmetic of p->precision (HH_BF16: the
 * tensor-core MLP used by the BF16 near field).  Asynchronous on stream. */
hh_status hh_eval_pairs(hh_ctx *ctx, const double *r_dev, int64_t n, const hh_params *p, void *stream,
                        double *K_dev);

/* Training loss of Eq. 5 (Section 2.3) and its gradient for a batch of
 * two-particle samples: r_dev [B, 3] separations (particle 1 minus particle
 * 2), e_dev [B, 3] unit forces on particle 2, U_dev [B, 3] teacher velocities
 * of particle 1 (NULL: the closed-form RPY velocity with radius a and
 * mu = 1, the stand-in for the paper's Stokesian-dynamics data); all FP64
 * device.  theta_dev: float32 packed parameters of 4 -> width -> width ->
 * width -> 6.  *loss (host) = (1/B) sum |U - K(r) e|^2 / |U|^2 with
 * K = S(MLP(f)) / |r|; grad_dev (float32, may be NULL) = dL/dtheta, summed in
 * sample order (reproducible).  Synchronises the stream. */
hh_status hh_train_loss_grad(hh_ctx *ctx, const float *theta_dev, int width, const double *r_dev,
                             const double *e_dev, const double *U_dev, int64_t batch, double radius,
                             float *grad_dev, void *stream, double *loss);

/* One training step: the loss and gradient above, then Adam (beta1 = 0.9,
 * beta2 = 0.999, eps = 1e-8, bias-corrected with step count step >= 1) on
 * theta_dev, m_dev, v_dev (float32, length of theta, caller-owned; zero m and
 * v before step 1).  *loss is the loss before the update. */
hh_status hh_train_step(hh_ctx *ctx, float *theta_dev, float *m_dev, float *v_dev, int64_t step, int width,
                        const double *r_dev, const double *e_dev, const double *U_dev, int64_t batch,
                        double radius, double lr, void *stream, double *loss);

/* Throughput probe of one arithmetic unit (measurement support for the
 * roofline of the activation-bound pair-kernel MLP; the paper has no
 * counterpart).  kind: 0 MUFU ex2.approx.f32, 1 MUFU rcp.approx.f32, 2 MUFU
 * tanh.approx.f32, 3 FP32 FMA, 4 FP64 FMA, 5 the SiLU of the tensor-core
 * epilogues (bias add, one ex2 and one rcp).  Runs iters dependent steps of 8
 * independent chains per thread on 8 CTAs x 256 threads per SM, timed with
 * CUDA events on stream; *ops_per_s receives operations per second (one FMA,
 * one MUFU op or one SiLU each).  Synchronises the stream.  HH_ERR_ARG for
 * kind outside [0, 5] or iters outside [1, 2^30]. */
hh_status hh_probe_throughput(hh_ctx *ctx, int32_t kind, int64_t iters, void *stream, double *ops_per_s);

/* Allocation-free product of one block.  The paper has no counterpart: this
 * is a service for callers that may not allocate device memory when they
 * call -- an application whose device memory is all handed to its own pool,
 * or a real-time step that must not risk the synchronisation or the failure
 * of a cudaMalloc.  y_dev [c, 3] FP64 = C (Q F), where C Q is the block
 * approximation hh_aca computes (same pivot and stopping rules; p->eps,
 * p->max_rank, p->j1_rule, p->kernel) of the block G(m, n) = K(Xt_m - Xs_n),
 * run by the SIMT kernels: p->precision HH_FP64 or HH_FP32 (HH_BF16 is
 * rejected with HH_ERR_ARG).  Xt_dev [c, 3], Xs_dev [q, 3], F_dev [q, 3]
 * FP64 device, caller-owned; rank_dev (int32, may be NULL) receives the rank
 * (rank == max_rank < min(c, q) means the block stopped at the rank cap;
 * this call returns HH_OK then, as it returns before the GPU has run).
 * 1 <= c, q <= 128 and max_rank <= 64, else HH_ERR_ARG; the current device
 * must be ctx's, else HH_ERR_ARG.  Every temporary lives in one fixed
 * 1,195,264-byte device array inside the library, held by every GPU that
 * loads it until exit: the call allocates nothing.  Each call looks up that
 * array's address on the current device; the first call on a device may load
 * the library's device code there, so make it before any stream capture.
 * Calls share the array: two calls that overlap on the GPU race.  ctx must
 * have been created (and hh_set_mlp called for the MLP kernel) beforehand;
 * the call is asynchronous on stream. */
hh_status hh_aca_block_apply_noalloc(hh_ctx *ctx, const double *Xt_dev, int32_t c, const double *Xs_dev, int32_t q,
                                     const double *F_dev, const hh_params *p, void *stream, double *y_dev,
                                     int32_t *rank_dev);

/* Adjoint of L = sum_i gU_i . U_i for U = alpha_1 F + M_H F built by hh_aca
 * with the MLP kernel (Section 3, Eqs. 4 and 8 differentiated; the paper
 * trains the MLP on pairs and has no H-matrix adjoint): gF_dev = alpha_1 gU
 * + M_H^T gU (FP64 [N,3]), gX_dev += dL/dX (FP64 [N,3]) and gtheta_dev +=
 * dL/dtheta (float32, length of theta), the last two with tree, partition
 * and ACA pivots frozen.  The admissible blocks are differentiated in FP64:
 * for an FP32 or BF16 h, along the pivots of the FP64 H-matrix on the same
 * tree and partition (its ACA, pivots only, is run inside the call; pivots
 * picked from low-precision residuals do not give a usable derivative of
 * the rank recursion).  The near-field entries are differentiated in the
 * precision the product used for them (FP64 for an FP64 h, else FP32).
 * When h holds pivots only, its FP64 factors are rebuilt group by group
 * (hh_params.mem_budget bounds the groups' buffers), and gF_dev's
 * admissible part comes from them: equal to the transposed product up to
 * summation order.  Every sum has a fixed order: repeated calls give the
 * same bits.  Any of gF_dev, gX_dev, gtheta_dev may be NULL; gX and gtheta
 * are accumulated into (zero them first).  Activations are recomputed, not
 * stored. */
hh_status hh_matvec_backward(hh_ctx *ctx, const hh_hmat *h, const double *gU_dev, const double *F_dev,
                             double *gF_dev, double *gX_dev, float *gtheta_dev, void *stream);

/* Copies the tree to host buffers (any pointer may be NULL).  perm[N]: input
 * row of each sorted position; codes[N]: sorted Morton codes; node arrays of
 * length n_nodes (child is [n_nodes, 2], -1 for leaves; lo/hi [n_nodes, 3]).
 * Synchronises the device. */
hh_status hh_export_tree(const hh_tree *tree, int32_t *perm, uint64_t *codes, int32_t *node_begin,
                         int32_t *node_end, int32_t *node_child, double *node_lo, double *node_hi,
                         int64_t *n_nodes, int64_t *n);

/* Copies the block lists ([n, 2] (target, source) node ids, sorted) to host
 * buffers (NULL pointers skipped).  Synchronises the device. */
hh_status hh_export_blocks(const hh_blocks *blocks, int32_t *PG, int64_t *nG, int32_t *PH, int64_t *nH);

/* The split of the work over n_shards shards (hh_params.shard_id /
 * n_shards; Section 3.3's workloads): block_owner[nG] receives the shard of
 * each admissible block (cut into contiguous ranges of equal cumulative
 * W^G = max(|tau|, |sigma|)), node_owner[n_nodes] the shard of each target
 * node's inadmissible blocks (contiguous ranges of equal cumulative W^H =
 * |tau| sum_sigma |sigma|).  Either pointer may be NULL (host buffers).
 * Synchronises the device. */
hh_status hh_shard_owners(const hh_blocks *blocks, int32_t n_shards, int32_t *block_owner, int32_t *node_owner);

/* Copies the per-block ACA ranks ([nG]) and pivots ([nG, max_rank]
 * block-local row / column indices, -1 past the rank) to host buffers. */
hh_status hh_export_aca(const hh_hmat *h, int32_t *ranks, int32_t *piv_rows, int32_t *piv_cols, int64_t *nG,
                        int32_t *max_rank);

/* Copies the stored ACA factors of Algorithm 2 to host buffers (Eq. 8: the
 * admissible block (tau, sigma) is C Q, C = [c_0 .. c_{l-1}], Q = [q_0 ..
 * q_{l-1}]).  fofs[nG + 1]: element offsets; block b's factors start at
 * element fofs[b] and hold C as [l][9][c] then Q as [l][9][q] (the 3x3
 * entries c_p(m)[u][v] at (p * 9 + 3u + v) * c + m, component-major), with l
 * = ranks[b], c = |tau|, q = |sigma|.  factors receives n_factor * 9 reals of
 * *real_bytes bytes each (8 for HH_FP64, else 4).  Pass NULL for fofs and
 * factors to query n_factor and real_bytes.  HH_ERR_ARG if h was built with
 * HH_FLAG_PIVOTS_ONLY.  Synchronises the device. */
hh_status hh_export_factors(const hh_hmat *h, int64_t *fofs, void *factors, int64_t *n_factor, int32_t *real_bytes);

typedef struct {
    double t_tree, t_part, t_near, t_aca, t_apply, t_acc; /* ms of the last call's stages (CUDA events) */
    int64_t n_near_pairs;   /* pair-kernel evaluations in inadmissible blocks */
    int64_t n_aca_queries;  /* pair-kernel evaluations inside ACA            */
    int64_t n_blocks_G, n_blocks_H, n_nodes;
    int64_t rank_hist[65];  /* rank_hist[min(rank, 64)] (hh_aca only)        */
    double t_kernel_aca;    /* ms inside the ACA team kernels (CUDA events)   */
    double t_kernel_near;   /* ms inside the near-field kernel (CUDA events)  */
    int64_t n_launches;     /* kernels this library launched in the call
                               (hh_filament_step: the whole step)            */
    double t_short;         /* ms of the short-range terms (0 when off)       */
    int64_t n_short_pairs;  /* neighbour pairs within R_cut (directed)        */
    int64_t mem_peak_bytes; /* high-water mark of the device's default memory
                               pool during the call: the library's stream-
                               ordered temporaries (plus any other user of
                               that pool); -1 if the driver does not report
                               it                                            */
    int64_t n_aca_rounds;   /* rounds of the BF16 block ACA (0 for the other
                               precisions)                                   */
    double t_aca_tiles;     /* ms in the BF16 ACA's tile kernels (CUDA events) */
    double t_aca_steps;     /* ms in its step kernels (CUDA events)            */
    int64_t n_aca_groups;   /* hh_predict: groups the admissible blocks ran in
                               (their partial outputs within half of
                               hh_params.mem_budget each)                    */
} hh_stats_t;

/* Short-range networks of Eq. 6 (Eq. 2 with the Eq. 4 normalisations; the
 * paper trains them on three-particle data, here they are caller-supplied):
 *   two-body self part  alpha_2^(s)(i, j) = (a/d)^4 / d * S(MLP_s([r/d, a/d])),
 *                       r = x_i - x_j, d = |r|, applied to F_i;
 *   three-body          alpha_3 = [S(o_0..5), S(o_6..11)] / (|x_j - x_k| |x_k - x_i|),
 *                       o = MLP_3([r_ji/|r_ji|, r_ki/|r_ki|, a/|x_j - x_k|]),
 *                       r_ji = x_j - x_i, r_ki = x_k - x_i, applied to [F_i; F_j],
 * summed over j in N(i) and over the 3-cliques (j, k, i) with i, j in N(k),
 * j != i, where N(i) = { j != i : |x_i - x_j| < r_cut } within one
 * suspension.  S(o) = [[o0,o3,o4],[o3,o1,o5],[o4,o5,o2]].  theta_s_dev:
 * MLP 4 -> width -> width -> width -> 6, theta_3_dev: MLP 7 -> width x 3 ->
 * 12, both float32 device arrays packed per layer as W[out, in] then b[out]
 * (copied; either may be NULL to leave its term out); width 32 or 64;
 * r_cut > 0.  Positions spanning more than 65535 r_cut per axis in one
 * suspension make the calls that use them fail with HH_ERR_NUMERIC. */
hh_status hh_set_short_range(hh_ctx *ctx, const float *theta_s_dev, const float *theta_3_dev, int width,
                             double r_cut, void *stream);

/* U_dev [N,3] FP64 (caller order) += the short-range terms above for X_dev,
 * F_dev [N,3] FP64, suspensions given by offsets (host, [batch+1]) as in
 * hh_predict; p->precision selects FP64 or FP32 arithmetic, p->radius is a.
 * Asynchronous on stream except for one size query. */
hh_status hh_short_range(hh_ctx *ctx, const double *X_dev, const double *F_dev, const int64_t *offsets,
                         int32_t batch, const hh_params *p, void *stream, double *U_dev);

/* Counters of the last hh_predict / hh_aca / hh_filament_step on ctx. */
hh_status hh_stats(hh_ctx *ctx, hh_stats_t *out);

/* Launch shape of the block-ACA and near-field kernels (the paper fixes
 * none; this is the B300 tuning surface).  0 in a field selects its default.
 *   small_max      blocks with both sides <= small_max go to warp teams (32
 *                  threads per block), the others to CTA teams; 32..512,
 *                  default 512
 *   aca_small_cps  CTAs per SM of the warp-team ACA kernel, 1..8, default 4
 *   aca_large_cps  CTAs per SM of the CTA-team ACA kernel, 1..8, default 2
 *                  (256-thread FP32 / FP64 kernel) or 4 (128-thread BF16
 *                  tensor-core kernel)
 *   near_cps       CTAs per SM of the tensor-core near-field kernel, 1..8,
 *                  default 5 (its 96 registers and shared tiles fit five)
 *   rounds_min_cq  (HH_BF16) admissible blocks with c + q above this value go
 *                  through the round-based ACA (every block of a size class
 *                  advancing one phase per round, its rows spread over the
 *                  whole GPU) instead of one CTA team each; 513..2^30, or 0
 *                  for the default 4096
 * Grids are further capped by the amount of work and the workspace budget;
 * the SM's occupancy limits how many CTAs actually run at once. */
typedef struct {
    int32_t small_max;
    int32_t aca_small_cps;
    int32_t aca_large_cps;
    int32_t near_cps;
    int32_t rounds_min_cq;
    int32_t reserved[3];   /* 0 */
} hh_launch_cfg;

/* Set / read ctx's launch shape (as stored: 0 = default).  Out-of-range
 * fields: HH_ERR_ARG, nothing changed. */
hh_status hh_set_launch(hh_ctx *ctx, const hh_launch_cfg *cfg);
hh_status hh_get_launch(hh_ctx *ctx, hh_launch_cfg *cfg);

/* Autotuner: times hh_predict on X_dev (FP64 [N,3] device, offsets / batch
 * as in hh_predict, every force (1, 1, 1)) under p for candidate launch
 * shapes and keeps the fastest on ctx (also written to *best when not NULL).
 * Coordinate descent from ctx's current shape: each field in turn is swept
 * over a fixed candidate list (small_max 128 / 256 / 512, aca_small_cps 1..4,
 * aca_large_cps 1 / 2 / 4, near_cps 2 / 4 / 5 / 8, rounds_min_cq 2048 / 4096 /
 * 16384) with the others held, and the
 * value of the smallest median time over reps (>= 1) predictions is kept.
 * Results do not depend on the launch shape beyond FP rounding order of the
 * per-block partial sums (none: each block's output is written once). */
hh_status hh_autotune(hh_ctx *ctx, const double *X_dev, const int64_t *offsets, int32_t batch, const hh_params *p,
                      int32_t reps, void *stream, hh_launch_cfg *best);

/* Filament suspension (the paper's filament application, Section 4.3).
 * Chains are `beads` consecutive rows of X (chain c = rows c*beads ..
 * c*beads + beads - 1, in order along the chain).  With r = x_{j+1} - x_j
 * and t = r / |r| along a chain, the bead forces are F = -grad E of
 *   E = sum_bonds (k_bond/2)(|r| - l0)^2            (the bond spring of Eq. 12)
 *     + sum_joints kappa (1 - t_j . t_{j+1})        (bending)
 *     - sum_beads g . x                             (uniform body force)
 * The paper prints a bending force whose form is garbled; this potential's
 * gradient is used instead. */
typedef struct {
    double k_bond;   /* bond stiffness k (100 in the 1M-bead suspension)   */
    double l0;       /* bond rest length (2.2 a)                            */
    double kappa;    /* bending stiffness (10)                              */
    double g[3];     /* force on every bead, e.g. gravity (0, 0, -1)        */
} hh_filament_params;

/* F_dev [n_chains * beads, 3] FP64 device (caller-owned) = the bead forces
 * above for X_dev (same layout).  n_chains >= 0, beads >= 1 (a one-bead
 * chain feels g only), n_chains * beads < 2^31.  A zero-length bond or a
 * non-finite result gives HH_ERR_NUMERIC (F then unspecified).
 * Synchronises the stream (status read-back). */
hh_status hh_filament_forces(hh_ctx *ctx, const double *X_dev, int64_t n_chains, int32_t beads,
                             const hh_filament_params *fp, void *stream, double *F_dev);

/* One explicit Euler step of the filament suspension (Section 2.5's time
 * step with the forces of Section 4.3's filaments), in place on X_dev:
 *   F = hh_filament_forces(X);  U = alpha_1 F + M_H(X) F  (hh_predict under p,
 *   one suspension);  X <- X + dt U.
 * F_dev and U_dev ([N, 3] FP64 device, caller-owned) receive the step's F
 * and U.  n_chains >= 1.  Errors as hh_filament_forces and hh_predict; on
 * an error X is unchanged.  HH_WARN_RANK_CAP from the prediction is passed
 * on (X is updated).  Synchronises as hh_predict does. */
hh_status hh_filament_step(hh_ctx *ctx, double *X_dev, int64_t n_chains, int32_t beads,
                           const hh_filament_params *fp, const hh_params *p, double dt, void *stream,
                           double *F_dev, double *U_dev);

/* A run of explicit Euler steps of a suspension of chains and free
 * particles (Section 2.5's time stepping; the drop and filament runs of
 * Section 4.3), in place on X_dev ([N, 3] FP64 device, N = n_chains * beads
 * + n_free): rows 0 .. n_chains * beads - 1 are chains as in
 * hh_filament_forces, the remaining n_free rows free particles that feel
 * fp->g only (a drop: n_chains = 0).  Each step k = 1 .. n_steps:
 *   F = forces(X);  U = alpha_1 F + M_H(X) F (hh_predict under p);  X += dt U.
 * With dump_every > 0, X_dump_host (host, caller-owned, FP64
 * [n_steps / dump_every + 1, N, 3]) receives the initial X in slot 0 and X
 * after step k in slot k / dump_every for every k divisible by dump_every.
 * t_step_ms (host, [n_steps], may be NULL) receives each step's device time
 * (CUDA events: forces through update).  Errors as hh_filament_step; an
 * error stops the run with X after the last completed step (the dumps up
 * to it written).  HH_WARN_RANK_CAP from any step is returned at the end.
 * Synchronises the device's work on stream before it returns. */
hh_status hh_simulate(hh_ctx *ctx, double *X_dev, int64_t n_chains, int32_t beads, int64_t n_free,
                      const hh_filament_params *fp, const hh_params *p, double dt, int32_t n_steps,
                      int32_t dump_every, double *X_dump_host, double *t_step_ms, void *stream);

/* Recompression of the stored ACA factors by truncated SVD (the paper
 * stores the ACA factors as they come; this lowers the bytes the low-rank
 * apply reads).  Per admissible block, M = sum_k C_k Q_k in scalar form
 * (3|tau| x 3|sigma|, scalar rank <= 3 rank) is replaced by U V with U
 * (3|tau| x r), V (r x 3|sigma|) and r the smallest rank whose discarded
 * singular values satisfy sum_{i>=r} s_i^2 <= eps_rc^2 sum_i s_i^2, so
 * ||M - U V||_F <= eps_rc ||M||_F (Eckart-Young; the singular values come
 * from FP64 Jacobi eigendecompositions of the factors' Gram matrices and a
 * 3 rank x 3 rank core, values below ~3e-8 of the largest count as zero).
 * U and V are stored in h's real type; the ACA factors are freed.  h must
 * hold factors (not HH_FLAG_PIVOTS_ONLY) and max_rank <= 64; eps_rc in
 * [0, 1).  hh_matvec then applies U V; hh_matvec_backward treats h as
 * pivots-only (rebuilds its FP64 factors).  Synchronises. */
hh_status hh_recompress(hh_ctx *ctx, hh_hmat *h, double eps_rc, void *stream);

/* Copies the recompressed factors to host buffers (NULL pointers skipped):
 * srank[nG] kept ranks, sofs[nG+1] offsets in reals, sfac[n_sfac] (block b
 * at sofs[b]: U row-major [r][3|tau|] -- row rho holds column rho of U --
 * then V [r][3|sigma|]; entry 3m + u of a U row is particle m, component u).
 * HH_ERR_ARG if h was not recompressed.  Synchronises the device. */
hh_status hh_export_recompressed(const hh_hmat *h, int32_t *srank, int64_t *sofs, void *sfac, int64_t *n_sfac,
                                 int32_t *real_bytes);

/* Test hooks for the failure paths (the paper has no counterpart).
 *
 * hh_debug_fail_alloc(n): the n-th device allocation made by the library
 * from now on (n >= 1; process-wide) fails as if the pool were exhausted;
 * the call that meets it returns HH_ERR_OOM after waiting for the device
 * and freeing every temporary it had made, so the pool's used memory
 * returns to its level before the call and the context stays usable.  n = 0
 * cancels a pending failure.
 *
 * hh_debug_stall_mma_waits(ctx, polls): polls > 0 makes every MMA
 * completion wait of this context's tensor-core kernels (HH_BF16) watch,
 * for `polls` polls, an mbarrier that nothing arrives at instead of the
 * MMA's own, so the wait runs out as it would for an MMA that never
 * completed: the kernel records HH_ERR_TIMEOUT and abandons its work, and
 * before it releases its accumulator memory it still waits, with the
 * built-in limit (2^26 polls), for the MMA it issued.  polls = 0 restores
 * normal waits.  Synchronises the device; HH_ERR_CUDA on a failed copy. */
void hh_debug_fail_alloc(int64_t n);
hh_status hh_debug_stall_mma_waits(hh_ctx *ctx, uint32_t polls);

void hh_tree_free(hh_tree *t);
void hh_blocks_free(hh_blocks *b);
void hh_hmat_free(hh_hmat *h);

#ifdef __cplusplus
}
#endif
#endif /* HHIGNN_H */
