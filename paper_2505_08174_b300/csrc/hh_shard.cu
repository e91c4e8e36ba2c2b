// hh_shard.cu -- the split of one prediction's work over shards (one per GPU)
// by the workloads of Section 3.3: the admissible blocks by the ACA workload
// W^G = max(|tau|, |sigma|) of each block, the inadmissible blocks by W^H =
// |tau| |sigma|, taken per target leaf (the near field's work unit).  Each
// list -- blocks in their (tau, sigma) order, nodes by number -- is cut into
// n_shards contiguous ranges of equal cumulative cost: item i of cost w_i,
// exclusive prefix P_i and total T belongs to shard
//   min(n - 1, floor(n (P_i + w_i / 2) / T)),
// so a shard's cost is within one item of T / n.  Every shard runs the same
// tree and partition (they are cheap); only these items are divided.
#include "hh_internal.h"

namespace {

__global__ void k_block_cost(const int32_t* __restrict__ PG, int64_t nG, const int32_t* __restrict__ nbeg,
                             const int32_t* __restrict__ nend, int64_t* __restrict__ cost)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nG) return;
    const int32_t c = nend[PG[2 * b]] - nbeg[PG[2 * b]], q = nend[PG[2 * b + 1]] - nbeg[PG[2 * b + 1]];
    cost[b] = max(c, q);
}

__global__ void k_node_cost(const int64_t* __restrict__ rowH, const int32_t* __restrict__ PH, int32_t n_nodes,
                            const int32_t* __restrict__ nbeg, const int32_t* __restrict__ nend,
                            int64_t* __restrict__ cost)
{
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nodes) return;
    int64_t q = 0;
    for (int64_t h = rowH[t]; h < rowH[t + 1]; ++h) q += nend[PH[2 * h + 1]] - nbeg[PH[2 * h + 1]];
    cost[t] = (int64_t)(nend[t] - nbeg[t]) * q;
}

__global__ void k_owner(const int64_t* __restrict__ excl, const int64_t* __restrict__ cost, int64_t n,
                        const int64_t* __restrict__ total, int n_shards, int32_t* __restrict__ owner)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double T = (double)*total;
    const double mid = (double)excl[i] + 0.5 * (double)cost[i];
    const int o = T > 0.0 ? (int)floor((double)n_shards * mid / T) : 0;
    owner[i] = min(max(o, 0), n_shards - 1);
}

__global__ void k_mine(const int32_t* __restrict__ owner, int64_t n, int shard, uint8_t* __restrict__ mine)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) mine[i] = owner[i] == shard;
}

// Owners of n items of the given costs (device arrays, n >= 1).
void owners(const int64_t* cost, int64_t n, int n_shards, int32_t* owner, cudaStream_t s)
{
    int64_t* excl = dev_alloc_t<int64_t>(n, s);
    int64_t* tot = dev_alloc_t<int64_t>(1, s);
    dev_scan_i64(cost, excl, n, tot, s);
    k_owner<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(excl, cost, n, tot, n_shards, owner);
    HH_CHECK_LAUNCH();
    dev_free(tot, s);
    dev_free(excl, s);
}

void block_owners(const hh_tree* t, const hh_blocks* b, int n_shards, int32_t* owner, cudaStream_t s)
{
    int64_t* cost = dev_alloc_t<int64_t>(b->nG, s);
    k_block_cost<<<(unsigned)ceil_div(b->nG, 256), 256, 0, s>>>(b->PG, b->nG, t->nbeg, t->nend, cost);
    HH_CHECK_LAUNCH();
    owners(cost, b->nG, n_shards, owner, s);
    dev_free(cost, s);
}

void node_owners(const hh_tree* t, const hh_blocks* b, int n_shards, int32_t* owner, cudaStream_t s)
{
    int64_t* cost = dev_alloc_t<int64_t>(t->n_nodes, s);
    k_node_cost<<<(unsigned)ceil_div(t->n_nodes, 256), 256, 0, s>>>(b->rowH, b->PH, t->n_nodes, t->nbeg, t->nend,
                                                                   cost);
    HH_CHECK_LAUNCH();
    owners(cost, t->n_nodes, n_shards, owner, s);
    dev_free(cost, s);
}

}  // namespace

uint8_t* shard_block_flags(const hh_tree* t, const hh_blocks* b, const hh_params& p, cudaStream_t s)
{
    if (p.n_shards <= 1 || b->nG == 0) return nullptr;
    int32_t* owner = dev_alloc_t<int32_t>(b->nG, s);
    block_owners(t, b, p.n_shards, owner, s);
    uint8_t* mine = dev_alloc_t<uint8_t>(b->nG, s);
    k_mine<<<(unsigned)ceil_div(b->nG, 256), 256, 0, s>>>(owner, b->nG, p.shard_id, mine);
    HH_CHECK_LAUNCH();
    dev_free(owner, s);
    return mine;
}

uint8_t* shard_node_flags(const hh_tree* t, const hh_blocks* b, const hh_params& p, cudaStream_t s)
{
    if (p.n_shards <= 1 || t->n_nodes == 0) return nullptr;
    int32_t* owner = dev_alloc_t<int32_t>(t->n_nodes, s);
    node_owners(t, b, p.n_shards, owner, s);
    uint8_t* mine = dev_alloc_t<uint8_t>(t->n_nodes, s);
    k_mine<<<(unsigned)ceil_div(t->n_nodes, 256), 256, 0, s>>>(owner, t->n_nodes, p.shard_id, mine);
    HH_CHECK_LAUNCH();
    dev_free(owner, s);
    return mine;
}

extern "C" hh_status hh_shard_owners(const hh_blocks* b, int32_t n_shards, int32_t* block_owner, int32_t* node_owner)
{
    if (!b || !b->tree) return HH_ERR_ARG;
    hh_ctx* ctx = b->tree->ctx;
    AllocScope scope;
    try {
        HH_REQUIRE(n_shards >= 1, HH_ERR_ARG, "n_shards must be >= 1");
        const hh_tree* t = b->tree;
        cudaStream_t s = 0;
        if (block_owner && b->nG > 0) {
            int32_t* o = dev_alloc_t<int32_t>(b->nG, s);
            block_owners(t, b, n_shards, o, s);
            HH_CUDA(cudaMemcpyAsync(block_owner, o, sizeof(int32_t) * b->nG, cudaMemcpyDeviceToHost, s));
            dev_free(o, s);
        }
        if (node_owner && t->n_nodes > 0) {
            int32_t* o = dev_alloc_t<int32_t>(t->n_nodes, s);
            node_owners(t, b, n_shards, o, s);
            HH_CUDA(cudaMemcpyAsync(node_owner, o, sizeof(int32_t) * t->n_nodes, cudaMemcpyDeviceToHost, s));
            dev_free(o, s);
        }
        HH_CUDA(cudaStreamSynchronize(s));
        if (ctx) ctx->err.clear();
        return HH_OK;
    } catch (const HHError& e) {
        scope.release();
        if (ctx) ctx->err = e.msg;
        return e.st;
    }
}
