// hh_noalloc.cu -- hh_aca_block_apply_noalloc: the low-rank product of one
// block through the block ACA team kernel, with no device allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// result: an application that has handed its whole device memory to its own
// pool, a real-time loop that must not risk the synchronisation or the
// failure a cudaMalloc can bring mid-step, or a host library that is only
// allowed to use memory it was given.  For them this entry point keeps every
// temporary -- the inputs staged contiguously, the one-block work lists, the
// team's C/Q workspace and the partial output -- in one file-scope device
// array of fixed size, so the call itself allocates nothing (it needs a
// context set up earlier for the network weights and its status word).
//
// The array's host-side name is not a device address.  Every call looks the
// address up with cudaGetSymbolAddress for the current device and passes it
// to the kernels (nothing is cached, so a device reset or a new primary
// context never leaves a stale address behind).  The first call on a device
// may also load the library's device code there, so make it before any
// stream capture.  All calls share the array; each call rewrites everything
// it reads (the work counter included), but two calls that overlap on the
// GPU -- on different streams, or from different threads -- race on it.
#include "hh_internal.h"

namespace {

constexpr int NA_MAX_SIDE = 128;   // targets and sources per call
constexpr int NA_MAX_RANK = 64;
// team workspace: C [rank][9][c] + Q [rank][9][q] in FP64 at the largest size
constexpr size_t NA_WS_BYTES = (size_t)2 * NA_MAX_SIDE * 9 * NA_MAX_RANK * sizeof(double);
constexpr size_t NA_POS_BYTES = (size_t)2 * NA_MAX_SIDE * 3 * sizeof(double);  // targets then sources
constexpr size_t NA_F_BYTES = NA_POS_BYTES;                                       // forces, same rows
constexpr size_t NA_PART_BYTES = (size_t)NA_MAX_SIDE * 3 * sizeof(double);
constexpr size_t NA_META_BYTES = 256;
constexpr size_t NA_OFF_POS = NA_WS_BYTES;
constexpr size_t NA_OFF_F = NA_OFF_POS + NA_POS_BYTES;
constexpr size_t NA_OFF_PART = NA_OFF_F + NA_F_BYTES;
constexpr size_t NA_OFF_META = NA_OFF_PART + NA_PART_BYTES;
constexpr size_t NA_TOTAL = NA_OFF_META + NA_META_BYTES;
static_assert(NA_TOTAL == 1195264, "the header states the array's size (1.2 MB)");

static __device__ __align__(256) unsigned char g_na_scratch[NA_TOTAL];

struct Meta {               // lives at NA_OFF_META
    unsigned long long counter;
    int64_t pofs[1];
    int32_t PG[2];
    int32_t nbeg[2];
    int32_t nend[2];
    int32_t work[1];
    int32_t rank[1];
};
static_assert(sizeof(Meta) <= NA_META_BYTES, "meta area too small");

// Stage the block: positions (targets then sources), forces (zero on the
// targets), one-block lists, zeroed work counter.
__global__ void k_na_stage(const double* __restrict__ Xt, int c, const double* __restrict__ Xsrc, int q,
                           const double* __restrict__ F, unsigned char* __restrict__ base)
{
    double* X = reinterpret_cast<double*>(base + NA_OFF_POS);
    double* Fs = reinterpret_cast<double*>(base + NA_OFF_F);
    for (int i = threadIdx.x; i < 3 * c; i += blockDim.x) {
        X[i] = Xt[i];
        Fs[i] = 0.0;
    }
    for (int i = threadIdx.x; i < 3 * q; i += blockDim.x) {
        X[3 * c + i] = Xsrc[i];
        Fs[3 * c + i] = F[i];
    }
    if (threadIdx.x == 0) {
        Meta* m = reinterpret_cast<Meta*>(base + NA_OFF_META);
        m->counter = 0;
        m->pofs[0] = 0;
        m->PG[0] = 0;
        m->PG[1] = 1;
        m->nbeg[0] = 0;
        m->nend[0] = c;
        m->nbeg[1] = c;
        m->nend[1] = c + q;
        m->work[0] = 0;
        m->rank[0] = 0;
    }
}

template <typename R>
__global__ void k_na_out(const unsigned char* __restrict__ base, int c, double* __restrict__ y,
                         int32_t* __restrict__ rank)
{
    const R* part = reinterpret_cast<const R*>(base + NA_OFF_PART);
    for (int i = threadIdx.x; i < 3 * c; i += blockDim.x) y[i] = (double)part[i];
    if (rank && threadIdx.x == 0) rank[0] = reinterpret_cast<const Meta*>(base + NA_OFF_META)->rank[0];
}

// Device address of g_na_scratch on the current device, which must be the
// context's device (the weights and the status word live there).
void* na_scratch_for_device(int ctx_device)
{
    int dev = -1;
    HH_CUDA(cudaGetDevice(&dev));
    HH_REQUIRE(dev == ctx_device, HH_ERR_ARG,
               "hh_aca_block_apply_noalloc: the current device is not the context's device");
    void* p = nullptr;
    HH_CUDA(cudaGetSymbolAddress(&p, g_na_scratch));
    HH_REQUIRE(p != nullptr, HH_ERR_CUDA, "cudaGetSymbolAddress returned NULL");
    return p;
}

}  // namespace

extern "C" hh_status hh_aca_block_apply_noalloc(hh_ctx* ctx, const double* Xt_dev, int32_t c, const double* Xs_dev,
                                                int32_t q, const double* F_dev, const hh_params* p, void* stream,
                                                double* y_dev, int32_t* rank_dev)
{
    if (!ctx) return HH_ERR_ARG;
    try {
        check_params_public(ctx, p);
        HH_REQUIRE(Xt_dev && Xs_dev && F_dev && y_dev, HH_ERR_ARG, "NULL argument");
        HH_REQUIRE(c >= 1 && q >= 1, HH_ERR_ARG, "block sides must be >= 1");
        HH_REQUIRE(c <= NA_MAX_SIDE && q <= NA_MAX_SIDE, HH_ERR_ARG,
                   "hh_aca_block_apply_noalloc: at most 128 targets and 128 sources per call");
        HH_REQUIRE(p->max_rank <= NA_MAX_RANK, HH_ERR_ARG, "max_rank must be <= 64");
        HH_REQUIRE(p->precision != HH_BF16, HH_ERR_ARG,
                   "hh_aca_block_apply_noalloc runs the SIMT kernels only: use HH_FP32 or HH_FP64");
        cudaStream_t s = (cudaStream_t)stream;
        unsigned char* base = static_cast<unsigned char*>(na_scratch_for_device(ctx->device));
        // the status bits of this call start from zero (a memset allocates nothing)
        HH_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), s));
        Meta* meta = reinterpret_cast<Meta*>(base + NA_OFF_META);
        k_na_stage<<<1, 256, 0, s>>>(Xt_dev, c, Xs_dev, q, F_dev, base);
        HH_CHECK_LAUNCH();
        aca_single_block_ws(ctx, *p, c, q, reinterpret_cast<const double*>(base + NA_OFF_POS),
                            reinterpret_cast<const double*>(base + NA_OFF_F), meta->PG, meta->nbeg, meta->nend,
                            meta->work, &meta->counter, base, base + NA_OFF_PART, meta->pofs, meta->rank, s);
        if (p->precision == HH_FP64) k_na_out<double><<<1, 256, 0, s>>>(base, c, y_dev, rank_dev);
        else k_na_out<float><<<1, 256, 0, s>>>(base, c, y_dev, rank_dev);
        HH_CHECK_LAUNCH();
        ctx->err.clear();
        return HH_OK;
    } catch (const HHError& e) {
        ctx->err = e.msg;
        return e.st;
    }
}
