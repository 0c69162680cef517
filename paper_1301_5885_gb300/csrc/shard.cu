// shard.cu -- row sharding of one solve over several GPUs (the multi-GPU
// direction the paper names in its conclusion, Section 4).
//
// The product y = A u of Eqs. (12)-(13) is split by target rows: rank p owns
// rows [p P, p P + n_p) of both row blocks, P = ceil(N / world), and holds
// the whole geometry (O(N), replicated).  Every product then needs the full
// u (which every rank has: GMRES runs replicated) and one exchange: each rank
// evaluates its rows (N P pair evaluations, the O(N^2 / world) part), the
// ranks allgather their 2 P row values, and every rank unpacks the gathered
// blocks into the full 2N vector.  GMRES itself (orthogonalisation, Givens,
// the true residual) then runs identically on every rank, on identical data
// in a fixed summation order, so no further collective is needed and every
// rank ends with the same x and energy.
//
// The library does not link a communication library: the caller passes an
// allgather callback (for example torch.distributed over NCCL) that the
// library calls, from the thread that called pb_solve_sharded, once per
// product.
#include <string.h>

#include "pb_internal.cuh"

namespace pb {
namespace {

// gathered layout: rank q's block is recv[q 2P .. (q+1) 2P), its phi rows
// first (P slots, n_q used), then its psi rows (P slots)
__global__ void shard_unpack_kernel(const double *__restrict__ recv, int64_t N, int world, int64_t per,
                                    double *__restrict__ y, const int *__restrict__ skip) {
    if (skip != nullptr && *((volatile const int *)skip)) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t q = i / per, t = i - q * per;
    const double *blk = recv + q * 2 * per;
    y[i] = blk[t];
    y[N + i] = blk[per + t];
}

__global__ void zero_kernel(double *p, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0.0;
}

void rows_of(int64_t N, int world, int rank, int64_t *row0, int64_t *nrows, int64_t *per) {
    const int64_t P = (N + world - 1) / world;
    int64_t r0 = (int64_t)rank * P;
    if (r0 > N) r0 = N;
    int64_t n = N - r0;
    if (n > P) n = P;
    *row0 = r0;
    *nrows = n;
    *per = P;
}

}  // namespace

pb_status shard_product(pb_ctx *ctx, const double *u, double *y, pb_precision prec, const int *skip_flag) {
    auto &sh = ctx->shard;
    if (prec != PB_FP32PAIR && prec != PB_FP64)
        return set_error(ctx, PB_ERR_ARG, "sharded product: FP32 pairs or FP64 only (not precision %d)", (int)prec);
    // own rows into the send block (phi rows, then psi rows, P slots each)
    pb_status s = matvec_rows_launch(ctx, u, sh.send, RowBlock{sh.row0, sh.nrows, sh.per}, prec, skip_flag);
    if (s != PB_OK) return s;
    const int rc = sh.fn(sh.user, sh.send, sh.recv, 2 * sh.per, (void *)ctx->stream);
    if (rc != 0) return set_error(ctx, PB_ERR_CUDA, "sharded product: the allgather callback returned %d", rc);
    sh.gathers += 1;
    const int threads = 256;
    shard_unpack_kernel<<<(unsigned)((ctx->N + threads - 1) / threads), threads, 0, ctx->stream>>>(
        sh.recv, ctx->N, sh.world, sh.per, y, skip_flag);
    PB_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PB_OK : cuda_error(ctx, e, "sharded product: unpack");
}

}  // namespace pb

using namespace pb;

extern "C" pb_status pb_shard_rows(int64_t N, int world, int rank, int64_t *row0, int64_t *nrows,
                                   int64_t *rows_per_rank) {
    if (N < 1 || world < 1 || rank < 0 || rank >= world || !row0 || !nrows || !rows_per_rank)
        return set_error(nullptr, PB_ERR_ARG, "pb_shard_rows: need N >= 1, 0 <= rank < world");
    rows_of(N, world, rank, row0, nrows, rows_per_rank);
    return PB_OK;
}

extern "C" pb_status pb_shard_unpack_host(const double *gathered, int64_t N, int world, double *y) {
    if (!gathered || !y || N < 1 || world < 1)
        return set_error(nullptr, PB_ERR_ARG, "pb_shard_unpack_host: bad arguments");
    const int64_t P = (N + world - 1) / world;
    for (int64_t i = 0; i < N; ++i) {
        const int64_t q = i / P, t = i - q * P;
        y[i] = gathered[q * 2 * P + t];
        y[N + i] = gathered[q * 2 * P + P + t];
    }
    return PB_OK;
}

extern "C" pb_status pb_matvec_rows(pb_ctx *ctx, const double *u, double *y_rows, int64_t row0, int64_t nrows,
                                    pb_precision prec) {
    if (!ctx || !u || !y_rows) return set_error(ctx, PB_ERR_ARG, "pb_matvec_rows: NULL argument");
    return matvec_rows_launch(ctx, u, y_rows, RowBlock{row0, nrows, nrows}, prec, nullptr);
}

extern "C" pb_status pb_solve_sharded(pb_ctx *ctx, const pb_solve_opts *opts, int rank, int world,
                                      pb_allgather_fn allgather, void *user, const double *x0, double *x_out,
                                      pb_solve_info *info) {
    if (!ctx) return set_error(nullptr, PB_ERR_ARG, "pb_solve_sharded: NULL context");
    if (!allgather || world < 1 || rank < 0 || rank >= world)
        return set_error(ctx, PB_ERR_ARG, "pb_solve_sharded: need an allgather callback and 0 <= rank < world");
    if (opts && (opts->prec == PB_FLOAT2 || (opts->refine > 0 && opts->refine_prec == PB_FLOAT2)))
        return set_error(ctx, PB_ERR_ARG, "pb_solve_sharded: the float-float product has no row-block form");
    auto &sh = ctx->shard;
    rows_of(ctx->N, world, rank, &sh.row0, &sh.nrows, &sh.per);
    const int64_t need = 2 * sh.per * (int64_t)world;
    if (need > sh.cap) {
        if (sh.send) ctx_free(ctx, sh.send);
        if (sh.recv) ctx_free(ctx, sh.recv);
        ctx->device_bytes -= sh.bytes;
        sh.send = sh.recv = nullptr;
        sh.cap = 0;
        sh.bytes = 0;
        pb_status s = ctx_alloc(ctx, (void **)&sh.send, 2 * sh.per * sizeof(double), "shard send block");
        if (s == PB_OK) s = ctx_alloc(ctx, (void **)&sh.recv, need * sizeof(double), "shard gather buffer");
        if (s != PB_OK) return s;
        sh.cap = need;
        sh.bytes = (int64_t)((2 * sh.per + need) * sizeof(double));
    }
    // the padding slots of the send block stay zero
    const int threads = 256;
    zero_kernel<<<(unsigned)((2 * sh.per + threads - 1) / threads), threads, 0, ctx->stream>>>(sh.send, 2 * sh.per);
    PB_LAUNCHED();
    sh.world = world;
    sh.rank = rank;
    sh.fn = allgather;
    sh.user = user;
    sh.gathers = 0;
    sh.on = true;
    pb_status s = pb_solve(ctx, opts, x0, x_out, info);
    sh.on = false;
    sh.fn = nullptr;
    sh.user = nullptr;
    return s;
}
