// pb_api.cu -- the extern "C" entry points of include/pb.h: argument checks,
// context memory, and the order of the device steps of a solve.
#include <atomic>
#include <math.h>
#include <new>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>

#include "pb_internal.cuh"

namespace pb {

static std::atomic<uint64_t> g_launches{0};
static thread_local char g_thread_error[512];

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

pb_status set_error(pb_ctx *ctx, pb_status s, const char *fmt, ...) {
    char *buf = ctx ? ctx->last_error : g_thread_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    if (ctx) memcpy(g_thread_error, ctx->last_error, sizeof(g_thread_error));
    return s;
}

pb_status cuda_error(pb_ctx *ctx, cudaError_t e, const char *what) {
    pb_status s = (e == cudaErrorMemoryAllocation) ? PB_ERR_OOM : PB_ERR_CUDA;
    return set_error(ctx, s, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

// ---- memory: a library-owned stream-ordered pool per device, and a cache of
// pinned host blocks.  The pool keeps freed memory (release threshold at its
// maximum) so that contexts created and destroyed in a loop reuse it instead
// of mapping it again; the pinned cache avoids a cudaMallocHost (and the
// device synchronisation of cudaFreeHost) per context.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};
static std::mutex g_pinned_mu;
static std::multimap<size_t, void *> g_pinned;

static size_t pinned_class(size_t bytes) {
    size_t c = 256;
    while (c < bytes) c <<= 1;
    return c;
}

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (dev >= 0 && dev < 64) {
            if (!g_pool[dev]) {
                cudaMemPoolProps props;
                memset(&props, 0, sizeof(props));
                props.allocType = cudaMemAllocationTypePinned;
                props.handleTypes = cudaMemHandleTypeNone;
                props.location.type = cudaMemLocationTypeDevice;
                props.location.id = dev;
                cudaMemPool_t created = nullptr;
                if (cudaMemPoolCreate(&created, &props) == cudaSuccess) {
                    uint64_t keep = UINT64_MAX;
                    cudaMemPoolSetAttribute(created, cudaMemPoolAttrReleaseThreshold, &keep);
                    g_pool[dev] = created;
                } else {
                    cudaGetLastError();
                }
            }
            pool = g_pool[dev];
        }
    }
    if (pool) return cudaMallocFromPoolAsync(p, bytes, pool, stream);
    return cudaMallocAsync(p, bytes, stream);
}

cudaError_t pinned_alloc(void **p, size_t bytes) {
    const size_t c = pinned_class(bytes);
    {
        std::lock_guard<std::mutex> lock(g_pinned_mu);
        auto it = g_pinned.find(c);
        if (it != g_pinned.end()) {
            *p = it->second;
            g_pinned.erase(it);
            return cudaSuccess;
        }
    }
    return cudaMallocHost(p, c);
}

void pinned_free(void *p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    g_pinned.emplace(pinned_class(bytes), p);
}

pb_status ctx_alloc(pb_ctx *ctx, void **p, size_t bytes, const char *what) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = pool_alloc(p, bytes, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(ctx, e == cudaErrorMemoryAllocation ? PB_ERR_OOM : PB_ERR_CUDA,
                         "allocating %zu bytes for %s: %s", bytes, what, cudaGetErrorString(e));
    }
    ctx->device_bytes += (int64_t)bytes;
    return PB_OK;
}

void ctx_free(pb_ctx *ctx, void *p) {
    if (p) cudaFreeAsync(p, ctx->stream);
}

pb_status profile_flush(pb_ctx *ctx) {
    if (ctx->prof_used == 0) return PB_OK;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "profile flush");
    for (int i = 0; i + 1 < ctx->prof_used; i += 2) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, ctx->prof_ev[i], ctx->prof_ev[i + 1]);
        if (e != cudaSuccess) return cuda_error(ctx, e, "profile event");
        ctx->prof_ms += ms;
    }
    ctx->prof_used = 0;
    return PB_OK;
}

}  // namespace pb

using namespace pb;

namespace {

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

// Copy n doubles from host or device memory into a fresh device buffer.
pb_status stage(pb_ctx *ctx, const double *src, int64_t n, double **dst, const char *what) {
    pb_status s = ctx_alloc(ctx, (void **)dst, (size_t)n * sizeof(double), what);
    if (s != PB_OK) return s;
    cudaError_t e = cudaMemcpyAsync(*dst, src, (size_t)n * sizeof(double), cudaMemcpyDefault, ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, what);
    return PB_OK;
}

void free_all(pb_ctx *ctx) {
    void *bufs[] = {ctx->g64, ctx->pos32, ctx->nrm32, ctx->charges, ctx->b, ctx->x, ctx->partials,
                    ctx->tile_counters, ctx->red, ctx->red_counter, ctx->scalar, ctx->V, ctx->w, ctx->r,
                    ctx->d, ctx->rres, ctx->st, ctx->sym_scratch, ctx->sym64_scratch, ctx->symff_scratch,
                    ctx->rows_partials, ctx->rows_counters, ctx->shard.send, ctx->shard.recv};
    for (void *p : bufs) ctx_free(ctx, p);
    cudaStreamSynchronize(ctx->stream);
    for (cudaEvent_t ev : ctx->prof_ev) cudaEventDestroy(ev);
    ctx->prof_ev.clear();
    for (cudaEvent_t &ev : ctx->band_ev) {
        if (ev) cudaEventDestroy(ev);
        ev = nullptr;
    }
    if (ctx->band_stream) cudaStreamDestroy(ctx->band_stream);
    ctx->band_stream = nullptr;
    pinned_free(ctx->host_scalar, 16 * sizeof(double));
    pinned_free(ctx->st_host, sizeof(GmresState));
}

pb_status ensure_charge_capacity(pb_ctx *ctx, int64_t nc) {
    if (nc <= ctx->nc_cap) return PB_OK;
    if (ctx->charges) ctx_free(ctx, ctx->charges);
    ctx->charges = nullptr;
    ctx->nc_cap = 0;
    pb_status s = ctx_alloc(ctx, (void **)&ctx->charges, (size_t)nc * sizeof(Charge4), "charges");
    if (s == PB_OK) ctx->nc_cap = nc;
    return s;
}

pb_status load_charges(pb_ctx *ctx, const double *charges, int64_t nc) {
    pb_status s = ensure_charge_capacity(ctx, nc > 0 ? nc : 1);
    if (s != PB_OK) return s;
    double *q = nullptr;
    if (nc > 0 && (s = stage(ctx, charges, 4 * nc, &q, "charge staging")) != PB_OK) return s;
    s = charges_prepare(ctx, q, nc);
    ctx_free(ctx, q);
    if (s != PB_OK) return s;
    double gmin = 0, gmax = 0;
    if ((s = gauss_check(ctx, &gmin, &gmax)) != PB_OK) return s;
    ctx->gauss_min = gmin;
    ctx->gauss_max = gmax;
    if (nc > 0 && !(gmin > -1.5 && gmax < -0.5))
        return set_error(ctx, PB_ERR_BADMESH,
                         "orientation check failed: Gauss sums at the charges lie in [%.4f, %.4f], expected about -1 "
                         "(charges outside the surface, an open surface, or inward normals)",
                         gmin, gmax);
    ctx->b_valid = false;
    ctx->x_valid = false;
    return PB_OK;
}

pb_status fill_opts(pb_ctx *ctx, const pb_solve_opts *in, pb_solve_opts *o) {
    pb_solve_opts d{10, 1e-4, 1000, PB_FP32PAIR, 0, PB_FP64};
    if (in) {
        d = *in;
        if (d.restart == 0) d.restart = 10;
        if (d.tol == 0.0) d.tol = 1e-4;
        if (d.maxit == 0) d.maxit = 1000;
    }
    if (d.restart < 1 || d.restart > kMaxRestart)
        return set_error(ctx, PB_ERR_ARG, "restart must be in [1, %d], got %d", kMaxRestart, d.restart);
    if (!(d.tol > 0.0) || !isfinite(d.tol)) return set_error(ctx, PB_ERR_ARG, "tol must be > 0");
    if (d.maxit < 1) return set_error(ctx, PB_ERR_ARG, "maxit must be >= 1");
    if (d.prec != PB_FP64 && d.prec != PB_FP32PAIR && d.prec != PB_FLOAT2)
        return set_error(ctx, PB_ERR_ARG, "unknown precision");
    if (d.refine_prec != PB_FP64 && d.refine_prec != PB_FLOAT2)
        return set_error(ctx, PB_ERR_ARG, "refine_prec must be PB_FP64 or PB_FLOAT2");
    if (d.refine < 0 || d.refine > 16) return set_error(ctx, PB_ERR_ARG, "refine must be in [0, 16]");
    *o = d;
    return PB_OK;
}

__global__ void sub_kernel(const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}
__global__ void add_kernel(double *__restrict__ x, const double *__restrict__ d, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += d[i];
}

pb_status launch_sub(pb_ctx *ctx, const double *a, const double *b, double *out) {
    sub_kernel<<<red_blocks(ctx, 2 * ctx->N), 256, 0, ctx->stream>>>(a, b, out, 2 * ctx->N);
    PB_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PB_OK : cuda_error(ctx, e, "sub kernel");
}

pb_status read_counter(pb_ctx *ctx, unsigned long long *host) {
    cudaError_t e = cudaMemcpyAsync(ctx->host_scalar + 8, ctx->mv_count, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "counter readback");
    memcpy(host, ctx->host_scalar + 8, sizeof(unsigned long long));
    return PB_OK;
}

pb_status read_scalar(pb_ctx *ctx, const double *dev, double *host) {
    cudaError_t e = cudaMemcpyAsync(ctx->host_scalar, dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "scalar readback");
    *host = ctx->host_scalar[0];
    return PB_OK;
}

}  // namespace

extern "C" {

const char *pb_status_string(pb_status s) {
    switch (s) {
        case PB_OK: return "PB_OK";
        case PB_ERR_ARG: return "PB_ERR_ARG";
        case PB_ERR_BADMESH: return "PB_ERR_BADMESH";
        case PB_ERR_OOM: return "PB_ERR_OOM";
        case PB_ERR_CUDA: return "PB_ERR_CUDA";
        case PB_ERR_NOCONV: return "PB_ERR_NOCONV";
        case PB_ERR_NAN: return "PB_ERR_NAN";
        case PB_ERR_TIMEOUT: return "PB_ERR_TIMEOUT";
        case PB_ERR_ADMIT: return "PB_ERR_ADMIT";
    }
    return "PB_UNKNOWN_STATUS";
}

const char *pb_last_error(const pb_ctx *ctx) { return ctx ? ctx->last_error : g_thread_error; }

uint64_t pb_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

pb_status pb_release_cached_memory(void) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_error(nullptr, e, "pb_release_cached_memory");
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (dev >= 0 && dev < 64) pool = g_pool[dev];
    }
    if (pool && (e = cudaMemPoolTrimTo(pool, 0)) != cudaSuccess)
        return cuda_error(nullptr, e, "pb_release_cached_memory: trim");
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    for (auto &kv : g_pinned) cudaFreeHost(kv.second);
    g_pinned.clear();
    return PB_OK;
}

pb_status pb_create(const double *centroids, const double *normals, const double *areas, int64_t N,
                    const double *charges, int64_t Nc, double eps1, double eps2, double kappa, void *cuda_stream,
                    pb_ctx **out) {
    if (!out) return set_error(nullptr, PB_ERR_ARG, "pb_create: out is NULL");
    *out = nullptr;
    if (!centroids || !normals || !areas) return set_error(nullptr, PB_ERR_ARG, "pb_create: NULL geometry pointer");
    if (N < 1 || N > ((int64_t)1 << 31) - 1)
        return set_error(nullptr, PB_ERR_ARG, "pb_create: N must be in [1, 2^31), got %lld", (long long)N);
    if (Nc < 0 || (Nc > 0 && !charges)) return set_error(nullptr, PB_ERR_ARG, "pb_create: bad charge arguments");
    if (!finite_pos(eps1) || !finite_pos(eps2) || !isfinite(kappa) || kappa < 0.0)
        return set_error(nullptr, PB_ERR_ARG, "pb_create: need eps1 > 0, eps2 > 0, kappa >= 0 (finite)");

    pb_ctx *ctx = new (std::nothrow) pb_ctx();
    if (!ctx) return set_error(nullptr, PB_ERR_OOM, "pb_create: host allocation failed");
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->N = N;
    ctx->eps1 = eps1;
    ctx->eps2 = eps2;
    ctx->eps = eps2 / eps1;
    ctx->kappa = kappa;
    pb_status s = PB_OK;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) s = cuda_error(ctx, e, "pb_create: device query");

    double *c_dev = nullptr, *n_dev = nullptr, *a_dev = nullptr;
    const int64_t N2 = 2 * N;
    int sym_default = 0, sym_cps = 0;
    if (s == PB_OK) {
        // scratch sized for every kernel variant at any CTA count per SM up to
        // its occupancy (fewer CTAs never need more segments)
        ctx->plan64 = make_plan(N, kF64TargetTile, kF64SourceTile, (int64_t)ctx->num_sms * matvec_occupancy(PB_FP64));
        ctx->partials_len = plan_partials(ctx->plan64, kF64TargetTile);
        ctx->counters_len = ctx->plan64.target_tiles;
        ctx->planff = matvec_ff_plan(ctx);
        if (plan_partials(ctx->planff, matvec_ff_target_tile()) > ctx->partials_len)
            ctx->partials_len = plan_partials(ctx->planff, matvec_ff_target_tile());
        if (ctx->planff.target_tiles > ctx->counters_len) ctx->counters_len = ctx->planff.target_tiles;
        for (int v = 1; v <= kNumF32Variants; ++v) {
            if (f32_variant_symmetric(v)) continue;   // own scratch, allocated when configured
            StreamKPlan pl = matvec_f32_plan(ctx, v, 0);
            int64_t need = plan_partials(pl, kF32Threads * f32_variant_targets(v));
            if (need > ctx->partials_len) ctx->partials_len = need;
            if (pl.target_tiles > ctx->counters_len) ctx->counters_len = pl.target_tiles;
        }
        int v = 0, cps = 0;
        default_f32_config(ctx, &v, &cps);
        ctx->plan32 = matvec_f32_plan(ctx, MV_F32_PACKED_T2, 0);
        ctx->f32_variant = MV_F32_PACKED_T2;
        if (!f32_variant_symmetric(v)) {
            ctx->f32_variant = v;
            ctx->f32_ctas_per_sm = cps;
            ctx->plan32 = matvec_f32_plan(ctx, v, cps);
        }
        sym_default = f32_variant_symmetric(v) ? v : 0;
        sym_cps = cps;
        ctx->red_len = (int64_t)(kMaxRestart + 1) * 2 * ctx->num_sms;
    }
    if (s == PB_OK) s = ctx_alloc(ctx, (void **)&ctx->g64, 7 * N * sizeof(double), "FP64 geometry");
    if (s == PB_OK) s = ctx_alloc(ctx, (void **)&ctx->pos32, N * sizeof(float4), "FP32 positions");
    if (s == PB_OK) s = ctx_alloc(ctx, (void **)&ctx->nrm32, N * sizeof(float4), "FP32 normals");
    if (s == PB_OK) s = ctx_alloc(ctx, (void **)&ctx->b, N2 * sizeof(double), "rhs");
    if (s == PB_OK) s = ctx_alloc(ctx, (void **)&ctx->x, N2 * sizeof(double), "solution");
    if (s == PB_OK) s = ctx_alloc(ctx, (void **)&ctx->partials, ctx->partials_len * sizeof(double), "matvec partials");
    if (s == PB_OK) s = ctx_alloc(ctx, (void **)&ctx->tile_counters, ctx->counters_len * sizeof(unsigned int), "tile counters");
    if (s == PB_OK) s = ctx_alloc(ctx, (void **)&ctx->red, ctx->red_len * sizeof(double), "reduction partials");
    if (s == PB_OK) s = ctx_alloc(ctx, (void **)&ctx->red_counter, 16 * sizeof(unsigned int), "reduction counters");
    if (s == PB_OK) s = ctx_alloc(ctx, (void **)&ctx->scalar, 16 * sizeof(double), "scalars");
    if (s == PB_OK) {
        e = pinned_alloc((void **)&ctx->host_scalar, 16 * sizeof(double));
        if (e != cudaSuccess) s = cuda_error(ctx, e, "pinned scalars");
    }
    if (s == PB_OK) {
        ctx->mv_count = (unsigned long long *)(ctx->scalar + 8);
        e = cudaMemsetAsync(ctx->tile_counters, 0, ctx->counters_len * sizeof(unsigned int), ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->red_counter, 0, 16 * sizeof(unsigned int), ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->scalar, 0, 16 * sizeof(double), ctx->stream);
        if (e != cudaSuccess) s = cuda_error(ctx, e, "counter reset");
    }
    if (s == PB_OK && sym_default) s = matvec_configure(ctx, sym_default, sym_cps);
    if (s == PB_OK) s = matvec_configure_fp64(ctx, default_f64_variant(N));
    if (s == PB_OK) s = stage(ctx, centroids, 3 * N, &c_dev, "centroid staging");
    if (s == PB_OK) s = stage(ctx, normals, 3 * N, &n_dev, "normal staging");
    if (s == PB_OK) s = stage(ctx, areas, N, &a_dev, "area staging");
    if (s == PB_OK) s = geometry_prepare(ctx, c_dev, n_dev, a_dev);
    ctx_free(ctx, c_dev);
    ctx_free(ctx, n_dev);
    ctx_free(ctx, a_dev);
    if (s == PB_OK) s = load_charges(ctx, charges, Nc);
    if (s == PB_OK) {
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) s = cuda_error(ctx, e, "pb_create");
    }
    if (s != PB_OK) {
        memcpy(g_thread_error, ctx->last_error, sizeof(g_thread_error));
        free_all(ctx);
        delete ctx;
        return s;
    }
    *out = ctx;
    return PB_OK;
}

pb_status pb_set_charges(pb_ctx *ctx, const double *charges, int64_t Nc) {
    if (!ctx) return set_error(nullptr, PB_ERR_ARG, "pb_set_charges: NULL context");
    if (Nc < 0 || (Nc > 0 && !charges)) return set_error(ctx, PB_ERR_ARG, "pb_set_charges: bad charge arguments");
    pb_status s = load_charges(ctx, charges, Nc);
    if (s != PB_OK) return s;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? PB_OK : cuda_error(ctx, e, "pb_set_charges");
}

pb_status pb_source(pb_ctx *ctx, double *b, pb_precision prec) {
    if (!ctx || !b) return set_error(ctx, PB_ERR_ARG, "pb_source: NULL argument");
    if (prec != PB_FP64 && prec != PB_FP32PAIR && prec != PB_FLOAT2)
        return set_error(ctx, PB_ERR_ARG, "pb_source: unknown precision");
    return source_launch(ctx, b, prec);
}

pb_status pb_matvec(pb_ctx *ctx, const double *u, double *y, pb_precision prec) {
    if (!ctx || !u || !y) return set_error(ctx, PB_ERR_ARG, "pb_matvec: NULL argument");
    if (u == y) return set_error(ctx, PB_ERR_ARG, "pb_matvec: u and y must not overlap");
    return matvec_launch(ctx, u, y, prec, nullptr);
}

pb_status pb_solve(pb_ctx *ctx, const pb_solve_opts *opts, const double *x0, double *x_out, pb_solve_info *info) {
    if (!ctx) return set_error(nullptr, PB_ERR_ARG, "pb_solve: NULL context");
    pb_solve_opts o;
    pb_status s = fill_opts(ctx, opts, &o);
    if (s != PB_OK) return s;
    const int64_t N2 = 2 * ctx->N;
    cudaError_t e;
    ctx->x_valid = false;
    // the source term and the energy: FP64 pairs on the plain FP64 path,
    // float-float pairs (FP64-level, on the FP32 pipe) otherwise
    const pb_precision side = o.prec == PB_FP64 ? PB_FP64 : PB_FLOAT2;
    if (!ctx->b_valid || ctx->b_prec != side) {
        if ((s = source_launch(ctx, ctx->b, side)) != PB_OK) return s;
        ctx->b_valid = true;
        ctx->b_prec = side;
    }
    if (x0) {
        e = cudaMemcpyAsync(ctx->x, x0, N2 * sizeof(double), cudaMemcpyDefault, ctx->stream);
    } else {
        e = cudaMemsetAsync(ctx->x, 0, N2 * sizeof(double), ctx->stream);
    }
    if (e != cudaSuccess) return cuda_error(ctx, e, "pb_solve: start vector");

    unsigned long long mv_before = 0, mv_after = 0;
    if ((s = read_counter(ctx, &mv_before)) != PB_OK) return s;
    int iters = 0, cycles = 0;
    double rel = 0.0;
    pb_status gs = gmres_solve(ctx, &o, ctx->b, ctx->x, x0 == nullptr, &iters, &cycles, &rel);
    if (gs != PB_OK && gs != PB_ERR_NOCONV) return gs;
    int total_it = iters, total_cy = cycles, refined = 0;
    double rel64 = -1.0;
    if (o.refine > 0 && o.prec == PB_FP32PAIR) {
        if (!ctx->d && (s = ctx_alloc(ctx, (void **)&ctx->d, N2 * sizeof(double), "refinement d")) != PB_OK) return s;
        if (!ctx->rres && (s = ctx_alloc(ctx, (void **)&ctx->rres, N2 * sizeof(double), "refinement r")) != PB_OK) return s;
        for (int step = 0; step < o.refine; ++step) {
            // r = b - A_fp64 x ; A d = r ; x += d   (the FP64 product uses ctx->w)
            if ((s = matvec_launch(ctx, ctx->x, ctx->rres, o.refine_prec, nullptr)) != PB_OK) return s;
            if ((s = launch_sub(ctx, ctx->b, ctx->rres, ctx->rres)) != PB_OK) return s;
            pb_solve_opts oi = o;
            int it2 = 0, cy2 = 0;
            double rel2 = 0.0;
            e = cudaMemsetAsync(ctx->d, 0, N2 * sizeof(double), ctx->stream);
            if (e != cudaSuccess) return cuda_error(ctx, e, "refinement");
            pb_status rs = gmres_solve(ctx, &oi, ctx->rres, ctx->d, true, &it2, &cy2, &rel2);
            if (rs != PB_OK && rs != PB_ERR_NOCONV) return rs;
            add_kernel<<<red_blocks(ctx, N2), 256, 0, ctx->stream>>>(ctx->x, ctx->d, N2);
            PB_LAUNCHED();
            total_it += it2;
            total_cy += cy2;
            refined += 1;
        }
        if ((s = matvec_launch(ctx, ctx->x, ctx->rres, o.refine_prec, nullptr)) != PB_OK) return s;
        if ((s = launch_sub(ctx, ctx->b, ctx->rres, ctx->rres)) != PB_OK) return s;
        if ((s = norm2_launch(ctx, ctx->rres, N2, ctx->scalar + 1)) != PB_OK) return s;
        if ((s = norm2_launch(ctx, ctx->b, N2, ctx->scalar + 2)) != PB_OK) return s;
        double rn = 0, bn = 0;
        if ((s = read_scalar(ctx, ctx->scalar + 1, &rn)) != PB_OK) return s;
        if ((s = read_scalar(ctx, ctx->scalar + 2, &bn)) != PB_OK) return s;
        rel64 = bn > 0 ? rn / bn : 0.0;
        gs = (rel64 <= o.tol) ? PB_OK : gs;
        rel = rel64;
    }
    double E = 0.0;
    if ((s = energy_launch(ctx, ctx->x, side, ctx->scalar)) != PB_OK) return s;
    ctx->e_prec = side;
    if ((s = read_scalar(ctx, ctx->scalar, &E)) != PB_OK) return s;
    if (x_out) {
        e = cudaMemcpyAsync(x_out, ctx->x, N2 * sizeof(double), cudaMemcpyDefault, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_error(ctx, e, "pb_solve: copy out");
    }
    ctx->x_valid = true;
    if ((s = read_counter(ctx, &mv_after)) != PB_OK) return s;
    if (ctx->prof_on && (s = profile_flush(ctx)) != PB_OK) return s;
    if (info) {
        info->matvecs = (int64_t)(mv_after - mv_before);
        info->iters = total_it;
        info->cycles = total_cy;
        info->rel_resid = rel;
        info->energy_kcal = E;
        info->rel_resid_fp64 = rel64;
        info->refine_steps = refined;
    }
    return gs;
}

pb_status pb_energy(pb_ctx *ctx, double *energy_kcal) {
    if (!ctx || !energy_kcal) return set_error(ctx, PB_ERR_ARG, "pb_energy: NULL argument");
    if (!ctx->x_valid) return set_error(ctx, PB_ERR_ARG, "pb_energy: no solution (call pb_solve first)");
    pb_status s = energy_launch(ctx, ctx->x, ctx->e_prec, ctx->scalar);
    if (s != PB_OK) return s;
    return read_scalar(ctx, ctx->scalar, energy_kcal);
}

pb_status pb_energy_of(pb_ctx *ctx, const double *u, pb_precision prec, double *energy_kcal) {
    if (!ctx || !u || !energy_kcal) return set_error(ctx, PB_ERR_ARG, "pb_energy_of: NULL argument");
    if (prec != PB_FP64 && prec != PB_FP32PAIR && prec != PB_FLOAT2)
        return set_error(ctx, PB_ERR_ARG, "pb_energy_of: unknown precision");
    pb_status s = energy_launch(ctx, u, prec, ctx->scalar);
    if (s != PB_OK) return s;
    return read_scalar(ctx, ctx->scalar, energy_kcal);
}

pb_status pb_get_info(pb_ctx *ctx, pb_ctx_info *info) {
    if (!ctx || !info) return set_error(ctx, PB_ERR_ARG, "pb_get_info: NULL argument");
    info->n = ctx->N;
    info->nc = ctx->Nc;
    info->eps1 = ctx->eps1;
    info->eps2 = ctx->eps2;
    info->kappa = ctx->kappa;
    for (int d = 0; d < 3; ++d) info->center[d] = ctx->center[d];
    info->gauss_min = ctx->gauss_min;
    info->gauss_max = ctx->gauss_max;
    info->device_bytes = ctx->device_bytes;
    return PB_OK;
}

pb_status pb_profile_enable(pb_ctx *ctx, int enable) {
    if (!ctx) return set_error(nullptr, PB_ERR_ARG, "pb_profile_enable: NULL context");
    if (enable && ctx->prof_ev.empty()) {
        ctx->prof_ev.resize(2 * 1024, nullptr);
        for (auto &ev : ctx->prof_ev) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) {
                ctx->prof_ev.clear();
                return cuda_error(ctx, e, "pb_profile_enable");
            }
        }
    }
    if (!enable) {
        pb_status s = profile_flush(ctx);
        if (s != PB_OK) return s;
    }
    ctx->prof_on = enable != 0;
    return PB_OK;
}

pb_status pb_profile_read(pb_ctx *ctx, double *matvec_ms, int64_t *timed_launches, int64_t *evaluated, int reset) {
    if (!ctx) return set_error(nullptr, PB_ERR_ARG, "pb_profile_read: NULL context");
    pb_status s = profile_flush(ctx);
    if (s != PB_OK) return s;
    unsigned long long n = 0;
    if ((s = read_counter(ctx, &n)) != PB_OK) return s;
    if (matvec_ms) *matvec_ms = ctx->prof_ms;
    if (timed_launches) *timed_launches = ctx->prof_launches;
    if (evaluated) *evaluated = (int64_t)(n - ctx->prof_count_base);
    if (reset) {
        ctx->prof_ms = 0.0;
        ctx->prof_launches = 0;
        ctx->prof_count_base = n;
    }
    return PB_OK;
}

void pb_destroy(pb_ctx *ctx) {
    if (!ctx) return;
    free_all(ctx);
    delete ctx;
}

}  // extern "C"
