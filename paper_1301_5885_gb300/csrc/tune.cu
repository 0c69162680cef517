// tune.cu -- choice of the FP32-pair matvec kernel variant and grid size.
//
// The variants (scalar or packed f32x2 arithmetic, 2 or 4 targets per thread)
// and the number of resident CTAs per SM trade registers, occupancy and
// instruction issue differently at different N.  pb_matvec_autotune times each
// candidate on the context's own geometry and keeps the fastest; the choice is
// also stored in a process-wide table keyed by (device, N bucket) so that later
// contexts of similar size start from it.  Without a stored choice a context
// uses the built-in default.
#include <math.h>
#include <mutex>

#include "pb_internal.cuh"

namespace pb {
namespace {

// Built-in default, from timings on GB300 (ordered pairs per second): the
// symmetric kernel with 4 targets per thread is fastest once the upper
// triangle of 512-point tile pairs fills the GPU (1168 Gpairs/s at
// N = 81,920 and 1190 at N = 327,680, against 790 for the packed kernel and
// 627 for the scalar one; 2212 against 1672 with kappa = 0); with 2 targets
// per thread it reaches 1041.  Small surfaces have too few tile pairs for
// either: at N = 5,120 the packed 2-target kernel gives 505 Gpairs/s, the
// symmetric ones 400 and 241.
constexpr int64_t kSymT4MinN = 40960;
constexpr int64_t kSymT2MinN = 16384;
// FP64 product: the symmetric kernel halves the FP64-pipe work; timed on
// GB300 at N = 5,120: 4.8 (plain), 11.8 (symmetric, 1 target per thread) and
// 9.2 Gpairs/s (2 targets); at N = 81,920: 8.2, 13.6 and 13.9.
constexpr int64_t kSym64T1MinN = 2048;
constexpr int64_t kSym64T2MinN = 65536;
constexpr int kBuckets = 256;

struct TuneEntry {
    bool set = false;
    int variant = 0;
    int ctas_per_sm = 0;
};
std::mutex g_tune_mu;
TuneEntry g_tune[8][kBuckets];   // [device % 8][bucket]

// quarter-octave bucket of N
int bucket_of(int64_t n) {
    int b = (int)floor(4.0 * log2((double)(n < 1 ? 1 : n)));
    return b < 0 ? 0 : (b >= kBuckets ? kBuckets - 1 : b);
}

}  // namespace

int default_f64_variant(int64_t n) {
    return n >= kSym64T2MinN ? MV_F64_SYM_T2 : (n >= kSym64T1MinN ? MV_F64_SYM_T1 : MV_F64_PLAIN);
}

int64_t default_scratch_bytes(int64_t n, int num_sms) {
    const int v = n >= kSymT4MinN ? MV_F32_SYM_T4 : (n >= kSymT2MinN ? MV_F32_SYM_T2 : 0);
    if (v == 0) return 0;
    const int tile = kF32Threads * f32_variant_targets(v);
    // one pass (the solve server's large requests take it while the lanes share the SMs)
    std::vector<int64_t> cuts;
    return sym_scratch_need(make_sym_plan(n, tile, (int64_t)num_sms * 4), tile, (int)sizeof(float),
                            kDefaultScratchLimit, 1, &cuts);
}

void default_f32_config(pb_ctx *ctx, int *variant, int *ctas_per_sm) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const TuneEntry &e = g_tune[ctx->device & 7][bucket_of(ctx->N)];
    if (e.set) {
        *variant = e.variant;
        *ctas_per_sm = e.ctas_per_sm;
    } else {
        *variant = ctx->N >= kSymT4MinN ? MV_F32_SYM_T4 : (ctx->N >= kSymT2MinN ? MV_F32_SYM_T2 : MV_F32_PACKED_T2);
        *ctas_per_sm = 0;
    }
}

}  // namespace pb

using namespace pb;

extern "C" {

pb_status pb_matvec_configure(pb_ctx *ctx, int variant, int ctas_per_sm) {
    if (!ctx) return set_error(nullptr, PB_ERR_ARG, "pb_matvec_configure: NULL context");
    if (variant == 0) {
        int v = 0, c = 0;
        default_f32_config(ctx, &v, &c);
        return matvec_configure(ctx, v, ctas_per_sm > 0 ? ctas_per_sm : c);
    }
    return matvec_configure(ctx, variant, ctas_per_sm);
}

pb_status pb_matvec_get_config(pb_ctx *ctx, int *variant, int *ctas_per_sm, int64_t *ctas) {
    if (!ctx) return set_error(nullptr, PB_ERR_ARG, "pb_matvec_get_config: NULL context");
    if (variant) *variant = ctx->f32_variant;
    if (ctas_per_sm) *ctas_per_sm = ctx->f32_ctas_per_sm;
    if (ctas) *ctas = f32_variant_symmetric(ctx->f32_variant) ? ctx->plansym.ctas : ctx->plan32.ctas;
    return PB_OK;
}

pb_status pb_matvec_configure_fp64(pb_ctx *ctx, int variant, int *variant_out) {
    if (!ctx) return set_error(nullptr, PB_ERR_ARG, "pb_matvec_configure_fp64: NULL context");
    if (variant == 0) variant = default_f64_variant(ctx->N);
    pb_status s = matvec_configure_fp64(ctx, variant);
    if (variant_out) *variant_out = ctx->f64_variant;
    return s;
}

pb_status pb_set_scratch_limit(pb_ctx *ctx, int64_t bytes) {
    if (!ctx) return set_error(nullptr, PB_ERR_ARG, "pb_set_scratch_limit: NULL context");
    if (bytes < 0) return set_error(ctx, PB_ERR_ARG, "pb_set_scratch_limit: negative bound %lld", (long long)bytes);
    // the next product of each kind allocates its scratch again (freed in stream order)
    void **bufs[3] = {&ctx->sym_scratch, &ctx->sym64_scratch, &ctx->symff_scratch};
    int64_t *lens[3] = {&ctx->sym_scratch_len, &ctx->sym64_scratch_len, &ctx->symff_scratch_len};
    for (int k = 0; k < 3; ++k) {
        if (*bufs[k]) ctx_free(ctx, *bufs[k]);
        ctx->device_bytes -= *lens[k];
        *bufs[k] = nullptr;
        *lens[k] = 0;
    }
    ctx->scratch_limit = bytes;
    return PB_OK;
}

pb_status pb_set_bands(pb_ctx *ctx, int bands) {
    if (!ctx) return set_error(nullptr, PB_ERR_ARG, "pb_set_bands: NULL context");
    if (bands < 0) return set_error(ctx, PB_ERR_ARG, "pb_set_bands: negative band count %d", bands);
    ctx->bands = bands;
    return PB_OK;
}

pb_status pb_scratch_plan(pb_ctx *ctx, pb_precision prec, int *bands, int64_t *bytes) {
    if (!ctx) return set_error(nullptr, PB_ERR_ARG, "pb_scratch_plan: NULL context");
    std::vector<int64_t> cuts;
    int64_t need = 0;
    if (prec == PB_FP32PAIR) {
        if (f32_variant_symmetric(ctx->f32_variant))
            need = sym_scratch_need(ctx->plansym, kF32Threads * f32_variant_targets(ctx->f32_variant),
                                    (int)sizeof(float), ctx->scratch_limit, ctx->bands, &cuts);
    } else if (prec == PB_FP64) {
        if (ctx->f64_variant != MV_F64_PLAIN)
            need = sym_scratch_need(ctx->plansym64, kF64Threads * (ctx->f64_variant == MV_F64_SYM_T2 ? 2 : 1),
                                    (int)sizeof(double), ctx->scratch_limit, ctx->bands, &cuts);
    } else if (prec == PB_FLOAT2) {
        need = ff_sym_scratch_need(ctx, &cuts);
    } else {
        return set_error(ctx, PB_ERR_ARG, "pb_scratch_plan: unknown precision %d", (int)prec);
    }
    if (bands) *bands = cuts.empty() ? 0 : (int)cuts.size() - 1;
    if (bytes) *bytes = need;
    return PB_OK;
}

pb_status pb_matvec_autotune(pb_ctx *ctx, int reps, int *variant, int *ctas_per_sm, double *best_ms) {
    if (!ctx) return set_error(nullptr, PB_ERR_ARG, "pb_matvec_autotune: NULL context");
    if (reps < 1) reps = 3;
    const int64_t n2 = 2 * ctx->N;
    double *u = nullptr, *y = nullptr;
    pb_status s = ctx_alloc(ctx, (void **)&u, n2 * sizeof(double), "autotune u");
    if (s == PB_OK) s = ctx_alloc(ctx, (void **)&y, n2 * sizeof(double), "autotune y");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaSuccess;
    if (s == PB_OK) {
        ce = cudaMemsetAsync(u, 0, n2 * sizeof(double), ctx->stream);
        if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
        if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
        if (ce != cudaSuccess) s = cuda_error(ctx, ce, "pb_matvec_autotune");
    }
    const int keep_v = ctx->f32_variant, keep_c = ctx->f32_ctas_per_sm;
    int best_v = keep_v, best_c = keep_c;
    double best = INFINITY;
    const bool prof = ctx->prof_on;
    ctx->prof_on = false;
    for (int v = 1; v <= kNumF32Variants && s == PB_OK; ++v) {
        const int occ = matvec_f32_occupancy(v);
        int tried[4], ntried = 0;
        const int cands[4] = {occ, occ - 1, 4, 2};
        for (int ci = 0; ci < 4 && s == PB_OK; ++ci) {
            const int c = cands[ci];
            if (c < 1 || c > occ) continue;
            bool dup = false;
            for (int k = 0; k < ntried; ++k) dup |= (tried[k] == c);
            if (dup) continue;
            tried[ntried++] = c;
            if ((s = matvec_configure(ctx, v, c)) != PB_OK) break;
            if ((s = matvec_launch(ctx, u, y, PB_FP32PAIR, nullptr)) != PB_OK) break;   // warm-up
            cudaEventRecord(e0, ctx->stream);
            for (int r = 0; r < reps && s == PB_OK; ++r) s = matvec_launch(ctx, u, y, PB_FP32PAIR, nullptr);
            cudaEventRecord(e1, ctx->stream);
            if (s != PB_OK) break;
            ce = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
            if (ce != cudaSuccess) {
                s = cuda_error(ctx, ce, "pb_matvec_autotune timing");
                break;
            }
            if (ms / reps < best) {
                best = ms / reps;
                best_v = v;
                best_c = c;
            }
        }
    }
    ctx->prof_on = prof;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ctx_free(ctx, u);
    ctx_free(ctx, y);
    if (s != PB_OK) {
        matvec_configure(ctx, keep_v, keep_c);
        return s;
    }
    if ((s = matvec_configure(ctx, best_v, best_c)) != PB_OK) return s;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        TuneEntry &e = g_tune[ctx->device & 7][bucket_of(ctx->N)];
        e.set = true;
        e.variant = best_v;
        e.ctas_per_sm = best_c;
    }
    if (variant) *variant = best_v;
    if (ctas_per_sm) *ctas_per_sm = best_c;
    if (best_ms) *best_ms = best;
    return PB_OK;
}

}  // extern "C"
