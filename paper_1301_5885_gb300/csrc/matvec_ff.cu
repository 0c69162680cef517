// matvec_ff.cu -- the product of Eqs. (12)-(13) in float-float arithmetic.
//
// Every real number of a pair evaluation is carried as an unevaluated sum of
// two FP32 numbers (hi + lo, about 44 significant bits), with the error-free
// transformations two-sum and two-product (the latter from one fused
// multiply-add); the row sums go to FP64 once per staged source tile.  This
// keeps the error of each pair term near 1e-12 of its size while running on the
// FP32 pipe, which on GB300 retires many times the FP64 rate: it serves the
// FP64 residual of iterative refinement and FP64-accuracy products.
//
// exp(-kappa rho) = 2^t, t = -kappa rho / ln 2, is evaluated as
// 2^n * 2^(k/64) * exp(g ln 2) with n = rint(t), k = rint(64 (t - n)) and
// |g| <= 1/128: the table holds 2^(k/64) as float-float numbers, the last
// factor is a degree-6 Taylor polynomial in u = g ln 2 (|u| < 0.0055, so the
// truncation error is below 4e-17), with its low-order terms in float-float.
// 1/rho comes from the MUFU rsqrt and one Newton step in float-float.  Sums
// that can cancel (x_i - x_j, 1 - e, eps e' - 1, e'/eps - 1, e' - 1,
// e p3 - 3 and the two parts of K4) are added accurately; the others with
// the quicker sum.
#include <math.h>

#include <mutex>

#include "fastmath.cuh"
#include "finish.cuh"
#include "pb_internal.cuh"

namespace pb {
namespace {

struct ff {
    float h, l;
};

__device__ __forceinline__ ff ff_make(double v) {
    const float h = (float)v;
    return ff{h, (float)(v - (double)h)};
}
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return ff{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = a + b;
    return ff{s, b - (s - a)};
}
// accurate sum (both parts two-summed)
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.h, b.h);
    const ff t = two_sum(a.l, b.l);
    s.l += t.h;
    s = fast_two_sum(s.h, s.l);
    s.l += t.l;
    return fast_two_sum(s.h, s.l);
}
// quick sum: error bounded relative to |a| + |b| (not to |a + b|); used where
// no cancellation has to be resolved (sums of squares, dot products, row
// accumulation, polynomial steps)
__device__ __forceinline__ ff ff_add_q(ff a, ff b) {
    ff s = two_sum(a.h, b.h);
    s.l += a.l + b.l;
    return fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.h, -a.l}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) {
    const float p = a.h * b;
    float e = fmaf(a.h, b, -p);
    e = fmaf(a.l, b, e);
    return fast_two_sum(p, e);
}

// 2^(k/64), k = -32..32, as float-float numbers (filled once per device)
__constant__ float2 c_exp2_table[65];

struct FFParams {
    ff eps, inv_eps, kappa, neg_kappa_log2e, ln2;
    double diag1, diag2;
};

// exp(-kappa rho) for t = -kappa rho / ln 2 (t <= 0)
__device__ __forceinline__ ff ff_exp2(ff t, const FFParams &p) {
    const float n = rintf(t.h);
    const ff f = fast_two_sum(t.h - n, t.l);
    const float kf = fminf(fmaxf(rintf(f.h * 64.f), -32.f), 32.f);   // |f| <= 1/2; the clamp bounds the index
    const ff g = fast_two_sum(f.h - kf * (1.f / 64.f), f.l);
    const ff u = ff_mul(g, p.ln2);
    const float r = fmaf(fmaf(u.h, 1.f / 720.f, 1.f / 120.f), u.h, 1.f / 24.f);
    const float t1 = fmaf(u.h, r, 1.f / 6.f);
    const ff t2 = ff_add_q(ff{0.5f, 0.f}, ff_mulf(u, t1));
    const ff t3 = ff_add_q(ff{1.f, 0.f}, ff_mul(u, t2));
    const ff pe = ff_add_q(ff{1.f, 0.f}, ff_mul(u, t3));
    const float2 tk = c_exp2_table[(int)kf + 32];
    const ff e = ff_mul(pe, ff{tk.x, tk.y});
    const int ni = (int)n;
    return ff{ldexpf(e.h, ni), ldexpf(e.l, ni)};
}

constexpr int kFFThreads = 128;
constexpr int kFFTargets = 2;
constexpr int kFFTargetTile = kFFThreads * kFFTargets;
constexpr int kFFSourceTile = 128;

__global__ void __launch_bounds__(kFFThreads)
matvec_ff_kernel(const double *__restrict__ g64, const double *__restrict__ u, int64_t N, FFParams prm,
                 StreamKPlan plan, double *__restrict__ partials, unsigned int *__restrict__ counters,
                 double *__restrict__ y, const int *__restrict__ skip, unsigned long long *__restrict__ evaluated) {
    constexpr int BS = kFFThreads, T = kFFTargets, TT = kFFTargetTile, TS = kFFSourceTile;
    if (skip != nullptr && *((volatile const int *)skip)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(evaluated, 1ull);
    // per source: position, normal and the two weights, each as (hi, lo)
    __shared__ float4 s_p[TS][4];
    const double *X = g64, *Y = g64 + N, *Z = g64 + 2 * N;
    const double *NX = g64 + 3 * N, *NY = g64 + 4 * N, *NZ = g64 + 5 * N, *W = g64 + 6 * N;
    const int tid = threadIdx.x;
    const int64_t c = blockIdx.x;
    const int64_t S = plan.source_tiles;
    int64_t p = sk_begin(c, plan.work, plan.ctas);
    const int64_t pend = sk_begin(c + 1, plan.work, plan.ctas);
    const ff one{1.f, 0.f}, three{3.f, 0.f};

    while (p < pend) {
        const int64_t a = p / S;
        const int64_t s_first = p % S;
        const int64_t s_end = (S < s_first + (pend - p)) ? S : s_first + (pend - p);
        ff xi[T], yi[T], zi[T], nxi[T], nyi[T], nzi[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            int64_t i = a * TT + t * BS + tid;
            if (i > N - 1) i = N - 1;
            xi[t] = ff_make(X[i]); yi[t] = ff_make(Y[i]); zi[t] = ff_make(Z[i]);
            nxi[t] = ff_make(NX[i]); nyi[t] = ff_make(NY[i]); nzi[t] = ff_make(NZ[i]);
        }
        double acc1[T], acc2[T];
#pragma unroll
        for (int t = 0; t < T; ++t) { acc1[t] = 0.0; acc2[t] = 0.0; }

        for (int64_t st = s_first; st < s_end; ++st) {
            __syncthreads();
            {
                const int64_t j = st * TS + tid;
                if (j < N) {
                    const ff x = ff_make(X[j]), yy = ff_make(Y[j]), z = ff_make(Z[j]);
                    const ff nx = ff_make(NX[j]), ny = ff_make(NY[j]), nz = ff_make(NZ[j]);
                    const double w = W[j] * kInv4Pi;
                    const ff wpsi = ff_make(w * u[N + j]), wphi = ff_make(w * u[j]);
                    s_p[tid][0] = make_float4(x.h, x.l, yy.h, yy.l);
                    s_p[tid][1] = make_float4(z.h, z.l, nx.h, nx.l);
                    s_p[tid][2] = make_float4(ny.h, ny.l, nz.h, nz.l);
                    s_p[tid][3] = make_float4(wpsi.h, wpsi.l, wphi.h, wphi.l);
                }
            }
            __syncthreads();
            const int cnt = (int)((N - st * TS) < TS ? (N - st * TS) : TS);
            ff f1[T], f2[T];
#pragma unroll
            for (int t = 0; t < T; ++t) { f1[t] = ff{0.f, 0.f}; f2[t] = ff{0.f, 0.f}; }
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 q0 = s_p[jj][0], q1 = s_p[jj][1], q2 = s_p[jj][2], q3 = s_p[jj][3];
                const ff sx{q0.x, q0.y}, sy{q0.z, q0.w}, sz{q1.x, q1.y};
                const ff snx{q1.z, q1.w}, sny{q2.x, q2.y}, snz{q2.z, q2.w};
                const ff wpsi{q3.x, q3.y}, wphi{q3.z, q3.w};
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const ff dx = ff_sub(xi[t], sx), dy = ff_sub(yi[t], sy), dz = ff_sub(zi[t], sz);
                    const ff r2 = ff_add_q(ff_add_q(ff_mul(dx, dx), ff_mul(dy, dy)), ff_mul(dz, dz));
                    if (r2.h > 0.f) {      // the self pair and pairs at zero distance are dropped
                        // 1/rho: MUFU rsqrt, then one Newton step in float-float
                        const float y0 = rsqrt_approx(r2.h);
                        const float y0y0 = y0 * y0;
                        const ff yy{y0y0, fmaf(y0, y0, -y0y0)};
                        const ff h = ff_mul(r2, yy);
                        const ff corr = ff_add_q(ff{1.5f, 0.f}, ff{-0.5f * h.h, -0.5f * h.l});
                        const ff inv = ff_mulf(corr, y0);
                        const ff rho = ff_mul(r2, inv);
                        const ff inv2 = ff_mul(inv, inv);
                        const ff inv3 = ff_mul(inv2, inv);
                        const ff cx = ff_add_q(ff_add_q(ff_mul(dx, nxi[t]), ff_mul(dy, nyi[t])), ff_mul(dz, nzi[t]));
                        const ff cy = ff_add_q(ff_add_q(ff_mul(dx, snx), ff_mul(dy, sny)), ff_mul(dz, snz));
                        const ff nn =
                            ff_add_q(ff_add_q(ff_mul(nxi[t], snx), ff_mul(nyi[t], sny)), ff_mul(nzi[t], snz));
                        const ff kr = ff_mul(prm.kappa, rho);
                        const ff e = ff_exp2(ff_mul(prm.neg_kappa_log2e, rho), prm);
                        const ff e1 = ff_add_q(e, ff_mul(e, kr));                        // e (1 + kappa rho)
                        const ff k1 = ff_mul(ff_sub(one, e), inv);
                        const ff k2 = ff_mul(ff_mul(ff_sub(ff_mul(prm.eps, e1), one), cy), inv3);
                        const ff k3 = ff_mul(ff_mul(ff_sub(ff_mul(prm.inv_eps, e1), one), cx), inv3);
                        const ff p3 = ff_add_q(ff_add_q(three, ff_mulf(kr, 3.f)), ff_mul(kr, kr));
                        const ff e3 = ff_sub(ff_mul(e, p3), three);
                        const ff k4 = ff_mul(ff_sub(ff_mul(ff_sub(e1, one), nn), ff_mul(ff_mul(ff_mul(e3, cx), cy), inv2)),
                                             inv3);
                        f1[t] = ff_add_q(f1[t], ff_add_q(ff_mul(k1, wpsi), ff_mul(k2, wphi)));
                        f2[t] = ff_add_q(f2[t], ff_add_q(ff_mul(k3, wpsi), ff_mul(k4, wphi)));
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < T; ++t) {
                acc1[t] += (double)f1[t].h + (double)f1[t].l;
                acc2[t] += (double)f2[t].h + (double)f2[t].l;
            }
        }
        finish_segment<TT, T, BS>(plan, a, c, acc1, acc2, u, N, prm.diag1, prm.diag2, partials, counters, y);
        p += s_end - s_first;
    }
}

std::mutex g_table_mu;
bool g_table_ready[64] = {};

}  // namespace

StreamKPlan matvec_ff_plan(pb_ctx *ctx) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, matvec_ff_kernel, kFFThreads, 0);
    if (occ < 1) occ = 1;
    return make_plan(ctx->N, kFFTargetTile, kFFSourceTile, (int64_t)ctx->num_sms * occ);
}

int matvec_ff_target_tile() { return kFFTargetTile; }

pb_status matvec_ff_enqueue(pb_ctx *ctx, const double *u, double *y, const int *skip_flag) {
    const int dev = ctx->device;
    {
        // the 2^(k/64) table, uploaded once per device (synchronously, so that
        // launches on any stream see it)
        std::lock_guard<std::mutex> lock(g_table_mu);
        if (dev < 0 || dev >= 64) return set_error(ctx, PB_ERR_ARG, "device index %d out of range", dev);
        if (!g_table_ready[dev]) {
            float2 tab[65];
            for (int k = -32; k <= 32; ++k) {
                const double v = exp2((double)k / 64.0);
                const float h = (float)v;
                tab[k + 32] = make_float2(h, (float)(v - (double)h));
            }
            cudaError_t e = cudaMemcpyToSymbol(c_exp2_table, tab, sizeof(tab));
            if (e != cudaSuccess) return cuda_error(ctx, e, "float-float exp table");
            g_table_ready[dev] = true;
        }
    }
    FFParams prm;
    auto mk = [](double v) {
        const float h = (float)v;
        return ff{h, (float)(v - (double)h)};
    };
    prm.eps = mk(ctx->eps);
    prm.inv_eps = mk(1.0 / ctx->eps);
    prm.kappa = mk(ctx->kappa);
    prm.neg_kappa_log2e = mk(-ctx->kappa / 0.69314718055994530942);
    prm.ln2 = mk(0.69314718055994530942);
    prm.diag1 = 0.5 * (1.0 + ctx->eps);
    prm.diag2 = 0.5 * (1.0 + 1.0 / ctx->eps);
    const StreamKPlan &pl = ctx->planff;
    matvec_ff_kernel<<<(unsigned)pl.ctas, kFFThreads, 0, ctx->stream>>>(
        ctx->g64, u, ctx->N, prm, pl, ctx->partials, ctx->tile_counters, y, skip_flag, ctx->mv_count);
    return PB_OK;
}

}  // namespace pb
