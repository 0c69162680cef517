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
#include <type_traits>

#include "fastmath.cuh"
#include "finish.cuh"
#include "pb_internal.cuh"
#include "reduce.cuh"
#include "sym.cuh"

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

// K1..K4 ingredients of one pair in float-float: K1 = k1, K2 = a c_y,
// K3 = b c_x, K4 = k4 (a, b and k4 already divided by rho^3).  Returns false
// for a pair at zero distance (the self pair), which is dropped.
struct FFPair {
    ff k1, a, b, k4, cx, cy;
};

__device__ __forceinline__ bool ff_pair(ff xi, ff yi, ff zi, ff nxi, ff nyi, ff nzi, ff sx, ff sy, ff sz, ff snx,
                                        ff sny, ff snz, const FFParams &prm, FFPair &o) {
    const ff one{1.f, 0.f}, three{3.f, 0.f};
    const ff dx = ff_sub(xi, sx), dy = ff_sub(yi, sy), dz = ff_sub(zi, sz);
    const ff r2 = ff_add_q(ff_add_q(ff_mul(dx, dx), ff_mul(dy, dy)), ff_mul(dz, dz));
    if (!(r2.h > 0.f)) return false;
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
    o.cx = ff_add_q(ff_add_q(ff_mul(dx, nxi), ff_mul(dy, nyi)), ff_mul(dz, nzi));
    o.cy = ff_add_q(ff_add_q(ff_mul(dx, snx), ff_mul(dy, sny)), ff_mul(dz, snz));
    const ff nn = ff_add_q(ff_add_q(ff_mul(nxi, snx), ff_mul(nyi, sny)), ff_mul(nzi, snz));
    const ff kr = ff_mul(prm.kappa, rho);
    const ff e = ff_exp2(ff_mul(prm.neg_kappa_log2e, rho), prm);
    const ff e1 = ff_add_q(e, ff_mul(e, kr));                        // e (1 + kappa rho)
    o.k1 = ff_mul(ff_sub(one, e), inv);
    o.a = ff_mul(ff_sub(ff_mul(prm.eps, e1), one), inv3);
    o.b = ff_mul(ff_sub(ff_mul(prm.inv_eps, e1), one), inv3);
    const ff p3 = ff_add_q(ff_add_q(three, ff_mulf(kr, 3.f)), ff_mul(kr, kr));
    const ff e3 = ff_sub(ff_mul(e, p3), three);
    o.k4 = ff_mul(ff_sub(ff_mul(ff_sub(e1, one), nn), ff_mul(ff_mul(ff_mul(e3, o.cx), o.cy), inv2)), inv3);
    return true;
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
                    FFPair q;
                    if (ff_pair(xi[t], yi[t], zi[t], nxi[t], nyi[t], nzi[t], sx, sy, sz, snx, sny, snz, prm, q)) {
                        const ff k2 = ff_mul(q.a, q.cy), k3 = ff_mul(q.b, q.cx);
                        f1[t] = ff_add_q(f1[t], ff_add_q(ff_mul(q.k1, wpsi), ff_mul(k2, wphi)));
                        f2[t] = ff_add_q(f2[t], ff_add_q(ff_mul(k3, wpsi), ff_mul(q.k4, wphi)));
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < T; ++t) {
                acc1[t] += (double)f1[t].h + (double)f1[t].l;
                acc2[t] += (double)f2[t].h + (double)f2[t].l;
            }
        }
        finish_segment<TT, T, BS>(plan, a, c, acc1, acc2, u, N, RowBlock{0, N, N}, prm.diag1, prm.diag2, partials,
                                  counters, y);
        p += s_end - s_first;
    }
}

// The float-float product evaluated symmetrically: the tiling, plan and
// finishing kernel of the symmetric FP32-pair and FP64 products, with each
// unordered pair evaluated once in float-float for both rows (row j gets
// K1 dphi_i - a c_x phi_i and -b c_y dphi_i + K4 phi_i).  Row sides are
// summed in float-float per 128-source stage and then in FP64; a source's
// column side is reduced over the warp in float-float (shuffling both parts)
// and stored in FP64.
template <int T>
__global__ void __launch_bounds__(kFFThreads)
matvec_ffsym_kernel(const double *__restrict__ g64, const double *__restrict__ u, int64_t N, FFParams prm,
                    SymPlan plan, double *__restrict__ islots, double *__restrict__ iside,
                    double *__restrict__ jpart, const int *__restrict__ skip,
                    unsigned long long *__restrict__ evaluated) {
    constexpr int BS = kFFThreads, B = BS * T, TS = BS, NW = BS / 32, STAGES = B / TS;
    if (skip != nullptr && *((volatile const int *)skip)) return;
    if (evaluated != nullptr && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(evaluated, 1ull);
    __shared__ float4 s_p[TS][4];
    __shared__ double s_col[NW][2][B];
    const double *X = g64, *Y = g64 + N, *Z = g64 + 2 * N;
    const double *NX = g64 + 3 * N, *NY = g64 + 4 * N, *NZ = g64 + 5 * N, *W = g64 + 6 * N;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool hi16 = (lane & 16) != 0;
    const int64_t c = blockIdx.x;
    const int64_t Tt = plan.tiles;
    const int64_t wb = plan.work_begin;   // first tile pair of this launch's band of rows
    int64_t p = wb + sk_begin(c, plan.work, plan.ctas);
    const int64_t pend = wb + sk_begin(c + 1, plan.work, plan.ctas);
    const int64_t I_first = sym_row_of(p, Tt);

    while (p < pend) {
        const int64_t I = sym_row_of(p, Tt);
        const int64_t row_end = sym_row_start(I + 1, Tt);
        const int64_t p_stop = pend < row_end ? pend : row_end;
        ff xi[T], yi[T], zi[T], nxi[T], nyi[T], nzi[T], wpi[T], wfi[T];
        double acc1[T], acc2[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int64_t i0 = I * B + t * BS + tid;
            const int64_t i = i0 < N ? i0 : N - 1;
            xi[t] = ff_make(X[i]); yi[t] = ff_make(Y[i]); zi[t] = ff_make(Z[i]);
            nxi[t] = ff_make(NX[i]); nyi[t] = ff_make(NY[i]); nzi[t] = ff_make(NZ[i]);
            const double w = i0 < N ? W[i] * kInv4Pi : 0.0;
            wpi[t] = ff_make(w * u[N + i]);
            wfi[t] = ff_make(w * u[i]);
            acc1[t] = 0.0;
            acc2[t] = 0.0;
        }
        for (; p < p_stop; ++p) {
            const int64_t J = I + (p - sym_row_start(I, Tt));
            const bool diag = (J == I);
            for (int stg = 0; stg < STAGES; ++stg) {
                const int64_t s0 = J * B + stg * TS;
                if (s0 >= N) break;
                __syncthreads();
                {
                    const int64_t j = s0 + tid;
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
                const int cnt = (int)((N - s0) < TS ? (N - s0) : TS);
                ff f1[T], f2[T];
#pragma unroll
                for (int t = 0; t < T; ++t) { f1[t] = ff{0.f, 0.f}; f2[t] = ff{0.f, 0.f}; }
                for (int jj = 0; jj < cnt; ++jj) {
                    const float4 q0 = s_p[jj][0], q1 = s_p[jj][1], q2 = s_p[jj][2], q3 = s_p[jj][3];
                    const ff sx{q0.x, q0.y}, sy{q0.z, q0.w}, sz{q1.x, q1.y};
                    const ff snx{q1.z, q1.w}, sny{q2.x, q2.y}, snz{q2.z, q2.w};
                    const ff wpsi{q3.x, q3.y}, wphi{q3.z, q3.w};
                    ff g1{0.f, 0.f}, g2{0.f, 0.f};     // column side of source jj
#pragma unroll
                    for (int t = 0; t < T; ++t) {
                        FFPair q;
                        if (ff_pair(xi[t], yi[t], zi[t], nxi[t], nyi[t], nzi[t], sx, sy, sz, snx, sny, snz, prm, q)) {
                            f1[t] = ff_add_q(f1[t], ff_add_q(ff_mul(q.k1, wpsi), ff_mul(ff_mul(q.a, q.cy), wphi)));
                            f2[t] = ff_add_q(f2[t], ff_add_q(ff_mul(ff_mul(q.b, q.cx), wpsi), ff_mul(q.k4, wphi)));
                            if (!diag) {
                                g1 = ff_add_q(g1, ff_sub(ff_mul(q.k1, wpi[t]), ff_mul(ff_mul(q.a, q.cx), wfi[t])));
                                g2 = ff_add_q(g2, ff_sub(ff_mul(q.k4, wfi[t]), ff_mul(ff_mul(q.b, q.cy), wpi[t])));
                            }
                        }
                    }
                    if (!diag) {
                        // lanes 0-15 end with the warp's sum of g1, 16-31 of g2,
                        // summed in float-float (the FP64 pipe is far slower)
                        ff keep = hi16 ? g2 : g1;
                        const ff send = hi16 ? g1 : g2;
                        keep = ff_add_q(keep, ff{__shfl_xor_sync(0xffffffffu, send.h, 16),
                                                 __shfl_xor_sync(0xffffffffu, send.l, 16)});
#pragma unroll
                        for (int off = 8; off >= 1; off >>= 1)
                            keep = ff_add_q(keep, ff{__shfl_xor_sync(0xffffffffu, keep.h, off),
                                                     __shfl_xor_sync(0xffffffffu, keep.l, off)});
                        if ((lane & 15) == 0) s_col[warp][lane >> 4][stg * TS + jj] = (double)keep.h + (double)keep.l;
                    }
                }
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    acc1[t] += (double)f1[t].h + (double)f1[t].l;
                    acc2[t] += (double)f2[t].h + (double)f2[t].l;
                }
            }
            if (!diag) {
                __syncthreads();
                double *dst = jpart + (sym_offdiag_index(I, J, Tt) - plan.joff) * 2 * B;
                for (int x = tid; x < 2 * B; x += BS) {
                    const int r = x / B, k = x - r * B;
                    double v = s_col[0][r][k];
#pragma unroll
                    for (int w2 = 1; w2 < NW; ++w2) v += s_col[w2][r][k];
                    dst[x] = v;
                }
            }
        }
        const int64_t c0 = sk_cta_of(sym_row_start(I, Tt) - wb, plan.work, plan.ctas);
        const int64_t c1 = sk_cta_of(row_end - 1 - wb, plan.work, plan.ctas);
        double *dst = (c0 == c1) ? iside + I * 2 * B : islots + (2 * c + (I == I_first ? 0 : 1)) * 2 * B;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            dst[t * BS + tid] = acc1[t];
            dst[B + t * BS + tid] = acc2[t];
        }
    }
}

std::mutex g_table_mu;
bool g_table_ready[64] = {};

}  // namespace

// the symmetric kernel from this N (below it the plain one balances better),
// with 2 targets per thread from kFFSymT2MinN
constexpr int64_t kFFSymMinN = 2048;
constexpr int64_t kFFSymT2MinN = 16384;

StreamKPlan matvec_ff_plan(pb_ctx *ctx) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, matvec_ff_kernel, kFFThreads, 0);
    if (occ < 1) occ = 1;
    if (ctx->N >= kFFSymMinN) {
        const int T = ctx->N >= kFFSymT2MinN ? 2 : 1;
        int occs = 0;
        if (T == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occs, matvec_ffsym_kernel<2>, kFFThreads, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occs, matvec_ffsym_kernel<1>, kFFThreads, 0);
        if (occs < 1) occs = 1;
        ctx->planffsym = make_sym_plan(ctx->N, kFFThreads * T, (int64_t)ctx->num_sms * occs);
    }
    return make_plan(ctx->N, kFFTargetTile, kFFSourceTile, (int64_t)ctx->num_sms * occ);
}

int matvec_ff_target_tile() { return kFFTargetTile; }

int64_t ff_sym_scratch_need(pb_ctx *ctx, std::vector<int64_t> *cuts) {
    cuts->clear();
    if (ctx->N < kFFSymMinN) return 0;
    const int B = kFFThreads * (ctx->N >= kFFSymT2MinN ? 2 : 1);
    return sym_scratch_need(ctx->planffsym, B, (int)sizeof(double), ctx->scratch_limit, ctx->bands, cuts);
}

// ---------------------------------------------------------------------------
// The source term of Eq. (11) and the energy of Eq. (14) in float-float: the
// same N x Nc pair sums as the FP64 kernels (source_energy.cu), with every
// pair quantity and the per-tile sums in float-float on the FP32 pipe and the
// final sums in FP64.
// ---------------------------------------------------------------------------
namespace {

constexpr int kFFChargeThreads = 256;
constexpr int kFFChargeTile = 256;

// charges as float-float {x, y}, {z, q} (hi, lo pairs)
__device__ __forceinline__ void ff_stage_charge(const Charge4 &q, float4 *dst) {
    const ff x = ff_make(q.x), y = ff_make(q.y), z = ff_make(q.z), w = ff_make(q.q);
    dst[0] = make_float4(x.h, x.l, y.h, y.l);
    dst[1] = make_float4(z.h, z.l, w.h, w.l);
}

// 1/rho from the MUFU rsqrt and one Newton step in float-float
__device__ __forceinline__ ff ff_rsqrt(ff r2) {
    const float y0 = rsqrt_approx(r2.h);
    const float y0y0 = y0 * y0;
    const ff yy{y0y0, fmaf(y0, y0, -y0y0)};
    const ff h = ff_mul(r2, yy);
    const ff corr = ff_add_q(ff{1.5f, 0.f}, ff{-0.5f * h.h, -0.5f * h.l});
    return ff_mulf(corr, y0);
}

// b_i = scale sum_k Q_k / rho_ik, b_{N+i} = scale sum_k -Q_k c_x / rho_ik^3
// (S1, S2 of Eq. (11) with scale = 1 / (4 pi eps1)); one thread per target
__global__ void __launch_bounds__(kFFChargeThreads)
ff_source_kernel(const double *__restrict__ g64, int64_t N, const Charge4 *__restrict__ ch, int64_t nc, double scale,
                 double *__restrict__ b) {
    __shared__ float4 s_q[kFFChargeTile][2];
    const int64_t i0 = blockIdx.x * (int64_t)kFFChargeThreads + threadIdx.x;
    const int64_t i = i0 < N ? i0 : N - 1;
    const ff xi = ff_make(g64[i]), yi = ff_make(g64[N + i]), zi = ff_make(g64[2 * N + i]);
    const ff nxi = ff_make(g64[3 * N + i]), nyi = ff_make(g64[4 * N + i]), nzi = ff_make(g64[5 * N + i]);
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k0 = 0; k0 < nc; k0 += kFFChargeTile) {
        __syncthreads();
        if (k0 + threadIdx.x < nc) ff_stage_charge(ch[k0 + threadIdx.x], s_q[threadIdx.x]);
        __syncthreads();
        const int cnt = (int)((nc - k0) < kFFChargeTile ? (nc - k0) : kFFChargeTile);
        ff a1{0.f, 0.f}, a2{0.f, 0.f};
        for (int k = 0; k < cnt; ++k) {
            const float4 A = s_q[k][0], B = s_q[k][1];
            const ff dx = ff_sub(xi, ff{A.x, A.y}), dy = ff_sub(yi, ff{A.z, A.w}), dz = ff_sub(zi, ff{B.x, B.y});
            const ff r2 = ff_add_q(ff_add_q(ff_mul(dx, dx), ff_mul(dy, dy)), ff_mul(dz, dz));
            if (!(r2.h > 0.f)) continue;
            const ff inv = ff_rsqrt(r2);
            const ff q{B.z, B.w};
            const ff cx = ff_add(ff_add(ff_mul(dx, nxi), ff_mul(dy, nyi)), ff_mul(dz, nzi));
            const ff inv3 = ff_mul(ff_mul(inv, inv), inv);
            a1 = ff_add(a1, ff_mul(q, inv));
            a2 = ff_sub(a2, ff_mul(ff_mul(q, cx), inv3));
        }
        s1 += (double)a1.h + (double)a1.l;
        s2 += (double)a2.h + (double)a2.l;
    }
    if (i0 < N) {
        b[i0] = scale * s1;
        b[N + i0] = scale * s2;
    }
}

// 1/2 sum_k Q_k sum_j W_j [K1(x_k, x_j) dphi_j + K2(x_k, x_j) phi_j] in kcal/mol
// (Eq. (14)); sources over blockIdx.x and threads, charges split over
// blockIdx.y; fixed-order two-stage reduction finished by the last block.
__global__ void __launch_bounds__(kFFChargeThreads)
ff_energy_kernel(const double *__restrict__ g64, int64_t N, const Charge4 *__restrict__ ch, int64_t nc,
                 const double *__restrict__ u, FFParams prm, double *__restrict__ red,
                 unsigned int *__restrict__ counter, double *__restrict__ out) {
    __shared__ float4 s_q[kFFChargeTile][2];
    const ff one{1.f, 0.f};
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kFFChargeThreads;
    const int64_t kchunk = (nc + gridDim.y - 1) / gridDim.y;
    const int64_t kbeg = blockIdx.y * kchunk, kend = (kbeg + kchunk < nc) ? kbeg + kchunk : nc;
    for (int64_t k0 = kbeg; k0 < kend; k0 += kFFChargeTile) {
        __syncthreads();
        if (k0 + threadIdx.x < kend) ff_stage_charge(ch[k0 + threadIdx.x], s_q[threadIdx.x]);
        __syncthreads();
        const int cnt = (int)((kend - k0) < kFFChargeTile ? (kend - k0) : kFFChargeTile);
        for (int64_t j = blockIdx.x * (int64_t)kFFChargeThreads + threadIdx.x; j < N; j += stride) {
            const ff xj = ff_make(g64[j]), yj = ff_make(g64[N + j]), zj = ff_make(g64[2 * N + j]);
            const ff nx = ff_make(g64[3 * N + j]), ny = ff_make(g64[4 * N + j]), nz = ff_make(g64[5 * N + j]);
            ff a1{0.f, 0.f}, a2{0.f, 0.f};   // sum_k Q_k K1, sum_k Q_k K2 (K without the 1/(4 pi))
            for (int k = 0; k < cnt; ++k) {
                const float4 A = s_q[k][0], B = s_q[k][1];
                const ff dx = ff_sub(ff{A.x, A.y}, xj), dy = ff_sub(ff{A.z, A.w}, yj), dz = ff_sub(ff{B.x, B.y}, zj);
                const ff r2 = ff_add_q(ff_add_q(ff_mul(dx, dx), ff_mul(dy, dy)), ff_mul(dz, dz));
                if (!(r2.h > 0.f)) continue;
                const ff inv = ff_rsqrt(r2);
                const ff rho = ff_mul(r2, inv);
                const ff e = ff_exp2(ff_mul(prm.neg_kappa_log2e, rho), prm);
                const ff e1 = ff_add_q(e, ff_mul(e, ff_mul(prm.kappa, rho)));     // e (1 + kappa rho)
                const ff cy = ff_add(ff_add(ff_mul(dx, nx), ff_mul(dy, ny)), ff_mul(dz, nz));
                const ff q{B.z, B.w};
                a1 = ff_add(a1, ff_mul(q, ff_mul(ff_sub(one, e), inv)));
                a2 = ff_add(a2, ff_mul(ff_mul(q, ff_sub(ff_mul(prm.eps, e1), one)),
                                       ff_mul(cy, ff_mul(ff_mul(inv, inv), inv))));
            }
            acc += g64[6 * N + j] * (((double)a1.h + (double)a1.l) * u[N + j] + ((double)a2.h + (double)a2.l) * u[j]);
        }
    }
    const double bs = block_sum<kFFChargeThreads>(acc);
    const unsigned int nblocks = gridDim.x * gridDim.y;
    if (threadIdx.x == 0) red[blockIdx.y * gridDim.x + blockIdx.x] = bs;
    if (last_block_arrived(counter, nblocks)) {
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (unsigned int b2 = 0; b2 < nblocks; ++b2) t += __ldcg(red + b2);
            out[0] = 0.5 * kCoulombKcal * t;
            *counter = 0u;
        }
    }
}

}  // namespace

namespace {

// The 2^(k/64) table (uploaded once per device) and the pair constants.
pb_status ff_setup(pb_ctx *ctx, FFParams *out) {
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
    *out = prm;
    return PB_OK;
}

}  // namespace

pb_status matvec_ff_enqueue(pb_ctx *ctx, const double *u, double *y, const int *skip_flag) {
    FFParams prm;
    pb_status fs = ff_setup(ctx, &prm);
    if (fs != PB_OK) return fs;
    if (ctx->N < kFFSymMinN) {
        const StreamKPlan &pl = ctx->planff;
        matvec_ff_kernel<<<(unsigned)pl.ctas, kFFThreads, 0, ctx->stream>>>(
            ctx->g64, u, ctx->N, prm, pl, ctx->partials, ctx->tile_counters, y, skip_flag, ctx->mv_count);
        return PB_OK;
    }
    const SymPlan &sp = ctx->planffsym;
    const int T = ctx->N >= kFFSymT2MinN ? 2 : 1;
    const int B = kFFThreads * T;
    const int64_t need = sym_scratch_need(sp, B, (int)sizeof(double), ctx->scratch_limit, ctx->bands, &ctx->cutsff);
    if (need > ctx->symff_scratch_len) {
        // the symmetric kernel's scratch, allocated by its first product
        if (ctx->symff_scratch) ctx_free(ctx, ctx->symff_scratch);
        ctx->device_bytes -= ctx->symff_scratch_len;
        ctx->symff_scratch = nullptr;
        ctx->symff_scratch_len = 0;
        pb_status s = ctx_alloc(ctx, &ctx->symff_scratch, (size_t)need, "symmetric float-float matvec scratch");
        if (s != PB_OK) return s;
        ctx->symff_scratch_len = need;
    }
    if (ctx->cutsff.size() > 2) {
        pb_status bs = ensure_band_streams(ctx);
        if (bs != PB_OK) return bs;
    }
    auto pair = [&](auto tag) {
        constexpr int TT = decltype(tag)::value;
        return [&](const SymPlan &bp, double *islots, double *iside, double *jpart, unsigned long long *ev,
                   cudaStream_t s) {
            matvec_ffsym_kernel<TT><<<(unsigned)bp.ctas, kFFThreads, 0, s>>>(
                ctx->g64, u, ctx->N, prm, bp, islots, iside, jpart, skip_flag, ev);
        };
    };
    cudaError_t e;
    if (T == 2)
        e = sym_enqueue<2 * kFFThreads, double>(sp, ctx->cutsff, ctx->symff_scratch, u, ctx->N, prm.diag1, prm.diag2,
                                                y, skip_flag, ctx->mv_count, ctx->stream, ctx->band_stream,
                                                ctx->band_ev, pair(std::integral_constant<int, 2>{}));
    else
        e = sym_enqueue<kFFThreads, double>(sp, ctx->cutsff, ctx->symff_scratch, u, ctx->N, prm.diag1, prm.diag2, y,
                                            skip_flag, ctx->mv_count, ctx->stream, ctx->band_stream, ctx->band_ev,
                                            pair(std::integral_constant<int, 1>{}));
    return e == cudaSuccess ? PB_OK : cuda_error(ctx, e, "symmetric float-float product bands");
}

pb_status source_ff_launch(pb_ctx *ctx, double *b) {
    FFParams prm;
    pb_status fs = ff_setup(ctx, &prm);
    if (fs != PB_OK) return fs;
    const unsigned blocks = (unsigned)((ctx->N + kFFChargeThreads - 1) / kFFChargeThreads);
    ff_source_kernel<<<blocks, kFFChargeThreads, 0, ctx->stream>>>(ctx->g64, ctx->N, ctx->charges, ctx->Nc,
                                                                  kInv4Pi / ctx->eps1, b);
    PB_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PB_OK : cuda_error(ctx, e, "float-float source kernel");
}

pb_status energy_ff_launch(pb_ctx *ctx, const double *u, double *dev_out) {
    FFParams prm;
    pb_status fs = ff_setup(ctx, &prm);
    if (fs != PB_OK) return fs;
    // the grid of the FP64 energy kernel: about 8 blocks per SM, charges
    // split over the second dimension; fixed for given N, Nc and SM count
    const int64_t want = 8 * (int64_t)ctx->num_sms;
    int64_t bx = red_blocks(ctx, ctx->N);
    int64_t by = want / bx;
    const int64_t ymax = (ctx->Nc + 31) / 32;
    if (by > ymax) by = ymax;
    if (by < 1) by = 1;
    if (bx * by > ctx->red_len) by = ctx->red_len / bx > 0 ? ctx->red_len / bx : 1;
    ff_energy_kernel<<<dim3((unsigned)bx, (unsigned)by), kFFChargeThreads, 0, ctx->stream>>>(
        ctx->g64, ctx->N, ctx->charges, ctx->Nc, u, prm, ctx->red, ctx->red_counter, dev_out);
    PB_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PB_OK : cuda_error(ctx, e, "float-float energy kernel");
}

}  // namespace pb
