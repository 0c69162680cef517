// matvec.cu -- the direct-sum matrix-vector product y = A u of Eqs. (12)-(13).
//
// For every centroid x_i (target) the kernels K1..K4 of Eq. (10) are summed
// over all other centroids x_j (sources), weighted by W_j = area_j and applied
// to u_j = (phi_j, dphi_j/dnu):
//   y_i     = (1 + eps)/2   phi_i  - sum_{j != i} W_j [K1 dphi_j + K2 phi_j]
//   y_{N+i} = (1 + 1/eps)/2 dphi_i - sum_{j != i} W_j [K3 dphi_j + K4 phi_j]
// With r = x_i - x_j, rho = |r|, e = exp(-kappa rho), c_x = r.nu_i,
// c_y = r.nu_j, n = nu_i.nu_j and the 1/(4 pi) folded into the source weights:
//   K1 = (1 - e)/rho
//   K2 = (eps e (1 + kappa rho) - 1) c_y / rho^3
//   K3 = (e (1 + kappa rho)/eps - 1) c_x / rho^3
//   K4 = (e (1 + kappa rho) - 1) n / rho^3 - (e (3 + 3 kappa rho + kappa^2 rho^2) - 3) c_x c_y / rho^5
// The singular j = i term is dropped (Section 2.2), and so is any pair at zero
// distance.
//
// Layout: the (target tile x source tile) iteration space is flattened and cut
// into equal contiguous ranges, one per persistent CTA, so every SM gets the
// same number of pair tiles whatever N is.  A CTA walks its range target tile
// by target tile; the source tiles it visits are staged in shared memory and
// read by all its threads (broadcast loads).  A target tile covered by several
// CTAs is finished by the last of them to arrive: it sums the per-CTA partial
// rows in CTA order (deterministic, no floating-point atomics) and adds the
// diagonal term.
#include <math.h>

#include "fastmath.cuh"
#include "pb_internal.cuh"

namespace pb {

StreamKPlan make_plan(int64_t n, int target_tile, int source_tile, int64_t ctas_wanted) {
    StreamKPlan p;
    p.target_tiles = (n + target_tile - 1) / target_tile;
    p.source_tiles = (n + source_tile - 1) / source_tile;
    p.work = p.target_tiles * p.source_tiles;
    p.ctas = ctas_wanted < 1 ? 1 : (ctas_wanted > p.work ? p.work : ctas_wanted);
    p.max_segments = 1;
    for (int64_t a = 0; a < p.target_tiles; ++a) {
        int64_t s = sk_cta_of(a * p.source_tiles + p.source_tiles - 1, p.work, p.ctas) -
                    sk_cta_of(a * p.source_tiles, p.work, p.ctas) + 1;
        if (s > p.max_segments) p.max_segments = s;
    }
    return p;
}

namespace {

struct F32Params {
    float eps, inv_eps, kappa, neg_kappa_log2e;
    double diag1, diag2;
};

// Finish a segment: either write y directly (one CTA covers the whole target
// tile) or publish partial rows and let the last arriving CTA reduce them.
template <int TT, int T, int BS>
__device__ __forceinline__ void finish_segment(const StreamKPlan &plan, int64_t a, int64_t c,
                                               const double (&acc1)[T], const double (&acc2)[T],
                                               const double *__restrict__ u, int64_t N, double diag1,
                                               double diag2, double *__restrict__ partials,
                                               unsigned int *__restrict__ counters, double *__restrict__ y) {
    const int64_t S = plan.source_tiles;
    const int64_t c0 = sk_cta_of(a * S, plan.work, plan.ctas);
    const int64_t c1 = sk_cta_of(a * S + S - 1, plan.work, plan.ctas);
    const int nseg = (int)(c1 - c0 + 1);
    const int tid = threadIdx.x;
    if (nseg == 1) {
#pragma unroll
        for (int t = 0; t < T; ++t) {
            int64_t i = a * TT + t * BS + tid;
            if (i < N) {
                y[i] = diag1 * u[i] - acc1[t];
                y[N + i] = diag2 * u[N + i] - acc2[t];
            }
        }
        return;
    }
    const int ord = (int)(c - c0);
    double *mine = partials + ((a * plan.max_segments + ord) * 2) * TT;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        mine[t * BS + tid] = acc1[t];
        mine[TT + t * BS + tid] = acc2[t];
    }
    __threadfence();
    __syncthreads();
    __shared__ int s_last;
    if (tid == 0) {
        unsigned int prev = atomicAdd(&counters[a], 1u);
        s_last = (prev == (unsigned int)(nseg - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
#pragma unroll
    for (int t = 0; t < T; ++t) {
        int64_t i = a * TT + t * BS + tid;
        double s1 = 0.0, s2 = 0.0;
        for (int o = 0; o < nseg; ++o) {
            const double *pp = partials + ((a * plan.max_segments + o) * 2) * TT;
            s1 += __ldcg(pp + t * BS + tid);
            s2 += __ldcg(pp + TT + t * BS + tid);
        }
        if (i < N) {
            y[i] = diag1 * u[i] - s1;
            y[N + i] = diag2 * u[N + i] - s2;
        }
    }
    if (tid == 0) counters[a] = 0u;   // ready for the next launch
}

// ---------------------------------------------------------------------------
// FP32 pair arithmetic, FP32 partial sums per source tile, FP64 row sums.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kF32Threads)
matvec_f32_kernel(const float4 *__restrict__ pos, const float4 *__restrict__ nrm,
                  const double *__restrict__ u, int64_t N, F32Params prm, StreamKPlan plan,
                  double *__restrict__ partials, unsigned int *__restrict__ counters,
                  double *__restrict__ y, const int *__restrict__ skip, unsigned long long *__restrict__ evaluated) {
    constexpr int BS = kF32Threads, T = kF32TargetsPerThread, TT = kF32TargetTile, TS = kF32SourceTile;
    if (skip != nullptr && *((volatile const int *)skip)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(evaluated, 1ull);
    __shared__ float4 s_pos[TS];   // x, y, z, W dphi / (4 pi)
    __shared__ float4 s_nrm[TS];   // nx, ny, nz, W phi / (4 pi)

    const int tid = threadIdx.x;
    const int64_t c = blockIdx.x;
    const int64_t S = plan.source_tiles;
    int64_t p = sk_begin(c, plan.work, plan.ctas);
    const int64_t pend = sk_begin(c + 1, plan.work, plan.ctas);

    while (p < pend) {
        const int64_t a = p / S;
        const int64_t s_first = p % S;
        const int64_t s_end = (S < s_first + (pend - p)) ? S : s_first + (pend - p);

        float xi[T], yi[T], zi[T], nxi[T], nyi[T], nzi[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            int64_t i = a * TT + t * BS + tid;
            if (i > N - 1) i = N - 1;
            float4 q = pos[i], n = nrm[i];
            xi[t] = q.x; yi[t] = q.y; zi[t] = q.z;
            nxi[t] = n.x; nyi[t] = n.y; nzi[t] = n.z;
        }
        double acc1[T], acc2[T];
#pragma unroll
        for (int t = 0; t < T; ++t) { acc1[t] = 0.0; acc2[t] = 0.0; }

        for (int64_t s = s_first; s < s_end; ++s) {
            __syncthreads();
            for (int jl = tid; jl < TS; jl += BS) {
                int64_t j = s * TS + jl;
                if (j < N) {
                    float4 q = pos[j], n = nrm[j];
                    float w = q.w;
                    s_pos[jl] = make_float4(q.x, q.y, q.z, (float)u[N + j] * w);
                    s_nrm[jl] = make_float4(n.x, n.y, n.z, (float)u[j] * w);
                }
            }
            __syncthreads();
            const int cnt = (int)((N - s * TS) < TS ? (N - s * TS) : TS);
            float f1[T], f2[T];
#pragma unroll
            for (int t = 0; t < T; ++t) { f1[t] = 0.f; f2[t] = 0.f; }
#pragma unroll 2
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 sp = s_pos[jj];
                const float4 sn = s_nrm[jj];
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const float dx = xi[t] - sp.x, dy = yi[t] - sp.y, dz = zi[t] - sp.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    float inv = rsqrt_approx(r2);
                    inv = (r2 > 0.f) ? inv : 0.f;             // drop j == i and coincident pairs
                    const float rho = r2 * inv;
                    const float e = exp2_approx(prm.neg_kappa_log2e * rho);
                    const float kr = prm.kappa * rho;
                    const float e1 = fmaf(e, kr, e);            // e (1 + kappa rho)
                    const float inv2 = inv * inv;
                    const float inv3 = inv2 * inv;
                    const float cx = fmaf(dx, nxi[t], fmaf(dy, nyi[t], dz * nzi[t]));
                    const float cy = fmaf(dx, sn.x, fmaf(dy, sn.y, dz * sn.z));
                    const float nn = fmaf(nxi[t], sn.x, fmaf(nyi[t], sn.y, nzi[t] * sn.z));
                    const float k1 = (1.f - e) * inv;
                    const float k2 = fmaf(prm.eps, e1, -1.f) * cy * inv3;
                    const float k3 = fmaf(e1, prm.inv_eps, -1.f) * cx * inv3;
                    const float p3 = fmaf(kr, kr + 3.f, 3.f);   // 3 + 3 kappa rho + kappa^2 rho^2
                    const float e3 = fmaf(e, p3, -3.f);
                    const float k4 = fmaf(-e3 * cx * cy, inv2, fmaf(e1, nn, -nn)) * inv3;
                    f1[t] = fmaf(k1, sp.w, fmaf(k2, sn.w, f1[t]));
                    f2[t] = fmaf(k3, sp.w, fmaf(k4, sn.w, f2[t]));
                }
            }
#pragma unroll
            for (int t = 0; t < T; ++t) { acc1[t] += (double)f1[t]; acc2[t] += (double)f2[t]; }
        }
        finish_segment<TT, T, BS>(plan, a, c, acc1, acc2, u, N, prm.diag1, prm.diag2, partials, counters, y);
        p += s_end - s_first;
    }
}

// ---------------------------------------------------------------------------
// The same FP32-pair product with packed f32x2 arithmetic: one instruction
// evaluates a step of two pairs (one target against two sources), which
// halves the issue slots of the FP32 work so that the FP32 pipe, not the
// instruction issue, bounds the kernel.  Sources are staged in shared memory
// as pairs (2q, 2q+1), four float4 per pair:
//   {-x0, -x1, -y0, -y1}  {-z0, -z1, nx0, nx1}  {ny0, ny1, nz0, nz1}  {Wdphi0, Wdphi1, Wphi0, Wphi1}
// (W carries the 1/(4 pi)).  Each thread owns T targets, duplicated into both
// halves of register pairs.  The singular self pair (and any pair at zero
// distance) is removed by clamping 1/rho at 1e12: then rho = r2 * (1/rho) is
// exactly 0, exp2(0) is exactly 1, c_x = c_y = 0, and every term of K1..K4 is an
// exact zero, with no infinity formed.  Real pairs have 1/rho < 1e12 (rho > 1e-12 A).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }

constexpr float kInvRhoMax = 1e12f;

template <int T>
__global__ void __launch_bounds__(kF32Threads)
matvec_f32x2_kernel(const float4 *__restrict__ pos, const float4 *__restrict__ nrm,
                    const double *__restrict__ u, int64_t N, F32Params prm, StreamKPlan plan,
                    double *__restrict__ partials, unsigned int *__restrict__ counters,
                    double *__restrict__ y, const int *__restrict__ skip, unsigned long long *__restrict__ evaluated) {
    constexpr int BS = kF32Threads, TT = BS * T, TS = kF32SourceTile, TQ = TS / 2;
    static_assert(TQ == BS, "one source pair per thread when staging");
    if (skip != nullptr && *((volatile const int *)skip)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(evaluated, 1ull);
    __shared__ float4 s_a[TQ], s_b[TQ], s_c[TQ], s_d[TQ];

    const int tid = threadIdx.x;
    const int64_t c = blockIdx.x;
    const int64_t S = plan.source_tiles;
    int64_t p = sk_begin(c, plan.work, plan.ctas);
    const int64_t pend = sk_begin(c + 1, plan.work, plan.ctas);
    const float2 eps2 = p_dup(prm.eps), ieps2 = p_dup(prm.inv_eps), kap2 = p_dup(prm.kappa);
    const float2 nk2 = p_dup(prm.neg_kappa_log2e);
    const float2 one2 = p_dup(1.f), mone2 = p_dup(-1.f), three2 = p_dup(3.f), mthree2 = p_dup(-3.f);

    while (p < pend) {
        const int64_t a = p / S;
        const int64_t s_first = p % S;
        const int64_t s_end = (S < s_first + (pend - p)) ? S : s_first + (pend - p);

        float2 xi[T], yi[T], zi[T], nxi[T], nyi[T], nzi[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            int64_t i = a * TT + t * BS + tid;
            if (i > N - 1) i = N - 1;
            const float4 q = pos[i], n = nrm[i];
            xi[t] = p_dup(q.x); yi[t] = p_dup(q.y); zi[t] = p_dup(q.z);
            nxi[t] = p_dup(n.x); nyi[t] = p_dup(n.y); nzi[t] = p_dup(n.z);
        }
        double acc1[T], acc2[T];
#pragma unroll
        for (int t = 0; t < T; ++t) { acc1[t] = 0.0; acc2[t] = 0.0; }

        for (int64_t s = s_first; s < s_end; ++s) {
            __syncthreads();
            {
                // stage source pair (2 tid, 2 tid + 1); a missing second source
                // repeats the first with zero weights
                const int64_t j0 = s * TS + 2 * tid;
                if (j0 < N) {
                    const int64_t j1 = (j0 + 1 < N) ? j0 + 1 : j0;
                    const float4 p0 = pos[j0], p1 = pos[j1], n0 = nrm[j0], n1 = nrm[j1];
                    const float w0 = p0.w, w1 = (j0 + 1 < N) ? p1.w : 0.f;
                    s_a[tid] = make_float4(-p0.x, -p1.x, -p0.y, -p1.y);
                    s_b[tid] = make_float4(-p0.z, -p1.z, n0.x, n1.x);
                    s_c[tid] = make_float4(n0.y, n1.y, n0.z, n1.z);
                    s_d[tid] = make_float4((float)u[N + j0] * w0, (float)u[N + j1] * w1, (float)u[j0] * w0,
                                           (float)u[j1] * w1);
                }
            }
            __syncthreads();
            const int64_t rem = N - s * TS;
            const int npairs = (int)(((rem < TS) ? rem : TS) + 1) / 2;
            float2 f1[T], f2[T];
#pragma unroll
            for (int t = 0; t < T; ++t) { f1[t] = p_dup(0.f); f2[t] = p_dup(0.f); }
#pragma unroll 2
            for (int q = 0; q < npairs; ++q) {
                const float4 A = s_a[q], B = s_b[q], C = s_c[q], D = s_d[q];
                const float2 mx = make_float2(A.x, A.y), my = make_float2(A.z, A.w), mz = make_float2(B.x, B.y);
                const float2 snx = make_float2(B.z, B.w), sny = make_float2(C.x, C.y), snz = make_float2(C.z, C.w);
                const float2 wpsi = make_float2(D.x, D.y), wphi = make_float2(D.z, D.w);
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const float2 dx = p_add(xi[t], mx), dy = p_add(yi[t], my), dz = p_add(zi[t], mz);
                    const float2 r2 = p_fma(dx, dx, p_fma(dy, dy, p_mul(dz, dz)));
                    float2 inv;
                    inv.x = fminf(rsqrt_approx(r2.x), kInvRhoMax);
                    inv.y = fminf(rsqrt_approx(r2.y), kInvRhoMax);
                    const float2 rho = p_mul(r2, inv);
                    const float2 arg = p_mul(nk2, rho);
                    float2 e;
                    e.x = exp2_approx(arg.x);
                    e.y = exp2_approx(arg.y);
                    const float2 kr = p_mul(kap2, rho);
                    const float2 e1 = p_fma(e, kr, e);                    // e (1 + kappa rho)
                    const float2 inv2 = p_mul(inv, inv);
                    const float2 inv3 = p_mul(inv2, inv);
                    const float2 cx = p_fma(dx, nxi[t], p_fma(dy, nyi[t], p_mul(dz, nzi[t])));
                    const float2 cy = p_fma(dx, snx, p_fma(dy, sny, p_mul(dz, snz)));
                    const float2 nn = p_fma(nxi[t], snx, p_fma(nyi[t], sny, p_mul(nzi[t], snz)));
                    const float2 k1 = p_mul(p_fma(e, mone2, one2), inv);   // (1 - e)/rho
                    const float2 k2 = p_mul(p_mul(p_fma(eps2, e1, mone2), cy), inv3);
                    const float2 k3 = p_mul(p_mul(p_fma(e1, ieps2, mone2), cx), inv3);
                    const float2 p3 = p_fma(kr, p_add(kr, three2), three2);   // 3 + 3 kr + kr^2
                    const float2 e3 = p_fma(e, p3, mthree2);
                    const float2 ccy = p_mul(p_mul(e3, cx), cy);
                    const float2 k4 = p_mul(p_fma(p_neg(ccy), inv2, p_fma(e1, nn, p_neg(nn))), inv3);
                    f1[t] = p_fma(k1, wpsi, p_fma(k2, wphi, f1[t]));
                    f2[t] = p_fma(k3, wpsi, p_fma(k4, wphi, f2[t]));
                }
            }
#pragma unroll
            for (int t = 0; t < T; ++t) {
                acc1[t] += (double)f1[t].x + (double)f1[t].y;
                acc2[t] += (double)f2[t].x + (double)f2[t].y;
            }
        }
        finish_segment<TT, T, BS>(plan, a, c, acc1, acc2, u, N, prm.diag1, prm.diag2, partials, counters, y);
        p += s_end - s_first;
    }
}

// ---------------------------------------------------------------------------
// Plain FP64 path: every pair and every sum in FP64.
// ---------------------------------------------------------------------------
struct F64Params {
    double eps, inv_eps, kappa, diag1, diag2;
};

__global__ void __launch_bounds__(kF64Threads)
matvec_f64_kernel(const double *__restrict__ g64, const double *__restrict__ u, int64_t N, F64Params prm,
                  StreamKPlan plan, double *__restrict__ partials, unsigned int *__restrict__ counters,
                  double *__restrict__ y, const int *__restrict__ skip, unsigned long long *__restrict__ evaluated) {
    constexpr int BS = kF64Threads, TT = kF64TargetTile, TS = kF64SourceTile;
    if (skip != nullptr && *((volatile const int *)skip)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(evaluated, 1ull);
    __shared__ double s_x[TS], s_y[TS], s_z[TS], s_nx[TS], s_ny[TS], s_nz[TS], s_wpsi[TS], s_wphi[TS];
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
        int64_t i = a * TT + tid;
        if (i > N - 1) i = N - 1;
        const double xi = X[i], yi = Y[i], zi = Z[i], nxi = NX[i], nyi = NY[i], nzi = NZ[i];
        double acc1[1] = {0.0}, acc2[1] = {0.0};

        for (int64_t s = s_first; s < s_end; ++s) {
            __syncthreads();
            for (int jl = tid; jl < TS; jl += BS) {
                int64_t j = s * TS + jl;
                if (j < N) {
                    double w = W[j] * kInv4Pi;
                    s_x[jl] = X[j]; s_y[jl] = Y[j]; s_z[jl] = Z[j];
                    s_nx[jl] = NX[j]; s_ny[jl] = NY[j]; s_nz[jl] = NZ[j];
                    s_wpsi[jl] = w * u[N + j];
                    s_wphi[jl] = w * u[j];
                }
            }
            __syncthreads();
            const int cnt = (int)((N - s * TS) < TS ? (N - s * TS) : TS);
            double a1 = acc1[0], a2 = acc2[0];
            for (int jj = 0; jj < cnt; ++jj) {
                const double dx = xi - s_x[jj], dy = yi - s_y[jj], dz = zi - s_z[jj];
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 > 0.0) {
                    const double inv = rsqrt(r2);
                    const double rho = r2 * inv;
                    const double kr = prm.kappa * rho;
                    const double e = exp(-kr);
                    const double e1 = e * (1.0 + kr);
                    const double inv2 = inv * inv;
                    const double inv3 = inv2 * inv;
                    const double cx = dx * nxi + dy * nyi + dz * nzi;
                    const double cy = dx * s_nx[jj] + dy * s_ny[jj] + dz * s_nz[jj];
                    const double nn = nxi * s_nx[jj] + nyi * s_ny[jj] + nzi * s_nz[jj];
                    const double k1 = (1.0 - e) * inv;
                    const double k2 = (prm.eps * e1 - 1.0) * cy * inv3;
                    const double k3 = (e1 * prm.inv_eps - 1.0) * cx * inv3;
                    const double k4 = ((e1 - 1.0) * nn - (e * (3.0 + 3.0 * kr + kr * kr) - 3.0) * cx * cy * inv2) * inv3;
                    a1 += k1 * s_wpsi[jj] + k2 * s_wphi[jj];
                    a2 += k3 * s_wpsi[jj] + k4 * s_wphi[jj];
                }
            }
            acc1[0] = a1; acc2[0] = a2;
        }
        finish_segment<TT, 1, BS>(plan, a, c, acc1, acc2, u, N, prm.diag1, prm.diag2, partials, counters, y);
        p += s_end - s_first;
    }
}

}  // namespace

pb_status matvec_launch(pb_ctx *ctx, const double *u, double *y, pb_precision prec, const int *skip_flag) {
    const double diag1 = 0.5 * (1.0 + ctx->eps), diag2 = 0.5 * (1.0 + 1.0 / ctx->eps);
    if (prec != PB_FP32PAIR && prec != PB_FP64)
        return set_error(ctx, PB_ERR_ARG, "pb_matvec: unknown precision %d", (int)prec);
    const bool timed = ctx->prof_on;
    if (timed) {
        if (ctx->prof_used + 2 > (int)ctx->prof_ev.size()) {
            pb_status fs = profile_flush(ctx);
            if (fs != PB_OK) return fs;
        }
        cudaEventRecord(ctx->prof_ev[ctx->prof_used], ctx->stream);
    }
    if (prec == PB_FP32PAIR) {
        F32Params prm;
        prm.eps = (float)ctx->eps;
        prm.inv_eps = (float)(1.0 / ctx->eps);
        prm.kappa = (float)ctx->kappa;
        prm.neg_kappa_log2e = (float)(-ctx->kappa * 1.4426950408889634);
        prm.diag1 = diag1;
        prm.diag2 = diag2;
        const StreamKPlan &pl = ctx->plan32;
        switch (ctx->f32_variant) {
            case MV_F32_SCALAR_T4:
                matvec_f32_kernel<<<(unsigned)pl.ctas, kF32Threads, 0, ctx->stream>>>(
                    ctx->pos32, ctx->nrm32, u, ctx->N, prm, pl, ctx->partials, ctx->tile_counters, y, skip_flag,
                    ctx->mv_count);
                break;
            case MV_F32_PACKED_T4:
                matvec_f32x2_kernel<4><<<(unsigned)pl.ctas, kF32Threads, 0, ctx->stream>>>(
                    ctx->pos32, ctx->nrm32, u, ctx->N, prm, pl, ctx->partials, ctx->tile_counters, y, skip_flag,
                    ctx->mv_count);
                break;
            default:
                matvec_f32x2_kernel<2><<<(unsigned)pl.ctas, kF32Threads, 0, ctx->stream>>>(
                    ctx->pos32, ctx->nrm32, u, ctx->N, prm, pl, ctx->partials, ctx->tile_counters, y, skip_flag,
                    ctx->mv_count);
                break;
        }
    } else {
        F64Params prm{ctx->eps, 1.0 / ctx->eps, ctx->kappa, diag1, diag2};
        const StreamKPlan &pl = ctx->plan64;
        matvec_f64_kernel<<<(unsigned)pl.ctas, kF64Threads, 0, ctx->stream>>>(
            ctx->g64, u, ctx->N, prm, pl, ctx->partials, ctx->tile_counters, y, skip_flag, ctx->mv_count);
    }
    PB_LAUNCHED();
    if (timed) {
        cudaEventRecord(ctx->prof_ev[ctx->prof_used + 1], ctx->stream);
        ctx->prof_used += 2;
        ctx->prof_launches += 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "matvec launch");
    return PB_OK;
}

// CTAs per SM for each matvec kernel, used to size the persistent grids.
int matvec_occupancy(pb_precision prec) {
    int n = 0;
    if (prec == PB_FP32PAIR)
        return matvec_f32_occupancy(MV_F32_PACKED_T2);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matvec_f64_kernel, kF64Threads, 0);
    return n < 1 ? 1 : n;
}

int matvec_f32_occupancy(int variant) {
    int n = 0;
    switch (variant) {
        case MV_F32_SCALAR_T4:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matvec_f32_kernel, kF32Threads, 0);
            break;
        case MV_F32_PACKED_T4:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matvec_f32x2_kernel<4>, kF32Threads, 0);
            break;
        default:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matvec_f32x2_kernel<2>, kF32Threads, 0);
            break;
    }
    return n < 1 ? 1 : n;
}

StreamKPlan matvec_f32_plan(pb_ctx *ctx, int variant, int ctas_per_sm) {
    int occ = matvec_f32_occupancy(variant);
    if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
    return make_plan(ctx->N, kF32Threads * f32_variant_targets(variant), kF32SourceTile, (int64_t)ctx->num_sms * occ);
}

int64_t plan_partials(const StreamKPlan &pl, int target_tile) {
    return pl.target_tiles * pl.max_segments * 2 * target_tile;
}

pb_status matvec_configure(pb_ctx *ctx, int variant, int ctas_per_sm) {
    if (variant < 1 || variant > kNumF32Variants)
        return set_error(ctx, PB_ERR_ARG, "matvec variant %d is not one of 1..%d", variant, kNumF32Variants);
    if (ctas_per_sm < 0) return set_error(ctx, PB_ERR_ARG, "ctas_per_sm must be >= 0");
    StreamKPlan pl = matvec_f32_plan(ctx, variant, ctas_per_sm);
    if (plan_partials(pl, kF32Threads * f32_variant_targets(variant)) > ctx->partials_len ||
        pl.target_tiles > ctx->counters_len)
        return set_error(ctx, PB_ERR_ARG, "matvec configuration exceeds the context's scratch");
    ctx->f32_variant = variant;
    ctx->f32_ctas_per_sm = ctas_per_sm;
    ctx->plan32 = pl;
    return PB_OK;
}

}  // namespace pb
