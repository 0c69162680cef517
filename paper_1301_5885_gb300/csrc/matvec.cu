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

__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float exp2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

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
        matvec_f32_kernel<<<(unsigned)pl.ctas, kF32Threads, 0, ctx->stream>>>(
            ctx->pos32, ctx->nrm32, u, ctx->N, prm, pl, ctx->partials, ctx->tile_counters, y, skip_flag,
            ctx->mv_count);
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
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matvec_f32_kernel, kF32Threads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matvec_f64_kernel, kF64Threads, 0);
    return n < 1 ? 1 : n;
}

}  // namespace pb
