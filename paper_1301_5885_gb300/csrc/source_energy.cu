// source_energy.cu -- the source term b of Eq. (11) and the solvation energy of
// Eq. (14).  Both are (targets x charges) pair sums like the matvec but with
// Nc << N, so one pass over the charges, staged in shared memory, suffices.
//
//   b_i     = 1/(4 pi eps1) sum_k Q_k / rho_ik                         (S1)
//   b_{N+i} = 1/(4 pi eps1) sum_k Q_k (-(x_i - x_k) . nu_i) / rho_ik^3  (S2)
//   E_sol   = 332.0636/2 sum_k Q_k sum_j W_j [K1~(x_k,x_j) dphi_j + K2~(x_k,x_j) phi_j]
// with K1~ = (1 - e)/rho, K2~ = (eps e (1 + kappa rho) - 1) c_y / rho^3
// (Eq. (10) times 4 pi), r = x_k - x_j, c_y = r . nu_j.  Pairs at zero
// distance are dropped.
#include <math.h>

#include "fastmath.cuh"
#include "pb_internal.cuh"
#include "reduce.cuh"

namespace pb {
namespace {

constexpr int kSrcThreads = 256;
constexpr int kChargeTile = 256;

template <bool F32>
__global__ void __launch_bounds__(kSrcThreads)
source_kernel(const double *__restrict__ g64, const float4 *__restrict__ pos32, const float4 *__restrict__ nrm32,
              int64_t N, const Charge4 *__restrict__ ch, int64_t nc, double scale, double *__restrict__ b) {
    __shared__ Charge4 s_q[kChargeTile];
    const int64_t i0 = blockIdx.x * (int64_t)kSrcThreads + threadIdx.x;
    const int64_t i = i0 < N ? i0 : N - 1;
    double xi, yi, zi, nxi, nyi, nzi;
    if (F32) {
        float4 p = pos32[i], n = nrm32[i];
        xi = p.x; yi = p.y; zi = p.z; nxi = n.x; nyi = n.y; nzi = n.z;
    } else {
        xi = g64[i]; yi = g64[N + i]; zi = g64[2 * N + i];
        nxi = g64[3 * N + i]; nyi = g64[4 * N + i]; nzi = g64[5 * N + i];
    }
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k0 = 0; k0 < nc; k0 += kChargeTile) {
        __syncthreads();
        if (k0 + threadIdx.x < nc) s_q[threadIdx.x] = ch[k0 + threadIdx.x];
        __syncthreads();
        const int cnt = (int)((nc - k0) < kChargeTile ? (nc - k0) : kChargeTile);
        if (F32) {
            const float fx = (float)xi, fy = (float)yi, fz = (float)zi;
            const float fnx = (float)nxi, fny = (float)nyi, fnz = (float)nzi;
            float a1 = 0.f, a2 = 0.f;
            for (int k = 0; k < cnt; ++k) {
                const Charge4 q = s_q[k];
                const float dx = fx - (float)q.x, dy = fy - (float)q.y, dz = fz - (float)q.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                float inv = rsqrt_approx(r2);
                inv = (r2 > 0.f) ? inv : 0.f;
                const float qq = (float)q.q;
                a1 = fmaf(qq, inv, a1);
                a2 = fmaf(-qq * fmaf(dx, fnx, fmaf(dy, fny, dz * fnz)), inv * inv * inv, a2);
            }
            s1 += a1;
            s2 += a2;
        } else {
            for (int k = 0; k < cnt; ++k) {
                const Charge4 q = s_q[k];
                const double dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 > 0.0) {
                    const double inv = rsqrt(r2);
                    s1 += q.q * inv;
                    s2 += -q.q * (dx * nxi + dy * nyi + dz * nzi) * inv * inv * inv;
                }
            }
        }
    }
    if (i0 < N) {
        b[i0] = scale * s1;
        b[N + i0] = scale * s2;
    }
}

template <bool F32>
__global__ void __launch_bounds__(kSrcThreads)
energy_kernel(const double *__restrict__ g64, const float4 *__restrict__ pos32, const float4 *__restrict__ nrm32,
              int64_t N, const Charge4 *__restrict__ ch, int64_t nc, const double *__restrict__ u, double eps,
              double kappa, double *__restrict__ red, unsigned int *__restrict__ counter, double *__restrict__ out) {
    __shared__ Charge4 s_q[kChargeTile];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kSrcThreads;
    // blockIdx.y takes the charges [kbeg, kend): a second grid dimension
    // keeps small surfaces from leaving most SMs idle
    const int64_t kchunk = (nc + gridDim.y - 1) / gridDim.y;
    const int64_t kbeg = blockIdx.y * kchunk, kend = (kbeg + kchunk < nc) ? kbeg + kchunk : nc;
    for (int64_t k0 = kbeg; k0 < kend; k0 += kChargeTile) {
        __syncthreads();
        if (k0 + threadIdx.x < kend) s_q[threadIdx.x] = ch[k0 + threadIdx.x];
        __syncthreads();
        const int cnt = (int)((kend - k0) < kChargeTile ? (kend - k0) : kChargeTile);
        for (int64_t j = blockIdx.x * (int64_t)kSrcThreads + threadIdx.x; j < N; j += stride) {
            const double phi = u[j], dphi = u[N + j];
            if (F32) {
                const float4 p = pos32[j], n = nrm32[j];
                const float fe = (float)eps, fk = (float)kappa, nk = (float)(-kappa * 1.4426950408889634);
                float a1 = 0.f, a2 = 0.f;   // sum_k Q_k K1~, sum_k Q_k K2~
                for (int k = 0; k < cnt; ++k) {
                    const Charge4 q = s_q[k];
                    const float dx = (float)q.x - p.x, dy = (float)q.y - p.y, dz = (float)q.z - p.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    float inv = rsqrt_approx(r2);
                    inv = (r2 > 0.f) ? inv : 0.f;
                    const float rho = r2 * inv;
                    const float e = exp2_approx(nk * rho);
                    const float e1 = fmaf(e, fk * rho, e);
                    const float cy = fmaf(dx, n.x, fmaf(dy, n.y, dz * n.z));
                    const float qq = (float)q.q;
                    a1 = fmaf(qq * (1.f - e), inv, a1);
                    a2 = fmaf(qq * fmaf(fe, e1, -1.f) * cy, inv * inv * inv, a2);
                }
                // pos32.w holds W/(4 pi)
                acc += 4.0 * kPi * (double)p.w * ((double)a1 * dphi + (double)a2 * phi);
            } else {
                const double xj = g64[j], yj = g64[N + j], zj = g64[2 * N + j];
                const double nx = g64[3 * N + j], ny = g64[4 * N + j], nz = g64[5 * N + j], w = g64[6 * N + j];
                double a1 = 0.0, a2 = 0.0;
                for (int k = 0; k < cnt; ++k) {
                    const Charge4 q = s_q[k];
                    const double dx = q.x - xj, dy = q.y - yj, dz = q.z - zj;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 > 0.0) {
                        const double inv = rsqrt(r2);
                        const double rho = r2 * inv;
                        const double e = exp(-kappa * rho);
                        const double e1 = e * (1.0 + kappa * rho);
                        const double cy = dx * nx + dy * ny + dz * nz;
                        a1 += q.q * (1.0 - e) * inv;
                        a2 += q.q * (eps * e1 - 1.0) * cy * inv * inv * inv;
                    }
                }
                acc += w * (a1 * dphi + a2 * phi);
            }
        }
    }
    const double bs = block_sum<kSrcThreads>(acc);
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

pb_status source_launch(pb_ctx *ctx, double *b, pb_precision prec) {
    if (prec == PB_FLOAT2) return source_ff_launch(ctx, b);
    const unsigned blocks = (unsigned)((ctx->N + kSrcThreads - 1) / kSrcThreads);
    const double scale = kInv4Pi / ctx->eps1;
    if (prec == PB_FP32PAIR)
        source_kernel<true><<<blocks, kSrcThreads, 0, ctx->stream>>>(ctx->g64, ctx->pos32, ctx->nrm32, ctx->N,
                                                                     ctx->charges, ctx->Nc, scale, b);
    else
        source_kernel<false><<<blocks, kSrcThreads, 0, ctx->stream>>>(ctx->g64, ctx->pos32, ctx->nrm32, ctx->N,
                                                                      ctx->charges, ctx->Nc, scale, b);
    PB_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "source kernel");
    return PB_OK;
}

pb_status energy_launch(pb_ctx *ctx, const double *u, pb_precision prec, double *dev_out) {
    if (prec == PB_FLOAT2) return energy_ff_launch(ctx, u, dev_out);
    // about 8 blocks per SM (FP64 pair arithmetic needs many warps to hide
    // its latency): source blocks first, then the charges split over a
    // second grid dimension (chunks of at least 32 charges); the grid depends
    // only on N, Nc and the SM count, so the summation order is fixed
    const int64_t want = 8 * (int64_t)ctx->num_sms;
    int64_t bx = red_blocks(ctx, ctx->N);
    int64_t by = want / bx;
    const int64_t ymax = (ctx->Nc + 31) / 32;
    if (by > ymax) by = ymax;
    if (by < 1) by = 1;
    if (bx * by > ctx->red_len) by = ctx->red_len / bx > 0 ? ctx->red_len / bx : 1;
    const dim3 blocks((unsigned)bx, (unsigned)by);
    if (prec == PB_FP32PAIR)
        energy_kernel<true><<<blocks, kSrcThreads, 0, ctx->stream>>>(ctx->g64, ctx->pos32, ctx->nrm32, ctx->N,
                                                                     ctx->charges, ctx->Nc, u, ctx->eps, ctx->kappa,
                                                                     ctx->red, ctx->red_counter, dev_out);
    else
        energy_kernel<false><<<blocks, kSrcThreads, 0, ctx->stream>>>(ctx->g64, ctx->pos32, ctx->nrm32, ctx->N,
                                                                      ctx->charges, ctx->Nc, u, ctx->eps, ctx->kappa,
                                                                      ctx->red, ctx->red_counter, dev_out);
    PB_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "energy kernel");
    return PB_OK;
}

}  // namespace pb
