// geom.cu -- geometry preprocessing for pb_create (Section 2.4: triangles are
// turned into centroids, normals and areas before the device computation).
//
// 1. bounding-box centre of the centroids (one block, FP64),
// 2. validate every element (area finite and > 0, normal within 1e-3 of unit
//    length), renormalise the normal, subtract the centre, and pack
//      - FP64 SoA x | y | z | nx | ny | nz | W for the FP64 path,
//      - FP32 float4 {x, y, z, W/(4 pi)} and {nx, ny, nz, 0} for the FP32 path,
// 3. shift the charges by the same centre,
// 4. orientation check: for each charge x_k the Gauss sum
//    sum_j W_j dG0(x_k, x_j)/dnu_j is -1 for a closed surface with outward
//    normals enclosing x_k.
#include <math.h>

#include "pb_internal.cuh"
#include "reduce.cuh"

namespace pb {
namespace {

constexpr int kBoxThreads = 512;

__global__ void __launch_bounds__(kBoxThreads) bbox_center_kernel(const double *__restrict__ c, int64_t N,
                                                                  double *__restrict__ center) {
    __shared__ double s_lo[3][kBoxThreads], s_hi[3][kBoxThreads];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = threadIdx.x; i < N; i += kBoxThreads) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double v = c[3 * i + d];
            lo[d] = fmin(lo[d], v);
            hi[d] = fmax(hi[d], v);
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) { s_lo[d][threadIdx.x] = lo[d]; s_hi[d][threadIdx.x] = hi[d]; }
    __syncthreads();
    for (int s = kBoxThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                s_lo[d][threadIdx.x] = fmin(s_lo[d][threadIdx.x], s_lo[d][threadIdx.x + s]);
                s_hi[d][threadIdx.x] = fmax(s_hi[d][threadIdx.x], s_hi[d][threadIdx.x + s]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) center[d] = 0.5 * (s_lo[d][0] + s_hi[d][0]);
    }
}

__global__ void pack_kernel(const double *__restrict__ c, const double *__restrict__ nrm,
                            const double *__restrict__ area, int64_t N, const double *__restrict__ center,
                            double *__restrict__ g64, float4 *__restrict__ pos32, float4 *__restrict__ nrm32,
                            unsigned int *__restrict__ bad) {
    const double cx = center[0], cy = center[1], cz = center[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double x = c[3 * i] - cx, y = c[3 * i + 1] - cy, z = c[3 * i + 2] - cz;
        double nx = nrm[3 * i], ny = nrm[3 * i + 1], nz = nrm[3 * i + 2];
        double w = area[i];
        double len = sqrt(nx * nx + ny * ny + nz * nz);
        bool ok = isfinite(w) && w > 0.0 && isfinite(len) && fabs(len - 1.0) <= 1e-3 && isfinite(x) &&
                  isfinite(y) && isfinite(z);
        if (!ok) {
            atomicAdd(bad, 1u);
            len = 1.0;
            if (!(isfinite(w) && w > 0.0)) w = 0.0;
        }
        nx /= len; ny /= len; nz /= len;
        g64[i] = x; g64[N + i] = y; g64[2 * N + i] = z;
        g64[3 * N + i] = nx; g64[4 * N + i] = ny; g64[5 * N + i] = nz;
        g64[6 * N + i] = w;
        pos32[i] = make_float4((float)x, (float)y, (float)z, (float)(w * kInv4Pi));
        nrm32[i] = make_float4((float)nx, (float)ny, (float)nz, 0.f);
    }
}

__global__ void shift_charges_kernel(const double *__restrict__ q, int64_t nc, double cx, double cy, double cz,
                                     Charge4 *__restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nc; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = Charge4{q[4 * k] - cx, q[4 * k + 1] - cy, q[4 * k + 2] - cz, q[4 * k + 3]};
}

// One block per charge (grid-stride over charges), FP32 pairs, FP64 block sum.
constexpr int kGaussThreads = 256;
__global__ void __launch_bounds__(kGaussThreads)
gauss_kernel(const float4 *__restrict__ pos32, const float4 *__restrict__ nrm32, int64_t N,
             const Charge4 *__restrict__ ch, int64_t nc, double *__restrict__ out) {
    for (int64_t k = blockIdx.x; k < nc; k += gridDim.x) {
        const Charge4 q = ch[k];
        const float qx = (float)q.x, qy = (float)q.y, qz = (float)q.z;
        float acc = 0.f;
        double accd = 0.0;
        int n_in = 0;
        for (int64_t j = threadIdx.x; j < N; j += kGaussThreads) {
            const float4 p = pos32[j], n = nrm32[j];
            const float dx = qx - p.x, dy = qy - p.y, dz = qz - p.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > 0.f) {
                const float inv = rsqrtf(r2);
                acc += p.w * (dx * n.x + dy * n.y + dz * n.z) * inv * inv * inv;
            }
            if (++n_in == 64) { accd += acc; acc = 0.f; n_in = 0; }
        }
        accd += acc;
        const double s = block_sum<kGaussThreads>(accd);
        if (threadIdx.x == 0) out[k] = s;
    }
}

}  // namespace

pb_status geometry_prepare(pb_ctx *ctx, const double *c_dev, const double *n_dev, const double *a_dev) {
    double *center_dev = ctx->scalar;   // scalar[0..2]
    unsigned int *bad = ctx->red_counter + 1;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "memset");
    bbox_center_kernel<<<1, kBoxThreads, 0, ctx->stream>>>(c_dev, ctx->N, center_dev);
    PB_LAUNCHED();
    int blocks = (int)((ctx->N + 255) / 256);
    if (blocks > 8 * ctx->num_sms) blocks = 8 * ctx->num_sms;
    pack_kernel<<<blocks, 256, 0, ctx->stream>>>(c_dev, n_dev, a_dev, ctx->N, center_dev, ctx->g64, ctx->pos32,
                                                 ctx->nrm32, bad);
    PB_LAUNCHED();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "geometry kernels");
    unsigned int nbad = 0;
    e = cudaMemcpyAsync(ctx->host_scalar, center_dev, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctx->host_scalar[3], bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "geometry readback");
    for (int d = 0; d < 3; ++d) ctx->center[d] = ctx->host_scalar[d];
    memcpy(&nbad, &ctx->host_scalar[3], sizeof(unsigned int));
    if (nbad != 0)
        return set_error(ctx, PB_ERR_BADMESH,
                         "pb_create: %u of %lld elements have a non-positive or non-finite area, a non-finite "
                         "centroid, or a normal more than 1e-3 away from unit length",
                         nbad, (long long)ctx->N);
    return PB_OK;
}

pb_status charges_prepare(pb_ctx *ctx, const double *q_dev, int64_t nc) {
    if (nc > 0) {
        int blocks = (int)((nc + 255) / 256);
        if (blocks > 4 * ctx->num_sms) blocks = 4 * ctx->num_sms;
        shift_charges_kernel<<<blocks, 256, 0, ctx->stream>>>(q_dev, nc, ctx->center[0], ctx->center[1],
                                                              ctx->center[2], ctx->charges);
        PB_LAUNCHED();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(ctx, e, "charges kernel");
    }
    ctx->Nc = nc;
    return PB_OK;
}

pb_status gauss_check(pb_ctx *ctx, double *gmin, double *gmax) {
    *gmin = 0.0;
    *gmax = 0.0;
    if (ctx->Nc == 0) return PB_OK;
    double *out = nullptr;
    pb_status s = ctx_alloc(ctx, (void **)&out, ctx->Nc * sizeof(double), "gauss sums");
    if (s != PB_OK) return s;
    int blocks = (int)(ctx->Nc < 65535 ? ctx->Nc : 65535);
    gauss_kernel<<<blocks, kGaussThreads, 0, ctx->stream>>>(ctx->pos32, ctx->nrm32, ctx->N, ctx->charges, ctx->Nc, out);
    PB_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    double *h = nullptr;
    if (e == cudaSuccess) e = pinned_alloc((void **)&h, ctx->Nc * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, ctx->Nc * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        pinned_free(h, ctx->Nc * sizeof(double));
        ctx_free(ctx, out);
        return cuda_error(ctx, e, "gauss check");
    }
    double lo = h[0], hi = h[0];
    for (int64_t k = 1; k < ctx->Nc; ++k) { lo = fmin(lo, h[k]); hi = fmax(hi, h[k]); }
    pinned_free(h, ctx->Nc * sizeof(double));
    ctx_free(ctx, out);
    *gmin = lo;
    *gmax = hi;
    return PB_OK;
}

}  // namespace pb
