// matvec_static.cu -- pb_matvec_f32_static: the FP32-pair matrix-vector product
// without any device allocation.
//
// Some callers cannot call cudaMalloc: for example code running under a
// framework whose caching allocator already owns all of the device memory, or
// code on a latency-critical path where an allocation (which may synchronise
// the device) is not acceptable.  They cannot create a pb_ctx, because
// pb_create allocates the geometry copies and the matvec scratch.  This entry
// point takes the caller's own device arrays instead and keeps the kernel's
// scratch (per-target-tile arrival counters and per-CTA partial rows) in one
// file-scope static device array of fixed size, kStaticScratchBytes (16 MiB).
// Every GPU that loads the library holds that array until the process exits.
// All calls share it: calls that overlap on the GPU (for example on two
// streams, or from two host threads) race on it and must be avoided.
//
// The arithmetic is the same as matvec_f32_kernel in matvec.cu (Eqs. (12)-(13),
// FP32 pairs with hardware rsqrt/exp2, FP32 partials per 256-source tile, FP64
// row sums, deterministic last-arriver reduction); only the input layout
// (FP64 arrays, converted while staging) and the home of the scratch differ.
#include <math.h>
#include <stdint.h>
#include <mutex>

#include "fastmath.cuh"
#include "pb_internal.cuh"

namespace pb {
namespace {

// 16 MiB: the arrival counters (one uint32 per 512-target tile, 256-byte
// aligned) followed by two partial slots per CTA (the CTA's first and last
// target tile; each slot holds the two rows of 512 doubles).  Partials are
// indexed by CTA here, not by (tile, segment) as in matvec.cu, so the scratch
// size depends on the grid, not on N.
constexpr size_t kStaticScratchBytes = size_t(16) << 20;
constexpr int64_t kStaticMaxN = int64_t(1) << 24;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
// Per-device launch shape, filled by the first call on a device.  The scratch
// address is not cached: it is resolved on every call, so that a module
// reloaded after cudaDeviceReset (which may place the array elsewhere) is
// still addressed correctly.
struct DeviceSetup {
    bool ready = false;
    int num_sms = 0;
    int occupancy = 0;
};
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

constexpr int BS = kF32Threads, T = kF32TargetsPerThread, TT = kF32TargetTile, TS = kF32SourceTile;

struct StaticParams {
    float eps, inv_eps, kappa, neg_kappa_log2e;
    double diag1, diag2;
    double cx, cy, cz;           // shift subtracted before the FP32 cast
};

__global__ void __launch_bounds__(BS)
matvec_f32_static_kernel(const double *__restrict__ c, const double *__restrict__ nrm,
                         const double *__restrict__ area, const double *__restrict__ u, int64_t N,
                         StaticParams prm, StreamKPlan plan, double *__restrict__ partials,
                         unsigned int *__restrict__ counters, double *__restrict__ y) {
    __shared__ float4 s_pos[TS];   // x, y, z, W dphi / (4 pi)
    __shared__ float4 s_nrm[TS];   // nx, ny, nz, W phi / (4 pi)
    __shared__ int s_last;
    const int tid = threadIdx.x;
    const int64_t cta = blockIdx.x;
    const int64_t S = plan.source_tiles;
    int64_t p = sk_begin(cta, plan.work, plan.ctas);
    const int64_t pend = sk_begin(cta + 1, plan.work, plan.ctas);

    while (p < pend) {
        const int64_t a = p / S;
        const int64_t s_first = p % S;
        const int64_t s_end = (S < s_first + (pend - p)) ? S : s_first + (pend - p);

        float xi[T], yi[T], zi[T], nxi[T], nyi[T], nzi[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            int64_t i = a * TT + t * BS + tid;
            if (i > N - 1) i = N - 1;
            xi[t] = (float)(c[3 * i] - prm.cx);
            yi[t] = (float)(c[3 * i + 1] - prm.cy);
            zi[t] = (float)(c[3 * i + 2] - prm.cz);
            nxi[t] = (float)nrm[3 * i];
            nyi[t] = (float)nrm[3 * i + 1];
            nzi[t] = (float)nrm[3 * i + 2];
        }
        double acc1[T], acc2[T];
#pragma unroll
        for (int t = 0; t < T; ++t) { acc1[t] = 0.0; acc2[t] = 0.0; }

        for (int64_t s = s_first; s < s_end; ++s) {
            __syncthreads();
            for (int jl = tid; jl < TS; jl += BS) {
                int64_t j = s * TS + jl;
                if (j < N) {
                    const float w = (float)(area[j] * kInv4Pi);
                    s_pos[jl] = make_float4((float)(c[3 * j] - prm.cx), (float)(c[3 * j + 1] - prm.cy),
                                            (float)(c[3 * j + 2] - prm.cz), (float)u[N + j] * w);
                    s_nrm[jl] = make_float4((float)nrm[3 * j], (float)nrm[3 * j + 1], (float)nrm[3 * j + 2],
                                            (float)u[j] * w);
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
                    inv = (r2 > 0.f) ? inv : 0.f;
                    const float rho = r2 * inv;
                    const float e = exp2_approx(prm.neg_kappa_log2e * rho);
                    const float kr = prm.kappa * rho;
                    const float e1 = fmaf(e, kr, e);
                    const float inv2 = inv * inv;
                    const float inv3 = inv2 * inv;
                    const float cxv = fmaf(dx, nxi[t], fmaf(dy, nyi[t], dz * nzi[t]));
                    const float cyv = fmaf(dx, sn.x, fmaf(dy, sn.y, dz * sn.z));
                    const float nn = fmaf(nxi[t], sn.x, fmaf(nyi[t], sn.y, nzi[t] * sn.z));
                    const float k1 = (1.f - e) * inv;
                    const float k2 = fmaf(prm.eps, e1, -1.f) * cyv * inv3;
                    const float k3 = fmaf(e1, prm.inv_eps, -1.f) * cxv * inv3;
                    const float p3 = fmaf(kr, kr + 3.f, 3.f);
                    const float e3 = fmaf(e, p3, -3.f);
                    const float k4 = fmaf(-e3 * cxv * cyv, inv2, fmaf(e1, nn, -nn)) * inv3;
                    f1[t] = fmaf(k1, sp.w, fmaf(k2, sn.w, f1[t]));
                    f2[t] = fmaf(k3, sp.w, fmaf(k4, sn.w, f2[t]));
                }
            }
#pragma unroll
            for (int t = 0; t < T; ++t) { acc1[t] += (double)f1[t]; acc2[t] += (double)f2[t]; }
        }

        // finish the segment (one CTA: write y; several: last arriver reduces)
        const int64_t c0 = sk_cta_of(a * S, plan.work, plan.ctas);
        const int64_t c1 = sk_cta_of(a * S + S - 1, plan.work, plan.ctas);
        const int nseg = (int)(c1 - c0 + 1);
        if (nseg == 1) {
#pragma unroll
            for (int t = 0; t < T; ++t) {
                int64_t i = a * TT + t * BS + tid;
                if (i < N) {
                    y[i] = prm.diag1 * u[i] - acc1[t];
                    y[N + i] = prm.diag2 * u[N + i] - acc2[t];
                }
            }
        } else {
            // slot 2c holds CTA c's first target tile, slot 2c+1 its last one
            const int64_t a_first = sk_begin(cta, plan.work, plan.ctas) / S;
            double *mine = partials + (2 * cta + (a == a_first ? 0 : 1)) * 2 * TT;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                mine[t * BS + tid] = acc1[t];
                mine[TT + t * BS + tid] = acc2[t];
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) s_last = (atomicAdd(&counters[a], 1u) == (unsigned int)(nseg - 1));
            __syncthreads();
            if (s_last) {
                __threadfence();
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    int64_t i = a * TT + t * BS + tid;
                    double s1 = 0.0, s2 = 0.0;
                    for (int o = 0; o < nseg; ++o) {
                        const int64_t co = c0 + o;
                        const int64_t co_first = sk_begin(co, plan.work, plan.ctas) / S;
                        const double *pp = partials + (2 * co + (a == co_first ? 0 : 1)) * 2 * TT;
                        s1 += __ldcg(pp + t * BS + tid);
                        s2 += __ldcg(pp + TT + t * BS + tid);
                    }
                    if (i < N) {
                        y[i] = prm.diag1 * u[i] - s1;
                        y[N + i] = prm.diag2 * u[N + i] - s2;
                    }
                }
                if (tid == 0) counters[a] = 0u;
            }
        }
        p += s_end - s_first;
    }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// true when the byte ranges [a, a + na) and [b, b + nb) intersect
bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb) {
    const uintptr_t pa = (uintptr_t)a, pb_ = (uintptr_t)b;
    return pa < pb_ + nb && pb_ < pa + na;
}

}  // namespace
}  // namespace pb

using namespace pb;

extern "C" pb_status pb_matvec_f32_static(const double *centroids, const double *normals, const double *areas,
                                          int64_t N, const double *center, double eps1, double eps2, double kappa,
                                          const double *u, double *y, void *cuda_stream) {
    if (!centroids || !normals || !areas || !u || !y)
        return set_error(nullptr, PB_ERR_ARG, "pb_matvec_f32_static: NULL pointer argument");
    if (N < 1) return set_error(nullptr, PB_ERR_ARG, "pb_matvec_f32_static: N must be >= 1");
    if (!(eps1 > 0.0) || !(eps2 > 0.0) || !isfinite(eps1) || !isfinite(eps2) || !(kappa >= 0.0) || !isfinite(kappa))
        return set_error(nullptr, PB_ERR_ARG, "pb_matvec_f32_static: need eps1 > 0, eps2 > 0, kappa >= 0 (finite)");
    if (N > kStaticMaxN)
        return set_error(nullptr, PB_ERR_ARG,
                         "pb_matvec_f32_static: N = %lld exceeds the maximum %lld of the fixed static scratch",
                         (long long)N, (long long)kStaticMaxN);
    {
        // y is written while other CTAs still read u and the geometry
        const size_t n = (size_t)N * sizeof(double);
        if (ranges_overlap(y, 2 * n, u, 2 * n) || ranges_overlap(y, 2 * n, centroids, 3 * n) ||
            ranges_overlap(y, 2 * n, normals, 3 * n) || ranges_overlap(y, 2 * n, areas, n))
            return set_error(nullptr, PB_ERR_ARG,
                             "pb_matvec_f32_static: y must not overlap u, centroids, normals or areas");
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(nullptr, e, "pb_matvec_f32_static: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(nullptr, PB_ERR_ARG, "pb_matvec_f32_static: device ordinal %d out of range", dev);
    DeviceSetup su;
    {
        // once per device, with that device current: size the persistent grid
        std::lock_guard<std::mutex> lock(g_setup_mu);
        DeviceSetup &g = g_setup[dev];
        if (!g.ready) {
            e = cudaDeviceGetAttribute(&g.num_sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return cuda_error(nullptr, e, "pb_matvec_f32_static: device query");
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.occupancy, matvec_f32_static_kernel, BS, 0);
            if (e != cudaSuccess) return cuda_error(nullptr, e, "pb_matvec_f32_static: occupancy query");
            if (g.occupancy < 1) g.occupancy = 1;
            g.ready = true;
        }
        su = g;
    }
    // the device address of the static scratch array on the current device
    // (host code must not use the symbol itself as a pointer); resolved on
    // every call, which allocates nothing
    unsigned char *scratch = nullptr;
    e = cudaGetSymbolAddress((void **)&scratch, g_static_scratch);
    if (e != cudaSuccess) return cuda_error(nullptr, e, "pb_matvec_f32_static: cudaGetSymbolAddress");

    // Persistent grid as for pb_matvec, capped so that two partial slots per
    // CTA fit in the static array after the counters.
    const int64_t target_tiles = (N + TT - 1) / TT;
    const size_t counter_bytes = align256((size_t)target_tiles * sizeof(unsigned int));
    const size_t slot_bytes = 2 * (size_t)TT * sizeof(double);
    const int64_t max_ctas = (int64_t)((kStaticScratchBytes - counter_bytes) / (2 * slot_bytes));
    int64_t ctas = (int64_t)su.num_sms * su.occupancy;
    if (ctas > max_ctas) ctas = max_ctas;
    const StreamKPlan plan = make_plan(N, TT, TS, ctas);

    cudaStream_t stream = (cudaStream_t)cuda_stream;
    unsigned int *counters = (unsigned int *)scratch;
    double *partials = (double *)(scratch + counter_bytes);
    // the counters must start at zero; the array keeps the last call's contents
    e = cudaMemsetAsync(counters, 0, (size_t)target_tiles * sizeof(unsigned int), stream);
    if (e != cudaSuccess) return cuda_error(nullptr, e, "pb_matvec_f32_static: clearing counters");

    StaticParams prm;
    const double eps = eps2 / eps1;
    prm.eps = (float)eps;
    prm.inv_eps = (float)(1.0 / eps);
    prm.kappa = (float)kappa;
    prm.neg_kappa_log2e = (float)(-kappa * 1.4426950408889634);
    prm.diag1 = 0.5 * (1.0 + eps);
    prm.diag2 = 0.5 * (1.0 + 1.0 / eps);
    prm.cx = center ? center[0] : 0.0;
    prm.cy = center ? center[1] : 0.0;
    prm.cz = center ? center[2] : 0.0;
    matvec_f32_static_kernel<<<(unsigned)plan.ctas, BS, 0, stream>>>(centroids, normals, areas, u, N, prm, plan,
                                                                      partials, counters, y);
    PB_LAUNCHED();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(nullptr, e, "pb_matvec_f32_static: launch");
    return PB_OK;
}
