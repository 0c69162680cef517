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

#include <type_traits>

#include "fastmath.cuh"
#include "finish.cuh"
#include "pb_internal.cuh"
#include "sym.cuh"

namespace pb {

StreamKPlan make_plan(int64_t n, int target_tile, int source_tile, int64_t ctas_wanted) {
    return make_plan_rows(n, n, target_tile, source_tile, ctas_wanted);
}

StreamKPlan make_plan_rows(int64_t n_targets, int64_t n_sources, int target_tile, int source_tile,
                           int64_t ctas_wanted) {
    StreamKPlan p;
    p.target_tiles = (n_targets + target_tile - 1) / target_tile;
    p.source_tiles = (n_sources + source_tile - 1) / source_tile;
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

SymPlan make_sym_plan(int64_t n, int tile, int64_t ctas_wanted) {
    SymPlan p;
    p.tiles = (n + tile - 1) / tile;
    p.work = p.tiles * (p.tiles + 1) / 2;
    p.ctas = ctas_wanted < 1 ? 1 : (ctas_wanted > p.work ? p.work : ctas_wanted);
    return p;
}

int64_t sym64_scratch_bytes(const SymPlan &pl, int tile) {
    return sym_layout(pl, tile, (int)sizeof(double), pl.work - pl.tiles, false).bytes;
}

int64_t sym_scratch_bytes(const SymPlan &pl, int tile) {
    return sym_layout(pl, tile, (int)sizeof(float), pl.work - pl.tiles, false).bytes;
}

int64_t sym_scratch_need(const SymPlan &pl, int tile, int elem, int64_t limit, int bands,
                         std::vector<int64_t> *cuts) {
    sym_band_cuts(pl, tile, elem, limit, bands, cuts);
    const bool banded = cuts->size() > 2;
    return sym_layout(pl, tile, elem, banded ? sym_max_band_slots(pl.tiles, *cuts) : pl.work - pl.tiles, banded)
        .bytes;
}

namespace {

struct F32Params {
    float eps, inv_eps, kappa, neg_kappa_log2e;
    double diag1, diag2;
};

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
        finish_segment<TT, T, BS>(plan, a, c, acc1, acc2, u, N, RowBlock{0, N, N}, prm.diag1, prm.diag2, partials,
                                  counters, y);
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
// distance) is removed by clamping r^2 from below at 1e-18 before the MUFU
// rsqrt and rcp (so 1/rho <= 1e9, 1/rho^2 <= 1e18): rho = r2 * (1/rho) with
// the unclamped r2 is exactly 0, exp2(0) is exactly 1, c_x = c_y = 0, and
// every term of K1..K4 is an exact zero.  The weights times 1/rho^3 <= 1e27
// stay finite for |W u| < 3e11, so no infinity is formed.  Real pairs have
// rho > 1e-9 A, where the clamp does nothing.
//
// Per pair and kappa > 0 the FP32 pipe does 39 operations: r (3), rho^2 (3),
// rho (1), the exp2 argument (1), kappa rho (1), e (1 + kappa rho) (1),
// 1/rho^3 (1), c_x c_y n (9), the weights folded with 1/rho and 1/rho^3 (3),
// K1 (2), K2 (3), K3 (3), K4 (5), 3 + 3 kappa rho + (kappa rho)^2 and e times
// it (3); 1/rho^2 comes from the MUFU reciprocal.  With kappa = 0, e = 1 makes
// K1 = K4 = 0 and K2, K3 reduce to (eps - 1) c_y / rho^3 and (1/eps - 1)
// c_x / rho^3 (the constants folded into the staged weights): 18 operations
// (r 3, rho^2 3, 1/rho^2 and 1/rho^3 2, c_x c_y 6, weights 2, sums 2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// r^2 is clamped from below before the MUFU rsqrt / rcp (the symmetric kernel
// adds it, one packed add instead of two max, the same for any r^2 of a
// mesh), so 1/rho <= 1e9 and 1/rho^2 <= 1e18; rho = r^2 (1/rho) takes the
// unclamped r^2 and is exactly 0 for a pair at zero distance.
constexpr float kRho2Min = 1e-18f;

template <int T, bool K0>
__global__ void __launch_bounds__(kF32Threads)
matvec_f32x2_kernel(const float4 *__restrict__ pos, const float4 *__restrict__ nrm,
                    const double *__restrict__ u, int64_t N, RowBlock rb, F32Params prm, StreamKPlan plan,
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
    // kappa = 0: the constant factors of K2 and K3, folded into the weights
    const float wphi_scale = K0 ? prm.eps - 1.f : 1.f, wpsi_scale = K0 ? prm.inv_eps - 1.f : 1.f;

    while (p < pend) {
        const int64_t a = p / S;
        const int64_t s_first = p % S;
        const int64_t s_end = (S < s_first + (pend - p)) ? S : s_first + (pend - p);

        float2 xi[T], yi[T], zi[T], nxi[T], nyi[T], nzi[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            int64_t i = a * TT + t * BS + tid;
            if (i > rb.nrows - 1) i = rb.nrows - 1;
            const float4 q = pos[rb.row0 + i], n = nrm[rb.row0 + i];
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
                    s_d[tid] = make_float4((float)u[N + j0] * (w0 * wpsi_scale), (float)u[N + j1] * (w1 * wpsi_scale),
                                           (float)u[j0] * (w0 * wphi_scale), (float)u[j1] * (w1 * wphi_scale));
                }
            }
            __syncthreads();
            const int64_t rem = N - s * TS;
            const int npairs = (int)(((rem < TS) ? rem : TS) + 1) / 2;
            float2 f1[T], f2[T];
#pragma unroll
            for (int t = 0; t < T; ++t) { f1[t] = p_dup(0.f); f2[t] = p_dup(0.f); }
#pragma unroll 4
            for (int q = 0; q < npairs; ++q) {
                const float4 A = s_a[q], B = s_b[q], C = s_c[q], D = s_d[q];
                const float2 mx = make_float2(A.x, A.y), my = make_float2(A.z, A.w), mz = make_float2(B.x, B.y);
                const float2 snx = make_float2(B.z, B.w), sny = make_float2(C.x, C.y), snz = make_float2(C.z, C.w);
                const float2 wpsi = make_float2(D.x, D.y), wphi = make_float2(D.z, D.w);
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const float2 dx = p_add(xi[t], mx), dy = p_add(yi[t], my), dz = p_add(zi[t], mz);
                    const float2 r2 = p_fma(dx, dx, p_fma(dy, dy, p_mul(dz, dz)));
                    float2 inv, inv2;
                    const float r2cx = fmaxf(r2.x, kRho2Min), r2cy = fmaxf(r2.y, kRho2Min);
                    inv.x = rsqrt_approx(r2cx);
                    inv.y = rsqrt_approx(r2cy);
                    if (K0) {
                        inv2 = p_mul(inv, inv);                // MUFU is busier than the FP32 pipe here
                    } else {
                        inv2.x = rcp_approx(r2cx);
                        inv2.y = rcp_approx(r2cy);
                    }
                    const float2 inv3 = p_mul(inv2, inv);
                    const float2 cx = p_fma(dx, nxi[t], p_fma(dy, nyi[t], p_mul(dz, nzi[t])));
                    const float2 cy = p_fma(dx, snx, p_fma(dy, sny, p_mul(dz, snz)));
                    const float2 wa = p_mul(inv3, wphi);       // W phi / rho^3
                    const float2 wb = p_mul(inv3, wpsi);       // W dphi / rho^3
                    if (K0) {
                        f1[t] = p_fma(cy, wa, f1[t]);          // (eps - 1) c_y / rho^3, constant in wphi
                        f2[t] = p_fma(cx, wb, f2[t]);          // (1/eps - 1) c_x / rho^3, constant in wpsi
                    } else {
                        const float2 rho = p_mul(r2, inv);
                        const float2 arg = p_mul(nk2, rho);
                        float2 e;
                        e.x = exp2_approx(arg.x);
                        e.y = exp2_approx(arg.y);
                        const float2 kr = p_mul(kap2, rho);
                        const float2 e1 = p_fma(e, kr, e);                    // e (1 + kappa rho)
                        const float2 nn = p_fma(nxi[t], snx, p_fma(nyi[t], sny, p_mul(nzi[t], snz)));
                        const float2 wc = p_mul(inv, wpsi);                   // W dphi / rho
                        f1[t] = p_fma(p_fma(e, mone2, one2), wc, f1[t]);     // K1
                        f1[t] = p_fma(p_mul(p_fma(eps2, e1, mone2), cy), wa, f1[t]);     // K2
                        f2[t] = p_fma(p_mul(p_fma(e1, ieps2, mone2), cx), wb, f2[t]);    // K3
                        const float2 p3 = p_fma(kr, p_add(kr, three2), three2);   // 3 + 3 kr + kr^2
                        const float2 e3 = p_fma(e, p3, mthree2);
                        const float2 ccy = p_mul(p_mul(e3, cx), cy);
                        f2[t] = p_fma(p_fma(p_neg(ccy), inv2, p_fma(e1, nn, p_neg(nn))), wa, f2[t]);   // K4
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < T; ++t) {
                acc1[t] += (double)f1[t].x + (double)f1[t].y;
                acc2[t] += (double)f2[t].x + (double)f2[t].y;
            }
        }
        finish_segment<TT, T, BS>(plan, a, c, acc1, acc2, u, N, rb, prm.diag1, prm.diag2, partials, counters, y);
        p += s_end - s_first;
    }
}

// ---------------------------------------------------------------------------
// Symmetric evaluation.  K1 and K4 do not change when the two points (with
// their normals) are exchanged, and the K2 / K3 of the reversed pair are the
// same scalars times -c_x and -c_y.  With r = x_i - x_j,
//   row i (source j): K1 dphi_j + a c_y phi_j,   b c_x dphi_j + K4 phi_j
//   row j (source i): K1 dphi_i - a c_x phi_i,  -b c_y dphi_i + K4 phi_i
// where a = (eps e (1 + kappa rho) - 1)/rho^3, b = (e (1 + kappa rho)/eps - 1)/rho^3,
// so one evaluation of the unordered pair serves both rows.
//
// The targets are cut into square tiles of B = 128 T points and the upper
// triangle of tile pairs (I <= J) is split evenly over persistent CTAs.  A
// diagonal pair (I, I) is evaluated plainly (every ordered pair, row side
// only).  For I < J the row-i side accumulates in registers across the J of
// a CTA's run, as in the plain kernel; the row-j ("column") side is summed
// over the thread's targets, then over the warp with a reduce-scatter (6
// shuffles per source pair), then over the 4 warps in shared memory, and
// stored per tile pair in FP32.  A second kernel adds, for every row, its row
// side and the column sides of all tile pairs above it in a fixed order:
// deterministic, no floating-point atomics.
//
// Signs are arranged so that no operand needs negating: the target normals
// are negated when loaded (c_x and n change sign), 1 - e (1 + kappa rho) is
// formed instead of e (1 + kappa rho) - 1, and b enters negated.  Per
// unordered pair and kappa > 0 the FP32 pipe does 46 operations (r 3,
// rho^2 3, 1/rho^3 1, c_x c_y n 9, rho, the exp2 argument and -kappa rho 3,
// 1 - e and 1 - e (1 + kappa rho) 2, K1 1, a 2, -b 2, K4 8, row side 6,
// column side 6): 23 per ordered pair against 39.  With kappa = 0 it is 20
// (r 3, rho^2 3, 1/rho^2 and 1/rho^3 2, c_x c_y 6, c/rho^3 2, four sums),
// the constants (eps - 1) and (1 - 1/eps) folded into the weights.
// ---------------------------------------------------------------------------
struct SymConsts {
    float2 nk2, mkap2, one2, mone2, mthree2, three2, meps2, epsm1, ieps2, omieps, rho2min;
};

// The warp reduce-scatter of four values (lanes 0-7 end with the total of the
// first, 8-15 of the second, 16-23 of the third, 24-31 of the fourth), cut
// into steps so that its shuffles can be interleaved with independent work:
// begin() exchanges halves across lanes 16 apart, step(1..4) finishes the
// previous exchange and starts the next (8, 4, 2, 1 lanes apart), end()
// adds the last one.  6 shuffles in all.
struct WarpReduce4 {
    float2 keep, recv;
    float k, o;
    __device__ __forceinline__ void begin(float2 g1, float2 g2, bool hi16) {
        keep = hi16 ? g2 : g1;
        const float2 send = hi16 ? g1 : g2;
        recv.x = __shfl_xor_sync(0xffffffffu, send.x, 16);
        recv.y = __shfl_xor_sync(0xffffffffu, send.y, 16);
    }
    __device__ __forceinline__ void step(int st, bool hi8) {
        if (st == 1) {
            keep = p_add(keep, recv);
            k = hi8 ? keep.y : keep.x;
            o = __shfl_xor_sync(0xffffffffu, hi8 ? keep.x : keep.y, 8);
        } else {
            k += o;
            o = __shfl_xor_sync(0xffffffffu, k, st == 2 ? 4 : (st == 3 ? 2 : 1));
        }
    }
    __device__ __forceinline__ float end() { return k + o; }
};

// One staged source tile against the thread's T targets: the row sides into
// f1, f2 and, with COL, the column sides of each source pair reduced over the
// warp into col (lanes 0-7: f1 side of the pair's first source, 8-15 of its
// second, 16-23 and 24-31: f2 side; col[k] and col[B + k] for source k of the
// tile).  The reduction of pair q runs during the arithmetic of pair q + 1,
// one shuffle step after each target, so that its latency is hidden.
template <int T, bool K0, bool COL>
__device__ __forceinline__ void sym_stage(const float4 *s_a, const float4 *s_b, const float4 *s_c,
                                          const float4 *s_d, int npairs, const float2 (&xi)[T],
                                          const float2 (&yi)[T], const float2 (&zi)[T], const float2 (&nxi)[T],
                                          const float2 (&nyi)[T], const float2 (&nzi)[T], const float2 (&wpi)[T],
                                          const float2 (&wfi)[T], float2 (&f1)[T], float2 (&f2)[T], float *col,
                                          const SymConsts &k) {
    constexpr int B = kF32Threads * T;
    const int lane = threadIdx.x & 31;
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    // this lane's slot for a reduced pair q: col[cbase + 2 q]
    const int cbase = (lane >> 4) * B + ((lane >> 3) & 1);
    const bool writer = (lane & 7) == 0;
    WarpReduce4 red;
    // source pairs unrolled 8-fold (measured: 1204 -> 1298 Gpairs/s from 1 to 8, 1004 at
    // 16), 16-fold for the shorter kappa = 0 body (+0.9 % over 8)
    constexpr int kUnr = K0 ? 16 : 8;
#pragma unroll kUnr
    for (int q = 0; q < npairs; ++q) {
        const float4 A = s_a[q], Bq = s_b[q], C = s_c[q], D = s_d[q];
        const float2 mx = make_float2(A.x, A.y), my = make_float2(A.z, A.w), mz = make_float2(Bq.x, Bq.y);
        const float2 snx = make_float2(Bq.z, Bq.w), sny = make_float2(C.x, C.y), snz = make_float2(C.z, C.w);
        const float2 wpsi = make_float2(D.x, D.y), wphi = make_float2(D.z, D.w);
        float2 g1 = p_dup(0.f), g2 = p_dup(0.f);     // column sides of the two sources
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float2 dx = p_add(xi[t], mx), dy = p_add(yi[t], my), dz = p_add(zi[t], mz);
            const float2 r2 = p_fma(dx, dx, p_fma(dy, dy, p_mul(dz, dz)));
            float2 inv, inv2;
            // r^2 + 1e-18: the same as the floor for any r^2 above 2e-11 and for r^2 = 0
            const float2 r2c = p_add(r2, k.rho2min);
            inv.x = rsqrt_approx(r2c.x);
            inv.y = rsqrt_approx(r2c.y);
            if (K0) {
                inv2 = p_mul(inv, inv);
            } else {
                inv2.x = rcp_approx(r2c.x);
                inv2.y = rcp_approx(r2c.y);
            }
            const float2 inv3 = p_mul(inv2, inv);
            const float2 ncx = p_fma(dx, nxi[t], p_fma(dy, nyi[t], p_mul(dz, nzi[t])));   // -c_x
            const float2 cy = p_fma(dx, snx, p_fma(dy, sny, p_mul(dz, snz)));
            if (K0) {
                const float2 ay = p_mul(cy, inv3), bx = p_mul(ncx, inv3);
                f1[t] = p_fma(ay, wphi, f1[t]);
                f2[t] = p_fma(bx, wpsi, f2[t]);
                if (COL) {
                    g1 = p_fma(bx, wfi[t], g1);
                    g2 = p_fma(ay, wpi[t], g2);
                }
            } else {
                const float2 rho = p_mul(r2, inv);
                float2 e;
                const float2 arg = p_mul(k.nk2, rho);
                e.x = exp2_approx(arg.x);
                e.y = exp2_approx(arg.y);
                const float2 mkr = p_mul(k.mkap2, rho);                             // -kappa rho
                const float2 nnn = p_fma(nxi[t], snx, p_fma(nyi[t], sny, p_mul(nzi[t], snz)));   // -n
                const float2 ome = p_fma(e, k.mone2, k.one2);                       // 1 - e
                const float2 ome1 = p_fma(e, mkr, ome);                             // 1 - e (1 + kappa rho)
                const float2 k1 = p_mul(ome, inv);
                const float2 al = p_mul(p_fma(ome1, k.meps2, k.epsm1), inv3);       // a
                const float2 nb = p_mul(p_fma(ome1, k.ieps2, k.omieps), inv3);      // -b
                const float2 p3 = p_fma(mkr, p_add(mkr, k.mthree2), k.three2);      // 3 + 3 kappa rho + (kappa rho)^2
                const float2 e3 = p_fma(e, p3, k.mthree2);
                const float2 ccy = p_mul(p_mul(e3, ncx), cy);                       // -e3 c_x c_y
                const float2 k4 = p_mul(p_fma(ccy, inv2, p_mul(ome1, nnn)), inv3);
                f1[t] = p_fma(k1, wpsi, p_fma(p_mul(al, cy), wphi, f1[t]));
                f2[t] = p_fma(p_mul(nb, ncx), wpsi, p_fma(k4, wphi, f2[t]));
                if (COL) {
                    g1 = p_fma(k1, wpi[t], p_fma(p_mul(al, ncx), wfi[t], g1));
                    g2 = p_fma(p_mul(nb, cy), wpi[t], p_fma(k4, wfi[t], g2));
                }
            }
            // one step of the previous pair's reduction per target (T >= 2)
            if (COL && q > 0) {
                if (T == 2) {
                    if (t == 0) { red.step(1, hi8); red.step(2, hi8); }
                    else { red.step(3, hi8); red.step(4, hi8); }
                } else if (t < 4) {
                    red.step(t + 1, hi8);
                }
            }
        }
        if (COL) {
            if (q > 0) {
                const float tot = red.end();
                if (writer) col[cbase + 2 * (q - 1)] = tot;
            }
            red.begin(g1, g2, hi16);
        }
    }
    if (COL && npairs > 0) {
        red.step(1, hi8);
        red.step(2, hi8);
        red.step(3, hi8);
        red.step(4, hi8);
        const float tot = red.end();
        if (writer) col[cbase + 2 * (npairs - 1)] = tot;
    }
}

template <int T, bool K0, int MINB>
__global__ void __launch_bounds__(kF32Threads, MINB)
matvec_sym_kernel(const float4 *__restrict__ pos, const float4 *__restrict__ nrm, const double *__restrict__ u,
                  int64_t N, F32Params prm, SymPlan plan, double *__restrict__ islots, double *__restrict__ iside,
                  float *__restrict__ jpart, const int *__restrict__ skip, unsigned long long *__restrict__ evaluated) {
    constexpr int BS = kF32Threads, B = BS * T, TS = kF32SourceTile, TQ = TS / 2, NW = BS / 32;
    constexpr int STAGES = B / TS;
    static_assert(TQ == BS && B % TS == 0, "tile shapes");
    if (skip != nullptr && *((volatile const int *)skip)) return;
    if (evaluated != nullptr && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(evaluated, 1ull);
    __shared__ float4 s_a[TQ], s_b[TQ], s_c[TQ], s_d[TQ];
    __shared__ float s_col[NW][2][B];     // per-warp column sides of the current tile pair

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t c = blockIdx.x;
    const int64_t Tt = plan.tiles;
    // tile pairs [work_begin, work_begin + work) (a band of whole rows, or all of them)
    const int64_t wb = plan.work_begin;
    int64_t p = wb + sk_begin(c, plan.work, plan.ctas);
    const int64_t pend = wb + sk_begin(c + 1, plan.work, plan.ctas);
    const int64_t I_first = sym_row_of(p, Tt);
    SymConsts c3;
    c3.nk2 = p_dup(prm.neg_kappa_log2e);
    c3.mkap2 = p_dup(-prm.kappa);
    c3.one2 = p_dup(1.f);
    c3.mone2 = p_dup(-1.f);
    c3.mthree2 = p_dup(-3.f);
    c3.three2 = p_dup(3.f);
    c3.meps2 = p_dup(-prm.eps);
    c3.epsm1 = p_dup(prm.eps - 1.f);
    c3.ieps2 = p_dup(prm.inv_eps);
    c3.omieps = p_dup(1.f - prm.inv_eps);
    c3.rho2min = p_dup(kRho2Min);
    // kappa = 0: a = (eps - 1)/rho^3 and -b = (1 - 1/eps)/rho^3, constants folded into the weights
    const float wphi_scale = K0 ? prm.eps - 1.f : 1.f, wpsi_scale = K0 ? 1.f - prm.inv_eps : 1.f;

    while (p < pend) {
        const int64_t I = sym_row_of(p, Tt);
        const int64_t row_end = sym_row_start(I + 1, Tt);
        const int64_t p_stop = pend < row_end ? pend : row_end;
        // row tile targets: position, negated normal, weights of their own u (column side)
        float2 xi[T], yi[T], zi[T], nxi[T], nyi[T], nzi[T], wpi[T], wfi[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int64_t i0 = I * B + t * BS + tid;
            const int64_t i = i0 < N ? i0 : N - 1;
            const float4 q = pos[i], n = nrm[i];
            xi[t] = p_dup(q.x); yi[t] = p_dup(q.y); zi[t] = p_dup(q.z);
            nxi[t] = p_dup(-n.x); nyi[t] = p_dup(-n.y); nzi[t] = p_dup(-n.z);
            const float w = i0 < N ? q.w : 0.f;
            wpi[t] = p_dup((float)u[N + i] * (w * wpsi_scale));
            wfi[t] = p_dup((float)u[i] * (w * wphi_scale));
        }
        double acc1[T], acc2[T];
#pragma unroll
        for (int t = 0; t < T; ++t) { acc1[t] = 0.0; acc2[t] = 0.0; }

        for (; p < p_stop; ++p) {
            const int64_t J = I + (p - sym_row_start(I, Tt));
            const bool diag = (J == I);
            for (int stg = 0; stg < STAGES; ++stg) {
                const int64_t s0 = J * B + stg * TS;
                if (s0 >= N) break;
                __syncthreads();
                {
                    const int64_t j0 = s0 + 2 * tid;
                    if (j0 < N) {
                        const int64_t j1 = (j0 + 1 < N) ? j0 + 1 : j0;
                        const float4 p0 = pos[j0], p1 = pos[j1], n0 = nrm[j0], n1 = nrm[j1];
                        const float w0 = p0.w, w1 = (j0 + 1 < N) ? p1.w : 0.f;
                        s_a[tid] = make_float4(-p0.x, -p1.x, -p0.y, -p1.y);
                        s_b[tid] = make_float4(-p0.z, -p1.z, n0.x, n1.x);
                        s_c[tid] = make_float4(n0.y, n1.y, n0.z, n1.z);
                        s_d[tid] = make_float4((float)u[N + j0] * (w0 * wpsi_scale),
                                               (float)u[N + j1] * (w1 * wpsi_scale),
                                               (float)u[j0] * (w0 * wphi_scale), (float)u[j1] * (w1 * wphi_scale));
                    }
                }
                __syncthreads();
                const int64_t rem = N - s0;
                const int npairs = (int)(((rem < TS) ? rem : TS) + 1) / 2;
                float2 f1[T], f2[T];
#pragma unroll
                for (int t = 0; t < T; ++t) { f1[t] = p_dup(0.f); f2[t] = p_dup(0.f); }
                if (diag)
                    sym_stage<T, K0, false>(s_a, s_b, s_c, s_d, npairs, xi, yi, zi, nxi, nyi, nzi, wpi, wfi, f1, f2,
                                            nullptr, c3);
                else
                    sym_stage<T, K0, true>(s_a, s_b, s_c, s_d, npairs, xi, yi, zi, nxi, nyi, nzi, wpi, wfi, f1, f2,
                                           &s_col[warp][0][stg * TS], c3);
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    acc1[t] += (double)f1[t].x + (double)f1[t].y;
                    acc2[t] += (double)f2[t].x + (double)f2[t].y;
                }
            }
            if (!diag) {
                // column side of tile pair (I, J): sum over the warps in a fixed order
                __syncthreads();
                float *dst = jpart + (sym_offdiag_index(I, J, Tt) - plan.joff) * 2 * B;
                for (int x = tid; x < 2 * B; x += BS) {
                    const int r = x / B, k = x - r * B;
                    float v = s_col[0][r][k];
#pragma unroll
                    for (int w2 = 1; w2 < NW; ++w2) v += s_col[w2][r][k];
                    dst[x] = v;
                }
            }
        }
        // row side of row tile I over this CTA's part of the row
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

// ---------------------------------------------------------------------------
// Plain FP64 path: every pair and every sum in FP64.
// ---------------------------------------------------------------------------
struct F64Params {
    double eps, inv_eps, kappa, diag1, diag2;
};

__global__ void __launch_bounds__(kF64Threads)
matvec_f64_kernel(const double *__restrict__ g64, const double *__restrict__ u, int64_t N, RowBlock rb,
                  F64Params prm, StreamKPlan plan, double *__restrict__ partials, unsigned int *__restrict__ counters,
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
        if (i > rb.nrows - 1) i = rb.nrows - 1;
        i += rb.row0;
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
        finish_segment<TT, 1, BS>(plan, a, c, acc1, acc2, u, N, rb, prm.diag1, prm.diag2, partials, counters, y);
        p += s_end - s_first;
    }
}


// ---------------------------------------------------------------------------
// Symmetric FP64 product: the plain path's arithmetic (every pair and every
// sum in FP64, the self pair and any pair at zero distance skipped), with each
// unordered pair evaluated once for both rows as in the FP32-pair symmetric
// kernel (same tiling, plan and finishing kernel; the column sides are kept in
// FP64).  On GB300 the FP64 pipe bounds this path, so halving the pair
// evaluations halves its time.  T targets per thread, B = 128 T, sources staged
// 128 at a time; the column side of a source is reduced over the warp with a
// reduce-scatter (xor 16, then 8, 4, 2, 1).
// ---------------------------------------------------------------------------
template <int T>
__global__ void __launch_bounds__(kF64Threads)
matvec_sym64_kernel(const double *__restrict__ g64, const double *__restrict__ u, int64_t N, F64Params prm,
                    SymPlan plan, double *__restrict__ islots, double *__restrict__ iside,
                    double *__restrict__ jpart, const int *__restrict__ skip,
                    unsigned long long *__restrict__ evaluated) {
    constexpr int BS = kF64Threads, B = BS * T, TS = BS, NW = BS / 32, STAGES = B / TS;
    if (skip != nullptr && *((volatile const int *)skip)) return;
    if (evaluated != nullptr && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(evaluated, 1ull);
    __shared__ double s_x[TS], s_y[TS], s_z[TS], s_nx[TS], s_ny[TS], s_nz[TS], s_wpsi[TS], s_wphi[TS];
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
        double xi[T], yi[T], zi[T], nxi[T], nyi[T], nzi[T], wpi[T], wfi[T], acc1[T], acc2[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int64_t i0 = I * B + t * BS + tid;
            const int64_t i = i0 < N ? i0 : N - 1;
            xi[t] = X[i]; yi[t] = Y[i]; zi[t] = Z[i];
            nxi[t] = NX[i]; nyi[t] = NY[i]; nzi[t] = NZ[i];
            const double w = i0 < N ? W[i] * kInv4Pi : 0.0;
            wpi[t] = w * u[N + i];
            wfi[t] = w * u[i];
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
                        const double w = W[j] * kInv4Pi;
                        s_x[tid] = X[j]; s_y[tid] = Y[j]; s_z[tid] = Z[j];
                        s_nx[tid] = NX[j]; s_ny[tid] = NY[j]; s_nz[tid] = NZ[j];
                        s_wpsi[tid] = w * u[N + j];
                        s_wphi[tid] = w * u[j];
                    }
                }
                __syncthreads();
                const int cnt = (int)((N - s0) < TS ? (N - s0) : TS);
                for (int jj = 0; jj < cnt; ++jj) {
                    double g1 = 0.0, g2 = 0.0;       // column side of source jj
#pragma unroll
                    for (int t = 0; t < T; ++t) {
                        const double dx = xi[t] - s_x[jj], dy = yi[t] - s_y[jj], dz = zi[t] - s_z[jj];
                        const double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 > 0.0) {
                            const double inv = rsqrt(r2);
                            const double rho = r2 * inv;
                            const double kr = prm.kappa * rho;
                            const double e = exp(-kr);
                            const double e1 = e * (1.0 + kr);
                            const double inv2 = inv * inv;
                            const double inv3 = inv2 * inv;
                            const double cx = dx * nxi[t] + dy * nyi[t] + dz * nzi[t];
                            const double cy = dx * s_nx[jj] + dy * s_ny[jj] + dz * s_nz[jj];
                            const double nn = nxi[t] * s_nx[jj] + nyi[t] * s_ny[jj] + nzi[t] * s_nz[jj];
                            const double k1 = (1.0 - e) * inv;
                            const double a = (prm.eps * e1 - 1.0) * inv3;
                            const double b = (e1 * prm.inv_eps - 1.0) * inv3;
                            const double k4 =
                                ((e1 - 1.0) * nn - (e * (3.0 + 3.0 * kr + kr * kr) - 3.0) * cx * cy * inv2) * inv3;
                            acc1[t] += k1 * s_wpsi[jj] + a * cy * s_wphi[jj];
                            acc2[t] += b * cx * s_wpsi[jj] + k4 * s_wphi[jj];
                            if (!diag) {
                                g1 += k1 * wpi[t] - a * cx * wfi[t];
                                g2 += k4 * wfi[t] - b * cy * wpi[t];
                            }
                        }
                    }
                    if (!diag) {
                        // lanes 0-15 end with the warp's sum of g1, 16-31 of g2
                        double keep = hi16 ? g2 : g1;
                        keep += __shfl_xor_sync(0xffffffffu, hi16 ? g1 : g2, 16);
                        keep += __shfl_xor_sync(0xffffffffu, keep, 8);
                        keep += __shfl_xor_sync(0xffffffffu, keep, 4);
                        keep += __shfl_xor_sync(0xffffffffu, keep, 2);
                        keep += __shfl_xor_sync(0xffffffffu, keep, 1);
                        if ((lane & 15) == 0) s_col[warp][lane >> 4][stg * TS + jj] = keep;
                    }
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

}  // namespace

pb_status matvec_rows_launch(pb_ctx *ctx, const double *u, double *y, RowBlock rb, pb_precision prec,
                             const int *skip_flag) {
    if (prec != PB_FP32PAIR && prec != PB_FP64)
        return set_error(ctx, PB_ERR_ARG, "row-block product: precision %d (FP32 pairs or FP64 only)", (int)prec);
    if (rb.row0 < 0 || rb.nrows < 0 || rb.row0 + rb.nrows > ctx->N || rb.ld < rb.nrows)
        return set_error(ctx, PB_ERR_ARG, "row-block product: rows [%lld, %lld) outside [0, %lld)",
                         (long long)rb.row0, (long long)(rb.row0 + rb.nrows), (long long)ctx->N);
    if (rb.nrows == 0) return PB_OK;
    const double diag1 = 0.5 * (1.0 + ctx->eps), diag2 = 0.5 * (1.0 + 1.0 / ctx->eps);
    // packed kernel with 4 targets per thread (2 for small blocks), or the plain FP64 kernel
    const int T = rb.nrows >= 4096 ? 4 : 2;
    const int tt = prec == PB_FP32PAIR ? kF32Threads * T : kF64TargetTile;
    const int ts = prec == PB_FP32PAIR ? kF32SourceTile : kF64SourceTile;
    const int occ = prec == PB_FP32PAIR ? matvec_f32_occupancy(T == 4 ? MV_F32_PACKED_T4 : MV_F32_PACKED_T2)
                                        : matvec_occupancy(PB_FP64);
    const StreamKPlan pl = make_plan_rows(rb.nrows, ctx->N, tt, ts, (int64_t)ctx->num_sms * occ);
    const int64_t need_p = plan_partials(pl, tt);
    if (need_p > ctx->rows_partials_len) {
        if (ctx->rows_partials) ctx_free(ctx, ctx->rows_partials);
        ctx->device_bytes -= ctx->rows_partials_len * (int64_t)sizeof(double);
        ctx->rows_partials = nullptr;
        ctx->rows_partials_len = 0;
        pb_status s = ctx_alloc(ctx, (void **)&ctx->rows_partials, (size_t)need_p * sizeof(double),
                                "row-block partials");
        if (s != PB_OK) return s;
        ctx->rows_partials_len = need_p;
    }
    if (pl.target_tiles > ctx->rows_counters_len) {
        if (ctx->rows_counters) ctx_free(ctx, ctx->rows_counters);
        ctx->device_bytes -= ctx->rows_counters_len * (int64_t)sizeof(unsigned int);
        ctx->rows_counters = nullptr;
        ctx->rows_counters_len = 0;
        pb_status s = ctx_alloc(ctx, (void **)&ctx->rows_counters, (size_t)pl.target_tiles * sizeof(unsigned int),
                                "row-block counters");
        if (s != PB_OK) return s;
        // the kernels leave every counter at zero after use
        cudaError_t e = cudaMemsetAsync(ctx->rows_counters, 0, pl.target_tiles * sizeof(unsigned int), ctx->stream);
        if (e != cudaSuccess) return cuda_error(ctx, e, "row-block counters");
        ctx->rows_counters_len = pl.target_tiles;
    }
    if (prec == PB_FP32PAIR) {
        F32Params prm;
        prm.eps = (float)ctx->eps;
        prm.inv_eps = (float)(1.0 / ctx->eps);
        prm.kappa = (float)ctx->kappa;
        prm.neg_kappa_log2e = (float)(-ctx->kappa * 1.4426950408889634);
        prm.diag1 = diag1;
        prm.diag2 = diag2;
        const bool k0 = ctx->kappa == 0.0;
#define PB_LAUNCH_ROWS(T_, K0_)                                                                                   \
    matvec_f32x2_kernel<T_, K0_><<<(unsigned)pl.ctas, kF32Threads, 0, ctx->stream>>>(                          \
        ctx->pos32, ctx->nrm32, u, ctx->N, rb, prm, pl, ctx->rows_partials, ctx->rows_counters, y, skip_flag,    \
        ctx->mv_count)
        if (T == 4) {
            if (k0) PB_LAUNCH_ROWS(4, true); else PB_LAUNCH_ROWS(4, false);
        } else {
            if (k0) PB_LAUNCH_ROWS(2, true); else PB_LAUNCH_ROWS(2, false);
        }
#undef PB_LAUNCH_ROWS
    } else {
        F64Params prm{ctx->eps, 1.0 / ctx->eps, ctx->kappa, diag1, diag2};
        matvec_f64_kernel<<<(unsigned)pl.ctas, kF64Threads, 0, ctx->stream>>>(
            ctx->g64, u, ctx->N, rb, prm, pl, ctx->rows_partials, ctx->rows_counters, y, skip_flag, ctx->mv_count);
    }
    PB_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PB_OK : cuda_error(ctx, e, "row-block product launch");
}

pb_status matvec_launch(pb_ctx *ctx, const double *u, double *y, pb_precision prec, const int *skip_flag) {
    const double diag1 = 0.5 * (1.0 + ctx->eps), diag2 = 0.5 * (1.0 + 1.0 / ctx->eps);
    if (prec != PB_FP32PAIR && prec != PB_FP64 && prec != PB_FLOAT2)
        return set_error(ctx, PB_ERR_ARG, "pb_matvec: unknown precision %d", (int)prec);
    if (ctx->shard.on) return shard_product(ctx, u, y, prec, skip_flag);
    {
        // the symmetric variants' scratch, allocated by the first product that needs it
        pb_status s = matvec_prepare(ctx);
        if (s != PB_OK) return s;
    }
    const bool timed = ctx->prof_on;
    if (timed) {
        if (ctx->prof_used + 2 > (int)ctx->prof_ev.size()) {
            pb_status fs = profile_flush(ctx);
            if (fs != PB_OK) return fs;
        }
        cudaEventRecord(ctx->prof_ev[ctx->prof_used], ctx->stream);
    }
    cudaError_t sym_e = cudaSuccess;
    if (prec == PB_FP32PAIR) {
        F32Params prm;
        prm.eps = (float)ctx->eps;
        prm.inv_eps = (float)(1.0 / ctx->eps);
        prm.kappa = (float)ctx->kappa;
        prm.neg_kappa_log2e = (float)(-ctx->kappa * 1.4426950408889634);
        prm.diag1 = diag1;
        prm.diag2 = diag2;
        const StreamKPlan &pl = ctx->plan32;
        const bool k0 = ctx->kappa == 0.0;
#define PB_LAUNCH_F32X2(T)                                                                                      \
    do {                                                                                                        \
        if (k0)                                                                                                 \
            matvec_f32x2_kernel<T, true><<<(unsigned)pl.ctas, kF32Threads, 0, ctx->stream>>>(                   \
                ctx->pos32, ctx->nrm32, u, ctx->N, RowBlock{0, ctx->N, ctx->N}, prm, pl, ctx->partials,                 \
                ctx->tile_counters, y, skip_flag,                                                               \
                ctx->mv_count);                                                                                 \
        else                                                                                                    \
            matvec_f32x2_kernel<T, false><<<(unsigned)pl.ctas, kF32Threads, 0, ctx->stream>>>(                  \
                ctx->pos32, ctx->nrm32, u, ctx->N, RowBlock{0, ctx->N, ctx->N}, prm, pl, ctx->partials,                 \
                ctx->tile_counters, y, skip_flag,                                                               \
                ctx->mv_count);                                                                                 \
    } while (0)
#define PB_LAUNCH_SYM(T, MINB)                                                                                  \
    do {                                                                                                        \
        auto pair = [&](const SymPlan &bp, double *islots, double *iside, float *jpart,                         \
                        unsigned long long *ev, cudaStream_t s) {                                               \
            if (k0)                                                                                             \
                matvec_sym_kernel<T, true, MINB><<<(unsigned)bp.ctas, kF32Threads, 0, s>>>(                     \
                    ctx->pos32, ctx->nrm32, u, ctx->N, prm, bp, islots, iside, jpart, skip_flag, ev);           \
            else                                                                                                \
                matvec_sym_kernel<T, false, MINB><<<(unsigned)bp.ctas, kF32Threads, 0, s>>>(                    \
                    ctx->pos32, ctx->nrm32, u, ctx->N, prm, bp, islots, iside, jpart, skip_flag, ev);           \
        };                                                                                                      \
        sym_e = sym_enqueue<kF32Threads * T, float>(ctx->plansym, ctx->cuts32, ctx->sym_scratch, u, ctx->N,     \
                                                    diag1, diag2, y, skip_flag, ctx->mv_count, ctx->stream,    \
                                                    ctx->band_stream, ctx->band_ev, pair);                     \
    } while (0)
        switch (ctx->f32_variant) {
            case MV_F32_SCALAR_T4:
                matvec_f32_kernel<<<(unsigned)pl.ctas, kF32Threads, 0, ctx->stream>>>(
                    ctx->pos32, ctx->nrm32, u, ctx->N, prm, pl, ctx->partials, ctx->tile_counters, y, skip_flag,
                    ctx->mv_count);
                break;
            case MV_F32_PACKED_T4: PB_LAUNCH_F32X2(4); break;
            case MV_F32_PACKED_T3: PB_LAUNCH_F32X2(3); break;
            case MV_F32_SYM_T2: PB_LAUNCH_SYM(2, 4); break;
            case MV_F32_SYM_T4: PB_LAUNCH_SYM(4, 3); break;
            default: PB_LAUNCH_F32X2(2); break;
        }
#undef PB_LAUNCH_F32X2
#undef PB_LAUNCH_SYM
    } else if (prec == PB_FLOAT2) {
        pb_status fs = matvec_ff_enqueue(ctx, u, y, skip_flag);
        if (fs != PB_OK) return fs;
    } else if (ctx->f64_variant == MV_F64_PLAIN) {
        F64Params prm{ctx->eps, 1.0 / ctx->eps, ctx->kappa, diag1, diag2};
        const StreamKPlan &pl = ctx->plan64;
        matvec_f64_kernel<<<(unsigned)pl.ctas, kF64Threads, 0, ctx->stream>>>(
            ctx->g64, u, ctx->N, RowBlock{0, ctx->N, ctx->N}, prm, pl, ctx->partials, ctx->tile_counters, y, skip_flag,
            ctx->mv_count);
    } else {
        F64Params prm{ctx->eps, 1.0 / ctx->eps, ctx->kappa, diag1, diag2};
        auto pair = [&](auto tag) {
            constexpr int T = decltype(tag)::value;
            return [&](const SymPlan &bp, double *islots, double *iside, double *jpart, unsigned long long *ev,
                       cudaStream_t s) {
                matvec_sym64_kernel<T><<<(unsigned)bp.ctas, kF64Threads, 0, s>>>(
                    ctx->g64, u, ctx->N, prm, bp, islots, iside, jpart, skip_flag, ev);
            };
        };
        if (ctx->f64_variant == MV_F64_SYM_T2)
            sym_e = sym_enqueue<2 * kF64Threads, double>(ctx->plansym64, ctx->cuts64, ctx->sym64_scratch, u, ctx->N,
                                                         diag1, diag2, y, skip_flag, ctx->mv_count, ctx->stream,
                                                         ctx->band_stream, ctx->band_ev,
                                                         pair(std::integral_constant<int, 2>{}));
        else
            sym_e = sym_enqueue<kF64Threads, double>(ctx->plansym64, ctx->cuts64, ctx->sym64_scratch, u, ctx->N,
                                                     diag1, diag2, y, skip_flag, ctx->mv_count, ctx->stream,
                                                     ctx->band_stream, ctx->band_ev,
                                                     pair(std::integral_constant<int, 1>{}));
    }
    if (sym_e != cudaSuccess) return cuda_error(ctx, sym_e, "symmetric product bands");
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
    // the kappa = 0 instantiations use fewer registers; size grids by the
    // general one so that one plan serves both
    int n = 0;
    switch (variant) {
        case MV_F32_SCALAR_T4:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matvec_f32_kernel, kF32Threads, 0);
            break;
        case MV_F32_PACKED_T4:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matvec_f32x2_kernel<4, false>, kF32Threads, 0);
            break;
        case MV_F32_PACKED_T3:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matvec_f32x2_kernel<3, false>, kF32Threads, 0);
            break;
        case MV_F32_SYM_T2:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matvec_sym_kernel<2, false, 4>, kF32Threads, 0);
            break;
        case MV_F32_SYM_T4:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matvec_sym_kernel<4, false, 3>, kF32Threads, 0);
            break;
        default:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matvec_f32x2_kernel<2, false>, kF32Threads, 0);
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

namespace {
pb_status ensure_scratch(pb_ctx *ctx, void **buf, int64_t *len, int64_t need, const char *what) {
    if (need <= *len) return PB_OK;
    if (*buf) ctx_free(ctx, *buf);
    ctx->device_bytes -= *len;
    *buf = nullptr;
    *len = 0;
    pb_status s = ctx_alloc(ctx, buf, (size_t)need, what);
    if (s != PB_OK) return s;
    *len = need;
    return PB_OK;
}
}  // namespace

pb_status ensure_band_streams(pb_ctx *ctx) {
    if (ctx->band_stream) return PB_OK;
    // the second stream of a banded product, at the priority of the context's stream
    int prio = 0;
    cudaError_t e = ctx->stream ? cudaStreamGetPriority(ctx->stream, &prio) : cudaSuccess;
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->band_stream, cudaStreamNonBlocking, prio);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&ctx->band_ev[k], cudaEventDisableTiming);
    return e == cudaSuccess ? PB_OK : cuda_error(ctx, e, "band streams");
}

pb_status matvec_prepare(pb_ctx *ctx) {
    pb_status s = PB_OK;
    if (f32_variant_symmetric(ctx->f32_variant))
        s = ensure_scratch(ctx, &ctx->sym_scratch, &ctx->sym_scratch_len,
                           sym_scratch_need(ctx->plansym, kF32Threads * f32_variant_targets(ctx->f32_variant),
                                            (int)sizeof(float), ctx->scratch_limit, ctx->bands, &ctx->cuts32),
                           "symmetric matvec scratch");
    if (s == PB_OK && ctx->f64_variant != MV_F64_PLAIN)
        s = ensure_scratch(ctx, &ctx->sym64_scratch, &ctx->sym64_scratch_len,
                           sym_scratch_need(ctx->plansym64, kF64Threads * (ctx->f64_variant == MV_F64_SYM_T2 ? 2 : 1),
                                            (int)sizeof(double), ctx->scratch_limit, ctx->bands, &ctx->cuts64),
                           "symmetric FP64 matvec scratch");
    if (s == PB_OK && (ctx->cuts32.size() > 2 || ctx->cuts64.size() > 2)) s = ensure_band_streams(ctx);
    return s;
}

pb_status matvec_configure_fp64(pb_ctx *ctx, int variant) {
    if (variant < 1 || variant > kNumF64Variants)
        return set_error(ctx, PB_ERR_ARG, "FP64 matvec variant %d is not one of 1..%d", variant, kNumF64Variants);
    if (variant != MV_F64_PLAIN) {
        const int T = variant == MV_F64_SYM_T2 ? 2 : 1;
        int occ = 0;
        if (T == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, matvec_sym64_kernel<2>, kF64Threads, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, matvec_sym64_kernel<1>, kF64Threads, 0);
        if (occ < 1) occ = 1;
        ctx->plansym64 = make_sym_plan(ctx->N, kF64Threads * T, (int64_t)ctx->num_sms * occ);
    } else if (ctx->sym64_scratch) {
        ctx_free(ctx, ctx->sym64_scratch);
        ctx->device_bytes -= ctx->sym64_scratch_len;
        ctx->sym64_scratch = nullptr;
        ctx->sym64_scratch_len = 0;
    }
    ctx->f64_variant = variant;
    return PB_OK;
}

pb_status matvec_configure(pb_ctx *ctx, int variant, int ctas_per_sm) {
    if (variant < 1 || variant > kNumF32Variants)
        return set_error(ctx, PB_ERR_ARG, "matvec variant %d is not one of 1..%d", variant, kNumF32Variants);
    if (ctas_per_sm < 0) return set_error(ctx, PB_ERR_ARG, "ctas_per_sm must be >= 0");
    if (f32_variant_symmetric(variant)) {
        int occ = matvec_f32_occupancy(variant);
        if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
        const int tile = kF32Threads * f32_variant_targets(variant);
        // the scratch is allocated by the first product that needs it
        ctx->plansym = make_sym_plan(ctx->N, tile, (int64_t)ctx->num_sms * occ);
    } else {
        StreamKPlan pl = matvec_f32_plan(ctx, variant, ctas_per_sm);
        if (plan_partials(pl, kF32Threads * f32_variant_targets(variant)) > ctx->partials_len ||
            pl.target_tiles > ctx->counters_len)
            return set_error(ctx, PB_ERR_ARG, "matvec configuration exceeds the context's scratch");
        ctx->plan32 = pl;
        if (ctx->sym_scratch) {
            ctx_free(ctx, ctx->sym_scratch);
            ctx->device_bytes -= ctx->sym_scratch_len;
            ctx->sym_scratch = nullptr;
            ctx->sym_scratch_len = 0;
        }
    }
    ctx->f32_variant = variant;
    ctx->f32_ctas_per_sm = ctas_per_sm;
    return PB_OK;
}

}  // namespace pb

extern "C" pb_status pb_sym_band_plan(int64_t n, int tile, int64_t ctas, int elem, int64_t limit, int bands,
                                      int64_t *cuts, int max_cuts, int *ncuts, int64_t *bytes) {
    if (n < 1 || tile < 128 || tile % 128 != 0 || ctas < 1 || (elem != 4 && elem != 8) || limit < 0 || bands < 0 ||
        max_cuts < 0 || (max_cuts > 0 && cuts == nullptr))
        return pb::set_error(nullptr, PB_ERR_ARG, "pb_sym_band_plan: bad argument");
    const pb::SymPlan pl = pb::make_sym_plan(n, tile, ctas);
    std::vector<int64_t> c;
    const int64_t need = pb::sym_scratch_need(pl, tile, elem, limit, bands, &c);
    for (int k = 0; k < max_cuts && k < (int)c.size(); ++k) cuts[k] = c[k];
    if (ncuts) *ncuts = (int)c.size();
    if (bytes) *bytes = need;
    return PB_OK;
}
