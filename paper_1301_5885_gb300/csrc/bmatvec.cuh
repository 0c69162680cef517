// bmatvec.cuh -- the multi-surface, multi-right-hand-side product of the
// batch engine (Eqs. (12)-(13) for every GMRES instance of a batch), its
// tables, and its tunable shapes.
//
// One persistent launch covers the flattened (surface, target tile, source
// tile) space of every surface in the batch.  Two choices shape the kernel
// and are picked per right-hand-side width R by the engine's autotuner
// (batch.cu):
//   - T, the targets per thread (target tile 128 T): more targets share each
//     staged source, fewer leave registers for the K1..K4 chains;
//   - where the thread's 2 R T row sums live and in what arithmetic: FP64 in
//     registers or in the thread's shared-memory slots, or float-float (an
//     unevaluated FP32 pair, about 48 bits) in registers or shared memory.
//     Each 256-source stage adds two FP32 half sums to every row sum; in FP64
//     that is 2 conversions and 2 additions on the FP64 pipe (a small
//     fraction of the FP32 rate on this GPU), in float-float 13 FP32
//     operations (two two-sums).
// The CTA count (CTAs per SM up to the kernel's occupancy) is the third knob.
//
// The kernels are instantiated in bmatvec_r12.cu, bmatvec_r4.cu and
// bmatvec_r8.cu (PB_BMATVEC_KERNELS defined) so that they compile in
// parallel; batch.cu sees only the declarations.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fastmath.cuh"
#include "pb_internal.cuh"

namespace pb {

constexpr int kBThreads = 128;          // product kernel threads
constexpr int kBSourceTile = 256;       // sources per staged tile (one pair per thread)

// placement and arithmetic of the row sums
enum BmvRowSums { BMV_FP64_REGISTERS = 0, BMV_FP64_SHARED = 1, BMV_FF_REGISTERS = 2, BMV_FF_SHARED = 3 };

struct BmvShape {
    int T;       // targets per thread
    int acc;     // BmvRowSums
};

struct BSurf {
    const float4 *pos;
    const float4 *nrm;
    int64_t N;
    float eps, inv_eps, kappa, nk;
    double diag1, diag2;
    int64_t tile_base;     // global index of this surface's first target tile
    int64_t work_base;     // global index of its first (target tile, source tile) pair, all surfaces active
    int64_t ntiles;        // its target tiles in the batched product (0 for a surface with its own launch)
    int64_t S;             // source tiles
    int inst0;             // first instance
    int nrhs;
};

struct BInst {
    double *b, *x, *w, *r, *V;   // V: (m+1) vectors of 2N
    GmresState *st;
    int64_t n2;
    int surf;
    int chunk0, nchunk;          // its chunks of the 2N vectors
};

struct BChunk {
    int inst;
    int len;
    int64_t start;               // relative to the instance's vectors
};

// Launch arguments of the product (see bmatvec_kernel).  wbase[s] is the
// first work item of surface s in the split of this launch and wbase[nsurf]
// the number of work items: bmv_plan_kernel writes them on the device before
// every launch, giving idle surfaces no work.
struct BmvArgs {
    const BSurf *surf;
    int nsurf;
    const BInst *inst;
    const int64_t *wbase;
    int64_t G;
    int usel, k;
    const int *active;
    double *partials;
    unsigned int *counters;
    unsigned long long *evaluated;
};

// Launches the product for R right-hand sides with shape (T, acc) on `grid`
// CTAs, or with occ != NULL only queries its occupancy (CTAs per SM).
// Returns cudaErrorInvalidValue for a shape that is not instantiated.
template <int R>
cudaError_t bmatvec_run(int T, int acc, const BmvArgs &a, unsigned grid, cudaStream_t s, int *occ);
template <>
cudaError_t bmatvec_run<1>(int T, int acc, const BmvArgs &a, unsigned grid, cudaStream_t s, int *occ);
template <>
cudaError_t bmatvec_run<2>(int T, int acc, const BmvArgs &a, unsigned grid, cudaStream_t s, int *occ);
template <>
cudaError_t bmatvec_run<4>(int T, int acc, const BmvArgs &a, unsigned grid, cudaStream_t s, int *occ);
template <>
cudaError_t bmatvec_run<8>(int T, int acc, const BmvArgs &a, unsigned grid, cudaStream_t s, int *occ);

// The shapes instantiated for each width R, (R, T, row sums); the first of
// each list is the built-in default.  At R = 8 the default keeps the FP64 row
// sums in shared memory (32 of them per thread leave too few registers).
#define PB_BMV_SHAPES_R1(X) X(1, 4, 0) X(1, 4, 2) X(1, 2, 0) X(1, 2, 2)
#define PB_BMV_SHAPES_R2(X) X(2, 2, 0) X(2, 2, 2) X(2, 4, 2) X(2, 4, 3) X(2, 1, 2)
#define PB_BMV_SHAPES_R4(X) X(4, 2, 0) X(4, 2, 2) X(4, 2, 3) X(4, 1, 2) X(4, 4, 3)
#define PB_BMV_SHAPES_R8(X) X(8, 2, 1) X(8, 2, 3) X(8, 2, 2) X(8, 1, 2) X(8, 1, 3)

// The shapes instantiated for width R, the built-in default first; returns
// their number (at most max_out are written).
inline int bmatvec_shapes(int R, BmvShape *out, int max_out) {
    int n = 0;
#define PB_BMV_LIST(R_, T_, A_) \
    if (R == R_) {                \
        if (n < max_out) out[n] = BmvShape{T_, A_}; \
        ++n;                      \
    }
    PB_BMV_SHAPES_R1(PB_BMV_LIST)
    PB_BMV_SHAPES_R2(PB_BMV_LIST)
    PB_BMV_SHAPES_R4(PB_BMV_LIST)
    PB_BMV_SHAPES_R8(PB_BMV_LIST)
#undef PB_BMV_LIST
    return n;
}

inline cudaError_t bmatvec_dispatch(int R, BmvShape sh, const BmvArgs &a, unsigned grid, cudaStream_t s, int *occ) {
    switch (R) {
        case 1: return bmatvec_run<1>(sh.T, sh.acc, a, grid, s, occ);
        case 2: return bmatvec_run<2>(sh.T, sh.acc, a, grid, s, occ);
        case 4: return bmatvec_run<4>(sh.T, sh.acc, a, grid, s, occ);
        case 8: return bmatvec_run<8>(sh.T, sh.acc, a, grid, s, occ);
        default: return cudaErrorInvalidValue;
    }
}

#ifdef PB_BMATVEC_KERNELS
namespace {

// hi + lo += a + b in float-float: Knuth's two-sum of a and b, then of hi
// and their sum; the two rounding errors go to lo.  Explicit round-to-nearest
// intrinsics keep the compiler from reassociating.
__device__ __forceinline__ void ff_add2(float &hi, float &lo, float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e1 = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    const float h = __fadd_rn(hi, s);
    const float cc = __fsub_rn(h, hi);
    const float e2 = __fadd_rn(__fsub_rn(hi, __fsub_rn(h, cc)), __fsub_rn(s, cc));
    hi = h;
    lo = __fadd_rn(lo, __fadd_rn(e1, e2));
}

__device__ __forceinline__ int bvol(const int *p) { return *((volatile const int *)p); }

// ---- the multi-surface, multi-right-hand-side product ------------------------
// the surface owning work item p: the last s with wbase[s] <= p (a surface
// without work shares its base with the next one, which is found instead)
__device__ __forceinline__ int find_surface(const int64_t *wbase, int nsurf, int64_t p) {
    int lo = 0, hi = nsurf - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (wbase[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct BConsts {
    float2 nk2, mkap2, one2, mone2, three2, mthree2, meps2, epsm1, ieps2, omieps;
};

// K1..K4 of one target against one staged source pair (K0: only K2 and K3,
// their constant factors being in the weights).
template <bool K0>
__device__ __forceinline__ void bcoef(const float4 &A, const float4 &Bq, const float4 &C, float2 x, float2 y,
                                      float2 z, float2 nx, float2 ny, float2 nz, const BConsts &k, float2 &k1,
                                      float2 &k2, float2 &k3, float2 &k4) {
    const float2 dx = p_add(x, make_float2(A.x, A.y)), dy = p_add(y, make_float2(A.z, A.w));
    const float2 dz = p_add(z, make_float2(Bq.x, Bq.y));
    const float2 snx = make_float2(Bq.z, Bq.w), sny = make_float2(C.x, C.y), snz = make_float2(C.z, C.w);
    const float2 r2 = p_fma(dx, dx, p_fma(dy, dy, p_mul(dz, dz)));
    float2 inv, inv2;
    // r^2 clamped below at 1e-18 for the MUFU; rho = r^2 (1/rho) uses the
    // unclamped r^2, exactly 0 for a pair at zero distance
    const float r2cx = fmaxf(r2.x, 1e-18f), r2cy = fmaxf(r2.y, 1e-18f);
    inv.x = rsqrt_approx(r2cx);
    inv.y = rsqrt_approx(r2cy);
    if (K0) {
        inv2 = p_mul(inv, inv);
    } else {
        inv2.x = rcp_approx(r2cx);
        inv2.y = rcp_approx(r2cy);
    }
    const float2 inv3 = p_mul(inv2, inv);
    const float2 ncx = p_fma(dx, nx, p_fma(dy, ny, p_mul(dz, nz)));   // -c_x
    const float2 cy = p_fma(dx, snx, p_fma(dy, sny, p_mul(dz, snz)));
    if (K0) {
        k2 = p_mul(cy, inv3);
        k3 = p_mul(ncx, inv3);
    } else {
        const float2 rho = p_mul(r2, inv);
        const float2 arg = p_mul(k.nk2, rho);
        float2 e;
        e.x = exp2_approx(arg.x);
        e.y = exp2_approx(arg.y);
        const float2 mkr = p_mul(k.mkap2, rho);
        const float2 nnn = p_fma(nx, snx, p_fma(ny, sny, p_mul(nz, snz)));   // -n
        const float2 ome = p_fma(e, k.mone2, k.one2);
        const float2 ome1 = p_fma(e, mkr, ome);                                // 1 - e (1 + kappa rho)
        k1 = p_mul(ome, inv);
        k2 = p_mul(p_mul(p_fma(ome1, k.meps2, k.epsm1), inv3), cy);
        k3 = p_mul(p_mul(p_fma(ome1, k.ieps2, k.omieps), inv3), ncx);
        const float2 p3 = p_fma(mkr, p_add(mkr, k.mthree2), k.three2);
        const float2 e3 = p_fma(e, p3, k.mthree2);
        const float2 ccy = p_mul(p_mul(e3, ncx), cy);
        k4 = p_mul(p_fma(ccy, inv2, p_mul(ome1, nnn)), inv3);
    }
}

// One staged source pair q against the thread's T targets, for the R
// right-hand sides of the surface.
template <int R, int T, bool K0>
__device__ __forceinline__ void bstep(const float4 *s_g, const float4 *s_w, int q, const BConsts &k,
                                      const float2 (&xi)[T], const float2 (&yi)[T], const float2 (&zi)[T],
                                      const float2 (&nxi)[T], const float2 (&nyi)[T], const float2 (&nzi)[T],
                                      float2 (&f1)[R][T], float2 (&f2)[R][T]) {
    constexpr int TQ = kBSourceTile / 2;
    float2 k1[T], k2[T], k3[T], k4[T];
    const float4 A = s_g[q], Bq = s_g[TQ + q], C = s_g[2 * TQ + q];
#pragma unroll
    for (int t = 0; t < T; ++t)
        bcoef<K0>(A, Bq, C, xi[t], yi[t], zi[t], nxi[t], nyi[t], nzi[t], k, k1[t], k2[t], k3[t], k4[t]);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float4 w = s_w[r * TQ + q];
        const float2 wpsi = make_float2(w.x, w.y), wphi = make_float2(w.z, w.w);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            if (K0) {
                f1[r][t] = p_fma(k2[t], wphi, f1[r][t]);
                f2[r][t] = p_fma(k3[t], wpsi, f2[r][t]);
            } else {
                f1[r][t] = p_fma(k1[t], wpsi, p_fma(k2[t], wphi, f1[r][t]));
                f2[r][t] = p_fma(k3[t], wpsi, p_fma(k4[t], wphi, f2[r][t]));
            }
        }
    }
}

// One staged tile of source pairs against the thread's T targets, for the R
// right-hand sides of the surface.  Packed f32x2: each instruction does a
// step of two pairs (one target, two sources).  The target normals arrive
// negated so that no operand needs a sign change: with c_x' = -c_x, n' = -n,
// 1 - e' = 1 - e (1 + kappa rho) and -b (b the K3 factor),
//   K1 = (1 - e)/rho,  K2 = a c_y,  K3 = (-b) c_x',
//   K4 = (-e3 c_x c_y / rho^2 + (e' - 1) n) / rho^3 = ((e3 c_x' c_y) / rho^2 + (1 - e') n') / rho^3
// with a = (eps e' - 1)/rho^3 and e3 = e (3 + 3 kappa rho + kappa^2 rho^2) - 3:
// 36 FP32 operations per pair for K1..K4 and 4 per right-hand side.  With
// kappa = 0 (K0), K1 = K4 = 0 and the constant factors of K2, K3 are folded
// into the staged weights: 16 operations per pair and 2 per right-hand side.
// The self pair is removed by the clamp of r^2 before the MUFU (every term
// an exact zero, as in the single-surface kernels).
template <int R, int T, bool K0>
__device__ __forceinline__ void bstage(const float4 *s_g, const float4 *s_w, int npairs, float eps, float inv_eps,
                                       float kappa, float nk, const float2 (&xi)[T], const float2 (&yi)[T],
                                       const float2 (&zi)[T], const float2 (&nxi)[T], const float2 (&nyi)[T],
                                       const float2 (&nzi)[T], float2 (&f1)[R][T], float2 (&f2)[R][T]) {
    BConsts k;
    k.nk2 = p_dup(nk);
    k.mkap2 = p_dup(-kappa);
    k.one2 = p_dup(1.f);
    k.mone2 = p_dup(-1.f);
    k.three2 = p_dup(3.f);
    k.mthree2 = p_dup(-3.f);
    k.meps2 = p_dup(-eps);
    k.epsm1 = p_dup(eps - 1.f);
    k.ieps2 = p_dup(inv_eps);
    k.omieps = p_dup(1.f - inv_eps);
#pragma unroll 1
    for (int q = 0; q < npairs; ++q) bstep<R, T, K0>(s_g, s_w, q, k, xi, yi, zi, nxi, nyi, nzi, f1, f2);
}

// y_q = A u_q for every instance q; u_q = x_q (usel 0) or V_q[k] (usel 1), y_q = w_q.
// CTA c owns the flattened (surface, target tile, source tile) range
// [c W / G, (c+1) W / G); a target tile split over several CTAs is finished
// by the last to arrive, which adds the partial rows in CTA order.
// T targets per thread (target tile 128 T); ACCM places the row sums of the
// thread's 2 R T rows (see BmvRowSums).
// Resident CTAs per SM the register allocation must allow (0: the compiler's
// choice).  Two targets per thread with 8 right-hand sides and float-float row
// sums in shared memory is held to 170 registers, three CTAs per SM; left to
// itself the allocation takes 186 and two.
constexpr int bmv_min_blocks(int R, int T, int ACCM) {
    return (R == 8 && T == 2 && ACCM == BMV_FF_SHARED) ? 3 : 0;
}

template <int R, int T, int ACCM>
__global__ void __launch_bounds__(kBThreads, bmv_min_blocks(R, T, ACCM))
bmatvec_kernel(const BSurf *__restrict__ surf, int nsurf, const BInst *__restrict__ inst,
               const int64_t *__restrict__ wbase, int64_t G,
               int usel, int k, const int *__restrict__ active, double *__restrict__ partials,
               unsigned int *__restrict__ counters, unsigned long long *__restrict__ evaluated) {
    constexpr int BS = kBThreads, TT = BS * T, TS = kBSourceTile, TQ = TS / 2;
    static_assert(TQ == BS, "one source pair per thread when staging");
    __shared__ float4 s_g[3 * TQ];       // {-x0,-x1,-y0,-y1}, {-z0,-z1,nx0,nx1}, {ny0,ny1,nz0,nz1}
    __shared__ float4 s_w[R * TQ];       // per right-hand side {W dphi0, W dphi1, W phi0, W phi1} / (4 pi)
    __shared__ const double *s_u[R];
    __shared__ double *s_y[R];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    // row sums (rows of phi: w = 0, of dphi: w = 1) of the thread's targets
    constexpr int NA = 2 * R * T;
    constexpr bool FF = ACCM >= BMV_FF_REGISTERS, SM = ACCM == BMV_FP64_SHARED || ACCM == BMV_FF_SHARED;
    __shared__ double s_a64[(SM && !FF) ? NA * BS : 1];
    __shared__ float s_ahi[(SM && FF) ? NA * BS : 1];
    __shared__ float s_alo[(SM && FF) ? NA * BS : 1];
    double r_a64[(!SM && !FF) ? NA : 1];
    float r_ahi[(!SM && FF) ? NA : 1], r_alo[(!SM && FF) ? NA : 1];
    // zero, add a stage's two FP32 half sums, read as FP64
    auto acc_zero = [&](int i) {
        if constexpr (!FF) {
            if constexpr (SM) s_a64[i * BS + tid] = 0.0; else r_a64[i] = 0.0;
        } else if constexpr (SM) {
            s_ahi[i * BS + tid] = 0.f;
            s_alo[i * BS + tid] = 0.f;
        } else {
            r_ahi[i] = 0.f;
            r_alo[i] = 0.f;
        }
    };
    auto acc_add = [&](int i, float a, float b) {
        if constexpr (!FF) {
            if constexpr (SM) s_a64[i * BS + tid] += (double)a + (double)b; else r_a64[i] += (double)a + (double)b;
        } else if constexpr (SM) {
            ff_add2(s_ahi[i * BS + tid], s_alo[i * BS + tid], a, b);
        } else {
            ff_add2(r_ahi[i], r_alo[i], a, b);
        }
    };
    auto acc_get = [&](int i) -> double {
        if constexpr (!FF) {
            if constexpr (SM) return s_a64[i * BS + tid]; else return r_a64[i];
        } else if constexpr (SM) {
            return (double)s_ahi[i * BS + tid] + (double)s_alo[i * BS + tid];
        } else {
            return (double)r_ahi[i] + (double)r_alo[i];
        }
    };
#define ACC_IDX(w, r, t) ((((w) * R + (r)) * T + (t)))
    const int64_t c = blockIdx.x;
    // this launch's work and grid: every CTA of the split must own at least
    // one work item (the last-arriver count covers every CTA between a
    // tile's first and last owner), so with less work than CTAs the surplus
    // CTAs leave at once
    const int64_t W = wbase[nsurf];
    const int64_t Gw = G < W ? G : W;
    if (c >= Gw) return;
    int64_t p = sk_begin(c, W, Gw);
    const int64_t pend = sk_begin(c + 1, W, Gw);
    // global target tile of this CTA's first pair (its partial slot 0)
    int64_t first_tile = -1;
    if (p < pend) {
        const int s0 = find_surface(wbase, nsurf, p);
        first_tile = surf[s0].tile_base + (p - wbase[s0]) / surf[s0].S;
    }

    while (p < pend) {
        const int si = find_surface(wbase, nsurf, p);
        const BSurf sf = surf[si];
        const int64_t local = p - wbase[si];
        const int64_t S = sf.S;
        const int64_t a = local / S;
        const int64_t s_first = local % S;
        const int64_t s_end = (S < s_first + (pend - p)) ? S : s_first + (pend - p);
        const int64_t N = sf.N;
        if (!bvol(active + si)) {          // every instance of this surface is idle
            p += s_end - s_first;
            continue;
        }
        if (local == 0 && tid == 0) atomicAdd(evaluated + si, 1ull);   // one product of this surface
        __syncthreads();                  // the previous segment is done with s_u / s_y
        if (tid < R) {
            if (tid < sf.nrhs) {
                const BInst in = inst[sf.inst0 + tid];
                s_u[tid] = usel ? in.V + (int64_t)k * in.n2 : in.x;
                s_y[tid] = in.w;
            } else {
                s_u[tid] = nullptr;
                s_y[tid] = nullptr;
            }
        }
        const bool k0 = sf.kappa == 0.f;
        // kappa = 0: (eps - 1) and (1/eps - 1) folded into the weights (K3 uses -c_x)
        const float wphi_scale = k0 ? sf.eps - 1.f : 1.f, wpsi_scale = k0 ? 1.f - sf.inv_eps : 1.f;
        float2 xi[T], yi[T], zi[T], nxi[T], nyi[T], nzi[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int64_t i = a * TT + t * BS + tid;
            const int64_t ic = i < N ? i : N - 1;
            const float4 q = sf.pos[ic], n = sf.nrm[ic];
            xi[t] = p_dup(q.x); yi[t] = p_dup(q.y); zi[t] = p_dup(q.z);
            nxi[t] = p_dup(-n.x); nyi[t] = p_dup(-n.y); nzi[t] = p_dup(-n.z);
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int t = 0; t < T; ++t) { acc_zero(ACC_IDX(0, r, t)); acc_zero(ACC_IDX(1, r, t)); }

        for (int64_t st = s_first; st < s_end; ++st) {
            __syncthreads();
            {
                // stage source pair (2 tid, 2 tid + 1); a missing second source
                // repeats the first with zero weights
                const int64_t j0 = st * TS + 2 * tid;
                if (j0 < N) {
                    const bool has1 = j0 + 1 < N;
                    const int64_t j1 = has1 ? j0 + 1 : j0;
                    const float4 p0 = sf.pos[j0], p1 = sf.pos[j1], n0 = sf.nrm[j0], n1 = sf.nrm[j1];
                    s_g[tid] = make_float4(-p0.x, -p1.x, -p0.y, -p1.y);
                    s_g[TQ + tid] = make_float4(-p0.z, -p1.z, n0.x, n1.x);
                    s_g[2 * TQ + tid] = make_float4(n0.y, n1.y, n0.z, n1.z);
                    const float w0 = p0.w, w1 = has1 ? p1.w : 0.f;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const double *u = s_u[r];
                        s_w[r * TQ + tid] = u ? make_float4((float)u[N + j0] * (w0 * wpsi_scale),
                                                            (float)u[N + j1] * (w1 * wpsi_scale),
                                                            (float)u[j0] * (w0 * wphi_scale),
                                                            (float)u[j1] * (w1 * wphi_scale))
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
            __syncthreads();
            const int64_t rem = N - st * TS;
            const int npairs = (int)(((rem < TS) ? rem : TS) + 1) / 2;
            float2 f1[R][T], f2[R][T];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int t = 0; t < T; ++t) { f1[r][t] = p_dup(0.f); f2[r][t] = p_dup(0.f); }
            if (k0)
                bstage<R, T, true>(s_g, s_w, npairs, sf.eps, sf.inv_eps, sf.kappa, sf.nk, xi, yi, zi, nxi, nyi, nzi,
                                   f1, f2);
            else
                bstage<R, T, false>(s_g, s_w, npairs, sf.eps, sf.inv_eps, sf.kappa, sf.nk, xi, yi, zi, nxi, nyi, nzi,
                                    f1, f2);
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    acc_add(ACC_IDX(0, r, t), f1[r][t].x, f1[r][t].y);
                    acc_add(ACC_IDX(1, r, t), f2[r][t].x, f2[r][t].y);
                }
        }

        const int64_t p_tile0 = wbase[si] + a * S;
        const int64_t c0 = sk_cta_of(p_tile0, W, Gw), c1 = sk_cta_of(p_tile0 + S - 1, W, Gw);
        const int nseg = (int)(c1 - c0 + 1);
        const int64_t gtile = sf.tile_base + a;
        if (nseg == 1) {
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const int64_t i = a * TT + t * BS + tid;
                if (i < N) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (s_y[r]) {
                            s_y[r][i] = sf.diag1 * s_u[r][i] - acc_get(ACC_IDX(0, r, t));
                            s_y[r][N + i] = sf.diag2 * s_u[r][N + i] - acc_get(ACC_IDX(1, r, t));
                        }
                    }
                }
            }
        } else {
            const int64_t slot = 2 * c + (gtile == first_tile ? 0 : 1);
            double *mine = partials + slot * (2 * R * TT);
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    mine[(2 * r) * TT + t * BS + tid] = acc_get(ACC_IDX(0, r, t));
                    mine[(2 * r + 1) * TT + t * BS + tid] = acc_get(ACC_IDX(1, r, t));
                }
            __threadfence();
            __syncthreads();
            if (tid == 0) s_last = (atomicAdd(&counters[gtile], 1u) == (unsigned int)(nseg - 1));
            __syncthreads();
            if (s_last) {
                __threadfence();
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    double s1[R], s2[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) { s1[r] = 0.0; s2[r] = 0.0; }
                    for (int o = 0; o < nseg; ++o) {
                        const int64_t co = c0 + o;
                        const int64_t pb0 = sk_begin(co, W, Gw);
                        const int sc = find_surface(wbase, nsurf, pb0);
                        const int64_t ft = surf[sc].tile_base + (pb0 - wbase[sc]) / surf[sc].S;
                        const double *pp = partials + (2 * co + (gtile == ft ? 0 : 1)) * (2 * R * TT);
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            s1[r] += __ldcg(pp + (2 * r) * TT + t * BS + tid);
                            s2[r] += __ldcg(pp + (2 * r + 1) * TT + t * BS + tid);
                        }
                    }
                    const int64_t i = a * TT + t * BS + tid;
                    if (i < N) {
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            if (s_y[r]) {
                                s_y[r][i] = sf.diag1 * s_u[r][i] - s1[r];
                                s_y[r][N + i] = sf.diag2 * s_u[r][N + i] - s2[r];
                            }
                        }
                    }
                }
                if (tid == 0) counters[gtile] = 0u;
            }
        }
        p += s_end - s_first;
    }
}

#undef ACC_IDX

template <int R, int T, int ACCM>
cudaError_t bmv_launch_or_query(const BmvArgs &a, unsigned grid, cudaStream_t s, int *occ) {
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, bmatvec_kernel<R, T, ACCM>, kBThreads, 0);
    bmatvec_kernel<R, T, ACCM><<<grid, kBThreads, 0, s>>>(a.surf, a.nsurf, a.inst, a.wbase, a.G, a.usel, a.k, a.active,
                                                           a.partials, a.counters, a.evaluated);
    return cudaSuccess;
}

}  // namespace

#define PB_BMV_SHAPE(R_, T_, A_) \
    if (T == T_ && acc == A_) return bmv_launch_or_query<R_, T_, A_>(a, grid, s, occ);
#endif  // PB_BMATVEC_KERNELS

}  // namespace pb
