// batch.cu -- many PB solves in lockstep: several surfaces of uneven N, each
// with up to 8 right-hand sides (charge sets), solved together.
//
// Every (surface, right-hand side) pair is one GMRES instance with its own
// Krylov basis, Hessenberg matrix and convergence state, all in device memory.
// The instances advance one Arnoldi step at a time in lockstep, so each step
// needs one product with A per instance.  Those products are evaluated by one
// persistent multi-right-hand-side launch over all surfaces: the (surface,
// target tile, source tile) iteration space is flattened and split evenly over
// the CTAs, and each pair's kernels K1..K4 (Eq. (10)) are evaluated once and
// applied to all R right-hand sides of that surface (Eqs. (12)-(13)).  The
// vector work of GMRES (Gram-Schmidt, norms, Givens, updates) runs in batched
// kernels over every instance's vectors, cut into chunks that never straddle
// two instances; per-instance sums are fixed-order two-stage reductions
// finished by the last chunk to arrive.  Instances that have converged are
// skipped, and a surface whose instances are all idle is skipped by the
// product.  Instances can join and leave between restart cycles (the solve
// server relies on this); with a fixed set, one restart cycle of the whole
// batch can be captured in a CUDA graph and replayed.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "engine.cuh"
#include "fastmath.cuh"
#include "pb_internal.cuh"
#include "reduce.cuh"

namespace pb {

constexpr int kBThreads = 128;          // product kernel threads
constexpr int kBSourceTile = 256;       // sources per staged tile (one pair per thread)
// targets per thread of the product kernel for R right-hand sides (more
// targets share each staged source when fewer accumulators are needed)
__host__ __device__ constexpr int bmatvec_targets(int R) { return R <= 1 ? 4 : 2; }
constexpr int kChunk = 4096;            // vector chunk (elements) of the GMRES kernels
constexpr int kVThreads = 256;
constexpr int LDH = kMaxRestart + 1;

struct BSurf {
    const float4 *pos;
    const float4 *nrm;
    int64_t N;
    float eps, inv_eps, kappa, nk;
    double diag1, diag2;
    int64_t tile_base;     // global index of this surface's first target tile
    int64_t work_base;     // global index of its first (target tile, source tile) pair
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

namespace {

__device__ __forceinline__ int vol(const int *p) { return *((volatile const int *)p); }

__device__ __forceinline__ bool inst_last(unsigned int *counter, unsigned int n) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == n - 1);
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// ---- the multi-surface, multi-right-hand-side product ------------------------
__device__ __forceinline__ int find_surface(const BSurf *surf, int nsurf, int64_t p) {
    int lo = 0, hi = nsurf - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (surf[mid].work_base <= p) lo = mid; else hi = mid - 1;
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
template <int R>
__global__ void __launch_bounds__(kBThreads)
bmatvec_kernel(const BSurf *__restrict__ surf, int nsurf, const BInst *__restrict__ inst, int64_t W, int64_t G,
               int usel, int k, const int *__restrict__ active, double *__restrict__ partials,
               unsigned int *__restrict__ counters, unsigned long long *__restrict__ evaluated) {
    constexpr int BS = kBThreads, T = bmatvec_targets(R), TT = BS * T, TS = kBSourceTile, TQ = TS / 2;
    static_assert(TQ == BS, "one source pair per thread when staging");
    __shared__ float4 s_g[3 * TQ];       // {-x0,-x1,-y0,-y1}, {-z0,-z1,nx0,nx1}, {ny0,ny1,nz0,nz1}
    __shared__ float4 s_w[R * TQ];       // per right-hand side {W dphi0, W dphi1, W phi0, W phi1} / (4 pi)
    __shared__ const double *s_u[R];
    __shared__ double *s_y[R];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    // FP64 row sums (rows of phi: w = 0, of dphi: w = 1): in registers, or in
    // this thread's own shared-memory slots when there are many of them
    constexpr bool SACC = R * T >= 16;
    __shared__ double s_acc[SACC ? 2 * R * T * BS : 1];
    double racc[SACC ? 1 : 2 * R * T];
#define ACC(w, r, t) (SACC ? s_acc[(((w) * R + (r)) * T + (t)) * BS + tid] : racc[((w) * R + (r)) * T + (t)])
    const int64_t c = blockIdx.x;
    int64_t p = sk_begin(c, W, G);
    const int64_t pend = sk_begin(c + 1, W, G);
    // global target tile of this CTA's first pair (its partial slot 0)
    int64_t first_tile = -1;
    if (p < pend) {
        const int s0 = find_surface(surf, nsurf, p);
        first_tile = surf[s0].tile_base + (p - surf[s0].work_base) / surf[s0].S;
    }

    while (p < pend) {
        const int si = find_surface(surf, nsurf, p);
        const BSurf sf = surf[si];
        const int64_t local = p - sf.work_base;
        const int64_t S = sf.S;
        const int64_t a = local / S;
        const int64_t s_first = local % S;
        const int64_t s_end = (S < s_first + (pend - p)) ? S : s_first + (pend - p);
        const int64_t N = sf.N;
        if (!vol(active + si)) {          // every instance of this surface is idle
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
            for (int t = 0; t < T; ++t) { ACC(0, r, t) = 0.0; ACC(1, r, t) = 0.0; }

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
                    ACC(0, r, t) += (double)f1[r][t].x + (double)f1[r][t].y;
                    ACC(1, r, t) += (double)f2[r][t].x + (double)f2[r][t].y;
                }
        }

        const int64_t p_tile0 = sf.work_base + a * S;
        const int64_t c0 = sk_cta_of(p_tile0, W, G), c1 = sk_cta_of(p_tile0 + S - 1, W, G);
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
                            s_y[r][i] = sf.diag1 * s_u[r][i] - ACC(0, r, t);
                            s_y[r][N + i] = sf.diag2 * s_u[r][N + i] - ACC(1, r, t);
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
                    mine[(2 * r) * TT + t * BS + tid] = ACC(0, r, t);
                    mine[(2 * r + 1) * TT + t * BS + tid] = ACC(1, r, t);
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
                        const int64_t pb0 = sk_begin(co, W, G);
                        const int sc = find_surface(surf, nsurf, pb0);
                        const int64_t ft = surf[sc].tile_base + (pb0 - surf[sc].work_base) / surf[sc].S;
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

#undef ACC

// ---- batched GMRES vector kernels (one block per chunk) ----------------------
__global__ void __launch_bounds__(kVThreads)
bg_cycle_start(int usex, const BChunk *__restrict__ ch, const BInst *__restrict__ inst, double *__restrict__ red,
               unsigned int *__restrict__ counters) {
    const BChunk c = ch[blockIdx.x];
    const BInst in = inst[c.inst];
    GmresState *g = in.st;
    if (vol(&g->done)) return;
    const bool zero = vol(&g->x_is_zero) != 0 || !usex;
    double s = 0.0;
    for (int k = threadIdx.x; k < c.len; k += kVThreads) {
        const int64_t e = c.start + k;
        const double ri = zero ? in.b[e] : in.b[e] - in.w[e];
        in.r[e] = ri;
        s += ri * ri;
    }
    s = block_sum<kVThreads>(s);
    if (threadIdx.x == 0) red[blockIdx.x] = s;
    if (inst_last(&counters[c.inst], in.nchunk) && threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < in.nchunk; ++b) t += __ldcg(red + in.chunk0 + b);
        counters[c.inst] = 0u;
        const double beta = sqrt(t);
        g->k = 0;
        g->beta = beta;
        g->rel_resid = g->bnorm > 0.0 ? beta / g->bnorm : 0.0;
        g->est_resid = g->rel_resid;
        if (!isfinite(beta)) {
            g->status = PB_ERR_NAN;
            g->done = 1;
        } else if (g->rel_resid <= g->tol) {
            g->converged = 1;
            g->status = PB_OK;
            g->done = 1;
        } else if (g->iters >= g->maxit) {
            g->status = PB_ERR_NOCONV;
            g->done = 1;
        } else {
            g->cycles += 1;
            g->g[0] = beta;
            for (int k = 1; k <= g->m; ++k) g->g[k] = 0.0;
        }
        g->cycle_done = 0;
        g->skip = g->done;
    }
}

// V[0] = r / beta (which = 0) or V[k+1] = w / H[k+1,k] (which = 1)
__global__ void __launch_bounds__(kVThreads)
bg_scale(int which, int k, const BChunk *__restrict__ ch, const BInst *__restrict__ inst) {
    const BChunk c = ch[blockIdx.x];
    const BInst in = inst[c.inst];
    const GmresState *g = in.st;
    if (vol(&g->skip)) return;
    const double *src = which ? in.w : in.r;
    double *dst = in.V + (which ? (int64_t)(k + 1) * in.n2 : 0);
    const double inv = 1.0 / (which ? g->hnext : g->beta);
    for (int e = threadIdx.x; e < c.len; e += kVThreads) dst[c.start + e] = src[c.start + e] * inv;
}

__global__ void __launch_bounds__(kVThreads)
bg_dots(int k, const BChunk *__restrict__ ch, const BInst *__restrict__ inst, double *__restrict__ red, int nchunks,
        unsigned int *__restrict__ counters) {
    const BChunk c = ch[blockIdx.x];
    const BInst in = inst[c.inst];
    GmresState *g = in.st;
    if (vol(&g->skip)) return;
    const int v = blockIdx.y;
    const double *Vv = in.V + (int64_t)v * in.n2;
    double s = 0.0;
    for (int e = threadIdx.x; e < c.len; e += kVThreads) s += Vv[c.start + e] * in.w[c.start + e];
    s = block_sum<kVThreads>(s);
    if (threadIdx.x == 0) red[(int64_t)v * nchunks + blockIdx.x] = s;
    if (inst_last(&counters[c.inst], in.nchunk * (k + 1))) {
        for (int vv = threadIdx.x; vv <= k; vv += kVThreads) {
            double t = 0.0;
            for (int b = 0; b < in.nchunk; ++b) t += __ldcg(red + (int64_t)vv * nchunks + in.chunk0 + b);
            g->h1[vv] = t;
        }
        if (threadIdx.x == 0) counters[c.inst] = 0u;
    }
}

__global__ void __launch_bounds__(kVThreads)
bg_orth1(int k, const BChunk *__restrict__ ch, const BInst *__restrict__ inst, double *__restrict__ red, int nchunks,
         unsigned int *__restrict__ counters) {
    const BChunk c = ch[blockIdx.x];
    const BInst in = inst[c.inst];
    GmresState *g = in.st;
    if (vol(&g->skip)) return;
    __shared__ double s_h[LDH];
    for (int v = threadIdx.x; v <= k; v += kVThreads) s_h[v] = g->h1[v];
    __syncthreads();
    for (int e = threadIdx.x; e < c.len; e += kVThreads) {
        const int64_t x = c.start + e;
        double wi = in.w[x];
        for (int v = 0; v <= k; ++v) wi -= s_h[v] * in.V[(int64_t)v * in.n2 + x];
        in.w[x] = wi;
    }
    for (int v = 0; v <= k; ++v) {
        double s = 0.0;
        for (int e = threadIdx.x; e < c.len; e += kVThreads)
            s += in.V[(int64_t)v * in.n2 + c.start + e] * in.w[c.start + e];
        s = block_sum<kVThreads>(s);
        if (threadIdx.x == 0) red[(int64_t)v * nchunks + blockIdx.x] = s;
    }
    if (inst_last(&counters[c.inst], in.nchunk)) {
        for (int vv = threadIdx.x; vv <= k; vv += kVThreads) {
            double t = 0.0;
            for (int b = 0; b < in.nchunk; ++b) t += __ldcg(red + (int64_t)vv * nchunks + in.chunk0 + b);
            g->h2[vv] = t;
        }
        if (threadIdx.x == 0) counters[c.inst] = 0u;
    }
}

__global__ void __launch_bounds__(kVThreads)
bg_orth2(int k, const BChunk *__restrict__ ch, const BInst *__restrict__ inst, double *__restrict__ red,
         unsigned int *__restrict__ counters) {
    const BChunk c = ch[blockIdx.x];
    const BInst in = inst[c.inst];
    GmresState *g = in.st;
    if (vol(&g->skip)) return;
    __shared__ double s_h[LDH];
    for (int v = threadIdx.x; v <= k; v += kVThreads) s_h[v] = g->h2[v];
    __syncthreads();
    double s = 0.0;
    for (int e = threadIdx.x; e < c.len; e += kVThreads) {
        const int64_t x = c.start + e;
        double wi = in.w[x];
        for (int v = 0; v <= k; ++v) wi -= s_h[v] * in.V[(int64_t)v * in.n2 + x];
        in.w[x] = wi;
        s += wi * wi;
    }
    s = block_sum<kVThreads>(s);
    if (threadIdx.x == 0) red[blockIdx.x] = s;
    if (inst_last(&counters[c.inst], in.nchunk) && threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < in.nchunk; ++b) t += __ldcg(red + in.chunk0 + b);
        counters[c.inst] = 0u;
        const double hn = sqrt(t);
        double *H = g->H;
        for (int v = 0; v <= k; ++v) H[v + k * LDH] = g->h1[v] + g->h2[v];
        H[k + 1 + k * LDH] = hn;
        g->hnext = hn;
        for (int i = 0; i < k; ++i) {
            const double a0 = H[i + k * LDH], b0 = H[i + 1 + k * LDH];
            H[i + k * LDH] = g->cs[i] * a0 + g->sn[i] * b0;
            H[i + 1 + k * LDH] = -g->sn[i] * a0 + g->cs[i] * b0;
        }
        const double a0 = H[k + k * LDH], b0 = H[k + 1 + k * LDH];
        const double d = hypot(a0, b0);
        const double cc = d > 0.0 ? a0 / d : 1.0, sn = d > 0.0 ? b0 / d : 0.0;
        g->cs[k] = cc;
        g->sn[k] = sn;
        H[k + k * LDH] = d;
        H[k + 1 + k * LDH] = 0.0;
        g->g[k + 1] = -sn * g->g[k];
        g->g[k] = cc * g->g[k];
        g->k = k + 1;
        g->iters += 1;
        const double est = fabs(g->g[k + 1]) / g->bnorm;
        g->est_resid = est;
        if (!isfinite(hn) || !isfinite(d) || !isfinite(est) || !(d > 0.0)) {
            g->status = PB_ERR_NAN;
            g->done = 1;
        }
        g->cycle_done = (est <= g->tol) || (g->iters >= g->maxit) || !(hn > 0.0) || (k + 1 >= g->m) || g->done;
        g->skip = g->done || g->cycle_done;
    }
}

// back substitution and x += V y, one block per chunk (block 0 of an instance
// solves the small triangular system into shared memory; every block redoes
// it, which is cheaper than another launch for k <= 64)
__global__ void __launch_bounds__(kVThreads)
bg_update_x(const BChunk *__restrict__ ch, const BInst *__restrict__ inst) {
    const BChunk c = ch[blockIdx.x];
    const BInst in = inst[c.inst];
    const GmresState *g = in.st;
    const int kk = g->k;
    if (kk == 0 || g->status != PB_OK || vol(&g->done)) return;
    __shared__ double s_y[kMaxRestart];
    if (threadIdx.x == 0) {
        const double *H = g->H;
        for (int i = kk - 1; i >= 0; --i) {
            double t = g->g[i];
            for (int j = i + 1; j < kk; ++j) t -= H[i + j * LDH] * s_y[j];
            s_y[i] = t / H[i + i * LDH];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < c.len; e += kVThreads) {
        const int64_t xi = c.start + e;
        double t = in.x[xi];
        for (int v = 0; v < kk; ++v) t += s_y[v] * in.V[(int64_t)v * in.n2 + xi];
        in.x[xi] = t;
    }
}

// per-surface activity flags for the product, and x_is_zero bookkeeping
// act_*: 1 when a surface's product is needed (read by the batched product);
// act_*[nsurf + s] holds the negation (the skip flag of a single-surface product).
__global__ void bg_flags(const BSurf *__restrict__ surf, int nsurf, const BInst *__restrict__ inst, int *act_step,
                         int *act_ax, int clear_x_zero) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsurf) return;
    const BSurf sf = surf[s];
    int step = 0, ax = 0;
    for (int r = 0; r < sf.nrhs; ++r) {
        GmresState *g = inst[sf.inst0 + r].st;
        if (clear_x_zero && g->k > 0 && g->status == PB_OK) g->x_is_zero = 0;
        step |= !g->skip;
        ax |= (!g->done && !g->x_is_zero);
    }
    act_step[s] = step;
    act_ax[s] = ax;
    act_step[nsurf + s] = !step;
    act_ax[nsurf + s] = !ax;
}

__global__ void bg_status(const BInst *__restrict__ inst, int nq, BStatus *out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const GmresState *g = inst[q].st;
    out[q] = BStatus{g->done, g->converged, g->status, g->iters, g->cycles, 0, g->rel_resid};
}

}  // namespace

// ---------------------------------------------------------------------------
// Engine
// ---------------------------------------------------------------------------
Engine::Engine(cudaStream_t stream, int device, int num_sms, int m, double tol, int maxit)
    : stream_(stream), device_(device), num_sms_(num_sms), m_(m), maxit_(maxit), tol_(tol) {}

Engine::~Engine() {
    for (EngineMember *mb : members_) {
        cudaFreeAsync(mb->q, stream_);
        cudaFreeAsync(mb->vec, stream_);
        cudaFreeAsync(mb->st, stream_);
        delete mb;
    }
    void *bufs[] = {d_surf_, d_inst_, d_ch_, cnt_inst_, cnt_tile_, evals_, act_step_, act_ax_, red_, part_, scalar_,
                    d_status_};
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, stream_);
    if (gexec_) cudaGraphExecDestroy(gexec_);
    if (graph_) cudaGraphDestroy(graph_);
    cudaStreamSynchronize(stream_);
    if (h_status_) cudaFreeHost(h_status_);
    for (cudaEvent_t e : ev_) cudaEventDestroy(e);
}

pb_status Engine::fail(pb_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(error, sizeof(error), fmt, ap);
    va_end(ap);
    return set_error(nullptr, s, "%s", error);
}

pb_status Engine::cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? PB_ERR_OOM : PB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

pb_status Engine::grow(void **p, size_t *cap, size_t need, size_t elem, const char *what) {
    if (need <= *cap && *p) return PB_OK;
    if (*p) cudaFreeAsync(*p, stream_);
    *p = nullptr;
    size_t n = need < 16 ? 16 : need + need / 2;
    cudaError_t e = pool_alloc(p, n * elem, stream_);
    if (e != cudaSuccess) {
        *cap = 0;
        *p = nullptr;
        return cuda_fail(e, what);
    }
    *cap = n;
    return PB_OK;
}

int64_t Engine::member_bytes(int64_t N, int nrhs, int m) {
    return (int64_t)nrhs * ((int64_t)(m + 5) * 2 * N * (int64_t)sizeof(double) + (int64_t)sizeof(GmresState));
}

EngineMember *Engine::add(pb_ctx *surf, const double *charges_host, int64_t nc, int nrhs, uint64_t tag,
                          pb_status *st) {
    *st = PB_OK;
    if (!surf || nrhs < 1 || nrhs > kEngineMaxRhs || nc < 0 || (nc > 0 && !charges_host)) {
        *st = fail(PB_ERR_ARG, "engine: bad member arguments");
        return nullptr;
    }
    EngineMember *mb = new EngineMember();
    mb->surf = surf;
    mb->nrhs = nrhs;
    mb->nc = nc;
    mb->tag = tag;
    const int64_t n2 = 2 * surf->N;
    const size_t per = (size_t)(m_ + 5) * n2;
    cudaError_t e = pool_alloc((void **)&mb->vec, per * nrhs * sizeof(double), stream_);
    if (e == cudaSuccess) e = pool_alloc((void **)&mb->st, nrhs * sizeof(GmresState), stream_);
    if (e == cudaSuccess) e = pool_alloc((void **)&mb->q, (nc > 0 ? nc * nrhs : 1) * sizeof(Charge4), stream_);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (mb->vec) cudaFreeAsync(mb->vec, stream_);
        if (mb->st) cudaFreeAsync(mb->st, stream_);
        if (mb->q) cudaFreeAsync(mb->q, stream_);
        delete mb;
        *st = cuda_fail(e, "engine member allocation");
        return nullptr;
    }
    mb->bytes = member_bytes(surf->N, nrhs, m_) + nc * nrhs * (int64_t)sizeof(Charge4);
    // charges, centred like the surface's geometry
    std::vector<Charge4> hq((size_t)(nc * nrhs));
    for (int64_t k = 0; k < nc * nrhs; ++k)
        hq[k] = Charge4{charges_host[4 * k] - surf->center[0], charges_host[4 * k + 1] - surf->center[1],
                        charges_host[4 * k + 2] - surf->center[2], charges_host[4 * k + 3]};
    if (nc > 0) e = cudaMemcpyAsync(mb->q, hq.data(), hq.size() * sizeof(Charge4), cudaMemcpyHostToDevice, stream_);
    // initial states (x0 = 0)
    GmresState init;
    memset(&init, 0, sizeof(init));
    init.m = m_;
    init.maxit = maxit_;
    init.tol = tol_;
    init.status = PB_OK;
    init.x_is_zero = 1;
    for (int r = 0; r < nrhs && e == cudaSuccess; ++r)
        e = cudaMemcpyAsync(mb->st + r, &init, sizeof(init), cudaMemcpyHostToDevice, stream_);
    if (e == cudaSuccess) e = cudaMemsetAsync(mb->vec, 0, per * nrhs * sizeof(double), stream_);
    // the host staging vector goes out of scope: finish the copies first
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
    // b = [S1; S2] and ||b|| for every set, through the context's FP64 kernels
    Charge4 *keep_q = surf->charges;
    const int64_t keep_nc = surf->Nc;
    const cudaStream_t keep_stream = surf->stream;
    surf->stream = stream_;
    for (int r = 0; r < nrhs && e == cudaSuccess && *st == PB_OK; ++r) {
        double *b = mb->vec + (size_t)r * per;
        surf->charges = mb->q + r * nc;
        surf->Nc = nc;
        *st = source_launch(surf, b, PB_FP64);
        if (*st == PB_OK) *st = norm2_launch(surf, b, n2, &mb->st[r].bnorm);
    }
    surf->charges = keep_q;
    surf->Nc = keep_nc;
    surf->stream = keep_stream;
    if (e != cudaSuccess && *st == PB_OK) *st = cuda_fail(e, "engine member initialisation");
    if (*st != PB_OK) {
        cudaFreeAsync(mb->vec, stream_);
        cudaFreeAsync(mb->st, stream_);
        cudaFreeAsync(mb->q, stream_);
        delete mb;
        return nullptr;
    }
    members_.push_back(mb);
    dirty_ = true;
    return mb;
}

void Engine::remove(EngineMember *mb) {
    for (size_t i = 0; i < members_.size(); ++i) {
        if (members_[i] == mb) {
            members_.erase(members_.begin() + i);
            break;
        }
    }
    cudaFreeAsync(mb->q, stream_);
    cudaFreeAsync(mb->vec, stream_);
    cudaFreeAsync(mb->st, stream_);
    delete mb;
    dirty_ = true;
}

pb_status Engine::rebuild() {
    std::vector<BSurf> hs;
    std::vector<BInst> hq;
    std::vector<BChunk> hch;
    surf_member_.clear();
    direct_.clear();
    int64_t tiles = 0, work = 0;
    int rmax = 1;
    for (EngineMember *mb : members_)
        if (!mb->finished && mb->nrhs > rmax) rmax = mb->nrhs;
    R_ = rmax <= 1 ? 1 : (rmax <= 2 ? 2 : (rmax <= 4 ? 4 : 8));
    const int64_t TT = (int64_t)kBThreads * bmatvec_targets(R_);
    for (size_t mi = 0; mi < members_.size(); ++mi) {
        EngineMember *mb = members_[mi];
        if (mb->finished) continue;
        pb_ctx *c = mb->surf;
        BSurf sf;
        sf.pos = c->pos32;
        sf.nrm = c->nrm32;
        sf.N = c->N;
        sf.eps = (float)c->eps;
        sf.inv_eps = (float)(1.0 / c->eps);
        sf.kappa = (float)c->kappa;
        sf.nk = (float)(-c->kappa * 1.4426950408889634);
        sf.diag1 = 0.5 * (1.0 + c->eps);
        sf.diag2 = 0.5 * (1.0 + 1.0 / c->eps);
        // a single charge set on a context whose product is the symmetric
        // kernel: its own launch of that kernel (about 23 FP32 operations per
        // ordered pair against 40 in the batched kernel); no batched work
        const bool direct = mb->nrhs == 1 && f32_variant_symmetric(c->f32_variant);
        const int64_t T = direct ? 0 : (c->N + TT - 1) / TT;
        sf.S = (c->N + kBSourceTile - 1) / kBSourceTile;
        if (direct) direct_.push_back((int)hs.size());
        sf.tile_base = tiles;
        sf.work_base = work;
        sf.inst0 = (int)hq.size();
        sf.nrhs = mb->nrhs;
        tiles += T;
        work += T * sf.S;
        const int64_t n2 = 2 * c->N;
        const size_t per = (size_t)(m_ + 5) * n2;
        for (int r = 0; r < mb->nrhs; ++r) {
            BInst in;
            double *base = mb->vec + (size_t)r * per;
            in.b = base;
            in.x = base + n2;
            in.w = base + 2 * n2;
            in.r = base + 3 * n2;
            in.V = base + 4 * n2;
            in.st = mb->st + r;
            in.n2 = n2;
            in.surf = (int)hs.size();
            in.chunk0 = (int)hch.size();
            for (int64_t s0 = 0; s0 < n2; s0 += kChunk)
                hch.push_back(BChunk{(int)hq.size(), (int)((n2 - s0) < kChunk ? (n2 - s0) : kChunk), s0});
            in.nchunk = (int)hch.size() - in.chunk0;
            hq.push_back(in);
        }
        hs.push_back(sf);
        surf_member_.push_back((int)mi);
    }
    nsurf_ = (int)hs.size();
    nq_ = (int)hq.size();
    nchunks_ = (int)hch.size();
    tiles_ = tiles;
    W_ = work;
    rhs_width = R_;
    if (gexec_) cudaGraphExecDestroy(gexec_);
    if (graph_) cudaGraphDestroy(graph_);
    gexec_ = nullptr;
    graph_ = nullptr;
    dirty_ = false;
    if (nsurf_ == 0) return PB_OK;
    int occ = 0;
    switch (R_) {
        case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bmatvec_kernel<1>, kBThreads, 0); break;
        case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bmatvec_kernel<2>, kBThreads, 0); break;
        case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bmatvec_kernel<4>, kBThreads, 0); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bmatvec_kernel<8>, kBThreads, 0); break;
    }
    if (occ < 1) occ = 1;
    G_ = (int64_t)num_sms_ * occ;
    if (G_ > W_) G_ = W_;
    ctas = G_;
    for (int si : direct_) {
        pb_ctx *c = members_[surf_member_[si]]->surf;
        const cudaStream_t keep_stream = c->stream;
        c->stream = stream_;
        pb_status ps = matvec_prepare(c);
        c->stream = keep_stream;
        if (ps != PB_OK) return fail(ps, "engine: %s", c->last_error);
    }
    pb_status s = PB_OK;
    if (s == PB_OK) s = grow((void **)&d_surf_, &cap_surf_, nsurf_, sizeof(BSurf), "engine surfaces");
    if (s == PB_OK) s = grow((void **)&d_inst_, &cap_inst_, nq_, sizeof(BInst), "engine instances");
    if (s == PB_OK) s = grow((void **)&d_ch_, &cap_ch_, nchunks_, sizeof(BChunk), "engine chunks");
    if (s == PB_OK) s = grow((void **)&cnt_inst_, &cap_cnt_inst_, nq_, sizeof(unsigned int), "engine counters");
    if (s == PB_OK) s = grow((void **)&cnt_tile_, &cap_cnt_tile_, tiles_, sizeof(unsigned int), "engine counters");
    if (s == PB_OK) s = grow((void **)&evals_, &cap_evals_, nsurf_, sizeof(unsigned long long), "engine counters");
    if (s == PB_OK) s = grow((void **)&act_step_, &cap_flags_, 2 * (size_t)nsurf_, sizeof(int), "engine flags");
    if (s == PB_OK) {
        size_t c2 = 0;
        if (act_ax_) cudaFreeAsync(act_ax_, stream_);
        act_ax_ = nullptr;
        s = grow((void **)&act_ax_, &c2, cap_flags_, sizeof(int), "engine flags");
    }
    if (s == PB_OK) s = grow((void **)&red_, &cap_red_, (size_t)(m_ + 1) * nchunks_, sizeof(double), "engine reductions");
    if (s == PB_OK) s = grow((void **)&part_, &cap_part_, (size_t)2 * G_ * 2 * R_ * TT, sizeof(double), "engine partials");
    if (s == PB_OK && !scalar_) {
        cudaError_t e = pool_alloc((void **)&scalar_, 64 * sizeof(double), stream_);
        if (e != cudaSuccess) s = cuda_fail(e, "engine scalars");
    }
    if (s == PB_OK && cap_status_ < (size_t)nq_) {
        if (d_status_) cudaFreeAsync(d_status_, stream_);
        d_status_ = nullptr;
        if (h_status_) {
            cudaStreamSynchronize(stream_);
            cudaFreeHost(h_status_);
            h_status_ = nullptr;
        }
        size_t cap = 0;
        s = grow((void **)&d_status_, &cap, nq_, sizeof(BStatus), "engine status");
        if (s == PB_OK) {
            cudaError_t e = cudaMallocHost((void **)&h_status_, cap * sizeof(BStatus));
            if (e != cudaSuccess) s = cuda_fail(e, "engine pinned status");
            else cap_status_ = cap;
        }
    }
    if (s != PB_OK) return s;
    cudaError_t e = cudaMemcpyAsync(d_surf_, hs.data(), nsurf_ * sizeof(BSurf), cudaMemcpyHostToDevice, stream_);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_inst_, hq.data(), nq_ * sizeof(BInst), cudaMemcpyHostToDevice, stream_);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ch_, hch.data(), nchunks_ * sizeof(BChunk), cudaMemcpyHostToDevice, stream_);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt_inst_, 0, nq_ * sizeof(unsigned int), stream_);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt_tile_, 0, tiles_ * sizeof(unsigned int), stream_);
    if (e == cudaSuccess) e = cudaMemsetAsync(evals_, 0, nsurf_ * sizeof(unsigned long long), stream_);
    // the staging vectors are pageable and local: wait for the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
    if (e != cudaSuccess) return cuda_fail(e, "engine table upload");
    last_evals_.assign(nsurf_, 0ull);
    // flags from the current states (members may be mid-solve)
    bg_flags<<<(nsurf_ + 127) / 128, 128, 0, stream_>>>(d_surf_, nsurf_, d_inst_, act_step_, act_ax_, 0);
    count_launch();
    e = cudaGetLastError();
    return e == cudaSuccess ? PB_OK : cuda_fail(e, "engine flags");
}

void Engine::enqueue_cycle() {
    const int sb = (nsurf_ + 127) / 128, qb = (nq_ + 127) / 128;
    auto mv = [&](int usel, int k, const int *act) {
        if (timing_ && ev_used_ + 2 <= (int)ev_.size()) cudaEventRecord(ev_[ev_used_], stream_);
        if (W_ > 0) {
            switch (R_) {
                case 1: bmatvec_kernel<1><<<(unsigned)G_, kBThreads, 0, stream_>>>(d_surf_, nsurf_, d_inst_, W_, G_, usel, k, act, part_, cnt_tile_, evals_); break;
                case 2: bmatvec_kernel<2><<<(unsigned)G_, kBThreads, 0, stream_>>>(d_surf_, nsurf_, d_inst_, W_, G_, usel, k, act, part_, cnt_tile_, evals_); break;
                case 4: bmatvec_kernel<4><<<(unsigned)G_, kBThreads, 0, stream_>>>(d_surf_, nsurf_, d_inst_, W_, G_, usel, k, act, part_, cnt_tile_, evals_); break;
                default: bmatvec_kernel<8><<<(unsigned)G_, kBThreads, 0, stream_>>>(d_surf_, nsurf_, d_inst_, W_, G_, usel, k, act, part_, cnt_tile_, evals_); break;
            }
            ++cycle_kernels_;
            ++cycle_mv_;
        }
        // single-surface symmetric products; their skip flag is the negated
        // activity flag, and their evaluation counter the engine's
        for (int si : direct_) {
            EngineMember *mb = members_[surf_member_[si]];
            pb_ctx *c = mb->surf;
            const int64_t n2 = 2 * c->N;
            const double *u = usel ? mb->vec + 4 * n2 + (int64_t)k * n2 : mb->vec + n2;   // V[k] or x
            double *y = mb->vec + 2 * n2;                                                  // w
            const cudaStream_t keep_stream = c->stream;
            unsigned long long *keep_count = c->mv_count;
            const bool keep_prof = c->prof_on;
            c->stream = stream_;
            c->mv_count = evals_ + si;
            c->prof_on = false;
            matvec_launch(c, u, y, PB_FP32PAIR, act + nsurf_ + si);
            c->stream = keep_stream;
            c->mv_count = keep_count;
            c->prof_on = keep_prof;
            cycle_kernels_ += 2;
            ++cycle_mv_;
        }
        if (timing_ && ev_used_ + 2 <= (int)ev_.size()) {
            cudaEventRecord(ev_[ev_used_ + 1], stream_);
            ev_used_ += 2;
        }
    };
    mv(0, 0, act_ax_);
    bg_cycle_start<<<nchunks_, kVThreads, 0, stream_>>>(1, d_ch_, d_inst_, red_, cnt_inst_);
    bg_scale<<<nchunks_, kVThreads, 0, stream_>>>(0, 0, d_ch_, d_inst_);
    bg_flags<<<sb, 128, 0, stream_>>>(d_surf_, nsurf_, d_inst_, act_step_, act_ax_, 0);
    cycle_kernels_ += 3;
    for (int k = 0; k < m_; ++k) {
        mv(1, k, act_step_);
        bg_dots<<<dim3(nchunks_, k + 1), kVThreads, 0, stream_>>>(k, d_ch_, d_inst_, red_, nchunks_, cnt_inst_);
        bg_orth1<<<nchunks_, kVThreads, 0, stream_>>>(k, d_ch_, d_inst_, red_, nchunks_, cnt_inst_);
        bg_orth2<<<nchunks_, kVThreads, 0, stream_>>>(k, d_ch_, d_inst_, red_, cnt_inst_);
        bg_scale<<<nchunks_, kVThreads, 0, stream_>>>(1, k, d_ch_, d_inst_);
        bg_flags<<<sb, 128, 0, stream_>>>(d_surf_, nsurf_, d_inst_, act_step_, act_ax_, 0);
        cycle_kernels_ += 5;
    }
    bg_update_x<<<nchunks_, kVThreads, 0, stream_>>>(d_ch_, d_inst_);
    bg_flags<<<sb, 128, 0, stream_>>>(d_surf_, nsurf_, d_inst_, act_step_, act_ax_, 1);
    bg_status<<<qb, 128, 0, stream_>>>(d_inst_, nq_, d_status_);
    cycle_kernels_ += 3;
}

pb_status Engine::cycle(bool use_graph, bool time_products) {
    pb_status s = PB_OK;
    if (dirty_ && (s = rebuild()) != PB_OK) return s;
    if (nsurf_ == 0) return PB_OK;
    cudaError_t e = cudaSuccess;
    if (time_products) {
        use_graph = false;
        if (ev_.empty()) {
            ev_.resize(2 * (m_ + 2), nullptr);
            for (auto &x : ev_)
                if ((e = cudaEventCreate(&x)) != cudaSuccess) return cuda_fail(e, "engine events");
        }
        ev_used_ = 0;
    }
    timing_ = time_products;
    if (use_graph && stream_ != nullptr && !gexec_) {
        cycle_kernels_ = 0;
        cycle_mv_ = 0;
        e = cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue_cycle();
            cudaError_t e2 = cudaStreamEndCapture(stream_, &graph_);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec_, graph_, 0);
        if (e != cudaSuccess) return cuda_fail(e, "engine graph capture");
        kernels_per_cycle_ = cycle_kernels_;
        mv_per_cycle_ = cycle_mv_;
    }
    if (use_graph && gexec_) {
        e = cudaGraphLaunch(gexec_, stream_);
        count_launches(kernels_per_cycle_);
        matvec_launches += mv_per_cycle_;
    } else {
        cycle_kernels_ = 0;
        cycle_mv_ = 0;
        enqueue_cycle();
        count_launches(cycle_kernels_);
        matvec_launches += cycle_mv_;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_status_, d_status_, nq_ * sizeof(BStatus), cudaMemcpyDeviceToHost, stream_);
    std::vector<unsigned long long> ev(nsurf_, 0ull);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ev.data(), evals_, nsurf_ * sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
    if (e != cudaSuccess) return cuda_fail(e, "engine cycle");
    for (int i = 0; timing_ && i + 1 < ev_used_; i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev_[i], ev_[i + 1]) == cudaSuccess) matvec_ms += ms;
    }
    timing_ = false;
    ++cycles_run;
    int q = 0;
    for (int si = 0; si < nsurf_; ++si) {
        EngineMember *mb = members_[surf_member_[si]];
        const int64_t pairs = mb->surf->N * (mb->surf->N - 1);
        pair_evals += (int64_t)(ev[si] - last_evals_[si]) * pairs;
        pair_products += (int64_t)(ev[si] - last_evals_[si]) * pairs * mb->nrhs;
        last_evals_[si] = ev[si];
        bool all = true;
        for (int r = 0; r < mb->nrhs; ++r, ++q) {
            mb->status[r] = h_status_[q];
            all &= h_status_[q].done != 0;
        }
        if (all && !mb->finished) {
            mb->finished = true;
            dirty_ = true;        // the next cycle's work split covers the running surfaces only
        }
    }
    return PB_OK;
}

pb_status Engine::energies(EngineMember *mb, double *out) {
    pb_ctx *c = mb->surf;
    const int64_t n2 = 2 * c->N;
    const size_t per = (size_t)(m_ + 5) * n2;
    if (!scalar_) {
        cudaError_t e = pool_alloc((void **)&scalar_, 64 * sizeof(double), stream_);
        if (e != cudaSuccess) return cuda_fail(e, "engine scalars");
    }
    Charge4 *keep_q = c->charges;
    const int64_t keep_nc = c->Nc;
    const cudaStream_t keep_stream = c->stream;
    c->stream = stream_;
    pb_status s = PB_OK;
    for (int r = 0; r < mb->nrhs && s == PB_OK; ++r) {
        c->charges = mb->q + r * mb->nc;
        c->Nc = mb->nc;
        s = energy_launch(c, mb->vec + (size_t)r * per + n2, PB_FP64, scalar_ + (r % 64));
    }
    c->charges = keep_q;
    c->Nc = keep_nc;
    c->stream = keep_stream;
    if (s != PB_OK) return s;
    cudaError_t e = cudaMemcpyAsync(out, scalar_, mb->nrhs * sizeof(double), cudaMemcpyDeviceToHost, stream_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
    return e == cudaSuccess ? PB_OK : cuda_fail(e, "engine energies");
}

}  // namespace pb

// ---------------------------------------------------------------------------
// pb_batch_solve: a fixed set of members solved to completion
// ---------------------------------------------------------------------------
using namespace pb;

extern "C" pb_status pb_batch_solve(pb_ctx *const *ctxs, int nsurf, const double *const *charges, const int64_t *nc,
                                    const int *nrhs, const pb_solve_opts *opts, int use_graph, double *energies,
                                    pb_batch_info *info) {
    if (!ctxs || nsurf < 1 || !charges || !nc || !nrhs || !energies)
        return set_error(nullptr, PB_ERR_ARG, "pb_batch_solve: NULL or empty argument");
    pb_ctx *lead = ctxs[0];
    if (!lead) return set_error(nullptr, PB_ERR_ARG, "pb_batch_solve: NULL context");
    pb_solve_opts o{10, 1e-4, 1000, PB_FP32PAIR, 0, PB_FP64};
    if (opts) {
        o = *opts;
        if (o.restart == 0) o.restart = 10;
        if (o.tol == 0.0) o.tol = 1e-4;
        if (o.maxit == 0) o.maxit = 1000;
    }
    if (o.restart < 1 || o.restart > kMaxRestart || !(o.tol > 0.0) || o.maxit < 1)
        return set_error(lead, PB_ERR_ARG, "pb_batch_solve: bad solve options");
    if (o.prec != PB_FP32PAIR)
        return set_error(lead, PB_ERR_ARG, "pb_batch_solve: the batched product is FP32-pair only");
    for (int s = 0; s < nsurf; ++s) {
        if (!ctxs[s] || ctxs[s]->device != lead->device)
            return set_error(lead, PB_ERR_ARG, "pb_batch_solve: context %d is NULL or on another device", s);
        if (nrhs[s] < 1 || nrhs[s] > kEngineMaxRhs)
            return set_error(lead, PB_ERR_ARG, "pb_batch_solve: nrhs[%d] = %d not in [1, %d]", s, nrhs[s],
                             kEngineMaxRhs);
        if (nc[s] < 0 || (nc[s] > 0 && !charges[s]))
            return set_error(lead, PB_ERR_ARG, "pb_batch_solve: bad charges for surface %d", s);
    }
    Engine eng(lead->stream, lead->device, lead->num_sms, o.restart, o.tol, o.maxit);
    std::vector<EngineMember *> mem(nsurf, nullptr);
    pb_status s = PB_OK;
    for (int i = 0; i < nsurf && s == PB_OK; ++i) mem[i] = eng.add(ctxs[i], charges[i], nc[i], nrhs[i], (uint64_t)i, &s);
    if (s != PB_OK) return set_error(lead, s, "%s", eng.error);
    bool all = false;
    for (int cyc = 0; cyc < o.maxit + 2 && s == PB_OK && !all; ++cyc) {
        s = eng.cycle(use_graph == 1, use_graph == 2);
        all = true;
        for (EngineMember *mb : mem) all &= mb->finished;
    }
    if (s != PB_OK) return set_error(lead, s, "%s", eng.error);
    int k = 0, nconv = 0, nq = 0, iters_max = 0;
    int64_t iters_sum = 0;
    double resid_max = 0.0;
    pb_status worst = PB_OK;
    for (int i = 0; i < nsurf && s == PB_OK; ++i) {
        s = eng.energies(mem[i], energies + k);
        for (int r = 0; r < nrhs[i]; ++r) {
            const BStatus &b = mem[i]->status[r];
            nconv += b.converged;
            ++nq;
            iters_max = b.iters > iters_max ? b.iters : iters_max;
            iters_sum += b.iters;
            resid_max = b.rel_resid > resid_max ? b.rel_resid : resid_max;
            if (b.status == PB_ERR_NAN) worst = PB_ERR_NAN;
            else if (!b.converged && worst == PB_OK) worst = PB_ERR_NOCONV;
        }
        k += nrhs[i];
    }
    if (s != PB_OK) return set_error(lead, s, "%s", eng.error);
    if (info) {
        info->instances = nq;
        info->converged = nconv;
        info->cycles = eng.cycles_run;
        info->iters_max = iters_max;
        info->iters_sum = iters_sum;
        info->rel_resid_max = resid_max;
        info->rhs_width = eng.rhs_width;
        info->ctas = eng.ctas;
        info->pair_evals = eng.pair_evals;
        info->pair_products = eng.pair_products;
        info->matvec_launches = eng.matvec_launches;
        info->matvec_ms = eng.matvec_ms;
    }
    if (worst != PB_OK)
        return set_error(lead, worst, "pb_batch_solve: %d of %d instances did not converge", nq - nconv, nq);
    return PB_OK;
}
