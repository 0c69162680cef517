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
// kernels over a flat concatenation of all instance vectors, cut into chunks
// that never straddle two instances; per-instance sums are fixed-order
// two-stage reductions finished by the last chunk to arrive.  Instances that
// have converged are skipped, and a surface whose instances are all idle is
// skipped by the product.  One restart cycle of the whole batch can be
// captured in a CUDA graph and replayed.
#include <math.h>
#include <string.h>

#include <vector>

#include "fastmath.cuh"
#include "pb_internal.cuh"
#include "reduce.cuh"

namespace pb {
namespace {

constexpr int kBThreads = 128;          // product kernel: one target per thread
constexpr int kBSourceTile = 128;
constexpr int kChunk = 4096;            // vector chunk (elements) of the GMRES kernels
constexpr int kVThreads = 256;
constexpr int kMaxRhs = 8;
constexpr int LDH = kMaxRestart + 1;

struct BSurf {
    const float4 *pos;
    const float4 *nrm;
    const double *g64;     // FP64 SoA geometry (source term)
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
    int64_t off;           // offset of the instance's 2N-vector in the flat arrays
    int64_t n;             // N of its surface
    int surf;
    int chunk0, nchunk;    // its chunks of the flat 2N vectors
    int schunk0, nschunk;  // its chunks over the N sources (energy)
    int64_t qoff;          // first charge
    int64_t nc;
};

struct BChunk {
    int inst;
    int len;
    int64_t start;         // flat index (vector chunks) or source index (source chunks)
};

struct BStatus {
    int done, converged, status, iters, cycles, pad;
    double rel_resid;
};

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

template <int R>
__global__ void __launch_bounds__(kBThreads)
bmatvec_kernel(const BSurf *__restrict__ surf, int nsurf, const BInst *__restrict__ inst, int64_t W, int64_t G,
               const double *__restrict__ u, double *__restrict__ y, const int *__restrict__ active,
               double *__restrict__ partials, unsigned int *__restrict__ counters,
               unsigned long long *__restrict__ evaluated) {
    constexpr int BS = kBThreads, TT = kBThreads, TS = kBSourceTile;
    __shared__ float4 s_pos[TS];
    __shared__ float4 s_nrm[TS];
    __shared__ float2 s_w[R][TS];        // (W dphi, W phi) / (4 pi) per right-hand side
    __shared__ int s_last;
    const int tid = threadIdx.x;
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
        int64_t i = a * TT + tid;
        const int64_t ic = i < N ? i : N - 1;
        const float4 qi = sf.pos[ic], ni = sf.nrm[ic];
        double acc1[R], acc2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { acc1[r] = 0.0; acc2[r] = 0.0; }

        for (int64_t st = s_first; st < s_end; ++st) {
            __syncthreads();
            {
                const int64_t j = st * TS + tid;
                if (j < N) {
                    const float4 q = sf.pos[j], n = sf.nrm[j];
                    s_pos[tid] = q;
                    s_nrm[tid] = n;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (r < sf.nrhs) {
                            const int64_t off = inst[sf.inst0 + r].off;
                            s_w[r][tid] = make_float2((float)u[off + N + j] * q.w, (float)u[off + j] * q.w);
                        } else {
                            s_w[r][tid] = make_float2(0.f, 0.f);
                        }
                    }
                }
            }
            __syncthreads();
            const int cnt = (int)((N - st * TS) < TS ? (N - st * TS) : TS);
            float f1[R], f2[R];
#pragma unroll
            for (int r = 0; r < R; ++r) { f1[r] = 0.f; f2[r] = 0.f; }
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 sp = s_pos[jj];
                const float4 sn = s_nrm[jj];
                const float dx = qi.x - sp.x, dy = qi.y - sp.y, dz = qi.z - sp.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float inv = fminf(rsqrt_approx(r2), 1e12f);   // self pair: every term exactly 0
                const float rho = r2 * inv;
                const float e = exp2_approx(sf.nk * rho);
                const float kr = sf.kappa * rho;
                const float e1 = fmaf(e, kr, e);
                const float inv2 = inv * inv;
                const float inv3 = inv2 * inv;
                const float cx = fmaf(dx, ni.x, fmaf(dy, ni.y, dz * ni.z));
                const float cy = fmaf(dx, sn.x, fmaf(dy, sn.y, dz * sn.z));
                const float nn = fmaf(ni.x, sn.x, fmaf(ni.y, sn.y, ni.z * sn.z));
                const float k1 = (1.f - e) * inv;
                const float k2 = fmaf(sf.eps, e1, -1.f) * cy * inv3;
                const float k3 = fmaf(e1, sf.inv_eps, -1.f) * cx * inv3;
                const float p3 = fmaf(kr, kr + 3.f, 3.f);
                const float e3 = fmaf(e, p3, -3.f);
                const float k4 = fmaf(-e3 * cx * cy, inv2, fmaf(e1, nn, -nn)) * inv3;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float2 w = s_w[r][jj];
                    f1[r] = fmaf(k1, w.x, fmaf(k2, w.y, f1[r]));
                    f2[r] = fmaf(k3, w.x, fmaf(k4, w.y, f2[r]));
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) { acc1[r] += (double)f1[r]; acc2[r] += (double)f2[r]; }
        }

        const int64_t p_tile0 = sf.work_base + a * S;
        const int64_t c0 = sk_cta_of(p_tile0, W, G), c1 = sk_cta_of(p_tile0 + S - 1, W, G);
        const int nseg = (int)(c1 - c0 + 1);
        const int64_t gtile = sf.tile_base + a;
        if (nseg == 1) {
            if (i < N) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r < sf.nrhs) {
                        const int64_t off = inst[sf.inst0 + r].off;
                        y[off + i] = sf.diag1 * u[off + i] - acc1[r];
                        y[off + N + i] = sf.diag2 * u[off + N + i] - acc2[r];
                    }
                }
            }
        } else {
            const int64_t slot = 2 * c + (gtile == first_tile ? 0 : 1);
            double *mine = partials + slot * (2 * R * TT);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                mine[(2 * r) * TT + tid] = acc1[r];
                mine[(2 * r + 1) * TT + tid] = acc2[r];
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) s_last = (atomicAdd(&counters[gtile], 1u) == (unsigned int)(nseg - 1));
            __syncthreads();
            if (s_last) {
                __threadfence();
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
                        s1[r] += __ldcg(pp + (2 * r) * TT + tid);
                        s2[r] += __ldcg(pp + (2 * r + 1) * TT + tid);
                    }
                }
                if (i < N) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (r < sf.nrhs) {
                            const int64_t off = inst[sf.inst0 + r].off;
                            y[off + i] = sf.diag1 * u[off + i] - s1[r];
                            y[off + N + i] = sf.diag2 * u[off + N + i] - s2[r];
                        }
                    }
                }
                if (tid == 0) counters[gtile] = 0u;
            }
        }
        p += s_end - s_first;
    }
}

// ---- batched GMRES vector kernels (one block per chunk) ----------------------
__global__ void __launch_bounds__(kVThreads)
bg_norm(const double *__restrict__ v, const BChunk *__restrict__ ch, const BInst *__restrict__ inst,
        double *__restrict__ red, unsigned int *__restrict__ counters, GmresState *st) {
    const BChunk c = ch[blockIdx.x];
    double s = 0.0;
    for (int k = threadIdx.x; k < c.len; k += kVThreads) { const double t = v[c.start + k]; s += t * t; }
    s = block_sum<kVThreads>(s);
    if (threadIdx.x == 0) red[blockIdx.x] = s;
    const BInst q = inst[c.inst];
    if (inst_last(&counters[c.inst], q.nchunk) && threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < q.nchunk; ++b) t += __ldcg(red + q.chunk0 + b);
        st[c.inst].bnorm = sqrt(t);
        counters[c.inst] = 0u;
    }
}

__global__ void __launch_bounds__(kVThreads)
bg_cycle_start(const double *__restrict__ rhs, const double *__restrict__ Ax, double *__restrict__ r,
               const BChunk *__restrict__ ch, const BInst *__restrict__ inst, double *__restrict__ red,
               unsigned int *__restrict__ counters, GmresState *st) {
    const BChunk c = ch[blockIdx.x];
    GmresState *g = st + c.inst;
    if (vol(&g->done)) return;
    const bool zero = vol(&g->x_is_zero) != 0;
    double s = 0.0;
    for (int k = threadIdx.x; k < c.len; k += kVThreads) {
        const int64_t e = c.start + k;
        const double ri = zero ? rhs[e] : rhs[e] - Ax[e];
        r[e] = ri;
        s += ri * ri;
    }
    s = block_sum<kVThreads>(s);
    if (threadIdx.x == 0) red[blockIdx.x] = s;
    const BInst q = inst[c.inst];
    if (inst_last(&counters[c.inst], q.nchunk) && threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < q.nchunk; ++b) t += __ldcg(red + q.chunk0 + b);
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

__global__ void __launch_bounds__(kVThreads)
bg_scale(const double *__restrict__ src, double *__restrict__ dst, const BChunk *__restrict__ ch,
         const GmresState *st, int which) {
    const BChunk c = ch[blockIdx.x];
    const GmresState *g = st + c.inst;
    if (vol(&g->skip)) return;
    const double inv = 1.0 / (which ? g->hnext : g->beta);
    for (int k = threadIdx.x; k < c.len; k += kVThreads) dst[c.start + k] = src[c.start + k] * inv;
}

__global__ void __launch_bounds__(kVThreads)
bg_dots(const double *__restrict__ V, int64_t L, const double *__restrict__ w, int k, const BChunk *__restrict__ ch,
        const BInst *__restrict__ inst, double *__restrict__ red, int nchunks, unsigned int *__restrict__ counters,
        GmresState *st) {
    const BChunk c = ch[blockIdx.x];
    GmresState *g = st + c.inst;
    if (vol(&g->skip)) return;
    const int v = blockIdx.y;
    const double *Vv = V + (int64_t)v * L;
    double s = 0.0;
    for (int e = threadIdx.x; e < c.len; e += kVThreads) s += Vv[c.start + e] * w[c.start + e];
    s = block_sum<kVThreads>(s);
    if (threadIdx.x == 0) red[(int64_t)v * nchunks + blockIdx.x] = s;
    const BInst q = inst[c.inst];
    if (inst_last(&counters[c.inst], q.nchunk * (k + 1))) {
        for (int vv = threadIdx.x; vv <= k; vv += kVThreads) {
            double t = 0.0;
            for (int b = 0; b < q.nchunk; ++b) t += __ldcg(red + (int64_t)vv * nchunks + q.chunk0 + b);
            g->h1[vv] = t;
        }
        if (threadIdx.x == 0) counters[c.inst] = 0u;
    }
}

__global__ void __launch_bounds__(kVThreads)
bg_orth1(const double *__restrict__ V, int64_t L, double *__restrict__ w, int k, const BChunk *__restrict__ ch,
         const BInst *__restrict__ inst, double *__restrict__ red, int nchunks, unsigned int *__restrict__ counters,
         GmresState *st) {
    const BChunk c = ch[blockIdx.x];
    GmresState *g = st + c.inst;
    if (vol(&g->skip)) return;
    __shared__ double s_h[LDH];
    for (int v = threadIdx.x; v <= k; v += kVThreads) s_h[v] = g->h1[v];
    __syncthreads();
    for (int e = threadIdx.x; e < c.len; e += kVThreads) {
        const int64_t x = c.start + e;
        double wi = w[x];
        for (int v = 0; v <= k; ++v) wi -= s_h[v] * V[(int64_t)v * L + x];
        w[x] = wi;
    }
    for (int v = 0; v <= k; ++v) {
        double s = 0.0;
        for (int e = threadIdx.x; e < c.len; e += kVThreads) s += V[(int64_t)v * L + c.start + e] * w[c.start + e];
        s = block_sum<kVThreads>(s);
        if (threadIdx.x == 0) red[(int64_t)v * nchunks + blockIdx.x] = s;
    }
    const BInst q = inst[c.inst];
    if (inst_last(&counters[c.inst], q.nchunk)) {
        for (int vv = threadIdx.x; vv <= k; vv += kVThreads) {
            double t = 0.0;
            for (int b = 0; b < q.nchunk; ++b) t += __ldcg(red + (int64_t)vv * nchunks + q.chunk0 + b);
            g->h2[vv] = t;
        }
        if (threadIdx.x == 0) counters[c.inst] = 0u;
    }
}

__global__ void __launch_bounds__(kVThreads)
bg_orth2(const double *__restrict__ V, int64_t L, double *__restrict__ w, int k, const BChunk *__restrict__ ch,
         const BInst *__restrict__ inst, double *__restrict__ red, unsigned int *__restrict__ counters, GmresState *st) {
    const BChunk c = ch[blockIdx.x];
    GmresState *g = st + c.inst;
    if (vol(&g->skip)) return;
    __shared__ double s_h[LDH];
    for (int v = threadIdx.x; v <= k; v += kVThreads) s_h[v] = g->h2[v];
    __syncthreads();
    double s = 0.0;
    for (int e = threadIdx.x; e < c.len; e += kVThreads) {
        const int64_t x = c.start + e;
        double wi = w[x];
        for (int v = 0; v <= k; ++v) wi -= s_h[v] * V[(int64_t)v * L + x];
        w[x] = wi;
        s += wi * wi;
    }
    s = block_sum<kVThreads>(s);
    if (threadIdx.x == 0) red[blockIdx.x] = s;
    const BInst q = inst[c.inst];
    if (inst_last(&counters[c.inst], q.nchunk) && threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < q.nchunk; ++b) t += __ldcg(red + q.chunk0 + b);
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

__global__ void bg_trisolve(GmresState *st, int nq) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    GmresState *g = st + q;
    const int kk = g->k;
    if (kk == 0 || g->status != PB_OK) return;
    const double *H = g->H;
    for (int i = kk - 1; i >= 0; --i) {
        double t = g->g[i];
        for (int j = i + 1; j < kk; ++j) t -= H[i + j * LDH] * g->y[j];
        g->y[i] = t / H[i + i * LDH];
    }
}

__global__ void __launch_bounds__(kVThreads)
bg_update_x(const double *__restrict__ V, int64_t L, double *__restrict__ x, const BChunk *__restrict__ ch,
            GmresState *st) {
    const BChunk c = ch[blockIdx.x];
    GmresState *g = st + c.inst;
    const int kk = g->k;
    if (kk == 0 || g->status != PB_OK || vol(&g->done)) return;
    __shared__ double s_y[kMaxRestart];
    for (int v = threadIdx.x; v < kk; v += kVThreads) s_y[v] = g->y[v];
    __syncthreads();
    for (int e = threadIdx.x; e < c.len; e += kVThreads) {
        const int64_t xi = c.start + e;
        double t = x[xi];
        for (int v = 0; v < kk; ++v) t += s_y[v] * V[(int64_t)v * L + xi];
        x[xi] = t;
    }
}

// per-surface activity flags for the product, and x_is_zero bookkeeping
__global__ void bg_flags(const BSurf *__restrict__ surf, int nsurf, GmresState *st, int *act_step, int *act_ax,
                         int clear_x_zero) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsurf) return;
    const BSurf sf = surf[s];
    int step = 0, ax = 0;
    for (int r = 0; r < sf.nrhs; ++r) {
        GmresState *g = st + sf.inst0 + r;
        if (clear_x_zero && g->k > 0) g->x_is_zero = 0;
        step |= !g->skip;
        ax |= (!g->done && !g->x_is_zero);
    }
    act_step[s] = step;
    act_ax[s] = ax;
}

__global__ void bg_status(const GmresState *st, int nq, BStatus *out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const GmresState *g = st + q;
    out[q] = BStatus{g->done, g->converged, g->status, g->iters, g->cycles, 0, g->rel_resid};
}

__global__ void bg_init(GmresState *st, int nq, int m, int maxit, double tol) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    GmresState *g = st + q;
    g->m = m;
    g->maxit = maxit;
    g->tol = tol;
    g->k = 0;
    g->iters = 0;
    g->cycles = 0;
    g->cycle_done = 0;
    g->done = 0;
    g->skip = 0;
    g->converged = 0;
    g->status = PB_OK;
    g->x_is_zero = 1;
    g->bnorm = 0.0;
}

// b = [S1; S2] (Eq. (11)) for every instance; one block per source chunk of 256 targets
__global__ void __launch_bounds__(kVThreads)
bg_source(const BChunk *__restrict__ sch, const BInst *__restrict__ inst, const BSurf *__restrict__ surf,
          const Charge4 *__restrict__ q, const double *__restrict__ inv_eps1, double *__restrict__ b) {
    const BChunk c = sch[blockIdx.x];
    const BInst in = inst[c.inst];
    const BSurf sf = surf[in.surf];
    const int64_t N = sf.N;
    const int64_t i = c.start + threadIdx.x;
    const bool on = threadIdx.x < c.len;
    const int64_t ic = on ? i : c.start;
    const double px = sf.g64[ic], py = sf.g64[N + ic], pz = sf.g64[2 * N + ic];
    const double nx = sf.g64[3 * N + ic], ny = sf.g64[4 * N + ic], nz = sf.g64[5 * N + ic];
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k = 0; k < in.nc; ++k) {
        const Charge4 ch = q[in.qoff + k];
        const double dx = px - ch.x, dy = py - ch.y, dz = pz - ch.z;
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 > 0.0) {
            const double inv = rsqrt(r2);
            s1 += ch.q * inv;
            s2 -= ch.q * (dx * nx + dy * ny + dz * nz) * inv * inv * inv;
        }
    }
    if (on) {
        const double sc = kInv4Pi * inv_eps1[in.surf];
        b[in.off + i] = sc * s1;
        b[in.off + in.n + i] = sc * s2;
    }
}

}  // namespace
}  // namespace pb

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using namespace pb;

namespace {

template <typename T>
pb_status dalloc(pb_ctx *owner, T **p, size_t n, const char *what) {
    return ctx_alloc(owner, (void **)p, n * sizeof(T), what);
}

}  // namespace

extern "C" pb_status pb_batch_solve(pb_ctx *const *ctxs, int nsurf, const double *const *charges, const int64_t *nc,
                                    const int *nrhs, const pb_solve_opts *opts, int use_graph, double *energies,
                                    pb_batch_info *info) {
    if (!ctxs || nsurf < 1 || !charges || !nc || !nrhs || !energies)
        return set_error(nullptr, PB_ERR_ARG, "pb_batch_solve: NULL or empty argument");
    pb_ctx *lead = ctxs[0];
    if (!lead) return set_error(nullptr, PB_ERR_ARG, "pb_batch_solve: NULL context");
    pb_solve_opts o{10, 1e-4, 1000, PB_FP32PAIR, 0};
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
    int rmax = 0, nq = 0;
    for (int s = 0; s < nsurf; ++s) {
        if (!ctxs[s] || ctxs[s]->device != lead->device)
            return set_error(lead, PB_ERR_ARG, "pb_batch_solve: context %d is NULL or on another device", s);
        if (nrhs[s] < 1 || nrhs[s] > kMaxRhs)
            return set_error(lead, PB_ERR_ARG, "pb_batch_solve: nrhs[%d] = %d not in [1, %d]", s, nrhs[s], kMaxRhs);
        if (nc[s] < 0 || (nc[s] > 0 && !charges[s]))
            return set_error(lead, PB_ERR_ARG, "pb_batch_solve: bad charges for surface %d", s);
        rmax = nrhs[s] > rmax ? nrhs[s] : rmax;
        nq += nrhs[s];
    }
    const int R = rmax <= 1 ? 1 : (rmax <= 2 ? 2 : (rmax <= 4 ? 4 : 8));
    const cudaStream_t stream = lead->stream;
    const int m = o.restart;

    // host tables
    std::vector<BSurf> hs(nsurf);
    std::vector<BInst> hq(nq);
    std::vector<BChunk> hch, hsch;
    std::vector<Charge4> hcharges;
    std::vector<double> h_inv_eps1(nsurf);
    int64_t L = 0, tiles = 0, work = 0;
    int qi = 0;
    for (int s = 0; s < nsurf; ++s) {
        pb_ctx *c = ctxs[s];
        BSurf &sf = hs[s];
        sf.pos = c->pos32;
        sf.nrm = c->nrm32;
        sf.g64 = c->g64;
        sf.N = c->N;
        sf.eps = (float)c->eps;
        sf.inv_eps = (float)(1.0 / c->eps);
        sf.kappa = (float)c->kappa;
        sf.nk = (float)(-c->kappa * 1.4426950408889634);
        sf.diag1 = 0.5 * (1.0 + c->eps);
        sf.diag2 = 0.5 * (1.0 + 1.0 / c->eps);
        const int64_t T = (c->N + kBThreads - 1) / kBThreads;
        sf.S = (c->N + kBSourceTile - 1) / kBSourceTile;
        sf.tile_base = tiles;
        sf.work_base = work;
        sf.inst0 = qi;
        sf.nrhs = nrhs[s];
        tiles += T;
        work += T * sf.S;
        h_inv_eps1[s] = 1.0 / c->eps1;
        for (int r = 0; r < nrhs[s]; ++r, ++qi) {
            BInst &in = hq[qi];
            in.off = L;
            in.n = c->N;
            in.surf = s;
            in.chunk0 = (int)hch.size();
            for (int64_t st = 0; st < 2 * c->N; st += kChunk)
                hch.push_back(BChunk{qi, (int)((2 * c->N - st) < kChunk ? (2 * c->N - st) : kChunk), L + st});
            in.nchunk = (int)hch.size() - in.chunk0;
            in.schunk0 = (int)hsch.size();
            for (int64_t st = 0; st < c->N; st += kVThreads)
                hsch.push_back(BChunk{qi, (int)((c->N - st) < kVThreads ? (c->N - st) : kVThreads), st});
            in.nschunk = (int)hsch.size() - in.schunk0;
            in.qoff = (int64_t)hcharges.size();
            in.nc = nc[s];
            const double *qs = charges[s] + (int64_t)r * nc[s] * 4;
            for (int64_t k = 0; k < nc[s]; ++k)
                hcharges.push_back(Charge4{qs[4 * k] - c->center[0], qs[4 * k + 1] - c->center[1],
                                           qs[4 * k + 2] - c->center[2], qs[4 * k + 3]});
            L += 2 * c->N;
        }
    }
    const int nchunks = (int)hch.size(), nschunks = (int)hsch.size();
    int occ = 0;
    switch (R) {
        case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bmatvec_kernel<1>, kBThreads, 0); break;
        case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bmatvec_kernel<2>, kBThreads, 0); break;
        case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bmatvec_kernel<4>, kBThreads, 0); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bmatvec_kernel<8>, kBThreads, 0); break;
    }
    if (occ < 1) occ = 1;
    int64_t G = (int64_t)lead->num_sms * occ;
    if (G > work) G = work;

    // device buffers (owned by the lead context's allocator, freed below)
    BSurf *d_surf = nullptr;
    BInst *d_inst = nullptr;
    BChunk *d_ch = nullptr, *d_sch = nullptr;
    Charge4 *d_q = nullptr;
    double *d_ie = nullptr, *b = nullptr, *x = nullptr, *w = nullptr, *r = nullptr, *V = nullptr, *red = nullptr,
           *part = nullptr, *en = nullptr;
    GmresState *st = nullptr;
    BStatus *d_status = nullptr, *h_status = nullptr;
    unsigned int *cnt_inst = nullptr, *cnt_tile = nullptr;
    unsigned long long *evals = nullptr;
    int *act_step = nullptr, *act_ax = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    pb_status s = PB_OK;
    cudaError_t e = cudaSuccess;
#define BA(ptr, n, what) \
    if (s == PB_OK) s = dalloc(lead, &ptr, (size_t)(n), what)
    BA(d_surf, nsurf, "batch surfaces");
    BA(d_inst, nq, "batch instances");
    BA(d_ch, nchunks, "batch chunks");
    BA(d_sch, nschunks, "batch source chunks");
    BA(d_q, hcharges.size() > 0 ? hcharges.size() : 1, "batch charges");
    BA(d_ie, nsurf, "batch 1/eps1");
    BA(b, L, "batch rhs");
    BA(x, L, "batch x");
    BA(w, L, "batch w");
    BA(r, L, "batch r");
    BA(V, (size_t)(m + 1) * L, "batch Krylov basis");
    BA(red, (size_t)(m + 1) * (nchunks > nschunks ? nchunks : nschunks), "batch reductions");
    BA(part, (size_t)2 * G * 2 * R * kBThreads, "batch partials");
    BA(en, nq, "batch energies");
    BA(st, nq, "batch states");
    BA(d_status, nq, "batch status");
    BA(cnt_inst, nq, "batch instance counters");
    BA(cnt_tile, tiles, "batch tile counters");
    BA(evals, nsurf, "batch product counters");
    BA(act_step, nsurf, "batch flags");
    BA(act_ax, nsurf, "batch flags");
#undef BA
    if (s == PB_OK) {
        e = cudaMallocHost((void **)&h_status, nq * sizeof(BStatus));
        if (e != cudaSuccess) s = cuda_error(lead, e, "batch pinned status");
    }
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (s == PB_OK && bytes) {
            e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) s = cuda_error(lead, e, "batch upload");
        }
    };
    up(d_surf, hs.data(), nsurf * sizeof(BSurf));
    up(d_inst, hq.data(), nq * sizeof(BInst));
    up(d_ch, hch.data(), nchunks * sizeof(BChunk));
    up(d_sch, hsch.data(), nschunks * sizeof(BChunk));
    up(d_q, hcharges.data(), hcharges.size() * sizeof(Charge4));
    up(d_ie, h_inv_eps1.data(), nsurf * sizeof(double));
    // the uploads read pageable host vectors: wait before they go out of scope
    if (s == PB_OK && (e = cudaStreamSynchronize(stream)) != cudaSuccess) s = cuda_error(lead, e, "batch upload");
    if (s == PB_OK) {
        e = cudaMemsetAsync(cnt_inst, 0, nq * sizeof(unsigned int), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt_tile, 0, tiles * sizeof(unsigned int), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, L * sizeof(double), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(w, 0, L * sizeof(double), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(evals, 0, nsurf * sizeof(unsigned long long), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(act_ax, 0, nsurf * sizeof(int), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(act_step, 0, nsurf * sizeof(int), stream);
        if (e != cudaSuccess) s = cuda_error(lead, e, "batch init");
    }
    const int qb = (nq + 127) / 128, sb = (nsurf + 127) / 128;
    int64_t matvec_launches = 0;
    int cycle_kernels = 0;

    auto launch_mv = [&](const double *uu, double *yy, const int *act) {
        switch (R) {
            case 1: bmatvec_kernel<1><<<(unsigned)G, kBThreads, 0, stream>>>(d_surf, nsurf, d_inst, work, G, uu, yy, act, part, cnt_tile, evals); break;
            case 2: bmatvec_kernel<2><<<(unsigned)G, kBThreads, 0, stream>>>(d_surf, nsurf, d_inst, work, G, uu, yy, act, part, cnt_tile, evals); break;
            case 4: bmatvec_kernel<4><<<(unsigned)G, kBThreads, 0, stream>>>(d_surf, nsurf, d_inst, work, G, uu, yy, act, part, cnt_tile, evals); break;
            default: bmatvec_kernel<8><<<(unsigned)G, kBThreads, 0, stream>>>(d_surf, nsurf, d_inst, work, G, uu, yy, act, part, cnt_tile, evals); break;
        }
        ++cycle_kernels;
        ++matvec_launches;
    };
    // one restart cycle of every instance
    auto enqueue_cycle = [&]() {
        launch_mv(x, w, act_ax);
        bg_cycle_start<<<nchunks, kVThreads, 0, stream>>>(b, w, r, d_ch, d_inst, red, cnt_inst, st);
        bg_scale<<<nchunks, kVThreads, 0, stream>>>(r, V, d_ch, st, 0);
        bg_flags<<<sb, 128, 0, stream>>>(d_surf, nsurf, st, act_step, act_ax, 0);
        cycle_kernels += 3;
        for (int k = 0; k < m; ++k) {
            double *vk = V + (int64_t)k * L;
            launch_mv(vk, w, act_step);
            bg_dots<<<dim3(nchunks, k + 1), kVThreads, 0, stream>>>(V, L, w, k, d_ch, d_inst, red, nchunks, cnt_inst, st);
            bg_orth1<<<nchunks, kVThreads, 0, stream>>>(V, L, w, k, d_ch, d_inst, red, nchunks, cnt_inst, st);
            bg_orth2<<<nchunks, kVThreads, 0, stream>>>(V, L, w, k, d_ch, d_inst, red, cnt_inst, st);
            bg_scale<<<nchunks, kVThreads, 0, stream>>>(w, vk + L, d_ch, st, 1);
            bg_flags<<<sb, 128, 0, stream>>>(d_surf, nsurf, st, act_step, act_ax, 0);
            cycle_kernels += 5;
        }
        bg_trisolve<<<qb, 128, 0, stream>>>(st, nq);
        bg_update_x<<<nchunks, kVThreads, 0, stream>>>(V, L, x, d_ch, st);
        bg_flags<<<sb, 128, 0, stream>>>(d_surf, nsurf, st, act_step, act_ax, 1);
        bg_status<<<qb, 128, 0, stream>>>(st, nq, d_status);
        cycle_kernels += 4;
    };

    int cycles_run = 0;
    if (s == PB_OK) {
        bg_init<<<qb, 128, 0, stream>>>(st, nq, m, o.maxit, o.tol);
        bg_source<<<nschunks, kVThreads, 0, stream>>>(d_sch, d_inst, d_surf, d_q, d_ie, b);
        bg_norm<<<nchunks, kVThreads, 0, stream>>>(b, d_ch, d_inst, red, cnt_inst, st);
        for (int q = 0; q < 3; ++q) PB_LAUNCHED();
        e = cudaGetLastError();
        if (e != cudaSuccess) s = cuda_error(lead, e, "batch setup kernels");
    }
    // a CUDA graph needs a capturable stream (not the legacy default stream)
    if (s == PB_OK && use_graph && stream != nullptr) {
        e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue_cycle();
            cudaError_t e2 = cudaStreamEndCapture(stream, &graph);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
        if (e != cudaSuccess) s = cuda_error(lead, e, "batch graph capture");
    }
    const int kernels_per_cycle = cycle_kernels;
    const int64_t mv_per_cycle = matvec_launches;
    matvec_launches = 0;
    const int max_cycles = o.maxit + 2;
    for (int cyc = 0; s == PB_OK && cyc < max_cycles; ++cyc) {
        if (gexec) {
            e = cudaGraphLaunch(gexec, stream);
            count_launches(kernels_per_cycle);
            matvec_launches += mv_per_cycle;
        } else {
            cycle_kernels = 0;
            enqueue_cycle();
            count_launches(cycle_kernels);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_status, d_status, nq * sizeof(BStatus), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            s = cuda_error(lead, e, "batch cycle");
            break;
        }
        ++cycles_run;
        bool all = true;
        for (int q = 0; q < nq; ++q) all &= (h_status[q].done != 0);
        if (all) break;
    }
    // energies (Eq. (14)) of every instance, FP64 pairs, through the per-context
    // kernel: point each context at the instance's charges and solution
    int nconv = 0, iters_max = 0, iters_sum = 0;
    double resid_max = 0.0;
    pb_status worst = PB_OK;
    if (s == PB_OK) {
        for (int q = 0; q < nq && s == PB_OK; ++q) {
            const BInst &in = hq[q];
            pb_ctx *c = ctxs[in.surf];
            // energy of instance q with its own charges: stage them in the context
            Charge4 *keep = c->charges;
            const int64_t keep_nc = c->Nc;
            const cudaStream_t keep_stream = c->stream;
            c->charges = d_q + in.qoff;
            c->Nc = in.nc;
            c->stream = stream;
            s = energy_launch(c, x + in.off, PB_FP64, en + q);
            c->charges = keep;
            c->Nc = keep_nc;
            c->stream = keep_stream;
        }
        if (s == PB_OK) {
            e = cudaMemcpyAsync(energies, en, nq * sizeof(double), cudaMemcpyDeviceToHost, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) s = cuda_error(lead, e, "batch energies");
        }
        for (int q = 0; q < nq; ++q) {
            nconv += h_status[q].converged;
            iters_max = h_status[q].iters > iters_max ? h_status[q].iters : iters_max;
            iters_sum += h_status[q].iters;
            resid_max = h_status[q].rel_resid > resid_max ? h_status[q].rel_resid : resid_max;
            if (h_status[q].status == PB_ERR_NAN) worst = PB_ERR_NAN;
            else if (!h_status[q].converged && worst == PB_OK) worst = PB_ERR_NOCONV;
        }
    }
    if (info) {
        info->instances = nq;
        info->converged = nconv;
        info->cycles = cycles_run;
        info->iters_max = iters_max;
        info->iters_sum = iters_sum;
        info->rel_resid_max = resid_max;
        info->rhs_width = R;
        info->ctas = G;
        info->pair_evals = 0;
        info->pair_products = 0;
        info->matvec_launches = matvec_launches;
        std::vector<unsigned long long> hev(nsurf, 0);
        if (s == PB_OK && cudaMemcpy(hev.data(), evals, nsurf * sizeof(unsigned long long), cudaMemcpyDeviceToHost) ==
                              cudaSuccess) {
            for (int sidx = 0; sidx < nsurf; ++sidx) {
                const int64_t pairs = hs[sidx].N * (hs[sidx].N - 1);
                info->pair_evals += (int64_t)hev[sidx] * pairs;
                info->pair_products += (int64_t)hev[sidx] * pairs * hs[sidx].nrhs;
            }
        }
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    void *bufs[] = {d_surf, d_inst, d_ch, d_sch, d_q, d_ie, b, x, w, r, V, red, part, en, st, d_status,
                    cnt_inst, cnt_tile, evals, act_step, act_ax};
    for (void *p : bufs) ctx_free(lead, p);
    cudaStreamSynchronize(stream);
    if (h_status) cudaFreeHost(h_status);
    if (s != PB_OK) return s;
    if (worst != PB_OK)
        return set_error(lead, worst, "pb_batch_solve: %d of %d instances did not converge", nq - nconv, nq);
    return PB_OK;
}
