// gmres.cu -- restarted GMRES (Saad & Schultz) on the device for A u = b.
//
// The paper runs GMRES on the host and moves y = A x across PCIe on every
// iteration (Section 2.4, the pseudo-code table).  Here every step stays on
// the GPU: the Arnoldi vectors V, the Hessenberg matrix, the Givens rotations
// and the convergence decision live in device memory, and the host only
// enqueues kernels and reads a small state record once per restart cycle.
//
// One Arnoldi step k of a cycle:
//   w = A v_k                          (matvec.cu)
//   h  = V_k^T w,  w -= V_k h          (classical Gram-Schmidt, pass 1)
//   h' = V_k^T w,  w -= V_k h'         (pass 2; H[:,k] = h + h')
//   H[k+1,k] = ||w||, v_{k+1} = w / H[k+1,k]
//   apply the previous Givens rotations to H[:,k], form rotation k, update g;
//   |g[k+1]| / ||b|| is the residual estimate.
// A cycle starts from the true residual r = b - A x (x = 0 at the first cycle
// unless a start vector is given, Section 2.4) and ends with x += V_k y,
// R y = g.  The solve stops when the true relative residual of a cycle start
// is <= tol.  Every reduction is a fixed-order two-stage sum (no float atomics).
#include <math.h>
#include <string.h>

#include "pb_internal.cuh"
#include "reduce.cuh"

namespace pb {

int red_blocks(pb_ctx *ctx, int64_t n) {
    int64_t b = (n + kRedThreads * 4 - 1) / (kRedThreads * 4);
    int64_t cap = 2 * (int64_t)ctx->num_sms;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

namespace {

constexpr int BS = kRedThreads;
constexpr int LDH = kMaxRestart + 1;

__device__ __forceinline__ int vol_int(const int *p) { return *((volatile const int *)p); }

__global__ void __launch_bounds__(BS) norm2_kernel(const double *__restrict__ v, int64_t n, double *__restrict__ red,
                                                   unsigned int *__restrict__ counter, double *__restrict__ out) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)BS + threadIdx.x; i < n; i += (int64_t)gridDim.x * BS) s += v[i] * v[i];
    s = block_sum<BS>(s);
    if (threadIdx.x == 0) red[blockIdx.x] = s;
    if (last_block_arrived(counter, gridDim.x) && threadIdx.x == 0) {
        double t = 0.0;
        for (unsigned int b = 0; b < gridDim.x; ++b) t += __ldcg(red + b);
        out[0] = sqrt(t);
        *counter = 0u;
    }
}

// r = rhs - Ax (Ax may be null: x = 0); beta = ||r||; decide convergence.
__global__ void __launch_bounds__(BS) cycle_start_kernel(const double *__restrict__ rhs, const double *__restrict__ Ax,
                                                         double *__restrict__ r, int64_t n, double *__restrict__ red,
                                                         unsigned int *__restrict__ counter, GmresState *st) {
    if (vol_int(&st->done)) return;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)BS + threadIdx.x; i < n; i += (int64_t)gridDim.x * BS) {
        double ri = Ax ? rhs[i] - Ax[i] : rhs[i];
        r[i] = ri;
        s += ri * ri;
    }
    s = block_sum<BS>(s);
    if (threadIdx.x == 0) red[blockIdx.x] = s;
    if (last_block_arrived(counter, gridDim.x) && threadIdx.x == 0) {
        double t = 0.0;
        for (unsigned int b = 0; b < gridDim.x; ++b) t += __ldcg(red + b);
        *counter = 0u;
        const double beta = sqrt(t);
        st->k = 0;
        st->beta = beta;
        st->rel_resid = beta / st->bnorm;
        st->est_resid = st->rel_resid;
        if (!isfinite(beta)) {
            st->status = PB_ERR_NAN;
            st->done = 1;
        } else if (st->rel_resid <= st->tol) {
            st->converged = 1;
            st->status = PB_OK;
            st->done = 1;
        } else if (st->iters >= st->maxit) {
            st->status = PB_ERR_NOCONV;
            st->done = 1;
        } else {
            st->cycles += 1;
            st->g[0] = beta;
            for (int i = 1; i <= st->m; ++i) st->g[i] = 0.0;
        }
        st->cycle_done = 0;
        st->skip = st->done;
    }
}

// dst = src / (which ? hnext : beta)
__global__ void __launch_bounds__(BS) scale_kernel(const double *__restrict__ src, double *__restrict__ dst, int64_t n,
                                                   const GmresState *st, int which) {
    if (vol_int(&st->skip)) return;
    const double inv = 1.0 / (which ? st->hnext : st->beta);
    for (int64_t i = blockIdx.x * (int64_t)BS + threadIdx.x; i < n; i += (int64_t)gridDim.x * BS) dst[i] = src[i] * inv;
}

// h1[v] = V_v . w for v = 0..k; grid (nb, k+1).
__global__ void __launch_bounds__(BS) dots_kernel(const double *__restrict__ V, const double *__restrict__ w, int64_t n,
                                                  int k, double *__restrict__ red, unsigned int *__restrict__ counter,
                                                  GmresState *st) {
    if (vol_int(&st->skip)) return;
    const int v = blockIdx.y;
    const int nb = gridDim.x;
    const double *Vv = V + (int64_t)v * n;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)BS + threadIdx.x; i < n; i += (int64_t)nb * BS) s += Vv[i] * w[i];
    s = block_sum<BS>(s);
    if (threadIdx.x == 0) red[v * nb + blockIdx.x] = s;
    if (last_block_arrived(counter, nb * (k + 1))) {
        for (int vv = threadIdx.x; vv <= k; vv += BS) {
            double t = 0.0;
            for (int b = 0; b < nb; ++b) t += __ldcg(red + vv * nb + b);
            st->h1[vv] = t;
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// w -= V h1; then h2[v] = V_v . w
__global__ void __launch_bounds__(BS) orth1_kernel(const double *__restrict__ V, double *__restrict__ w, int64_t n, int k,
                                                   double *__restrict__ red, unsigned int *__restrict__ counter,
                                                   GmresState *st) {
    if (vol_int(&st->skip)) return;
    __shared__ double s_h[LDH];
    for (int v = threadIdx.x; v <= k; v += BS) s_h[v] = st->h1[v];
    __syncthreads();
    const int nb = gridDim.x;
    for (int64_t i = blockIdx.x * (int64_t)BS + threadIdx.x; i < n; i += (int64_t)nb * BS) {
        double wi = w[i];
        for (int v = 0; v <= k; ++v) wi -= s_h[v] * V[(int64_t)v * n + i];
        w[i] = wi;
    }
    for (int v = 0; v <= k; ++v) {
        double s = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)BS + threadIdx.x; i < n; i += (int64_t)nb * BS)
            s += V[(int64_t)v * n + i] * w[i];
        s = block_sum<BS>(s);
        if (threadIdx.x == 0) red[v * nb + blockIdx.x] = s;
    }
    if (last_block_arrived(counter, nb)) {
        for (int vv = threadIdx.x; vv <= k; vv += BS) {
            double t = 0.0;
            for (int b = 0; b < nb; ++b) t += __ldcg(red + vv * nb + b);
            st->h2[vv] = t;
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// w -= V h2; H[:,k] = h1 + h2, H[k+1,k] = ||w||; Givens update and decisions.
__global__ void __launch_bounds__(BS) orth2_kernel(const double *__restrict__ V, double *__restrict__ w, int64_t n, int k,
                                                   double *__restrict__ red, unsigned int *__restrict__ counter,
                                                   GmresState *st) {
    if (vol_int(&st->skip)) return;
    __shared__ double s_h[LDH];
    for (int v = threadIdx.x; v <= k; v += BS) s_h[v] = st->h2[v];
    __syncthreads();
    const int nb = gridDim.x;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)BS + threadIdx.x; i < n; i += (int64_t)nb * BS) {
        double wi = w[i];
        for (int v = 0; v <= k; ++v) wi -= s_h[v] * V[(int64_t)v * n + i];
        w[i] = wi;
        s += wi * wi;
    }
    s = block_sum<BS>(s);
    if (threadIdx.x == 0) red[blockIdx.x] = s;
    if (last_block_arrived(counter, nb) && threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += __ldcg(red + b);
        *counter = 0u;
        const double hn = sqrt(t);
        double *H = st->H;
        for (int v = 0; v <= k; ++v) H[v + k * LDH] = st->h1[v] + st->h2[v];
        H[k + 1 + k * LDH] = hn;
        st->hnext = hn;
        for (int i = 0; i < k; ++i) {
            const double a = H[i + k * LDH], b = H[i + 1 + k * LDH];
            H[i + k * LDH] = st->cs[i] * a + st->sn[i] * b;
            H[i + 1 + k * LDH] = -st->sn[i] * a + st->cs[i] * b;
        }
        const double a = H[k + k * LDH], b = H[k + 1 + k * LDH];
        const double d = hypot(a, b);
        const double c = d > 0.0 ? a / d : 1.0, sn = d > 0.0 ? b / d : 0.0;
        st->cs[k] = c;
        st->sn[k] = sn;
        H[k + k * LDH] = d;
        H[k + 1 + k * LDH] = 0.0;
        st->g[k + 1] = -sn * st->g[k];
        st->g[k] = c * st->g[k];
        st->k = k + 1;
        st->iters += 1;
        const double est = fabs(st->g[k + 1]) / st->bnorm;
        st->est_resid = est;
        if (!isfinite(hn) || !isfinite(d) || !isfinite(est) || !(d > 0.0)) {
            // non-finite data, or an exactly singular projected matrix
            st->status = PB_ERR_NAN;
            st->done = 1;
        }
        const bool breakdown = !(hn > 0.0);
        st->cycle_done = (est <= st->tol) || (st->iters >= st->maxit) || breakdown || (k + 1 >= st->m) || st->done;
        st->skip = st->done || st->cycle_done;
    }
}

// Back substitution R y = g over the k columns of this cycle.
__global__ void trisolve_kernel(GmresState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int kk = st->k;
    if (kk == 0 || st->status != PB_OK) return;
    const double *H = st->H;
    for (int i = kk - 1; i >= 0; --i) {
        double t = st->g[i];
        for (int j = i + 1; j < kk; ++j) t -= H[i + j * LDH] * st->y[j];
        st->y[i] = t / H[i + i * LDH];
    }
}

// x += V_k y
__global__ void __launch_bounds__(BS) update_x_kernel(const double *__restrict__ V, double *__restrict__ x, int64_t n,
                                                      GmresState *st) {
    const int kk = st->k;
    if (kk == 0 || st->status != PB_OK) return;
    __shared__ double s_y[kMaxRestart];
    for (int v = threadIdx.x; v < kk; v += BS) s_y[v] = st->y[v];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)BS + threadIdx.x; i < n; i += (int64_t)gridDim.x * BS) {
        double xi = x[i];
        for (int v = 0; v < kk; ++v) xi += s_y[v] * V[(int64_t)v * n + i];
        x[i] = xi;
    }
}

}  // namespace

pb_status norm2_launch(pb_ctx *ctx, const double *v, int64_t n, double *dev_out) {
    norm2_kernel<<<red_blocks(ctx, n), BS, 0, ctx->stream>>>(v, n, ctx->red, ctx->red_counter, dev_out);
    PB_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PB_OK : cuda_error(ctx, e, "norm kernel");
}

static pb_status ensure_workspace(pb_ctx *ctx, int m) {
    const int64_t n2 = 2 * ctx->N;
    pb_status s;
    if (ctx->gm_m < m) {
        if (ctx->V) ctx_free(ctx, ctx->V);
        ctx->V = nullptr;
        ctx->gm_m = 0;
        if ((s = ctx_alloc(ctx, (void **)&ctx->V, (size_t)(m + 1) * n2 * sizeof(double), "Krylov basis")) != PB_OK)
            return s;
        ctx->gm_m = m;
    }
    if (!ctx->w && (s = ctx_alloc(ctx, (void **)&ctx->w, n2 * sizeof(double), "gmres w")) != PB_OK) return s;
    if (!ctx->r && (s = ctx_alloc(ctx, (void **)&ctx->r, n2 * sizeof(double), "gmres r")) != PB_OK) return s;
    if (!ctx->st && (s = ctx_alloc(ctx, (void **)&ctx->st, sizeof(GmresState), "gmres state")) != PB_OK) return s;
    if (!ctx->st_host) {
        cudaError_t e = pinned_alloc((void **)&ctx->st_host, sizeof(GmresState));
        if (e != cudaSuccess) return cuda_error(ctx, e, "pinned gmres state");
    }
    return PB_OK;
}

static pb_status launch_cycle_start(pb_ctx *ctx, const double *rhs, const double *x, bool x_zero, pb_precision prec) {
    const int64_t n2 = 2 * ctx->N;
    pb_status s;
    if (!x_zero && (s = matvec_launch(ctx, x, ctx->w, prec, &ctx->st->done)) != PB_OK) return s;
    cycle_start_kernel<<<red_blocks(ctx, n2), BS, 0, ctx->stream>>>(rhs, x_zero ? nullptr : ctx->w, ctx->r, n2, ctx->red,
                                                                    ctx->red_counter, ctx->st);
    PB_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PB_OK : cuda_error(ctx, e, "gmres cycle start");
}

static pb_status read_state(pb_ctx *ctx) {
    cudaError_t e = cudaMemcpyAsync(ctx->st_host, ctx->st, sizeof(GmresState), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? PB_OK : cuda_error(ctx, e, "gmres state readback");
}

pb_status gmres_solve(pb_ctx *ctx, const pb_solve_opts *o, const double *rhs, double *x, bool x_is_zero, int *iters,
                      int *cycles, double *rel_resid) {
    const int m = o->restart;
    const int64_t n2 = 2 * ctx->N;
    pb_status s = ensure_workspace(ctx, m);
    if (s != PB_OK) return s;

    GmresState *h = ctx->st_host;
    memset(h, 0, sizeof(GmresState));
    h->m = m;
    h->maxit = o->maxit;
    h->tol = o->tol;
    h->status = PB_OK;
    cudaError_t e = cudaMemcpyAsync(ctx->st, h, sizeof(GmresState), cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "gmres state upload");
    if ((s = norm2_launch(ctx, rhs, n2, &ctx->st->bnorm)) != PB_OK) return s;
    if ((s = read_state(ctx)) != PB_OK) return s;
    if (!(h->bnorm > 0.0) || !isfinite(h->bnorm)) {
        if (!isfinite(h->bnorm)) return set_error(ctx, PB_ERR_NAN, "gmres: right-hand side is not finite");
        // b = 0: the solution is x = 0
        e = cudaMemsetAsync(x, 0, n2 * sizeof(double), ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_error(ctx, e, "gmres zero solution");
        *iters = 0;
        *cycles = 0;
        *rel_resid = 0.0;
        return PB_OK;
    }

    const int nb = red_blocks(ctx, n2);
    bool started = false;
    bool x_zero = x_is_zero;
    for (int cyc = 0; cyc < o->maxit + 2; ++cyc) {
        if (!started && (s = launch_cycle_start(ctx, rhs, x, x_zero, o->prec)) != PB_OK) return s;
        started = false;
        x_zero = false;
        scale_kernel<<<nb, BS, 0, ctx->stream>>>(ctx->r, ctx->V, n2, ctx->st, 0);
        PB_LAUNCHED();
        for (int k = 0; k < m; ++k) {
            double *vk = ctx->V + (int64_t)k * n2;
            if ((s = matvec_launch(ctx, vk, ctx->w, o->prec, &ctx->st->skip)) != PB_OK) return s;
            dots_kernel<<<dim3(nb, k + 1), BS, 0, ctx->stream>>>(ctx->V, ctx->w, n2, k, ctx->red, ctx->red_counter,
                                                                 ctx->st);
            orth1_kernel<<<nb, BS, 0, ctx->stream>>>(ctx->V, ctx->w, n2, k, ctx->red, ctx->red_counter, ctx->st);
            orth2_kernel<<<nb, BS, 0, ctx->stream>>>(ctx->V, ctx->w, n2, k, ctx->red, ctx->red_counter, ctx->st);
            scale_kernel<<<nb, BS, 0, ctx->stream>>>(ctx->w, vk + n2, n2, ctx->st, 1);
            for (int q = 0; q < 4; ++q) PB_LAUNCHED();
        }
        trisolve_kernel<<<1, 32, 0, ctx->stream>>>(ctx->st);
        update_x_kernel<<<nb, BS, 0, ctx->stream>>>(ctx->V, x, n2, ctx->st);
        PB_LAUNCHED();
        PB_LAUNCHED();
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(ctx, e, "gmres kernels");
        if ((s = read_state(ctx)) != PB_OK) return s;
        if (h->done) break;
        if (h->est_resid <= o->tol || h->iters >= o->maxit) {
            // the Givens estimate says this may be the last cycle: test the
            // true residual now instead of enqueueing a full cycle
            if ((s = launch_cycle_start(ctx, rhs, x, false, o->prec)) != PB_OK) return s;
            if ((s = read_state(ctx)) != PB_OK) return s;
            if (h->done) break;
            started = true;
        }
    }
    *iters = h->iters;
    *cycles = h->cycles;
    *rel_resid = h->rel_resid;
    if (h->status == PB_ERR_NAN) return set_error(ctx, PB_ERR_NAN, "gmres: non-finite residual after %d iterations", h->iters);
    if (!h->converged)
        return set_error(ctx, PB_ERR_NOCONV, "gmres: relative residual %.3e > tol %.3e after %d iterations",
                         h->rel_resid, o->tol, h->iters);
    return PB_OK;
}

}  // namespace pb
