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

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "bmatvec.cuh"
#include "engine.cuh"
#include "fastmath.cuh"
#include "pb_internal.cuh"
#include "reduce.cuh"

namespace pb {

constexpr int kChunk = 4096;            // vector chunk (elements) of the GMRES kernels
constexpr int kVThreads = 256;
constexpr int LDH = kMaxRestart + 1;


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

// The work split of one batched product over the surfaces with a running
// instance: wbase[s] = sum of ntiles S over the active surfaces before s,
// wbase[nsurf] = the total (surfaces without a running instance get none, so
// the product's CTAs share only live work).  One block; a prefix sum over
// shared-memory chunks by one thread.
__global__ void bmv_plan_kernel(const BSurf *__restrict__ surf, int nsurf, const int *__restrict__ act,
                                int64_t *__restrict__ wbase) {
    constexpr int CH = 1024;
    __shared__ int64_t s_w[CH];
    __shared__ int64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    for (int c0 = 0; c0 < nsurf; c0 += CH) {
        __syncthreads();
        for (int i = threadIdx.x; i < CH; i += blockDim.x) {
            const int s = c0 + i;
            s_w[i] = (s < nsurf && vol(act + s)) ? surf[s].ntiles * surf[s].S : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t c = s_carry;
            const int n = (nsurf - c0) < CH ? (nsurf - c0) : CH;
            for (int i = 0; i < n; ++i) {
                wbase[c0 + i] = c;
                c += s_w[i];
            }
            s_carry = c;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) wbase[nsurf] = s_carry;
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
                    d_status_, d_wbase_};
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, stream_);
    if (gexec_) cudaGraphExecDestroy(gexec_);
    if (graph_) cudaGraphDestroy(graph_);
    cudaStreamSynchronize(stream_);
    if (h_status_) cudaFreeHost(h_status_);
    if (h_evals_) cudaFreeHost(h_evals_);
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
        *st = source_launch(surf, b, PB_FLOAT2);
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

// ---------------------------------------------------------------------------
// Batched-product tuning: process-wide mode, forced shapes and tuned choices
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
int g_tune_mode = 1;                                   // 0 built-in defaults, 1 autotune
BmvConfig g_forced[kEngineMaxRhs + 1];                 // by width (T == 0: none)
std::map<std::tuple<int, int, int64_t>, BmvConfig> g_tuned;   // (device, width, size class)

double wall_seconds() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

BmvConfig default_config(int R) {
    BmvShape sh[16];
    bmatvec_shapes(R, sh, 16);
    BmvConfig c;
    c.T = sh[0].T;
    c.acc = sh[0].acc;
    c.ctas_per_sm = 0;
    return c;
}

BmvArgs bmv_args(const BSurf *surf, int nsurf, const BInst *inst, const int64_t *wbase, int64_t G, int usel, int k,
                 const int *act, double *part, unsigned int *cnt, unsigned long long *evals) {
    BmvArgs a;
    a.surf = surf;
    a.nsurf = nsurf;
    a.inst = inst;
    a.wbase = wbase;
    a.G = G;
    a.usel = usel;
    a.k = k;
    a.active = act;
    a.partials = part;
    a.counters = cnt;
    a.evaluated = evals;
    return a;
}
}  // namespace

void Engine::retile(std::vector<BSurf> &hs, const std::vector<char> &direct, int64_t TT, int64_t *tiles,
                    int64_t *work) {
    int64_t t = 0, w = 0;
    for (size_t i = 0; i < hs.size(); ++i) {
        const int64_t nt = direct[i] ? 0 : (hs[i].N + TT - 1) / TT;
        hs[i].tile_base = t;
        hs[i].work_base = w;
        hs[i].ntiles = nt;
        t += nt;
        w += nt * hs[i].S;
    }
    *tiles = t;
    *work = w;
}

// Times every instantiated shape of width R_ at every CTA count up to its
// occupancy on the current work list (two launches each after one warm-up,
// CUDA events on the engine's stream) and keeps the fastest.  The launches
// read x and write w of the running instances, which the next cycle
// recomputes first; the evaluation counters are cleared afterwards.
pb_status Engine::tune(std::vector<BSurf> &hs, const std::vector<char> &direct, int64_t size_class) {
    const double t0 = wall_seconds();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    BmvShape sh[16];
    const int nsh = bmatvec_shapes(R_, sh, 16);
    BmvConfig best = config;
    float best_ms = 1e30f;
    int tried = 0;
    for (int i = 0; i < nsh && e == cudaSuccess; ++i) {
        int occ = 0;
        e = bmatvec_dispatch(R_, sh[i], BmvArgs{}, 0, stream_, &occ);
        if (e != cudaSuccess) break;
        if (occ < 1) continue;
        int64_t tiles = 0, W = 0;
        retile(hs, direct, (int64_t)kBThreads * sh[i].T, &tiles, &W);
        if (W == 0) break;
        e = cudaMemcpyAsync(d_surf_, hs.data(), hs.size() * sizeof(BSurf), cudaMemcpyHostToDevice, stream_);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
        for (int cps = 1; cps <= occ && e == cudaSuccess; ++cps) {
            int64_t G = (int64_t)num_sms_ * cps;
            if (G > W) G = W;
            // every surface with a running instance takes part (the Arnoldi-step
            // flags; the x-product flags are off for instances that start at x = 0)
            const BmvArgs a = bmv_args(d_surf_, nsurf_, d_inst_, d_wbase_, G, 0, 0, act_step_, part_, cnt_tile_,
                                       evals_);
            bmv_plan_kernel<<<1, 256, 0, stream_>>>(d_surf_, nsurf_, act_step_, d_wbase_);
            count_launch();
            e = bmatvec_dispatch(R_, sh[i], a, (unsigned)G, stream_, nullptr);
            if (e == cudaSuccess) e = cudaEventRecord(e0, stream_);
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) e = bmatvec_dispatch(R_, sh[i], a, (unsigned)G, stream_, nullptr);
            count_launches(3);
            if (e == cudaSuccess) e = cudaEventRecord(e1, stream_);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaGetLastError();
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            ++tried;
            if (e == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                best.T = sh[i].T;
                best.acc = sh[i].acc;
                best.ctas_per_sm = cps;
            }
            if (G == W) break;               // more CTAs than work items change nothing
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "engine: tuning the batched product");
    config = best;
    tuned = true;
    tune_candidates = tried;
    tune_ms = 1e3 * (wall_seconds() - t0);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned[std::make_tuple(device_, R_, size_class)] = best;
    }
    return PB_OK;
}

pb_status Engine::rebuild() {
    std::vector<BSurf> hs;
    std::vector<BInst> hq;
    std::vector<BChunk> hch;
    std::vector<char> direct_flag;
    surf_member_.clear();
    direct_.clear();
    tuned = false;
    int rmax = 1;
    for (EngineMember *mb : members_)
        if (!mb->finished && mb->nrhs > rmax) rmax = mb->nrhs;
    R_ = rmax <= 1 ? 1 : (rmax <= 2 ? 2 : (rmax <= 4 ? 4 : 8));
    double pairs = 0.0;      // pair evaluations of one batched launch (its size class)
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
        sf.S = (c->N + kBSourceTile - 1) / kBSourceTile;
        if (direct) direct_.push_back((int)hs.size());
        else pairs += (double)c->N * (double)c->N;
        sf.inst0 = (int)hq.size();
        sf.nrhs = mb->nrhs;
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
        direct_flag.push_back(direct ? 1 : 0);
        surf_member_.push_back((int)mi);
    }
    nsurf_ = (int)hs.size();
    nq_ = (int)hq.size();
    nchunks_ = (int)hch.size();
    rhs_width = R_;
    if (gexec_) cudaGraphExecDestroy(gexec_);
    if (graph_) cudaGraphDestroy(graph_);
    gexec_ = nullptr;
    graph_ = nullptr;
    dirty_ = false;
    if (nsurf_ == 0) return PB_OK;

    // the product's shape: forced; the one this engine tuned or looked up
    // first for this width (a batch keeps it as its members finish); tuned
    // for this size class; tuned for the nearest size class within an
    // octave; else the built-in default
    const int64_t size_class = pairs > 1.0 ? (int64_t)floor(4.0 * log2(pairs)) : 0;
    bool need_tune = false, forced = false;
    config = default_config(R_);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        if (g_forced[R_].T > 0) {
            config = g_forced[R_];
            forced = true;
        } else if (g_tune_mode == 1 && kept_R_ == R_) {
            config = kept_;
        } else if (g_tune_mode == 1) {
            auto it = g_tuned.find(std::make_tuple(device_, R_, size_class));
            if (it != g_tuned.end()) {
                config = it->second;
            } else if (autotune && pairs > 0.0) {
                need_tune = true;
            } else {
                int64_t best_d = 5;
                for (const auto &kv : g_tuned) {
                    if (std::get<0>(kv.first) != device_ || std::get<1>(kv.first) != R_) continue;
                    const int64_t d0 = std::get<2>(kv.first) - size_class, d = d0 < 0 ? -d0 : d0;
                    if (d < best_d) {
                        best_d = d;
                        config = kv.second;
                    }
                }
            }
        }
    }
    // buffer sizes cover every shape the tuner may try
    int occ = 0;
    cudaError_t qe = bmatvec_dispatch(R_, BmvShape{config.T, config.acc}, BmvArgs{}, 0, stream_, &occ);
    if (qe != cudaSuccess) return cuda_fail(qe, "engine: batched product shape");
    if (occ < 1) occ = 1;
    size_t part_need = 0;
    int64_t tiles_need = 0;
    {
        BmvShape sh[16];
        const int nsh = need_tune ? bmatvec_shapes(R_, sh, 16) : 1;
        if (!need_tune) sh[0] = BmvShape{config.T, config.acc};
        for (int i = 0; i < nsh; ++i) {
            int o = occ;
            if (need_tune && bmatvec_dispatch(R_, sh[i], BmvArgs{}, 0, stream_, &o) != cudaSuccess) o = 1;
            if (!need_tune && config.ctas_per_sm > 0 && config.ctas_per_sm < o) o = config.ctas_per_sm;
            const int64_t TTi = (int64_t)kBThreads * sh[i].T;
            const size_t need = (size_t)2 * num_sms_ * (o < 1 ? 1 : o) * 2 * R_ * TTi;
            part_need = need > part_need ? need : part_need;
            int64_t t = 0, w = 0;
            retile(hs, direct_flag, TTi, &t, &w);
            tiles_need = t > tiles_need ? t : tiles_need;
        }
    }
    const int64_t TT = (int64_t)kBThreads * config.T;
    int64_t tiles = 0, work = 0;
    retile(hs, direct_flag, TT, &tiles, &work);
    tiles_ = tiles;
    W_ = work;
    int cps = (config.ctas_per_sm > 0 && config.ctas_per_sm < occ) ? config.ctas_per_sm : occ;
    if (cta_cap_ > 0 && cps > cta_cap_) cps = cta_cap_;
    G_ = (int64_t)num_sms_ * cps;
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
    if (s == PB_OK) s = grow((void **)&d_wbase_, &cap_wbase_, nsurf_ + 1, sizeof(int64_t), "engine work split");
    if (s == PB_OK) s = grow((void **)&d_inst_, &cap_inst_, nq_, sizeof(BInst), "engine instances");
    if (s == PB_OK) s = grow((void **)&d_ch_, &cap_ch_, nchunks_, sizeof(BChunk), "engine chunks");
    if (s == PB_OK) s = grow((void **)&cnt_inst_, &cap_cnt_inst_, nq_, sizeof(unsigned int), "engine counters");
    if (s == PB_OK) s = grow((void **)&cnt_tile_, &cap_cnt_tile_, tiles_need, sizeof(unsigned int), "engine counters");
    if (s == PB_OK) s = grow((void **)&evals_, &cap_evals_, nsurf_, sizeof(unsigned long long), "engine counters");
    if (s == PB_OK) s = grow((void **)&act_step_, &cap_flags_, 2 * (size_t)nsurf_, sizeof(int), "engine flags");
    if (s == PB_OK) {
        size_t c2 = 0;
        if (act_ax_) cudaFreeAsync(act_ax_, stream_);
        act_ax_ = nullptr;
        s = grow((void **)&act_ax_, &c2, cap_flags_, sizeof(int), "engine flags");
    }
    if (s == PB_OK) s = grow((void **)&red_, &cap_red_, (size_t)(m_ + 1) * nchunks_, sizeof(double), "engine reductions");
    if (s == PB_OK) s = grow((void **)&part_, &cap_part_, part_need, sizeof(double), "engine partials");
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
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt_tile_, 0, tiles_need * sizeof(unsigned int), stream_);
    if (e == cudaSuccess) e = cudaMemsetAsync(evals_, 0, nsurf_ * sizeof(unsigned long long), stream_);
    // the staging vectors are pageable and local: wait for the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
    if (e != cudaSuccess) return cuda_fail(e, "engine table upload");
    last_evals_.assign(nsurf_, 0ull);
    // flags from the current states (members may be mid-solve)
    bg_flags<<<(nsurf_ + 127) / 128, 128, 0, stream_>>>(d_surf_, nsurf_, d_inst_, act_step_, act_ax_, 0);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "engine flags");
    if (!need_tune) {
        if (autotune && !forced) {
            kept_ = config;
            kept_R_ = R_;
        }
        return PB_OK;
    }

    // tune on this work list, then install the choice
    if ((s = tune(hs, direct_flag, size_class)) != PB_OK) return s;
    kept_ = config;
    kept_R_ = R_;
    retile(hs, direct_flag, (int64_t)kBThreads * config.T, &tiles, &work);
    tiles_ = tiles;
    W_ = work;
    occ = 1;
    e = bmatvec_dispatch(R_, BmvShape{config.T, config.acc}, BmvArgs{}, 0, stream_, &occ);
    if (e != cudaSuccess) return cuda_fail(e, "engine: batched product shape");
    {
        int cps2 = (config.ctas_per_sm > 0 && config.ctas_per_sm < occ) ? config.ctas_per_sm : occ;
        if (cta_cap_ > 0 && cps2 > cta_cap_) cps2 = cta_cap_;
        G_ = (int64_t)num_sms_ * cps2;
    }
    if (G_ > W_) G_ = W_;
    ctas = G_;
    e = cudaMemcpyAsync(d_surf_, hs.data(), nsurf_ * sizeof(BSurf), cudaMemcpyHostToDevice, stream_);
    if (e == cudaSuccess) e = cudaMemsetAsync(evals_, 0, nsurf_ * sizeof(unsigned long long), stream_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
    return e == cudaSuccess ? PB_OK : cuda_fail(e, "engine table upload");
}

void Engine::enqueue_cycle() {
    const int sb = (nsurf_ + 127) / 128, qb = (nq_ + 127) / 128;
    auto mv = [&](int usel, int k, const int *act) {
        if (timing_ && ev_used_ + 2 <= (int)ev_.size()) cudaEventRecord(ev_[ev_used_], stream_);
        if (W_ > 0) {
            bmv_plan_kernel<<<1, 256, 0, stream_>>>(d_surf_, nsurf_, act, d_wbase_);
            bmatvec_dispatch(R_, BmvShape{config.T, config.acc},
                             bmv_args(d_surf_, nsurf_, d_inst_, d_wbase_, G_, usel, k, act, part_, cnt_tile_, evals_),
                             (unsigned)G_, stream_, nullptr);
            cycle_kernels_ += 2;
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

pb_status Engine::prepare() {
    pb_status s = PB_OK;
    if (dirty_ && (s = rebuild()) != PB_OK) return s;
    if (cap_h_evals_ < (size_t)nsurf_) {
        if (h_evals_) {
            cudaStreamSynchronize(stream_);
            cudaFreeHost(h_evals_);
            h_evals_ = nullptr;
            cap_h_evals_ = 0;
        }
        const size_t cap = (size_t)nsurf_ + 16;
        cudaError_t e = cudaMallocHost((void **)&h_evals_, cap * sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(e, "engine pinned counters");
        cap_h_evals_ = cap;
    }
    return PB_OK;
}

pb_status Engine::cycle(bool use_graph, bool time_products) {
    pb_status s = launch_cycle(use_graph, time_products);
    return s != PB_OK ? s : finish_cycle();
}

pb_status Engine::launch_cycle(bool use_graph, bool time_products) {
    pb_status s = prepare();
    if (s != PB_OK) return s;
    launched_ = false;
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
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_evals_, evals_, nsurf_ * sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream_);
    if (e != cudaSuccess) return cuda_fail(e, "engine cycle");
    launched_ = true;
    return PB_OK;
}

pb_status Engine::finish_cycle() {
    if (!launched_) return PB_OK;
    launched_ = false;
    cudaError_t e = cudaStreamSynchronize(stream_);
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
        pair_evals += (int64_t)(h_evals_[si] - last_evals_[si]) * pairs;
        pair_products += (int64_t)(h_evals_[si] - last_evals_[si]) * pairs * mb->nrhs;
        last_evals_[si] = h_evals_[si];
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
        s = energy_launch(c, mb->vec + (size_t)r * per + n2, PB_FLOAT2, scalar_ + (r % 64));
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

namespace {
std::atomic<int> g_batch_streams{2};   // engines (streams) of pb_batch_solve
}  // namespace

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
    const double t_begin = wall_seconds();
    // Two engines on two streams (the members split in two halves of about
    // equal pair work) run their restart cycles at the same time, so that one
    // engine's launches fill the SMs the other's leave idle (the tail of each
    // persistent product launch, the short orthogonalisation kernels).
    const int neng = (g_batch_streams >= 2 && nsurf >= 2) ? 2 : 1;
    cudaStream_t side = nullptr;
    if (neng == 2) {
        int prio = 0;
        cudaError_t e = lead->stream ? cudaStreamGetPriority(lead->stream, &prio) : cudaSuccess;
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, prio);
        if (e != cudaSuccess) return cuda_error(lead, e, "pb_batch_solve: second stream");
        // the inputs the caller enqueued on its stream come first
        cudaEvent_t ready = nullptr;
        e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ready, lead->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ready, 0);
        if (ready) cudaEventDestroy(ready);
        if (e != cudaSuccess) {
            cudaStreamDestroy(side);
            return cuda_error(lead, e, "pb_batch_solve: second stream");
        }
    }
    std::vector<std::unique_ptr<Engine>> engs;
    for (int k = 0; k < neng; ++k) {
        engs.emplace_back(new Engine(k == 0 ? lead->stream : side, lead->device, lead->num_sms, o.restart, o.tol,
                                     o.maxit));
        engs.back()->autotune = true;
    }
    // members to engines: by pair work, largest first, each to the lighter engine
    std::vector<int> owner(nsurf, 0);
    if (neng == 2) {
        std::vector<int> order(nsurf);
        for (int i = 0; i < nsurf; ++i) order[i] = i;
        auto work = [&](int i) { return (double)ctxs[i]->N * (double)ctxs[i]->N * (double)nrhs[i]; };
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
        double load[2] = {0.0, 0.0};
        for (int i : order) {
            const int k = load[1] < load[0] ? 1 : 0;
            owner[i] = k;
            load[k] += work(i);
        }
    }
    std::vector<EngineMember *> mem(nsurf, nullptr);
    pb_status s = PB_OK;
    for (int i = 0; i < nsurf && s == PB_OK; ++i)
        mem[i] = engs[owner[i]]->add(ctxs[i], charges[i], nc[i], nrhs[i], (uint64_t)i, &s);
    auto finish_engines = [&]() {
        engs.clear();
        if (side) {
            cudaStreamSynchronize(side);
            cudaStreamDestroy(side);
            side = nullptr;
        }
    };
    auto engine_error = [&]() -> const char * {
        for (auto &e : engs)
            if (e->error[0]) return e->error;
        return "engine error";
    };
    if (s != PB_OK) {
        set_error(lead, s, "%s", engine_error());
        finish_engines();
        return s;
    }
    const double t_setup = wall_seconds();
    bool all = false;
    int tuned_any = 0, tune_candidates = 0;
    double tune_ms = 0.0;
    for (int cyc = 0; cyc < o.maxit + 2 && s == PB_OK && !all; ++cyc) {
        // tables and tuning first (nothing in flight), then both cycles at once
        for (auto &e : engs)
            if (s == PB_OK) s = e->prepare();
        for (auto &e : engs)
            if (s == PB_OK) s = e->launch_cycle(use_graph == 1, use_graph == 2);
        for (auto &e : engs) {
            const pb_status fs = e->finish_cycle();
            if (s == PB_OK) s = fs;
            if (e->tuned) {
                tuned_any = 1;
                tune_candidates += e->tune_candidates;
                tune_ms += e->tune_ms;
                e->tuned = false;
            }
        }
        all = true;
        for (EngineMember *mb : mem) all &= mb->finished;
    }
    if (s != PB_OK) {
        set_error(lead, s, "%s", engine_error());
        finish_engines();
        return s;
    }
    const double t_cycles = wall_seconds();
    int k = 0, nconv = 0, nq = 0, iters_max = 0;
    int64_t iters_sum = 0;
    double resid_max = 0.0;
    pb_status worst = PB_OK;
    for (int i = 0; i < nsurf && s == PB_OK; ++i) {
        s = engs[owner[i]]->energies(mem[i], energies + k);
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
    if (s != PB_OK) {
        set_error(lead, s, "%s", engine_error());
        finish_engines();
        return s;
    }
    const double t_end = wall_seconds();
    if (info) {
        const Engine &eng = *engs[0];
        info->setup_ms = 1e3 * (t_setup - t_begin);
        info->cycles_ms = 1e3 * (t_cycles - t_setup);
        info->energy_ms = 1e3 * (t_end - t_cycles);
        info->instances = nq;
        info->converged = nconv;
        info->cycles = 0;
        info->pair_evals = info->pair_products = info->matvec_launches = 0;
        info->matvec_ms = 0.0;
        info->rhs_width = 0;
        for (auto &e : engs) {
            info->cycles = e->cycles_run > info->cycles ? e->cycles_run : info->cycles;
            info->pair_evals += e->pair_evals;
            info->pair_products += e->pair_products;
            info->matvec_launches += e->matvec_launches;
            info->matvec_ms += e->matvec_ms;
            info->rhs_width = e->rhs_width > info->rhs_width ? e->rhs_width : info->rhs_width;
        }
        info->iters_max = iters_max;
        info->iters_sum = iters_sum;
        info->rel_resid_max = resid_max;
        info->ctas = eng.ctas;
        info->targets_per_thread = eng.config.T;
        info->row_sums = eng.config.acc;
        info->ctas_per_sm = eng.config.ctas_per_sm;
        info->tuned = tuned_any;
        info->tune_candidates = tune_candidates;
        info->tune_ms = tune_ms;
        info->streams = neng;
    }
    finish_engines();
    if (worst != PB_OK)
        return set_error(lead, worst, "pb_batch_solve: %d of %d instances did not converge", nq - nconv, nq);
    return PB_OK;
}

extern "C" pb_status pb_batch_set_streams(int n) {
    if (n != 1 && n != 2) return set_error(nullptr, PB_ERR_ARG, "pb_batch_set_streams: n must be 1 or 2");
    g_batch_streams = n;
    return PB_OK;
}

extern "C" pb_status pb_batch_set_tuning(int mode) {
    if (mode != 0 && mode != 1) return set_error(nullptr, PB_ERR_ARG, "pb_batch_set_tuning: mode must be 0 or 1");
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_mode = mode;
    return PB_OK;
}

extern "C" pb_status pb_batch_force_shape(int rhs_width, int targets_per_thread, int row_sums, int ctas_per_sm) {
    if (rhs_width != 1 && rhs_width != 2 && rhs_width != 4 && rhs_width != 8)
        return set_error(nullptr, PB_ERR_ARG, "pb_batch_force_shape: width must be 1, 2, 4 or 8");
    if (ctas_per_sm < 0) return set_error(nullptr, PB_ERR_ARG, "pb_batch_force_shape: ctas_per_sm < 0");
    BmvConfig c;
    if (targets_per_thread > 0) {
        BmvShape sh[16];
        const int n = bmatvec_shapes(rhs_width, sh, 16);
        bool found = false;
        for (int i = 0; i < n; ++i) found |= sh[i].T == targets_per_thread && sh[i].acc == row_sums;
        if (!found)
            return set_error(nullptr, PB_ERR_ARG,
                             "pb_batch_force_shape: (targets %d, row sums %d) is not a shape of width %d",
                             targets_per_thread, row_sums, rhs_width);
        c.T = targets_per_thread;
        c.acc = row_sums;
        c.ctas_per_sm = ctas_per_sm;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_forced[rhs_width] = c;
    return PB_OK;
}

extern "C" pb_status pb_batch_clear_tuning(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned.clear();
    return PB_OK;
}

extern "C" int pb_batch_shapes(int rhs_width, int *targets_per_thread, int *row_sums, int max_out) {
    BmvShape sh[16];
    const int n = bmatvec_shapes(rhs_width, sh, 16);
    for (int i = 0; i < n && i < max_out; ++i) {
        if (targets_per_thread) targets_per_thread[i] = sh[i].T;
        if (row_sums) row_sums[i] = sh[i].acc;
    }
    return n;
}
