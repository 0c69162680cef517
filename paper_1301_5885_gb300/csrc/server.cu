// server.cu -- a solve server with continuous batching.
//
// Clients submit PB solve requests (a surface, a charge set and the physical
// constants) from any thread.  Requests go to one of two lanes by size: small
// surfaces (N < split_n), whose products share one batched launch, and large
// ones, each with its own symmetric product.  Each lane has a worker thread,
// a CUDA stream and the lockstep engine of batch.cu; the small lane's stream
// has the higher priority.  Between two restart cycles a worker
//   - finishes every request of its lane whose instance has converged (or
//     failed): energy (Eq. (14)), result with its latency, and release of its
//     device memory;
//   - admits its lane's queued requests in arrival order while the lane has
//     fewer than max_active running and their estimated device footprint fits
//     the memory budget shared by both lanes (a request larger than the whole
//     budget is rejected with PB_ERR_ADMIT);
// so requests that arrive while others are on the GPU join the running batch
// at the next cycle boundary and their products share the same launches.
// A large request's product fills every SM with persistent CTAs; while small
// requests are running, the large lane launches its products with one CTA
// per SM fewer, so that the small lane's kernels find free slots and its
// requests are not held to the large products' step time.  Every wait is
// bounded; no request ever waits on the GPU with a lock held.
#include <math.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "engine.cuh"
#include "pb_internal.cuh"

using namespace pb;

namespace {

using Clock = std::chrono::steady_clock;
constexpr int64_t kDefaultSplitN = 16384;   // from here a context's product is the symmetric one

struct Request {
    uint64_t id = 0;
    std::vector<double> c, n, a, q;
    int64_t N = 0, Nc = 0;
    double eps1 = 1, eps2 = 1, kappa = 0;
    Clock::time_point t_submit, t_admit;
    int64_t bytes = 0;
    pb_ctx *ctx = nullptr;
    EngineMember *member = nullptr;
    int cps = 0;                  // CTAs per SM its symmetric product is configured with (0: occupancy)
};

struct Lane {
    int index = 0;
    cudaStream_t stream = nullptr;
    Engine *eng = nullptr;
    std::thread worker;
    std::deque<Request *> pending;
    std::vector<Request *> active;
    std::atomic<int> n_active{0};
};

}  // namespace

struct pb_server {
    pb_server_opts opts{};
    int device = 0;
    int num_sms = 0;
    int nlanes = 2;
    int64_t split_n = kDefaultSplitN;
    Lane lanes[2];
    std::mutex mu;
    std::condition_variable cv;
    std::deque<pb_server_result> done;
    bool stop = false;
    uint64_t next_id = 1;
    int64_t used_bytes = 0;
    pb_server_stats stats{};
    int64_t lane_evals[2] = {0, 0}, lane_products[2] = {0, 0};
    Clock::time_point t0;
};

namespace {

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// Estimated device bytes of one request: its context (geometry in FP64 and
// FP32, right-hand side and solution, matvec scratch) plus the engine member
// (Krylov basis and work vectors).
int64_t footprint(int64_t N, int64_t Nc, int m, int num_sms) {
    const int64_t ctx_bytes = N * (7 * 8 + 2 * 16 + 4 * 8) + Nc * 32 + ((int64_t)4 << 20);
    return ctx_bytes + default_scratch_bytes(N, num_sms) + Engine::member_bytes(N, 1, m) + Nc * 32;
}

void finish(pb_server *sv, Lane &L, Request *r, int status, double energy, int iters) {
    pb_server_result res;
    memset(&res, 0, sizeof(res));
    res.id = r->id;
    res.status = status;
    res.energy_kcal = energy;
    res.iters = iters;
    res.n = r->N;
    const Clock::time_point now = Clock::now();
    res.latency_ms = ms_between(r->t_submit, now);
    res.queue_ms = r->member ? ms_between(r->t_submit, r->t_admit) : res.latency_ms;
    if (r->member) {
        L.eng->remove(r->member);
        r->member = nullptr;
    }
    if (r->ctx) {
        pb_destroy(r->ctx);
        r->ctx = nullptr;
    }
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->used_bytes -= r->bytes;
    sv->stats.completed += 1;
    if (status != PB_OK) sv->stats.failed += 1;
    sv->done.push_back(res);
    sv->cv.notify_all();
    delete r;
}

// Admit a lane's queued requests that fit; runs on the lane's worker.
void admit(pb_server *sv, Lane &L) {
    for (;;) {
        Request *r = nullptr;
        bool too_big = false;
        {
            std::lock_guard<std::mutex> lock(sv->mu);
            if (L.pending.empty() || (int)L.active.size() >= sv->opts.max_active) return;
            Request *head = L.pending.front();
            too_big = head->bytes > sv->opts.hbm_budget_bytes;
            if (!too_big && sv->used_bytes + head->bytes > sv->opts.hbm_budget_bytes) return;   // wait for memory
            L.pending.pop_front();
            r = head;
            sv->used_bytes += r->bytes;            // released by finish()
            if (too_big) sv->stats.rejected += 1;
            else sv->stats.admitted += 1;
        }
        if (too_big) {
            finish(sv, L, r, PB_ERR_ADMIT, 0.0, 0);
            continue;
        }
        r->t_admit = Clock::now();
        pb_status s = pb_create(r->c.data(), r->n.data(), r->a.data(), r->N, r->Nc > 0 ? r->q.data() : nullptr, r->Nc,
                                r->eps1, r->eps2, r->kappa, L.stream, &r->ctx);
        if (s != PB_OK) {
            finish(sv, L, r, s, 0.0, 0);
            continue;
        }
        r->member = L.eng->add(r->ctx, r->q.data(), r->Nc, 1, r->id, &s);
        if (s != PB_OK || !r->member) {
            r->member = nullptr;
            finish(sv, L, r, s == PB_OK ? PB_ERR_CUDA : s, 0.0, 0);
            continue;
        }
        // the context now holds the geometry: drop the host copies
        std::vector<double>().swap(r->c);
        std::vector<double>().swap(r->n);
        std::vector<double>().swap(r->a);
        std::lock_guard<std::mutex> lock(sv->mu);
        L.active.push_back(r);
        L.n_active.store((int)L.active.size());
    }
}

// Large lane: while the small lane runs requests, symmetric products use one
// CTA per SM fewer than their occupancy in one pass (no bands: the launches
// of overlapping bands would take the slots), so small-lane kernels find
// slots; otherwise their default bands.
pb_status set_yield(Lane &L, bool yield) {
    for (Request *r : L.active) {
        pb_ctx *c = r->ctx;
        if (!c || !f32_variant_symmetric(c->f32_variant)) continue;
        c->bands = yield ? 1 : 0;
        const int occ = matvec_f32_occupancy(c->f32_variant);
        const int want = (yield && occ > 1) ? occ - 1 : 0;
        if (want == r->cps) continue;
        pb_status s = matvec_configure(c, c->f32_variant, want);
        if (s == PB_OK) s = matvec_prepare(c);
        if (s != PB_OK) return s;
        r->cps = want;
    }
    return PB_OK;
}

void worker_main(pb_server *sv, int li) {
    cudaSetDevice(sv->device);
    Lane &L = sv->lanes[li];
    Lane *other = (sv->nlanes == 2) ? &sv->lanes[1 - li] : nullptr;
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(sv->mu);
            if (sv->stop && L.pending.empty() && L.active.empty()) break;
            if (L.active.empty() && L.pending.empty()) sv->cv.wait_for(lock, std::chrono::milliseconds(2));
        }
        admit(sv, L);
        std::vector<Request *> act;
        {
            std::lock_guard<std::mutex> lock(sv->mu);
            act = L.active;
        }
        if (act.empty()) continue;
        pb_status s = PB_OK;
        // the two lanes share the SMs while both run: the large lane's
        // symmetric products leave one CTA slot per SM, the small lane's
        // batched product uses one CTA per SM (so it fits in those slots)
        if (li == 1 && other) s = set_yield(L, other->n_active.load() > 0);
        if (li == 0 && other) L.eng->set_cta_cap(other->n_active.load() > 0 ? 1 : 0);
        if (s == PB_OK) s = L.eng->cycle(false);
        {
            std::lock_guard<std::mutex> lock(sv->mu);
            sv->stats.cycles += 1;
            sv->lane_evals[li] = L.eng->pair_evals;
            sv->lane_products[li] = L.eng->pair_products;
            sv->stats.pair_evals = sv->lane_evals[0] + sv->lane_evals[1];
            sv->stats.pair_products = sv->lane_products[0] + sv->lane_products[1];
            const int total = (int)(sv->lanes[0].active.size() + (sv->nlanes == 2 ? sv->lanes[1].active.size() : 0));
            if (total > sv->stats.max_active_seen) sv->stats.max_active_seen = total;
        }
        for (Request *r : act) {
            bool fin = (s != PB_OK) || r->member->finished;
            if (!fin) continue;
            int st = s;
            double e = 0.0;
            int it = r->member->status[0].iters;
            if (s == PB_OK) {
                st = r->member->status[0].converged ? PB_OK
                                                    : (r->member->status[0].status == PB_OK ? PB_ERR_NOCONV
                                                                                            : r->member->status[0].status);
                pb_status es = L.eng->energies(r->member, &e);
                if (es != PB_OK) st = es;
            }
            {
                std::lock_guard<std::mutex> lock(sv->mu);
                for (size_t i = 0; i < L.active.size(); ++i)
                    if (L.active[i] == r) {
                        L.active.erase(L.active.begin() + i);
                        break;
                    }
                L.n_active.store((int)L.active.size());
            }
            finish(sv, L, r, st, e, it);
        }
    }
}

}  // namespace

extern "C" {

pb_status pb_server_create(const pb_server_opts *opts, pb_server **out) {
    if (!out) return set_error(nullptr, PB_ERR_ARG, "pb_server_create: out is NULL");
    *out = nullptr;
    pb_server_opts o{8, (int64_t)8 << 30, 10, 1e-4, 1000, 0};
    if (opts) {
        o = *opts;
        if (o.max_active <= 0) o.max_active = 8;
        if (o.hbm_budget_bytes <= 0) o.hbm_budget_bytes = (int64_t)8 << 30;
        if (o.restart <= 0) o.restart = 10;
        if (!(o.tol > 0.0)) o.tol = 1e-4;
        if (o.maxit <= 0) o.maxit = 1000;
    }
    if (o.restart > kMaxRestart) return set_error(nullptr, PB_ERR_ARG, "pb_server_create: restart > %d", kMaxRestart);
    pb_server *sv = new pb_server();
    sv->opts = o;
    sv->nlanes = o.split_n < 0 ? 1 : 2;
    sv->split_n = o.split_n > 0 ? o.split_n : kDefaultSplitN;
    int lo = 0, hi = 0;
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sv->num_sms, cudaDevAttrMultiProcessorCount, sv->device);
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo, &hi);   // hi: the highest priority
    for (int li = 0; li < sv->nlanes && e == cudaSuccess; ++li)
        e = cudaStreamCreateWithPriority(&sv->lanes[li].stream, cudaStreamNonBlocking, li == 0 ? hi : lo);
    if (e != cudaSuccess) {
        for (int li = 0; li < 2; ++li)
            if (sv->lanes[li].stream) cudaStreamDestroy(sv->lanes[li].stream);
        delete sv;
        return cuda_error(nullptr, e, "pb_server_create");
    }
    for (int li = 0; li < sv->nlanes; ++li) {
        sv->lanes[li].index = li;
        sv->lanes[li].eng = new Engine(sv->lanes[li].stream, sv->device, sv->num_sms, o.restart, o.tol, o.maxit);
    }
    sv->t0 = Clock::now();
    for (int li = 0; li < sv->nlanes; ++li) sv->lanes[li].worker = std::thread(worker_main, sv, li);
    *out = sv;
    return PB_OK;
}

pb_status pb_server_submit(pb_server *sv, const double *centroids, const double *normals, const double *areas,
                           int64_t N, const double *charges, int64_t Nc, double eps1, double eps2, double kappa,
                           uint64_t *id) {
    if (!sv || !centroids || !normals || !areas || N < 1 || Nc < 0 || (Nc > 0 && !charges))
        return set_error(nullptr, PB_ERR_ARG, "pb_server_submit: bad arguments");
    if (!(eps1 > 0.0) || !(eps2 > 0.0) || !(kappa >= 0.0))
        return set_error(nullptr, PB_ERR_ARG, "pb_server_submit: need eps1 > 0, eps2 > 0, kappa >= 0");
    Request *r = new Request();
    r->c.assign(centroids, centroids + 3 * N);
    r->n.assign(normals, normals + 3 * N);
    r->a.assign(areas, areas + N);
    if (Nc > 0) r->q.assign(charges, charges + 4 * Nc);
    r->N = N;
    r->Nc = Nc;
    r->eps1 = eps1;
    r->eps2 = eps2;
    r->kappa = kappa;
    r->bytes = footprint(N, Nc, sv->opts.restart, sv->num_sms);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        if (sv->stop) {
            delete r;
            return set_error(nullptr, PB_ERR_ARG, "pb_server_submit: server is shutting down");
        }
        r->id = sv->next_id++;
        sv->lanes[(sv->nlanes == 2 && N >= sv->split_n) ? 1 : 0].pending.push_back(r);
        sv->stats.submitted += 1;
        if (id) *id = r->id;
    }
    sv->cv.notify_all();
    return PB_OK;
}

int pb_server_poll(pb_server *sv, pb_server_result *out, int max) {
    if (!sv || !out || max <= 0) return 0;
    std::lock_guard<std::mutex> lock(sv->mu);
    int n = 0;
    while (n < max && !sv->done.empty()) {
        out[n++] = sv->done.front();
        sv->done.pop_front();
    }
    return n;
}

pb_status pb_server_wait(pb_server *sv, int64_t n_results, double timeout_s) {
    if (!sv) return set_error(nullptr, PB_ERR_ARG, "pb_server_wait: NULL server");
    std::unique_lock<std::mutex> lock(sv->mu);
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
    while ((int64_t)sv->done.size() < n_results) {
        if (sv->cv.wait_until(lock, until) == std::cv_status::timeout && (int64_t)sv->done.size() < n_results)
            return set_error(nullptr, PB_ERR_TIMEOUT, "pb_server_wait: %lld of %lld results after %.3f s",
                             (long long)sv->done.size(), (long long)n_results, timeout_s);
    }
    return PB_OK;
}

pb_status pb_server_get_stats(pb_server *sv, pb_server_stats *out) {
    if (!sv || !out) return set_error(nullptr, PB_ERR_ARG, "pb_server_get_stats: NULL argument");
    std::lock_guard<std::mutex> lock(sv->mu);
    *out = sv->stats;
    out->active = 0;
    out->pending = 0;
    for (int li = 0; li < sv->nlanes; ++li) {
        out->active += (int)sv->lanes[li].active.size();
        out->pending += (int)sv->lanes[li].pending.size();
    }
    out->used_bytes = sv->used_bytes;
    return PB_OK;
}

void pb_server_destroy(pb_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        // drop requests that were never admitted
        for (int li = 0; li < sv->nlanes; ++li) {
            while (!sv->lanes[li].pending.empty()) {
                delete sv->lanes[li].pending.front();
                sv->lanes[li].pending.pop_front();
            }
        }
    }
    sv->cv.notify_all();
    for (int li = 0; li < sv->nlanes; ++li)
        if (sv->lanes[li].worker.joinable()) sv->lanes[li].worker.join();   // finishes the active requests
    for (int li = 0; li < sv->nlanes; ++li) {
        delete sv->lanes[li].eng;
        cudaStreamDestroy(sv->lanes[li].stream);
    }
    delete sv;
}

}  // extern "C"
