// engine.cuh -- the lockstep solver engine behind pb_batch_solve and the
// solve server: a changing set of GMRES instances (one per surface and charge
// set) advanced one restart cycle at a time with batched kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pb_internal.cuh"

namespace pb {

constexpr int kEngineMaxRhs = 8;

struct BSurf;
struct BInst;
struct BChunk;

// Shape and grid of the batched product (bmatvec.cuh): targets per thread,
// placement and arithmetic of the row sums, CTAs per SM (0: the occupancy).
struct BmvConfig {
    int T = 0;
    int acc = 0;
    int ctas_per_sm = 0;
};

struct BStatus {
    int done, converged, status, iters, cycles, pad;
    double rel_resid;
};

// One surface with its charge sets (one GMRES instance per set).
struct EngineMember {
    pb_ctx *surf = nullptr;      // geometry (not owned)
    int nrhs = 0;
    int64_t nc = 0;
    Charge4 *q = nullptr;        // device, nrhs x nc, centred like the surface
    double *vec = nullptr;       // device, per set: b, x, w, r, V((m+1) x 2N)
    GmresState *st = nullptr;    // device, nrhs states
    BStatus status[kEngineMaxRhs] = {};
    bool finished = false;
    uint64_t tag = 0;
    int64_t bytes = 0;           // device bytes held by this member
};

class Engine {
  public:
    Engine(cudaStream_t stream, int device, int num_sms, int m, double tol, int maxit);
    ~Engine();

    // Adds a surface with nrhs host charge sets of nc rows (x, y, z, Q):
    // allocates its vectors, computes b = [S1; S2] (Eq. (11), float-float
    // pairs) and ||b||, and
    // initialises its GMRES states (x0 = 0).  Returns the member, or null.
    EngineMember *add(pb_ctx *surf, const double *charges_host, int64_t nc, int nrhs, uint64_t tag, pb_status *st);
    // Frees a member's device memory and drops it from the set.
    void remove(EngineMember *m);
    // One restart cycle of every unfinished instance (lockstep).  Fills the
    // members' status and marks members whose instances are all done.  With
    // time_products (no graph), the product launches are bracketed by CUDA
    // events and their time is added to matvec_ms.
    pb_status cycle(bool use_graph, bool time_products = false);
    // The same in two halves, so that several engines on their own streams
    // can run their cycles at the same time: prepare() rebuilds the tables
    // (and tunes) if the member set changed, launch_cycle() enqueues the cycle
    // and the copies of its results without waiting, finish_cycle() waits for
    // them and updates the members.
    pb_status prepare();
    pb_status launch_cycle(bool use_graph, bool time_products = false);
    pb_status finish_cycle();
    // Caps the batched product's CTAs per SM (0: no cap); takes effect at the
    // next cycle (the tables are rebuilt).
    void set_cta_cap(int cap) {
        if (cap != cta_cap_) {
            cta_cap_ = cap;
            dirty_ = true;
        }
    }
    // Eq. (14) for every instance of a member (float-float pairs), kcal/mol.
    pb_status energies(EngineMember *m, double *out);
    // Bytes one member of N triangles with nrhs sets needs (vectors and states).
    static int64_t member_bytes(int64_t N, int nrhs, int m);

    const std::vector<EngineMember *> &members() const { return members_; }
    int64_t matvec_launches = 0;
    double matvec_ms = 0.0;      // event time of timed product launches
    int64_t pair_evals = 0;      // K1..K4 pair evaluations of the products
    int64_t pair_products = 0;   // times the charge sets they served
    int cycles_run = 0;
    int rhs_width = 1;
    int64_t ctas = 0;
    // batched-product shape: with autotune, a batch whose (width, size class)
    // has no cached choice is tuned when its tables are built (every shape at
    // every CTA count, timed on the batch's own work list); otherwise the
    // cached choice of the nearest size class, else the built-in default
    bool autotune = false;
    BmvConfig config;
    bool tuned = false;           // the last rebuild ran the tuner
    int tune_candidates = 0;
    double tune_ms = 0.0;         // host time spent tuning
    char error[512] = {0};

  private:
    pb_status rebuild();
    pb_status tune(std::vector<BSurf> &hs, const std::vector<char> &direct, int64_t size_class);
    void retile(std::vector<BSurf> &hs, const std::vector<char> &direct, int64_t TT, int64_t *tiles, int64_t *work);
    pb_status grow(void **p, size_t *cap, size_t need, size_t elem, const char *what);
    void enqueue_cycle();
    pb_status fail(pb_status s, const char *fmt, ...);
    pb_status cuda_fail(cudaError_t e, const char *what);

    cudaStream_t stream_;
    int device_, num_sms_, m_, maxit_;
    double tol_;
    std::vector<EngineMember *> members_;
    bool dirty_ = true;
    // current tables
    int nsurf_ = 0, nq_ = 0, nchunks_ = 0, R_ = 1;
    int64_t W_ = 0, G_ = 0, tiles_ = 0;
    std::vector<int> surf_member_;     // table surface -> member index
    std::vector<int> direct_;          // table surfaces with their own symmetric product
    BSurf *d_surf_ = nullptr;
    int64_t *d_wbase_ = nullptr;       // the work split of the current product (bmv_plan_kernel)
    size_t cap_wbase_ = 0;
    BInst *d_inst_ = nullptr;
    BChunk *d_ch_ = nullptr;
    unsigned int *cnt_inst_ = nullptr, *cnt_tile_ = nullptr;
    unsigned long long *evals_ = nullptr;
    int *act_step_ = nullptr, *act_ax_ = nullptr;
    double *red_ = nullptr, *part_ = nullptr, *scalar_ = nullptr;
    BStatus *d_status_ = nullptr, *h_status_ = nullptr;
    size_t cap_surf_ = 0, cap_inst_ = 0, cap_ch_ = 0, cap_cnt_inst_ = 0, cap_cnt_tile_ = 0, cap_evals_ = 0,
           cap_flags_ = 0, cap_red_ = 0, cap_part_ = 0, cap_status_ = 0;
    std::vector<unsigned long long> last_evals_;
    unsigned long long *h_evals_ = nullptr;   // pinned copy of the product counters
    size_t cap_h_evals_ = 0;
    bool launched_ = false;                   // a cycle was launched and not finished
    cudaGraphExec_t gexec_ = nullptr;
    cudaGraph_t graph_ = nullptr;
    int kernels_per_cycle_ = 0, mv_per_cycle_ = 0, cycle_kernels_ = 0, cycle_mv_ = 0;
    bool timing_ = false;
    int cta_cap_ = 0;            // CTAs per SM of the batched product at most (0: none)
    BmvConfig kept_;             // an autotuning engine's choice, kept across rebuilds
    int kept_R_ = 0;
    std::vector<cudaEvent_t> ev_;
    int ev_used_ = 0;
};

}  // namespace pb
