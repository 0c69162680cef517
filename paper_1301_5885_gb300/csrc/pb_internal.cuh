// pb_internal.cuh -- shared declarations of the CUDA library behind include/pb.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pb.h"

namespace pb {

// e_c^2 / (4 pi eps_0 * 1 Angstrom) in kcal/mol (the energy unit of Eq. (14)).
constexpr double kCoulombKcal = 332.0636;
constexpr double kPi = 3.14159265358979323846;
constexpr double kInv4Pi = 1.0 / (4.0 * kPi);

constexpr int kMaxRestart = 64;       // largest GMRES restart length supported

// One point charge (centred position and charge in e_c), 32-byte aligned so a
// warp loads it with two 16-byte transactions per lane.
struct alignas(32) Charge4 {
    double x, y, z, q;
};

// ---- matvec tiling ---------------------------------------------------------
// FP32-pair kernel: 128 threads x 4 targets = 512 targets per target tile,
// 256 sources per shared-memory source tile.
constexpr int kF32Threads = 128;
constexpr int kF32TargetsPerThread = 4;
constexpr int kF32TargetTile = kF32Threads * kF32TargetsPerThread;
constexpr int kF32SourceTile = 256;
// FP32-pair kernel variants (one is chosen per context, by default or by the
// autotuner): targets per thread and scalar or packed f32x2 arithmetic.
// The symmetric variants evaluate each unordered pair once for both rows.
enum MatvecVariant {
    MV_F32_SCALAR_T4 = 1,
    MV_F32_PACKED_T2 = 2,
    MV_F32_PACKED_T4 = 3,
    MV_F32_PACKED_T3 = 4,
    MV_F32_SYM_T2 = 5,
    MV_F32_SYM_T4 = 6
};
constexpr int kNumF32Variants = 6;
__host__ __device__ constexpr int f32_variant_targets(int v) {
    return (v == MV_F32_PACKED_T2 || v == MV_F32_SYM_T2) ? 2 : (v == MV_F32_PACKED_T3 ? 3 : 4);
}
__host__ __device__ constexpr bool f32_variant_symmetric(int v) {
    return v == MV_F32_SYM_T2 || v == MV_F32_SYM_T4;
}
// FP64 product variants: the plain stream-K kernel, or the symmetric one with
// 1 or 2 targets per thread.
enum Matvec64Variant { MV_F64_PLAIN = 1, MV_F64_SYM_T1 = 2, MV_F64_SYM_T2 = 3 };
constexpr int kNumF64Variants = 3;
// FP64 kernel: 128 threads x 1 target, 128 sources per source tile.
constexpr int kF64Threads = 128;
constexpr int kF64TargetTile = kF64Threads;
constexpr int kF64SourceTile = 128;

// Stream-K style split of the (target tile x source tile) iteration space over
// a fixed number of persistent CTAs.  CTA c owns the flattened tile-pair range
// [c*W/G, (c+1)*W/G); target tile a is covered by the contiguous CTAs
// cta_of(a*S) .. cta_of(a*S + S - 1).
struct StreamKPlan {
    int64_t target_tiles;   // T
    int64_t source_tiles;   // S
    int64_t work;           // W = T * S
    int64_t ctas;           // G, 1 <= G <= W
    int64_t max_segments;   // largest number of CTAs covering one target tile
};

__host__ __device__ inline int64_t sk_begin(int64_t c, int64_t W, int64_t G) { return (c * W) / G; }
// the CTA whose range contains tile-pair p: ceil((p+1) G / W) - 1
__host__ __device__ inline int64_t sk_cta_of(int64_t p, int64_t W, int64_t G) {
    return ((p + 1) * G + W - 1) / W - 1;
}

StreamKPlan make_plan(int64_t n, int target_tile, int source_tile, int64_t ctas_wanted);
// the same split for n_targets target rows against n_sources sources
StreamKPlan make_plan_rows(int64_t n_targets, int64_t n_sources, int target_tile, int source_tile,
                           int64_t ctas_wanted);

// Target rows of a plain product: rows [row0, row0 + nrows) of both row
// blocks of A u, the phi rows written to y[0, nrows) and the psi rows to
// y[ld, ld + nrows); {0, N, N} is the whole product.
struct RowBlock {
    int64_t row0, nrows, ld;
};

// Split of the upper triangle of square tile pairs (I <= J, numbered row by
// row) of the symmetric product over persistent CTAs, with the same range
// rule as StreamKPlan.
struct SymPlan {
    int64_t tiles;          // square tiles of the targets
    int64_t work;           // tile pairs of this launch (all tiles (tiles + 1) / 2 of them unbanded)
    int64_t ctas;
    int64_t work_begin = 0; // first tile pair of this launch (a band of rows)
    int64_t joff = 0;       // off-diagonal index of the band's first column side (its slot 0)
};
SymPlan make_sym_plan(int64_t n, int tile, int64_t ctas_wanted);
// a new context's bound on each symmetric product's scratch: 1 GiB (the
// FP32-pair product stays in one band up to about 365,000 triangles)
constexpr int64_t kDefaultScratchLimit = int64_t(1) << 30;
// device bytes of the symmetric product's scratch (row sides, split-row
// slots, column sides per off-diagonal tile pair)
int64_t sym_scratch_bytes(const SymPlan &pl, int tile);
// the same under a bound of limit bytes (0: none) for column sides of elem
// bytes; cuts receives the band cuts of row tiles (two entries: one band)
int64_t sym_scratch_need(const SymPlan &pl, int tile, int elem, int64_t limit, int bands,
                         std::vector<int64_t> *cuts);

// ---- GMRES device state ----------------------------------------------------
struct GmresState {
    double H[(kMaxRestart + 1) * kMaxRestart];   // column-major, ld = kMaxRestart + 1
    double cs[kMaxRestart], sn[kMaxRestart];
    double g[kMaxRestart + 1];
    double h1[kMaxRestart + 1];   // first Gram-Schmidt pass coefficients
    double h2[kMaxRestart + 1];   // second pass
    double y[kMaxRestart];
    double bnorm;
    double beta;                  // ||r0|| of the current cycle
    double hnext;                 // H[k+1][k] of the current step
    double rel_resid;             // last true relative residual
    double est_resid;             // Givens estimate |g[k+1]| / bnorm
    double tol;
    int m;                        // restart length
    int maxit;
    int k;                        // Arnoldi columns completed in this cycle
    int iters;                    // total Arnoldi steps
    int cycles;
    int cycle_done;               // 1: remaining steps of this cycle are skipped
    int done;                     // 1: converged or stopped; every kernel is skipped
    int skip;                     // done || cycle_done (read by the matvec kernels)
    int converged;
    int status;                   // pb_status
    int x_is_zero;                // the current x is exactly zero (skip A x)
};

}  // namespace pb

// ---- context -----------------------------------------------------------------
struct pb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t N = 0, Nc = 0;
    double eps1 = 1, eps2 = 1, eps = 1, kappa = 0;
    double center[3] = {0, 0, 0};
    double gauss_min = 0, gauss_max = 0;
    int num_sms = 0;

    // geometry, shifted by center
    double *g64 = nullptr;       // SoA 7N: x | y | z | nx | ny | nz | W
    float4 *pos32 = nullptr;     // {x, y, z, W / (4 pi)}
    float4 *nrm32 = nullptr;     // {nx, ny, nz, 0}
    pb::Charge4 *charges = nullptr;  // {x, y, z, Q}, Nc entries (capacity nc_cap)
    int64_t nc_cap = 0;

    // vectors (2N each)
    double *b = nullptr;         // right-hand side for the current charges
    double *x = nullptr;         // last solution
    bool b_valid = false, x_valid = false;
    pb_precision b_prec = PB_FP64;   // pair arithmetic of the stored b
    pb_precision e_prec = PB_FP64;   // of the last solve's energy (pb_energy repeats it)

    // matvec scratch: per (target tile, segment) partial row sums, and one
    // arrival counter per target tile (left at zero between launches)
    pb::StreamKPlan plan32{}, plan64{};
    int f32_variant = 0;         // MatvecVariant of the FP32-pair product
    int f32_ctas_per_sm = 0;
    double *partials = nullptr;
    int64_t partials_len = 0;
    // symmetric variants: their plan and scratch (allocated when configured)
    pb::SymPlan plansym{};
    void *sym_scratch = nullptr;
    int64_t sym_scratch_len = 0;   // bytes
    // float-float product (PB_FLOAT2): the plain plan (shares partials and
    // tile counters) and the symmetric one's plan and scratch
    pb::StreamKPlan planff{};
    pb::SymPlan planffsym{};
    void *symff_scratch = nullptr;
    int64_t symff_scratch_len = 0;
    // FP64 product variant (Matvec64Variant) and the symmetric one's plan and scratch
    int f64_variant = 1;
    pb::SymPlan plansym64{};
    void *sym64_scratch = nullptr;
    int64_t sym64_scratch_len = 0;
    // bound on each symmetric product's scratch (bytes, 0: none) and the band
    // cuts of row tiles each product runs in (FP32 pairs, FP64, float-float)
    int64_t scratch_limit = pb::kDefaultScratchLimit;
    int bands = 0;                 // requested bands: 0 automatic, 1 none, n >= 2 at least n
    std::vector<int64_t> cuts32, cuts64, cutsff;
    // second stream and events of a banded product (created by its first one)
    cudaStream_t band_stream = nullptr;
    cudaEvent_t band_ev[3] = {nullptr, nullptr, nullptr};
    unsigned int *tile_counters = nullptr;
    int64_t counters_len = 0;

    // reductions
    double *red = nullptr;       // block partials
    int64_t red_len = 0;
    unsigned int *red_counter = nullptr;
    double *scalar = nullptr;    // device scalars (energy, norms)
    double *host_scalar = nullptr;   // pinned

    // GMRES workspace
    int gm_m = 0;
    double *V = nullptr;         // (m+1) x 2N
    double *w = nullptr;         // 2N
    double *r = nullptr;         // 2N
    double *d = nullptr;         // 2N (refinement correction)
    double *rres = nullptr;      // 2N (refinement residual b - A_fp64 x)
    pb::GmresState *st = nullptr;
    pb::GmresState *st_host = nullptr;   // pinned

    // device count of evaluated matrix-vector products (scalar[8] as uint64)
    unsigned long long *mv_count = nullptr;

    // optional event timing of the matvec launches (pb_profile_enable)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;
    int prof_used = 0;
    double prof_ms = 0.0;
    int64_t prof_launches = 0;
    unsigned long long prof_count_base = 0;

    // row-block products (pb_matvec_rows and the sharded solve): their own
    // stream-K partials and tile counters
    double *rows_partials = nullptr;
    int64_t rows_partials_len = 0;   // doubles
    unsigned int *rows_counters = nullptr;
    int64_t rows_counters_len = 0;

    // row-sharded solve (pb_solve_sharded): while on, every FP32-pair or FP64
    // product computes this rank's rows, gathers all ranks' rows through the
    // caller's allgather and unpacks them into the full 2N vector
    struct Shard {
        bool on = false;
        int world = 1, rank = 0;
        int64_t row0 = 0, nrows = 0, per = 0;   // this rank's rows; rows per rank (padded)
        pb_allgather_fn fn = nullptr;
        void *user = nullptr;
        double *send = nullptr, *recv = nullptr;
        int64_t cap = 0;                        // doubles in recv
        int64_t bytes = 0;                      // device bytes of send and recv
        int64_t gathers = 0;
    } shard;

    int64_t device_bytes = 0;
    char last_error[512] = {0};
};

namespace pb {

// error helpers (pb_api.cu)
pb_status set_error(pb_ctx *ctx, pb_status s, const char *fmt, ...);
pb_status cuda_error(pb_ctx *ctx, cudaError_t e, const char *what);
void count_launch();
void count_launches(int n);
#define PB_LAUNCHED() ::pb::count_launch()

// stream-ordered allocation from the library's pool of the current device
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t stream);
// pinned host blocks, cached for reuse (pinned_free returns a block to the cache)
cudaError_t pinned_alloc(void **p, size_t bytes);
void pinned_free(void *p, size_t bytes);
// allocation on the context's stream (stream-ordered pool)
pb_status ctx_alloc(pb_ctx *ctx, void **p, size_t bytes, const char *what);
void ctx_free(pb_ctx *ctx, void *p);

// geom.cu
pb_status geometry_prepare(pb_ctx *ctx, const double *c_dev, const double *n_dev, const double *a_dev);
pb_status charges_prepare(pb_ctx *ctx, const double *q_dev, int64_t nc);
pb_status gauss_check(pb_ctx *ctx, double *gmin, double *gmax);

// matvec.cu
pb_status matvec_launch(pb_ctx *ctx, const double *u, double *y, pb_precision prec, const int *skip_flag);
int matvec_occupancy(pb_precision prec);
int matvec_f32_occupancy(int variant);
// plan of an FP32 variant at a CTA count per SM (0 = the variant's occupancy)
StreamKPlan matvec_f32_plan(pb_ctx *ctx, int variant, int ctas_per_sm);
// partial-row capacity (doubles) a plan needs
int64_t plan_partials(const StreamKPlan &pl, int target_tile);
pb_status matvec_configure(pb_ctx *ctx, int variant, int ctas_per_sm);
// allocates the scratch the configured FP32 variant needs (on ctx->stream), so
// that later products allocate nothing (for example inside a stream capture)
pb_status matvec_prepare(pb_ctx *ctx);
// rows [rb.row0, rb.row0 + rb.nrows) of both blocks of A u into y (2 nrows:
// phi rows, then psi rows), FP32 pairs (packed kernel) or FP64 (plain kernel)
pb_status matvec_rows_launch(pb_ctx *ctx, const double *u, double *y, RowBlock rb, pb_precision prec,
                             const int *skip_flag);
// the sharded product: own rows, the caller's allgather, unpack (shard.cu)
pb_status shard_product(pb_ctx *ctx, const double *u, double *y, pb_precision prec, const int *skip_flag);
// matvec_ff.cu: the float-float product (PB_FLOAT2)
StreamKPlan matvec_ff_plan(pb_ctx *ctx);
int matvec_ff_target_tile();
// the second stream and events of banded symmetric products (matvec.cu)
pb_status ensure_band_streams(pb_ctx *ctx);
// scratch bytes and band cuts of the symmetric float-float product (0 and no
// cuts below the size that uses it)
int64_t ff_sym_scratch_need(pb_ctx *ctx, std::vector<int64_t> *cuts);
pb_status matvec_ff_enqueue(pb_ctx *ctx, const double *u, double *y, const int *skip_flag);
// Eq. (11) and Eq. (14) with float-float pair arithmetic (matvec_ff.cu)
pb_status source_ff_launch(pb_ctx *ctx, double *b);
pb_status energy_ff_launch(pb_ctx *ctx, const double *u, double *dev_out);
// FP64 product variant (Matvec64Variant); the symmetric ones allocate their
// scratch with their first product
pb_status matvec_configure_fp64(pb_ctx *ctx, int variant);
int64_t sym64_scratch_bytes(const SymPlan &pl, int tile);
// tune.cu: the stored or built-in FP32 kernel choice for this context's size
void default_f32_config(pb_ctx *ctx, int *variant, int *ctas_per_sm);
// built-in FP64 product variant for n points
int default_f64_variant(int64_t n);
// device scratch of the built-in default product for n points (an estimate
// for admission control; the symmetric variants' scratch, else 0)
int64_t default_scratch_bytes(int64_t n, int num_sms);

// pb_api.cu: fold recorded matvec event pairs into ctx->prof_ms (syncs the stream)
pb_status profile_flush(pb_ctx *ctx);

// source_energy.cu
pb_status source_launch(pb_ctx *ctx, double *b, pb_precision prec);
pb_status energy_launch(pb_ctx *ctx, const double *u, pb_precision prec, double *dev_out);

// gmres.cu
pb_status gmres_solve(pb_ctx *ctx, const pb_solve_opts *o, const double *rhs, double *x, bool x_is_zero,
                      int *iters, int *cycles, double *rel_resid);
pb_status norm2_launch(pb_ctx *ctx, const double *v, int64_t n, double *dev_out);

// reduction sizing shared by the kernels
constexpr int kRedThreads = 256;
int red_blocks(pb_ctx *ctx, int64_t n);

}  // namespace pb
