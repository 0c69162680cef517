/*
 * pb.h -- C ABI of the GB300 direct-sum boundary-integral linear
 * Poisson-Boltzmann library (the well-conditioned formulation of Geng & Jacob,
 * "A GPU-accelerated Direct-sum Boundary Integral Poisson-Boltzmann Solver").
 *
 * The problem (Section 1, Eqs. (1)-(4)): a solute region Omega_1 with dielectric
 * constant eps1 holding Nc point charges, bounded by a closed surface Gamma,
 * inside a solvent with dielectric constant eps2 and inverse Debye length
 * kappa.  Gamma is given as N flat triangles with centroid collocation
 * (Section 2.2): centroid x_i, unit outward normal nu_i, area W_i.
 *
 * The unknowns are u = [phi_1..phi_N, dphi/dnu_1..dphi/dnu_N] at the centroids;
 * the system A u = b is Eqs. (12)-(13) with the kernels K1..K4 of Eq. (10)
 * (eps = eps2/eps1), and b = [S1(x_i); S2(x_i)] of Eq. (11) with each charge
 * divided by eps1.  The electrostatic solvation energy is Eq. (14), reported in
 * kcal/mol (332.0636 kcal/mol per e_c^2/(4 pi eps_0 Angstrom)).
 *
 * Conventions for every entry point:
 *  - Lengths in Angstrom, charges in e_c, energies in kcal/mol.
 *  - Vectors of length 2N are FP64, contiguous, device memory owned by the
 *    caller (for example a torch tensor's data_ptr()).
 *  - All GPU work of a context is ordered on the CUDA stream given to
 *    pb_create (a banded symmetric product forks part of its launches to a
 *    second stream of the context and joins it back on that stream; see
 *    pb_set_bands).  pb_matvec and pb_source only enqueue work; pb_solve, pb_energy,
 *    pb_energy_of and pb_create return after the stream has finished the work
 *    they enqueued.
 *  - Every call returns a pb_status and never aborts, traps or exits.  On
 *    failure pb_last_error(ctx) (or pb_last_error(NULL) when no context
 *    exists) holds a one-line message.
 *  - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef PB_H
#define PB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pb_ctx pb_ctx;   /* opaque; owns all the device memory it allocates */

typedef enum {
    PB_OK = 0,
    PB_ERR_ARG = 1,       /* invalid argument (NULL pointer, N <= 0, eps <= 0, ...) */
    PB_ERR_BADMESH = 2,   /* area <= 0 or non-finite, normal far from unit length,
                             or the Gauss orientation check failed */
    PB_ERR_OOM = 3,       /* device allocation failed */
    PB_ERR_CUDA = 4,      /* a CUDA runtime call failed */
    PB_ERR_NOCONV = 5,    /* GMRES reached maxit without meeting tol */
    PB_ERR_NAN = 6,       /* a non-finite residual or Hessenberg entry appeared */
    PB_ERR_TIMEOUT = 7,   /* a bounded wait gave up */
    PB_ERR_ADMIT = 8      /* a request does not fit the memory budget */
} pb_status;

typedef enum {
    PB_FP64 = 0,          /* every pair in FP64, FP64 accumulation */
    PB_FP32PAIR = 1,      /* pair arithmetic in FP32 (hardware rsqrt/exp2),
                             FP32 partial sums per source tile, FP64 row sums */
    PB_FLOAT2 = 2         /* pair arithmetic in float-float (each value the
                             unevaluated sum of two FP32 numbers, about 44
                             bits; about 1e-12 relative per pair term) on the
                             FP32 pipe, FP64 row sums: FP64-level products at
                             several times the FP64 kernel's speed where the
                             FP64 rate is a small fraction of FP32.  From
                             N = 2,048 each unordered pair is evaluated once
                             for both rows, with device scratch of about
                             8 N^2 / 256 bytes in one pass (less in bands,
                             see pb_set_bands) allocated by the first such
                             product.  Accepted by pb_matvec, pb_solve
                             (prec, refine_prec), pb_source and pb_energy_of
                             (the N x Nc pair sums of Eqs. (11) and (14)). */
} pb_precision;

typedef struct {
    int restart;          /* GMRES restart length m (>= 1); 10 if 0 */
    double tol;           /* stop when ||b - A x||_2 / ||b||_2 <= tol; 1e-4 if 0 */
    int maxit;            /* maximum Arnoldi steps (products with A); 1000 if 0 */
    pb_precision prec;    /* precision of the products with A inside GMRES */
    int refine;           /* number of FP64 iterative-refinement steps after a
                             PB_FP32PAIR solve: r = b - A_fp64 x, solve A d = r
                             with the same options, x += d.  0 = none */
    pb_precision refine_prec; /* precision of the refinement residual product
                             (and of the final residual check): PB_FP64 (the
                             default, 0) or PB_FLOAT2 */
} pb_solve_opts;

typedef struct {
    int iters;            /* Arnoldi steps taken, all refinement passes included */
    int cycles;           /* GMRES restart cycles */
    double rel_resid;     /* final true relative residual, in the precision of
                             the last product used to measure it */
    double energy_kcal;   /* E_sol of Eq. (14) for the solution, FP64 reduction */
    double rel_resid_fp64;/* ||b - A_fp64 x|| / ||b|| when refine > 0, else -1 */
    int refine_steps;     /* refinement steps taken */
    int64_t matvecs;      /* products with A the device actually evaluated
                             (Arnoldi steps, true residuals, refinement) */
} pb_solve_info;

typedef struct {
    int64_t n;            /* triangles */
    int64_t nc;           /* charges */
    double eps1, eps2, kappa;
    double center[3];     /* the shift subtracted from every coordinate (bounding-box centre) */
    double gauss_min, gauss_max; /* min / max over charges of sum_j W_j dG0(x_k, x_j)/dnu_j
                                    (about -1 for charges inside a closed outward surface) */
    int64_t device_bytes; /* device memory held by the context */
} pb_ctx_info;

/* Create a context for one surface and one charge set (Sections 2.2 and 2.4).
 * centroids, normals: N x 3 row-major; areas: N; charges: Nc x 4 rows (x, y, z, Q).
 * Each pointer may be host or device memory (detected per pointer); the data
 * are copied, the caller keeps ownership.  The geometry is validated (areas
 * finite and > 0, normals within 1e-3 of unit length; normals are then
 * renormalised), shifted by the bounding-box centre, packed into FP64 and FP32
 * device arrays, and checked for orientation: every charge must see a Gauss
 * sum in (-1.5, -0.5).  Nc may be 0 (then charges may be NULL).
 * cuda_stream: a cudaStream_t, or NULL for the legacy default stream.
 * Errors: PB_ERR_ARG, PB_ERR_BADMESH, PB_ERR_OOM, PB_ERR_CUDA; *out is NULL then. */
pb_status pb_create(const double *centroids, const double *normals, const double *areas, int64_t N,
                    const double *charges, int64_t Nc, double eps1, double eps2, double kappa,
                    void *cuda_stream, pb_ctx **out);

/* Replace the charge set (a new right-hand side on the same surface; Eq. (11)).
 * Same pointer rules as pb_create.  Invalidates the stored solution. */
pb_status pb_set_charges(pb_ctx *ctx, const double *charges, int64_t Nc);

/* b = [S1(x_i); S2(x_i)] of Eq. (11) into the caller's device buffer b (2N). */
pb_status pb_source(pb_ctx *ctx, double *b, pb_precision prec);

/* y = A u, Eqs. (12)-(13).  u, y: device, 2N each, must not overlap.  Enqueued
 * on the context's stream.  Uses the context's scratch memory, so calls on one
 * context are serialised by its stream.  prec: PB_FP32PAIR (the kernel chosen
 * by pb_matvec_configure), PB_FP64 (the one chosen by
 * pb_matvec_configure_fp64) or PB_FLOAT2; a symmetric kernel's scratch is
 * allocated by its first product (PB_ERR_OOM if that fails). */
pb_status pb_matvec(pb_ctx *ctx, const double *u, double *y, pb_precision prec);

/* Solve A u = b with restarted GMRES on the device (Section 2.4; x0 = 0 unless
 * x0 is given, restarts continue from the current approximation), then
 * evaluate Eq. (14).  The source term b and the energy take FP64 pairs when
 * prec is PB_FP64 (the plain path) and float-float pairs otherwise (about
 * 1e-12 relative per pair term, on the FP32 pipe).  x0: device 2N or NULL.  x_out: device 2N or NULL; the
 * solution is also kept in the context for pb_energy.  info may be NULL.
 * Returns PB_ERR_NOCONV (solution and info still filled) if maxit is reached. */
pb_status pb_solve(pb_ctx *ctx, const pb_solve_opts *opts, const double *x0, double *x_out,
                   pb_solve_info *info);

/* Eq. (14) for the solution of the last successful pb_solve, in the pair
 * arithmetic that solve used for its energy. */
pb_status pb_energy(pb_ctx *ctx, double *energy_kcal);

/* Eq. (14) for an arbitrary device vector u (2N): (1/2) sum_k Q_k phi_reac(x_k). */
pb_status pb_energy_of(pb_ctx *ctx, const double *u, pb_precision prec, double *energy_kcal);

/* Context facts (sizes, centring shift, Gauss orientation sums, memory). */
pb_status pb_get_info(pb_ctx *ctx, pb_ctx_info *info);

/* Free all device memory of the context.  NULL is accepted. */
void pb_destroy(pb_ctx *ctx);

/* Static string for a status code. */
const char *pb_status_string(pb_status s);

/* Last error message of a context, or of the calling thread when ctx is NULL. */
const char *pb_last_error(const pb_ctx *ctx);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t pb_kernel_launches(void);

/* Device memory of contexts, batches and servers comes from a library-owned
 * stream-ordered pool per device that keeps freed memory for reuse.  This
 * returns the pool's unused memory of the current device to the driver
 * (after synchronising the device) and frees the cached pinned host blocks
 * that no context holds.  Memory in use is not affected.  A library
 * convenience; the paper has no counterpart. */
pb_status pb_release_cached_memory(void);

/* Kernel timing for measurement (not part of the method).  While enabled,
 * every matrix-vector product launched by this context is bracketed by CUDA
 * events recorded on the context's stream.  pb_profile_read waits for the
 * stream, then returns the summed event time of those launches in ms, the
 * number of timed launches, and the number of products the device actually
 * evaluated (launches whose GMRES state said "skip" return at once and are
 * timed but not counted there).  reset != 0 clears the totals. */
pb_status pb_profile_enable(pb_ctx *ctx, int enable);
pb_status pb_profile_read(pb_ctx *ctx, double *matvec_ms, int64_t *timed_launches, int64_t *evaluated,
                          int reset);

/* Batched solves (many surfaces of uneven N, each with 1..8 charge sets).
 * ctxs[s]: a context per surface (its geometry is used; its own charges are
 * not); charges[s]: host array of nrhs[s] charge sets of nc[s] rows each
 * (nrhs[s] x nc[s] x 4, rows x, y, z, Q).  Every (surface, charge set) pair is
 * a GMRES instance (Section 2.4, restarted, x0 = 0) solved with FP32-pair
 * products; all instances advance in lockstep and each lockstep product is one
 * persistent launch over all surfaces that evaluates K1..K4 once per pair for
 * all charge sets of a surface; a surface with a single charge set whose
 * context is configured for a symmetric product variant (the default for
 * N >= 16,384) takes its own launch of that product instead.  The members
 * are split into two halves of about equal pair work, each run by its own
 * engine: one on ctxs[0]'s stream, one on a second stream of the same
 * priority created for the call (it waits for the work enqueued on ctxs[0]'s
 * stream before the call, and the call returns after both are done), their
 * restart cycles launched together so that each fills the SMs the other's
 * launches leave idle (pb_batch_set_streams(1): one engine on ctxs[0]'s
 * stream).  The other contexts must not be in use meanwhile.  use_graph = 1 captures one restart
 * cycle of the whole batch in a CUDA graph and replays it (ignored on the
 * legacy default stream); 0 launches the kernels one by one; 2 launches them
 * one by one and times every product launch with CUDA events (matvec_ms).
 * energies: host array of sum(nrhs) doubles (kcal/mol,
 * Eq. (14)), in surface-major order.  Returns PB_ERR_NOCONV if an instance
 * reached maxit (energies still filled).  This is a library extension for
 * throughput; the paper solves one molecule per run. */
typedef struct {
    int instances;        /* sum of nrhs */
    int converged;
    int cycles;           /* lockstep restart cycles */
    int iters_max;        /* largest Arnoldi step count of an instance */
    int64_t iters_sum;
    double rel_resid_max; /* largest final true relative residual */
    int rhs_width;        /* charge sets per product kernel (1, 2, 4 or 8) */
    int64_t ctas;         /* persistent CTAs of the product kernel */
    int64_t pair_evals;   /* K1..K4 pair evaluations, sum over products of N(N-1) */
    int64_t pair_products;/* pair evaluations times the charge sets they served */
    int64_t matvec_launches;
    double matvec_ms;     /* summed CUDA-event time of the product launches
                             (only measured when use_graph == 2) */
    int targets_per_thread; /* shape of the batched product in the last cycle */
    int row_sums;           /* PB_ROWSUM_* of that shape */
    int ctas_per_sm;        /* 0: the kernel's occupancy */
    int tuned;              /* 1 if the autotuner ran during this call */
    int tune_candidates;    /* (shape, CTA count) pairs it timed */
    double tune_ms;         /* host time it took */
    double setup_ms;        /* host time of the set-up: vectors, source terms, norms */
    double cycles_ms;       /* host time of the restart cycles (tuning included) */
    double energy_ms;       /* host time of the energies (Eq. (14), FP64) */
    int streams;            /* engines (streams) the call ran: 1 or 2 */
} pb_batch_info;

pb_status pb_batch_solve(pb_ctx *const *ctxs, int nsurf, const double *const *charges, const int64_t *nc,
                         const int *nrhs, const pb_solve_opts *opts, int use_graph, double *energies,
                         pb_batch_info *info);
/* Engines of pb_batch_solve: 2 (default; one engine when nsurf is 1) or 1.
 * Other n: PB_ERR_ARG. */
pb_status pb_batch_set_streams(int n);

/* Shapes of the batched product (a library extension; the paper has a single
 * one-target-per-thread kernel).  A shape is (targets per thread, row sums):
 * more targets per thread share each staged source among more targets; the
 * row sums of every target row are kept in FP64 or in float-float (an
 * unevaluated sum of two FP32 numbers, about 48 significant bits), in
 * registers or in the thread's shared-memory slots.  Every shape computes the
 * same Eqs. (12)-(13) with FP32 pair terms summed per 256-source stage; they
 * differ only in summation arithmetic (results agree to the FP32-pair
 * tolerance).  The third knob is the number of CTAs per SM.
 *
 * pb_batch_solve tunes by default: the first batch of a (width, size class)
 * (size class: a quarter octave of the summed N^2 of its batched surfaces)
 * times every instantiated shape at every CTA count on its own work list
 * (two launches each after a warm-up) when its tables are built, and caches
 * the fastest per device; later batches, and the solve server, use the cached
 * choice of the nearest size class within an octave (the server never tunes
 * inline), else the built-in default.  pb_batch_info reports the shape used.
 *
 * pb_batch_set_tuning: mode 1 = as above (default); 0 = built-in defaults only.
 * pb_batch_force_shape: use (targets_per_thread, row_sums, ctas_per_sm) for
 *   every batch of this width; targets_per_thread = 0 removes the override.
 *   PB_ERR_ARG for a shape that is not instantiated.
 * pb_batch_clear_tuning: forget the cached choices.
 * pb_batch_shapes: the instantiated shapes of a width (the default first);
 *   returns their number, writes at most max_out. */
enum { PB_ROWSUM_FP64_REGISTERS = 0, PB_ROWSUM_FP64_SHARED = 1, PB_ROWSUM_FF_REGISTERS = 2,
       PB_ROWSUM_FF_SHARED = 3 };
pb_status pb_batch_set_tuning(int mode);
pb_status pb_batch_force_shape(int rhs_width, int targets_per_thread, int row_sums, int ctas_per_sm);
pb_status pb_batch_clear_tuning(void);
int pb_batch_shapes(int rhs_width, int *targets_per_thread, int *row_sums, int max_out);

/* Solve server with continuous batching (a library extension for serving;
 * the paper runs one molecule per run).  pb_server_create starts a worker
 * thread with its own CUDA stream on the current device.  pb_server_submit
 * (any thread) copies a request (host arrays, same layout as pb_create) into
 * the queue and returns its id.  The worker admits queued requests in arrival
 * order while fewer than max_active are running and their estimated device
 * footprint fits hbm_budget_bytes (larger than the whole budget: result
 * status PB_ERR_ADMIT), and advances all running requests together one GMRES
 * restart cycle at a time (FP32-pair products, FP64 Krylov arithmetic), so
 * requests that arrive while others run join at the next cycle boundary.
 * Results (energy of Eq. (14), status, latency from submit to result, time
 * queued) are collected with pb_server_poll; pb_server_wait blocks until at
 * least n results are waiting or the timeout passes (PB_ERR_TIMEOUT).
 * pb_server_destroy drops requests not yet admitted, finishes the running
 * ones, and frees everything.
 * Two lanes (split_n >= 0): requests with N < split_n (whose products share
 * one batched launch) and the others (each with its own symmetric product)
 * run on two worker threads and streams, the small lane's with the higher
 * priority; max_active applies per lane and the budget to both together.
 * While small requests run, the large lane's products use one CTA per SM
 * fewer than their occupancy, which leaves the small lane's kernels room to
 * run at the same time. */
typedef struct pb_server pb_server;
typedef struct {
    int max_active;           /* running requests at most (8 if <= 0) */
    int64_t hbm_budget_bytes; /* device memory for running requests (8 GiB if <= 0) */
    int restart;              /* GMRES restart (10 if <= 0) */
    double tol;               /* relative residual (1e-4 if <= 0) */
    int maxit;                /* Arnoldi steps per request (1000 if <= 0) */
    int64_t split_n;          /* requests with N >= split_n go to the large lane (16,384 if 0; < 0: one lane) */
} pb_server_opts;
typedef struct {
    uint64_t id;
    int status;               /* pb_status of the request */
    int iters;
    double energy_kcal;
    double latency_ms;        /* submit -> result */
    double queue_ms;          /* submit -> admission */
    int64_t n;
} pb_server_result;
typedef struct {
    int64_t submitted, admitted, rejected, completed, failed;
    int64_t cycles;
    int64_t pair_evals, pair_products;
    int active, pending, max_active_seen;
    int64_t used_bytes;
} pb_server_stats;

pb_status pb_server_create(const pb_server_opts *opts, pb_server **out);
pb_status pb_server_submit(pb_server *sv, const double *centroids, const double *normals, const double *areas,
                           int64_t N, const double *charges, int64_t Nc, double eps1, double eps2, double kappa,
                           uint64_t *id);
int pb_server_poll(pb_server *sv, pb_server_result *out, int max);
pb_status pb_server_wait(pb_server *sv, int64_t n_results, double timeout_s);
pb_status pb_server_get_stats(pb_server *sv, pb_server_stats *out);
void pb_server_destroy(pb_server *sv);

/* Kernel choice for the FP32-pair product (a tuning knob of this library; the
 * paper has a single FP64 kernel).  variant: 1 = scalar FP32, 4 targets per
 * thread; 2 = packed f32x2, 2 targets per thread; 3 = packed f32x2, 4 targets
 * per thread; 4 = packed f32x2, 3 targets per thread; 5 and 6 = symmetric
 * packed f32x2 with 2 and 4 targets per thread (each unordered pair of
 * Eqs. (12)-(13) evaluated once for both of its rows, using K1(i,j) = K1(j,i),
 * K4(i,j) = K4(j,i) and the sign change of c_x, c_y under the exchange; two
 * kernel launches per product in one pass, two per band in bands (see
 * pb_set_bands); device scratch of about 4 N^2 / (128 t) bytes in one pass,
 * t the targets per thread, less in bands, allocated by the first product that uses the
 * variant and freed when another variant is configured; that product returns
 * PB_ERR_OOM if it cannot be allocated); 0 = the
 * stored or built-in default.  The packed variants use a kappa = 0
 * specialisation when the context's kappa is 0.  ctas_per_sm: resident CTAs
 * per SM of the persistent grid, 0 = as many as fit.  Results differ between
 * variants only by FP32 rounding.  pb_matvec_autotune times every candidate
 * (reps launches each) on the context's geometry, keeps the fastest, and
 * stores the choice for later contexts of similar N on the same device. */
pb_status pb_matvec_configure(pb_ctx *ctx, int variant, int ctas_per_sm);
pb_status pb_matvec_get_config(pb_ctx *ctx, int *variant, int *ctas_per_sm, int64_t *ctas);
pb_status pb_matvec_autotune(pb_ctx *ctx, int reps, int *variant, int *ctas_per_sm, double *best_ms);

/* Kernel choice for the FP64 product (PB_FP64 in pb_matvec, and the residual
 * of the refinement in pb_solve).  variant: 1 = plain (every ordered pair);
 * 2 and 3 = symmetric with 1 and 2 targets per thread (each unordered pair of
 * Eqs. (12)-(13) evaluated once for both rows, as in the FP32-pair variants
 * 5 and 6, with FP64 column sides; scratch of about 8 N^2 / (128 t) bytes in
 * one pass, t the targets per thread, less in bands (see pb_set_bands),
 * allocated by the first product and freed when
 * the plain variant is configured); 0 = the built-in default for the
 * context's N (symmetric from N = 2,048, with 2 targets per thread from
 * 65,536; pb_create applies it).  All variants do every pair and every sum in FP64; results
 * differ only by summation order.  *variant_out (may be NULL) receives the
 * variant now in use. */
pb_status pb_matvec_configure_fp64(pb_ctx *ctx, int variant, int *variant_out);

/* Bands of the symmetric products (FP32-pair variants 5 and 6, FP64
 * variants 2 and 3, the float-float product).  Their column sides take about
 * 4 N^2 / B bytes of device scratch in one pass (B the targets of a tile;
 * 8 N^2 / B with FP64 column sides).  In bands, the product runs over whole
 * row tiles at a time, with about equal numbers of column sides per band:
 * each band's pair kernel is followed by a finishing kernel that completes
 * the band's rows and adds its column sides of the later row tiles to FP64
 * accumulators (16 N bytes), and consecutive bands alternate between the
 * context's stream and a second one (created by the first banded product),
 * so that a band's pair kernel fills the SMs that the previous one's last
 * CTAs leave idle; two sets of slots and column sides are kept for that.
 * Every row is still summed in a fixed order: results are deterministic and
 * differ from the one-pass product only by the rounding of that order.
 *
 * pb_set_scratch_limit: bound on each symmetric product's scratch in bytes;
 * 0: none.  pb_create sets 1 GiB, under which the FP32-pair product of up to
 * about 365,000 triangles needs no band for memory (the FP64 and float-float
 * ones to about 180,000).  Bands take as many column sides as the bound leaves
 * room for after the parts that grow with N only, and at least one row tile
 * each (so a bound below one row's column sides is exceeded).  Frees the
 * context's current symmetric scratch (the next product allocates it again).
 * bytes < 0: PB_ERR_ARG.
 *
 * pb_set_bands: bands requested besides the bound.  0 (the default):
 * automatic, as many as give every CTA of the product's persistent grid at
 * least 5 tile pairs per band, at most 72 requested (for the FP32-pair
 * product: one pass below about 28,000 triangles, 6 bands at 81,920, 79 at
 * 300,176);
 * 1: none; n >= 2: at least n (or one row tile per band where the row
 * tiles are fewer).  Except for n >= 2, a product takes one pass
 * whenever bands would need more scratch than one pass.  Takes effect at the
 * next product.  bands < 0: PB_ERR_ARG. */
pb_status pb_set_scratch_limit(pb_ctx *ctx, int64_t bytes);
pb_status pb_set_bands(pb_ctx *ctx, int bands);

/* The band plan of a symmetric product without a context (host only, no
 * GPU): n targets in square tiles of `tile` targets (a multiple of 128),
 * `ctas` persistent CTAs, column sides of elem bytes (4: FP32 pairs, 8: FP64
 * and float-float), a scratch bound `limit` (0: none) and a band request as
 * for pb_set_bands.  cuts receives up to max_cuts row-tile boundaries
 * 0 = R_0 < R_1 < ... < R_m = tiles (band k holds row tiles [R_k, R_k+1));
 * *ncuts = m + 1 and *bytes = the scratch (either may be NULL).  This is the
 * plan pb_matvec uses for a context with that kernel choice, bound and
 * request.  Bad arguments: PB_ERR_ARG. */
pb_status pb_sym_band_plan(int64_t n, int tile, int64_t ctas, int elem, int64_t limit, int bands,
                           int64_t *cuts, int max_cuts, int *ncuts, int64_t *bytes);

/* Bands and scratch bytes of the symmetric product of precision prec at the
 * context's current kernel choice, bound and band request; 0 and 0 when that
 * product is not a symmetric one.  Either pointer may be NULL.  Unknown prec:
 * PB_ERR_ARG. */
pb_status pb_scratch_plan(pb_ctx *ctx, pb_precision prec, int *bands, int64_t *bytes);

/* Row-block product: rows [row0, row0 + nrows) of both row blocks of
 * Eqs. (12)-(13), y_rows[t] = (A u)_{row0 + t} and y_rows[nrows + t] =
 * (A u)_{N + row0 + t} for t < nrows.  u: device, 2N FP64 (all of it is
 * read); y_rows: device, 2 nrows FP64, caller-owned, must not overlap u.
 * prec: PB_FP32PAIR (the packed stream-K kernel) or PB_FP64 (the plain FP64
 * kernel); PB_ERR_ARG for PB_FLOAT2 or rows outside [0, N).  The same sums
 * as the plain full product restricted to those rows (the symmetric
 * variants have no row-block form).  Scratch grows on first use. */
pb_status pb_matvec_rows(pb_ctx *ctx, const double *u, double *y_rows, int64_t row0, int64_t nrows,
                         pb_precision prec);

/* Row-sharded solve over `world` ranks, one GPU each (a library extension;
 * the paper names multiple GPUs as future work, Section 4).  Rank p owns
 * rows [p P, p P + n_p), P = ceil(N / world) (pb_shard_rows).  Every rank
 * creates its own context with the whole surface and the same charges and
 * calls pb_solve_sharded with the same options; GMRES, the source term and
 * the energy run replicated, and each product of A evaluates only the rank's
 * rows, then calls
 *     allgather(user, send, recv, count, cuda_stream)
 * with send: device, count = 2P doubles (the rank's phi rows in the first P
 * slots, its psi rows in the next P; unused slots zero) and recv: device,
 * world x count doubles to be filled in rank order; the callback must enqueue
 * the collective so that it is ordered after the work already on cuda_stream
 * and before work enqueued after it returns (NCCL on that stream does this),
 * and return 0 on success (anything else ends the solve with PB_ERR_CUDA).
 * It is called from the calling thread, once per product.  The gathered rows
 * are unpacked into the full 2N vector on every rank, so every rank holds the
 * same x, info and energy.  Options, x0, x_out, info and errors as for
 * pb_solve; PB_FP32PAIR or PB_FP64 products only (PB_ERR_ARG for PB_FLOAT2,
 * including as the refinement precision). */
typedef int (*pb_allgather_fn)(void *user, const double *send, double *recv, int64_t count, void *cuda_stream);
pb_status pb_solve_sharded(pb_ctx *ctx, const pb_solve_opts *opts, int rank, int world, pb_allgather_fn allgather,
                           void *user, const double *x0, double *x_out, pb_solve_info *info);

/* Host helpers of the sharded layout (no GPU needed): the rows of a rank,
 * and the unpacking of a gathered buffer (world blocks of 2P doubles, as
 * above) into the 2N vector [phi; psi]. */
pb_status pb_shard_rows(int64_t N, int world, int rank, int64_t *row0, int64_t *nrows, int64_t *rows_per_rank);
pb_status pb_shard_unpack_host(const double *gathered, int64_t N, int world, double *y);

/* No-allocation matrix-vector product.  The paper has no counterpart: this is
 * a library convenience for callers that cannot call cudaMalloc (for example
 * code running under a framework whose caching allocator already owns all of
 * the device memory, or a latency-critical path where an allocation, which may
 * synchronise the device, is not acceptable).  It computes the same y = A u as
 * pb_matvec(..., PB_FP32PAIR) without a pb_ctx and without allocating:
 *  - centroids, normals: device, N x 3 row-major FP64; areas: device, N FP64;
 *    normals must already be unit length and areas > 0 (no validation pass);
 *  - center: host, 3 doubles subtracted from every centroid before the FP32
 *    cast (pass the bounding-box centre, as pb_create does; NULL = origin);
 *  - u, y: device, 2N FP64 each; the caller owns them.  y must not overlap
 *    u or any geometry array (other CTAs still read them while y is written):
 *    such calls are rejected with PB_ERR_ARG;
 *  - the work is enqueued on cuda_stream (NULL = legacy default stream).
 * Scratch lives in one 16 MiB file-scope static device array that every GPU
 * loading the library keeps until the process exits.  Its arrival counters are
 * cleared by every call; every call shares the array, so calls that overlap
 * on the GPU race and must not be issued.  Every call resolves the array's
 * device address (cudaGetSymbolAddress, no allocation) with the caller's
 * device current, and the first call on a device also queries its SM count
 * and the kernel's occupancy; make that first call before any stream capture.
 * N above 2^24 = 16,777,216 is rejected with PB_ERR_ARG (a fixed limit of the
 * static scratch).  Errors: PB_ERR_ARG, PB_ERR_CUDA; messages via
 * pb_last_error(NULL). */
pb_status pb_matvec_f32_static(const double *centroids, const double *normals, const double *areas, int64_t N,
                               const double *center, double eps1, double eps2, double kappa, const double *u,
                               double *y, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PB_H */
