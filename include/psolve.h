/*
 * psolve.h -- C ABI of libpsolve, a single-GPU (B300, sm_103a) solver for the
 * 3-D Poisson equation -Laplace(phi) = f (Eq. 1) discretised with the
 * second-order 7-point finite-difference operator (Eq. 3, Eq. 6) and zero
 * Dirichlet boundaries (the 1-D matrix D of Eq. 4), by preconditioned
 * Bi-CGSTAB (Algorithm 1) with Chebyshev-iteration preconditioners (Eq. 15,
 * Algorithm 2) on the whole grid, G(CI), or per block, BJ(CI) and
 * GNoComm(CI) (Eq. 12-14 and the preconditioner summary, Table 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid vectors are contiguous arrays of n = nx*ny*nz doubles, x fastest:
 *     index(i, j, k) = i + nx * (j + ny * k),  0 <= i < nx, ...
 * (a torch tensor of shape [nz, ny, nx], float64, contiguous).  Unless an
 * entry point says "host", every vector pointer is a DEVICE pointer on the
 * current CUDA device, 8-byte aligned, owned by the caller, and must stay
 * valid until the call returns (or, for psolve_submit, until psolve_poll
 * reports a status other than PSOLVE_PENDING).
 *
 * Grid spacing h[3] = (hx, hy, hz) > 0; the interior points are
 * x_i = (i + 1) hx etc. (the unit cube has h_d = 1/(n_d + 1)).
 *
 * All work is ordered on the CUDA stream passed at creation (a cudaStream_t
 * cast to uintptr_t; 0 = the legacy default stream).  Solves are
 * synchronous: they return after the result is known.  A context is not
 * thread-safe: use one context per host thread.
 *
 * Every call returns a psolve_status and never aborts the process; on error
 * psolve_last_error() gives a message for the calling thread.  There is no
 * CPU fallback: without a usable CUDA device the calls return
 * PSOLVE_E_CUDA.
 */
#ifndef PSOLVE_H
#define PSOLVE_H

#include <stdint.h>

#if defined(__GNUC__)
#define PSOLVE_API __attribute__((visibility("default")))
#else
#define PSOLVE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PSOLVE_OK = 0,            /* converged (or nothing to do)                 */
    PSOLVE_E_ARG = 1,         /* invalid argument; nothing was launched       */
    PSOLVE_E_OOM = 2,         /* device or pinned allocation failed           */
    PSOLVE_E_CUDA = 3,        /* a CUDA runtime call failed                   */
    PSOLVE_NOT_CONVERGED = 4, /* maxit reached; x holds the last iterate      */
    PSOLVE_BREAKDOWN = 5,     /* r~.w, t.t, omega or rho became exactly zero  */
    PSOLVE_NONFINITE = 6,     /* NaN/Inf met in a reduction                   */
    PSOLVE_TIMEOUT = 7,       /* a bounded wait gave up                       */
    PSOLVE_PENDING = 8,       /* psolve_poll: request not finished yet        */
    PSOLVE_REJECTED = 9       /* psolve_submit: exceeds the memory budget     */
} psolve_status;

/* Preconditioner M of Algorithm 1 (Table 1). */
typedef enum {
    PSOLVE_PC_NONE = 0,         /* M = I: plain Bi-CGSTAB                         */
    PSOLVE_PC_CHEB = 1,         /* G(CI): Chebyshev iteration on the whole grid   */
    PSOLVE_PC_BJ_CHEB = 2,      /* BJ(CI): Chebyshev per block (Eq. 14), bounds
                                   of one block                                   */
    PSOLVE_PC_GNOCOMM_CHEB = 3, /* GNoComm(CI): per block, bounds of the whole
                                   grid                                           */
    PSOLVE_PC_G_BICGS = 4,      /* G(BiCGS): an inner Bi-CGSTAB solve of A z = v
                                   on the whole grid (opts.inner_rtol,
                                   inner_maxit); the outer iteration is then the
                                   flexible Bi-CGSTAB (FBiCGS) of the paper       */
    PSOLVE_PC_BJ_BICGS = 5      /* BJ(BiCGS): inner Bi-CGSTAB solves on each block
                                   (Eq. 13-14), all blocks in one batched solve   */
} psolve_precond;

/* Storage precision of the Chebyshev preconditioner's vectors.  The outer
 * Bi-CGSTAB vectors, its dot products and alpha/omega/beta stay FP64. */
typedef enum {
    PSOLVE_FP64 = 0,  /* everything FP64                                    */
    PSOLVE_FP32 = 1,  /* Chebyshev vectors FP32, FP32 arithmetic             */
    PSOLVE_BF16 = 2   /* Chebyshev vectors stored BF16, FP32 arithmetic      */
} psolve_prec;

typedef struct {
    /* Chebyshev interval [a, b] = [lmin_scale * lambda_min, lmax_scale *
     * lambda_max], lambda from the closed form (Eq. 9-11).  1, 1 = exact
     * bounds.  The experimental set-up's rescaling for G(CI)/GNoComm(CI) is
     * lmin_scale = 100, lmax_scale = 1 - 1e-4. */
    double lmin_scale;
    double lmax_scale;
    /* Number of equal blocks along x, y, z for BJ(CI) / GNoComm(CI); each
     * must divide the grid size on its axis. */
    int32_t blocks[3];
    int32_t cheb_prec;       /* psolve_prec                                  */
    int32_t half_step_check; /* 1: exit after the alpha half-step when
                                ||s||/||b|| <= rtol (Algorithm 1); 0: never */
    int32_t use_x0;          /* 1: x_dev holds the initial guess x0; 0: x0 = 0 */
    int32_t poll_every;      /* outer iterations per host status check; 0 = auto */
    int32_t use_graph;       /* 1: replay captured CUDA graphs; 0: plain launches */
    int32_t timing;          /* 1: time each kernel class with CUDA events
                                (plain launches); see psolve_result           */
    int32_t true_residual;   /* 1: recompute ||b - A x||/||b|| at exit        */
    int32_t rr_every;        /* residual replacement: after the update of
                                every outer iteration that is a multiple of
                                rr_every, replace the recursive r by the true
                                b - A x, rescale beta and rho to it (rho =
                                r~ . r) and take the stop test on its norm
                                (0 = never).  Meant for the mixed-precision
                                forms; not part of the paper's method.       */
    int32_t engine;          /* stencil kernels: 0 = TMA ring where possible
                                (16-byte aligned vectors; when nx is not a
                                multiple of 8 the context lays its vectors out
                                with rows padded to one and copies b and x
                                through padded staging vectors), else the
                                general engine; 1 = always the general engine
                                (no tensor copies, no padding)                */
    int32_t persistent;      /* 1: run the whole solve (r0, every outer
                                iteration, the exit true residual) as ONE
                                cooperative kernel launch whose phases are
                                separated by grid barriers, captured in a
                                CUDA graph when use_graph = 1.  Results are
                                bitwise those of the per-kernel path.  Not
                                with timing = 1.  A barrier wait that gives up
                                (4 s) ends the solve with PSOLVE_TIMEOUT.     */
    int32_t autotune;        /* 1: pick the slab depth (z planes per work
                                unit) and the stencil engine of each grid
                                shape by timing candidates on the GPU (at
                                psolve_create, or per shape in a batch);
                                decisions are cached per process and, when
                                the environment variable PSOLVE_TUNE_CACHE
                                names a file, in that file across processes.
                                0: built-in rule.                            */
    int32_t inner_maxit;     /* G(BiCGS) / BJ(BiCGS): inner iteration limit
                                (default 500)                                */
    int32_t record_history;  /* 1: psolve_solve records the relative residual
                                norms ||s_i||/||b|| (after the alpha half step)
                                and ||r_i||/||b|| (after the update) of every
                                outer iteration i of Algorithm 1 -- the
                                convergence history the paper plots -- for
                                psolve_history.  The device writes one double
                                per norm from the reduction that computes it
                                (no extra pass, no host round trip); the
                                context keeps a buffer of 2 * maxit doubles,
                                grown when a solve asks for more iterations.
                                Contexts only (not batch or server).         */
    int32_t slab_share;      /* how many grids of this shape the slab-depth
                                rule takes to share every launch: the more,
                                the deeper the slabs (z planes per work unit)
                                it picks, hence fewer units and less
                                per-unit overhead when many grids fill the
                                GPU together.  0 = the entry point's own: 1
                                (a grid alone) for psolve_create,
                                PSOLVE_SHARED_SLAB_SHARE for
                                psolve_solve_batch and psolve_submit.  The
                                decomposition fixes the order of every
                                reduction, so a batched or served problem's
                                result is bitwise that of a context created
                                with the same slab_share (and otherwise the
                                same options).  Ignored with autotune = 1.   */
    double inner_rtol;       /* and inner relative tolerance; 0 = the
                                experimental set-up's 1e-2 for G(BiCGS) and
                                1e-6 for BJ(BiCGS)                           */
} psolve_opts;

/* Fill *o with the defaults: scales 1, 1; blocks 1,1,1; FP64; half-step check
 * on; x0 = 0; poll auto; graphs on; timing off; true residual on; rr off;
 * engine auto; per-kernel launches (persistent off); autotune off; inner
 * solves (G(BiCGS), BJ(BiCGS)) at the set-up's tolerances, 500 iterations;
 * no residual history; slab_share 0 (the entry point's own). */
PSOLVE_API void psolve_opts_default(psolve_opts *o);

/* Kernel classes reported by timing mode (psolve_result.kclass_*). */
enum {
    PSOLVE_K_INIT = 0,        /* r0 and norms                                  */
    PSOLVE_K_CI_FIRST = 1,    /* direction / half-step update fused with CI
                                 sweep 1                                       */
    PSOLVE_K_CI_SWEEP3 = 2,   /* CI sweep k = 2 (reads 2 vectors, writes 1)     */
    PSOLVE_K_CI_SWEEP4 = 3,   /* CI sweeps k >= 3 (reads 3 vectors, writes 1)   */
    PSOLVE_K_STENCIL_DOT = 4, /* w = A p^, r~.w                                */
    PSOLVE_K_STENCIL_2DOT = 5,/* t = A r^, t.s, t.t                            */
    PSOLVE_K_UPDATE = 6,      /* x, r update with r~.r, r.r                    */
    PSOLVE_K_OTHER = 7,       /* true residual, unpreconditioned updates, ...  */
    PSOLVE_K_NCLASS = 8
};

typedef struct {
    int32_t status;            /* psolve_status of the solve                   */
    int32_t iterations;        /* outer index i at exit (0 if r0 passes)       */
    int32_t half_step_exit;    /* 1 if the exit was the ||s|| half-step test   */
    int32_t engine;            /* stencil engine used: 1 TMA ring, 0 general   */
    int32_t slab_planes;       /* z planes per work unit of the grid          */
    int32_t tuned;             /* 1: slab and engine chosen by the autotuner,
                                  2: taken from its on-disk cache, 0: rule    */
    double rel_res_recursive;  /* ||r||/||b|| of the recursive residual        */
    double rel_res_true;       /* ||b - A x||/||b|| at exit (if enabled)       */
    double seconds;            /* wall time of the call                        */
    double model_bytes;        /* algorithmic HBM bytes of the work done       */
    int64_t kernel_launches;   /* kernels launched by this call (incl. no-ops) */
    int64_t inner_iterations;  /* G(BiCGS) / BJ(BiCGS): inner Bi-CGSTAB
                                  iterations over all inner solves (for BJ the
                                  largest block count of each solve)          */
    /* timing mode only: per kernel class, summed CUDA-event milliseconds,
     * number of launches that did work, and algorithmic bytes they moved. */
    double kclass_ms[PSOLVE_K_NCLASS];
    int64_t kclass_launches[PSOLVE_K_NCLASS];
    double kclass_bytes[PSOLVE_K_NCLASS];
} psolve_result;

typedef struct psolve_ctx psolve_ctx;

/* Create a solver for one grid.
 *   grid[3] = (nx, ny, nz) unknowns per axis, each >= 1, product < 2^31.
 *   h[3]    = (hx, hy, hz) > 0.
 *   bc[6]   = condition on the faces x-, x+, y-, y+, z-, z+: 0 zero Dirichlet
 *             (the boundary node is known and 0; matrix D, Eq. 4), 1 zero-flux
 *             Neumann (the boundary node is the first / last unknown and its
 *             outside neighbour equals its inside one; matrix N, Eq. 5).  A
 *             Neumann face needs at least 2 unknowns on its axis (and 2 per
 *             block for BJ/GNoComm); at least one face must be Dirichlet.
 *             NULL means all Dirichlet.  The Chebyshev bounds use the closed
 *             form of each axis's spectrum (D: Eq. 9; N with one Neumann face:
 *             4 sin^2((2i-1) pi / (4n)); Neumann on both faces: [0, 4]).
 *   opts    = NULL for psolve_opts_default().
 *   stream  = cudaStream_t (as uintptr_t) that orders all work.
 * Allocates the device workspace (at most 12 grid vectors) once; returns
 * PSOLVE_E_ARG for bad sizes, blocks < 1 or bad face conditions, PSOLVE_E_OOM if
 * it does not fit.  *out is set only on success. */
PSOLVE_API psolve_status psolve_create(const int64_t grid[3], const double h[3], const int32_t bc[6],
                            const psolve_opts *opts, uintptr_t stream, psolve_ctx **out);

/* Solve A x = b (Algorithm 1) to ||r||/||b|| <= rtol or maxit iterations.
 *   rhs_dev : b (device, read only).
 *   x_dev   : out: x.  In: x0 if opts.use_x0, else ignored (x0 = 0).
 *   rtol >= 0 (0 runs exactly maxit iterations unless a residual is 0).
 *   maxit >= 0.
 *   precond : psolve_precond; degree = Chebyshev iterations d of Algorithm 2
 *             (0 <= d <= 64; = number of A applications; 0 gives b/theta).
 *             Ignored by G(BiCGS) and BJ(BiCGS).  For GNoComm(CI) the paper
 *             bounds useful degrees by N_s/2, N_s the block side (beyond it
 *             the error from the frozen block ghosts has reached every point):
 *             a degree above half the smallest block side still runs, and
 *             psolve_last_error() then holds a "warning: ..." message while
 *             the status is that of the solve.
 * G(BiCGS) / BJ(BiCGS) run the flexible Bi-CGSTAB: x is updated with the
 * preconditioned vectors themselves, each an inner Bi-CGSTAB solve from x0 = 0
 * with the half-step test, stopped at opts.inner_rtol or opts.inner_maxit (an
 * inner solve that runs out of iterations still counts as an approximation;
 * an inner breakdown or non-finite value ends the solve with that status).
 * They need cheb_prec = PSOLVE_FP64, persistent = 0, timing = 0 and
 * rr_every = 0, and allocate their inner workspaces (for BJ: one per block
 * plus two block-ordered copies of a grid vector) at the first such solve.
 * Returns the solve's status (also in res->status; res may be NULL).
 * PSOLVE_E_ARG: bad rtol/maxit/precond/degree, blocks not dividing the grid
 * for BJ/GNoComm/BJ(BiCGS), an empty Chebyshev interval (scaled lambda_min >=
 * scaled lambda_max), or a flexible form with an option it does not take. */
PSOLVE_API psolve_status psolve_solve(psolve_ctx *ctx, const double *rhs_dev, double *x_dev, double rtol,
                           int32_t maxit, int32_t precond, int32_t degree, psolve_result *res);

/* Residual history of the context's last psolve_solve, recorded when the
 * context was created with opts.record_history = 1 (Algorithm 1's relative
 * residuals, the quantity of the paper's convergence plots).  Copies
 * min(*count, capacity) entries into the host arrays (either may be NULL):
 *   rel_s[i-1] = ||s_i||/||b||, the half-step residual of outer iteration i;
 *   rel_r[i-1] = ||r_i||/||b||, the residual after its update (the true
 *                residual b - A x when residual replacement ran at i);
 * NaN where iteration i did not produce the value (after a half-step exit
 * there is no r_i; a solve that stopped on a breakdown leaves later entries).
 * *count = the last solve's iteration count.  PSOLVE_E_ARG without
 * record_history, before the first solve, or after a Chebyshev
 * psolve_precond_apply (which reuses the solve's scalar state). */
PSOLVE_API psolve_status psolve_history(psolve_ctx *ctx, int32_t capacity, double *rel_s, double *rel_r,
                                        int32_t *count);

/* The same solve from HOST memory: copies rhs_host (n doubles) to the device,
 * solves, and copies x back to x_host (n doubles; read as x0 when
 * opts.use_x0).  Host buffers may be pageable or pinned (pinned is faster).
 * The copies are ordered on the context's stream; the device copies of b and
 * x are owned by the context. */
PSOLVE_API psolve_status psolve_solve_host(psolve_ctx *ctx, const double *rhs_host, double *x_host,
                                double rtol, int32_t maxit, int32_t precond, int32_t degree,
                                psolve_result *res);

PSOLVE_API void psolve_destroy(psolve_ctx *ctx);

/* ---- building blocks of the hot path, exposed for parity testing ------- */

/* out = A u (Eq. 6).  block_restricted != 0 applies R_s A R_s^T per block
 * (Eq. 14) with the context's opts.blocks.  u and out must not overlap. */
PSOLVE_API psolve_status psolve_apply_A(psolve_ctx *ctx, const double *u_dev, double *out_dev,
                             int32_t block_restricted);

/* out = M^{-1} v for the preconditioner (precond, degree) exactly as
 * psolve_solve applies it: for the Chebyshev forms at the context's
 * opts.cheb_prec (the result is widened to double); for G(BiCGS) / BJ(BiCGS)
 * one inner solve (or one per block) at opts.inner_rtol and inner_maxit.
 * precond must not be PSOLVE_PC_NONE.  v and out must not overlap. */
PSOLVE_API psolve_status psolve_precond_apply(psolve_ctx *ctx, const double *v_dev, double *out_dev,
                                   int32_t precond, int32_t degree);

/* *result_host = a . b with the solver's deterministic device reduction. */
PSOLVE_API psolve_status psolve_dot(psolve_ctx *ctx, const double *a_dev, const double *b_dev,
                         double *result_host);

/* Closed-form Chebyshev interval [a, b] that psolve_solve hands to the
 * preconditioner (Eq. 9-11 with the context's scales and blocks). */
PSOLVE_API psolve_status psolve_cheb_interval(psolve_ctx *ctx, int32_t precond, double *a, double *b);

/* *result_host = a . b over a grid of grid[3] = (nx, ny, nz) points, the same
 * deterministic reduction as psolve_dot of a context created without
 * opts.autotune (bitwise the same value), without any context and without
 * allocating device memory.  The paper has no counterpart: this exists for
 * callers that must not allocate, e.g. code running while a framework's
 * caching allocator or a serving process owns the device memory budget, or
 * host paths that cannot afford the synchronisation cudaMalloc/cudaFree may
 * cause.  Its scratch (descriptor, scalars, per-unit partial sums) is one
 * fixed 4 MiB device array inside the library, held by every GPU that loads
 * it until the process exits; grids whose partial sums do not fit (more than
 * about 2.6e5 work units: a unit is a 32 x 8 tile of columns times up to 32
 * planes, so very flat grids reach the limit first) return PSOLVE_E_ARG.  Every
 * call looks the array's address up on the current device
 * (cudaGetSymbolAddress), stages its small descriptor from host memory and
 * waits for the result, so no call can be made inside a stream capture.  All
 * calls share the array: calls that overlap on the GPU (other streams, other
 * host threads) race.  a_dev,
 * b_dev: device vectors of nx*ny*nz doubles; work is ordered on `stream`
 * and the call returns after the result is copied to *result_host. */
PSOLVE_API psolve_status psolve_dot_noalloc(const int64_t grid[3], const double *a_dev,
                                            const double *b_dev, uintptr_t stream,
                                            double *result_host);

/* Self-check of the library's exact FP32<->FP64 conversions.  B300 runs FP64
 * conversion instructions on its narrow FP64 pipe, so the mixed-precision
 * kernels widen and round with integer bit operations instead (IEEE-754
 * round to nearest even); this compares them bit for bit with the hardware
 * conversions on `count` seeded bit patterns (including rounding ties) and
 * stores the number of differences in *mismatches (0 expected).  No
 * counterpart in the paper (an implementation check). */
PSOLVE_API psolve_status psolve_selfcheck_conversions(uint64_t seed, int64_t count, int64_t *mismatches);

/* Self-check of the bounded waits: a kernel waits, with the same bounded wait
 * the TMA ring uses, on a shared-memory barrier that nothing completes, and
 * gives up after limit_cycles clock cycles (<= 2^34).  *status receives
 * PSOLVE_TIMEOUT when the wait gave up as designed.  No counterpart in the
 * paper (failure detection without a GPU fault). */
PSOLVE_API psolve_status psolve_selfcheck_wait_timeout(int64_t limit_cycles, int32_t *status);

/* Self-check of the persistent kernel's grid barrier: a cooperative launch of
 * *ctas small CTAs meets once at the same bounded grid barrier the persistent
 * solve uses, with a wait limit of limit_ns nanoseconds (1e3 .. 2e9), while
 * CTA absent_cta never arrives (absent_cta < 0: every CTA arrives).  On
 * return *passed CTAs got through, *gave_up CTAs timed out and *error_word
 * is the barrier's error word (1 after a time-out).  Expected: absent_cta < 0
 * gives passed = ctas, gave_up = 0, error_word = 0; absent_cta >= 0 gives
 * passed = 0, gave_up = ctas - 1, error_word = 1, within about limit_ns.  No
 * counterpart in the paper (failure detection without a GPU fault). */
PSOLVE_API psolve_status psolve_selfcheck_grid_timeout(int64_t limit_ns, int32_t absent_cta, int32_t *ctas,
                                                       int32_t *passed, int32_t *gave_up, int32_t *error_word);

/* Measured FP64 instruction throughput of this GPU: a kernel in which every
 * thread of 8 CTAs of 256 threads per SM runs 8 independent chains of
 * `iters` (1 .. 2^24) dependent FP64 instructions, fused multiply-adds (kind
 * 0) or adds (kind 1), timed with CUDA events on `stream` after one warm-up
 * run.  *instr_per_s receives the FP64 instructions (thread level) executed
 * per second, *ms_out (may be NULL) the timed run's duration and *sm_mhz (may
 * be NULL) the SM clock one CTA saw (clock cycles over global-timer time).
 * The FP64 kernels of the solver are bound by this rate rather than by HBM
 * bandwidth, so it is the roofline their achieved rate is divided by.  No
 * counterpart in the paper (a measurement of the hardware). */
PSOLVE_API psolve_status psolve_measure_fp64_rate(int32_t kind, int64_t iters, uintptr_t stream,
                                                  double *instr_per_s, double *ms_out, double *sm_mhz);

/* ---- many independent grids at once ----------------------------------- */

/* Solve `count` independent problems of (possibly) different sizes together:
 * every kernel launch processes the units of all unfinished problems, and
 * the iteration loop is replayed from one CUDA graph.  Problem q has grid
 * grids[3q..3q+2] = (nx, ny, nz), spacing h[3q..3q+2], right-hand side
 * rhs_dev[q] and solution x_dev[q] (device, caller-owned, same conventions as
 * psolve_solve).  All problems share rtol, maxit, precond, degree and opts;
 * precond is PSOLVE_PC_NONE or one of the Chebyshev forms.
 * results[q] receives problem q's result.  Each problem's iterates are
 * bitwise the same as when it is solved alone in a context created with the
 * same opts and the batch's slab share (opts.slab_share, by default
 * PSOLVE_SHARED_SLAB_SHARE). */
PSOLVE_API psolve_status psolve_solve_batch(int32_t count, const int64_t *grids, const double *h,
                                 const double *const *rhs_dev, double *const *x_dev, double rtol,
                                 int32_t maxit, int32_t precond, int32_t degree,
                                 const psolve_opts *opts, uintptr_t stream,
                                 psolve_result *results);

/* ---- continuous-batching server ---------------------------------------- */

typedef struct psolve_server psolve_server;

/* The slab-depth rule's default share for batched and served problems
 * (opts.slab_share = 0 in psolve_solve_batch and psolve_submit): they share
 * every launch with the other problems of the batch or the admitted
 * requests. */
#define PSOLVE_SHARED_SLAB_SHARE 16

/* A server owns a device memory pool of hbm_budget_bytes, a request queue
 * and a host thread that advances all admitted problems together, a few
 * outer iterations per round, admitting queued requests at round boundaries
 * as slots (max_slots) and memory free up.  Requests that share the
 * preconditioner (precond, degree, cheb_prec) share every kernel launch of a
 * round; each distinct preconditioner is a launch group of its own in the
 * same round (at most 32 distinct ones per server).  The server's kernels
 * run on `stream`. */
PSOLVE_API psolve_status psolve_server_create(double hbm_budget_bytes, int32_t max_slots, uintptr_t stream,
                                              psolve_server **out);

/* Queue one solve (Algorithm 1, as psolve_solve).  grid/h as in
 * psolve_create; rhs_dev/x_dev device pointers that stay valid until
 * psolve_poll returns non-PENDING.  precond is PSOLVE_PC_NONE or a Chebyshev
 * form (G(CI), BJ(CI), GNoComm(CI)) with degree as in psolve_solve.  opts may
 * be NULL; taken from it: cheb_prec, blocks (dividing the grid for BJ /
 * GNoComm) and the half-step check; x0 = 0; its Chebyshev scales must be
 * 1, 1 (served problems use the exact closed-form bounds, which makes the
 * sweeps of every request of a group the same kernels), else PSOLVE_E_ARG.
 * *ticket identifies the request.  PSOLVE_REJECTED if the request alone
 * exceeds the memory budget. */
PSOLVE_API psolve_status psolve_submit(psolve_server *srv, const int64_t grid[3], const double h[3],
                                       const double *rhs_dev, double *x_dev, double rtol, int32_t maxit,
                                       int32_t precond, int32_t degree, const psolve_opts *opts,
                                       uint64_t *ticket);

/* PSOLVE_PENDING while the request runs; otherwise its final status, with
 * *res filled (res may be NULL) and the ticket released. */
PSOLVE_API psolve_status psolve_poll(psolve_server *srv, uint64_t ticket, psolve_result *res);

/* Stops the host thread after the running round and frees everything;
 * requests still queued or running end with PSOLVE_TIMEOUT. */
PSOLVE_API void psolve_server_destroy(psolve_server *srv);

/* Message describing the last error on the calling thread ("" if none). */
PSOLVE_API const char *psolve_last_error(void);

/* Library version string. */
PSOLVE_API const char *psolve_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PSOLVE_H */
