// psolve_engine.cuh -- host-side engine shared by the single-grid context, the
// batched solve and the server: per-problem workspaces and descriptors,
// kernel sequencing for one outer iteration and per-kernel-class accounting.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/psolve.h"
#include "psolve_program.cuh"

namespace psolve {

// A named range on the calling host thread for profilers that read NVTX
// annotations (ncu --nvtx, nsys); without such a tool attached it costs a
// call that returns at once.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// ---------------------------------------------------------------- errors --
void set_error(const char *fmt, ...);
void clear_error();
const char *last_error();

#define PS_CK(call)                                                                      \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            psolve::set_error("%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                              __LINE__);                                                 \
            return PSOLVE_E_CUDA;                                                        \
        }                                                                                \
    } while (0)

// ------------------------------------------------------------ device info --
struct DevInfo {
    int dev = -1;
    int sms = 0;
};
psolve_status device_info(DevInfo *out);

// ------------------------------------------------------------- the plan --
// Static description of the kernels of one outer iteration.
struct Plan {
    int precond = PSOLVE_PC_NONE;
    int degree = 0;
    int prec = PSOLVE_FP64;
    bool exact_bounds = false; // scales (1, 1): the sweeps' y coefficient is zero
    int rr_every = 0;          // residual replacement period (0: none)
    bool neumann = false;      // the grid has zero-flux Neumann faces
    int split = 1;             // sub-units per work unit for the Chebyshev sweeps (see sweep_split)
    bool wide = false;         // Chebyshev sweeps in the two-points-per-thread form (see wide_sweeps)
    bool operator==(const Plan &o) const
    {
        return precond == o.precond && degree == o.degree && prec == o.prec && exact_bounds == o.exact_bounds &&
               rr_every == o.rr_every && neumann == o.neumann && split == o.split && wide == o.wide;
    }
};

// Whether the Chebyshev sweeps of `plan` run two x-adjacent points per thread
// (OpCiSweepW): FP32 or BF16 vectors, G(CI) (no block restriction), no
// Neumann face, and every problem of the launch list on the TMA ring
// (all_tma).  The FP32 sweeps are limited by instruction issue at one point
// per thread; the FP64 sweeps are bound by the FP64 pipe and keep one.
inline bool wide_sweeps(const Plan &p, bool all_tma)
{
    return all_tma && p.prec != PSOLVE_FP64 && p.precond == PSOLVE_PC_CHEB && !p.neumann;
}

// Sub-units per work unit for the Chebyshev sweeps of a launch list whose
// smallest slab is min_zc planes.  The FP64 sweeps are bound by the FP64
// pipe, to which a unit's two extra halo planes add no work, so halving a
// 32-plane unit only evens out the end of each launch (256^3: 247 -> 230 us
// per sweep); the FP32/BF16 sweeps keep whole units (the wide 256^3 FP32
// sweep measured 53.2 us whole against 55.2 us halved).
inline int sweep_split(int prec, int min_zc) { return (prec == PSOLVE_FP64 && min_zc >= 32) ? 2 : 1; }

inline size_t ci_elem_bytes(int prec) { return prec == PSOLVE_FP64 ? 8 : (prec == PSOLVE_FP32 ? 4 : 2); }

// One kernel launch as the host sees it (for timing and byte accounting).
struct LaunchRec {
    int cls;
    int side;          // 0: always runs; 1: skipped after a passed half-step test;
                       // 2: runs on iterations that are multiples of rr_every
    int iter;          // outer iteration (1-based); 0 = set-up, -1 = after the loop
    int is_update;
    int rr_every;
    double bytes;      // algorithmic bytes if the kernel does its full work
    double bytes_half; // update kernel after a passed half-step test
    cudaEvent_t ev0, ev1;
};

// Issues kernels (or only records what it would issue, dry = true).
struct Launcher {
    static constexpr bool WIDE_SWEEPS = true; // runs the wide sweeps of a plan that allows them
    cudaStream_t stream = 0;
    int sms = 1;               // SMs of the device
    long long units = 1;       // units of the launch list (upper bound)
    bool configure = false;    // only set up the kernels' launch attributes
    const Desc *d_desc = nullptr;
    const int32_t *d_list = nullptr;
    bool dry = false;
    bool timing = false;
    int iter = 0;       // outer iteration being issued (byte model only)
    int rr_every = 0;   // residual replacement period (byte model only)
    int64_t launches = 0;
    double npts = 0;    // points per problem for the byte model
    std::vector<LaunchRec> *recs = nullptr;
    std::vector<cudaEvent_t> *event_pool = nullptr;
    size_t *event_next = nullptr;
    cudaError_t err = cudaSuccess;

    cudaEvent_t next_event();
    template <class Op>
    void go(int cls, int side, KArgs a, double bytes_per_pt, double half_bytes_per_pt = 0.0,
            int is_update = 0);
};

// ----------------------------------------------------------- a problem --
struct Problem {
    int64_t n[3] = {0, 0, 0};
    double h[3] = {0, 0, 0};
    int blocks[3] = {1, 1, 1};
    int bc[6] = {0, 0, 0, 0, 0, 0}; // face conditions x-, x+, y-, y+, z-, z+ (0 Dirichlet, 1 Neumann)
    int prec = PSOLVE_FP64;
    bool have_rt = false;  // r~ buffer allocated (x0 != 0 support)
    int tuned = 0;         // slab/engine from the autotuner: 1 measured, 2 cached, 0 rule
    Desc desc{};           // host copy (vec[] of b, x filled per solve)
    char *mem = nullptr;   // one device allocation for all workspace vectors
    size_t mem_bytes = 0;
    Scal *d_sc = nullptr;
    double *d_partials = nullptr;
    // Row pitch of the workspace vectors in elements (0: nx).  A problem
    // whose nx is not a multiple of 8 can be laid out with rows padded to one
    // (padded_pitch), so that the tensor copies run on it; the caller's b and
    // x (rows of nx) are then copied into d_bst / d_xst (rows of px) before a
    // solve and x back after it.
    int64_t px = 0;
    bool no_stage = false; // padded, but bound only to other padded vectors (no staging copies)
    double *d_bst = nullptr, *d_xst = nullptr;
    int64_t pitch() const { return px ? px : n[0]; }
    bool staged() const { return pitch() != n[0] && !no_stage; }
    int64_t npts() const { return n[0] * n[1] * n[2]; }
    int64_t nvec() const { return pitch() * n[1] * n[2]; } // elements one vector holds
};

// nx rounded up to a multiple of 8: rows of 8-, 4- and 2-byte elements then
// all start on 16-byte boundaries.
inline int64_t padded_pitch(int64_t nx) { return (nx + 7) / 8 * 8; }

// Copy a vector with rows of nx (a caller's, `src`) into one with rows of
// P.pitch() (`dst`), or back; `kind` says which sides are on the host.
cudaError_t copy_to_pitched(const Problem &P, double *dst, const double *src, cudaStream_t s,
                            cudaMemcpyKind kind = cudaMemcpyDeviceToDevice);
cudaError_t copy_from_pitched(const Problem &P, double *dst, const double *src, cudaStream_t s,
                              cudaMemcpyKind kind = cudaMemcpyDeviceToDevice);

// Bytes one problem's workspace needs (vectors + partials + scalars), for
// vectors with rows of px elements (0: n[0]); a padded pitch adds the two
// staging vectors of b and x unless no_stage.
size_t problem_bytes(const int64_t n[3], int prec, bool with_rt, int sms, int64_t px = 0, bool no_stage = false);
// Fill the geometry fields of P.desc from P.n, P.h, P.blocks.  The slab depth
// (planes per unit) is zc_choice when > 0 (a tuned value, at most nz), else
// the built-in rule, applied to `copies` such problems sharing every launch.
void problem_geometry(Problem &P, int sms, int zc_choice = 0, int copies = 1);
// Lay out P's workspace inside `base` (device, problem_bytes long).
void problem_bind(Problem &P, char *base);
// Chebyshev interval [a, b] (Eq. 9-11 times the scales) for precond.
psolve_status cheb_interval(const Problem &P, int precond, double lmin_scale, double lmax_scale,
                            double *a, double *b);
// Chebyshev coefficients for (precond, degree) into P.desc.
psolve_status problem_set_cheb(Problem &P, int precond, int degree, double lmin_scale,
                               double lmax_scale);

// Enqueue the kernels of one outer iteration for `plan`.
void enqueue_iteration(Launcher &L, const Plan &plan);
void enqueue_init(Launcher &L, bool use_x0);
void enqueue_true_residual(Launcher &L);
void enqueue_apply_A(Launcher &L, bool blocked);
void enqueue_dot(Launcher &L);
void enqueue_precond(Launcher &L, const Plan &plan);
// Outer phases of the flexible Bi-CGSTAB (G(BiCGS), BJ(BiCGS)): the inner
// solves between them write p^ (ROLE_PH) and r^ (ROLE_RH) in FP64.
enum FlexPhase {
    FLEX_PUPDATE = 0, // p = r + beta (p - omega w), in place (p = r first)
    FLEX_W,           // w = A p^, r~ . w -> alpha
    FLEX_S,           // s = r - alpha w, ||s||^2 -> half-step test
    FLEX_T,           // t = A r^, t.s, t.t -> omega
    FLEX_UPDATE       // x, r and r~.r, r.r -> beta, stop test
};
void enqueue_flex_phase(Launcher &L, int phase);
// Gather a grid vector into block-contiguous storage (block q = Bx + bx (By +
// by Bz), x fastest inside a block) and back.
void enqueue_gather_blocks(cudaStream_t s, const double *src, double *dst, const int64_t n[3], int64_t px,
                           const int blocks[3], bool to_blocks);

// The autotuner's probe kernels (a sweep, a stencil with two dots, an update)
// for Chebyshev vectors of precision `prec`; needs every role bound.  split:
// the sweep's sub-units per work unit (sweep_split).
void enqueue_tune_probe(Launcher &L, int prec, bool blk, int split);

// What problem_encode_tmaps last wrote into one maps array: the vectors it
// encoded, `allow`, the resulting P.desc.tma, and the roles [lo, hi) whose
// maps the last call rewrote (empty: the array is unchanged).
struct TmapCache {
    bool valid = false;
    bool allow = false;
    int tma = 0;
    void *vec[NROLES] = {};
    int lo = 0, hi = 0;
};

// Encode the tensor maps of every bound vector of P into
// maps[0..TMAPS_PER_PROBLEM) and set P.desc.tma (1 when the TMA engine can run
// this problem: a row pitch that is a multiple of 8, every vector 16-byte
// aligned, and `allow`; the maps span nx columns, so a copy reads zeros for
// the padding columns as for any cell outside the grid).  With
// a cache, the maps of roles whose vector is the one encoded last time are
// kept as they are (the grid and the precision of a Problem never change), and
// cache->lo/hi name the roles rewritten.
void problem_encode_tmaps(Problem &P, CUtensorMap *maps, bool allow, TmapCache *cache = nullptr);

// Algorithmic bytes of the launches in `recs` that did work, given the exit
// iteration and whether it was a half-step exit.
double model_bytes_for(const std::vector<LaunchRec> &recs, int final_iter, int half_exit);
// Whether a recorded launch did work.
bool launch_did_work(const LaunchRec &r, int final_iter, int half_exit);

} // namespace psolve
