// psolve_types.cuh -- device-side data structures shared by the kernels and
// the host driver of libpsolve.
//
// A "problem" is one grid with its own Krylov state.  The kernels process a
// list of problems (one for a single solve, many for batched and served
// solves).  Each problem's grid is cut into work units: an xy tile of
// TILE_X x TILE_Y columns times a chunk of `zc` consecutive z planes.  Units
// are the scheduling granule (CTAs take contiguous unit ranges) and the
// reduction granule (one partial sum per unit, summed in unit order by the
// last CTA to finish the problem), so every reduction result depends only on
// the problem's own shape, never on the launch size or the batch mix.
#pragma once
#include <cuda.h> // CUtensorMap (type only; the library does not link libcuda)

#include <cstdint>

namespace psolve {

constexpr int TILE_X = 32;                // columns along x per CTA tile (one warp)
constexpr int TILE_Y = 8;                 // columns along y per CTA tile
constexpr int NTHREADS = TILE_X * TILE_Y; // threads per CTA, one z column each
constexpr int MAX_DEGREE = 64;            // largest Chebyshev degree accepted
constexpr int MAX_DOTS = 2;               // reductions fused into one kernel

// Roles of the per-problem vectors.  FP64 roles hold doubles; CI roles hold
// the Chebyshev storage type (double, float or bf16).
enum Role : int {
    ROLE_R = 0, // residual r (FP64)
    ROLE_P,     // search direction p, one parity (FP64)
    ROLE_P2,    // search direction p, other parity (FP64); must follow ROLE_P
    ROLE_W,     // w = A p^ (FP64)
    ROLE_S,     // half-step residual s (FP64)
    ROLE_T,     // t = A r^ (FP64)
    ROLE_RT,    // shadow residual r~ (FP64; aliases b when x0 = 0)
    ROLE_X,     // solution x (FP64, caller's buffer)
    ROLE_B,     // right-hand side b (FP64, caller's buffer)
    ROLE_PH,    // p^ = M^-1 p (CI type)
    ROLE_RH,    // r^ = M^-1 s (CI type)
    ROLE_YA,    // Chebyshev work vector (CI type)
    ROLE_YB,    // Chebyshev work vector (CI type)
    ROLE_BC,    // CI right-hand side rounded to the CI type (mixed only)
    ROLE_YC,    // Chebyshev work vectors of the paired sweeps (CI type, mixed only):
    ROLE_YD,    // two sweeps per pass read their inputs with a halo, so none is overwritten in place
    ROLE_U,     // input of the building-block entry points (FP64)
    ROLE_V,     // output of the building-block entry points (FP64)
    NROLES,
    // Virtual roles resolved per problem from its iteration parity: the
    // direction update reads p_{i-2} and writes p_{i-1} into the other buffer
    // (it reads p at stencil neighbours, so it cannot update in place).
    ROLE_PCUR = 100, // buffer holding p_{i-1} during outer iteration i
    ROLE_POLD = 101  // buffer holding p_{i-2} during outer iteration i
};

// Per-problem scalar state, updated on the device by the last CTA of each
// reducing kernel.  The host only reads it when it polls.
struct Scal {
    double rho;      // rho_{i-1} = r~ . r
    double alpha;
    double omega;
    double beta;
    double nb2;      // ||b||^2
    double thr2;     // (rtol ||b||)^2
    double rr;       // ||r||^2 of the latest recursive residual
    double ss;       // ||s||^2 of the latest half step
    double true_rr;  // ||b - A x||^2 (true residual at exit)
    double red[MAX_DOTS]; // raw values of the latest reduction (building blocks)
    int32_t status;  // psolve_status once stop != 0
    int32_t stop;    // nonzero: every later kernel skips this problem
    int32_t half;    // the half-step test passed in this iteration
    int32_t iter;    // completed outer iterations
    int32_t maxit;
    int32_t first;   // 1 until the first direction update (beta unused)
    int32_t half_exit;
    int32_t zero_x;  // b == 0 with an initial guess: host must zero x
    uint32_t ticket; // units finished in the running reduction
    int32_t pad_[3];
};

struct Desc {
    // geometry
    int32_t nx, ny, nz;
    // row pitch of every vector in elements (element (i, j, k) is at
    // i + px (j + ny k)): nx, or nx rounded up to a multiple of 8 so that the
    // rows of every precision start on 16-byte boundaries for the tensor maps;
    // the columns i >= nx are never read as grid values
    int32_t px;
    int32_t tiles_x, tiles_y;
    int32_t zc;         // planes per unit chunk
    int32_t nzc;        // chunks along z
    int32_t units;      // tiles_x * tiles_y * nzc
    int32_t bx, by, bz; // block sizes of the restricted operator
    int32_t half_check;
    int32_t maxit;
    int32_t degree;
    double rtol;
    double cx, cy, cz, cc; // 1/hx^2, 1/hy^2, 1/hz^2, 2 (cx + cy + cz)
    // Chebyshev (Eq. 15): 1/theta, 2/delta, 2 sigma and rho_0..rho_d
    double theta_inv, two_over_delta, two_sigma;
    double rho[MAX_DEGREE + 1];
    // the same folded into per-sweep coefficients on the host, so that a
    // kernel spends no FP64 instruction on them: CI sweep 1 (a_u, a_x, a_y,
    // a_z) and sweep k >= 2 (c_y, c_b, c_z, c_x, c_yy, c_zz)
    double ci1[4];
    double cik[MAX_DEGREE + 1][6];
    // the same rounded to FP32 (nearest) for the FP32-arithmetic sweeps, which
    // would otherwise convert them per work unit on the FP64 pipe
    float ci1f[4];
    float cikf[MAX_DEGREE + 1][6];
    float theta_inv_f;
    // p^ and r^ are stored divided by hat (1 unless FP64 Chebyshev vectors and
    // degree >= 2); w and t are stored as A (stored vector) / cc, and
    // wcx.. = -(cx, cy, cz) / cc are that operator's neighbour coefficients
    double hat, inv_cc, wcx, wcy, wcz;
    void *vec[NROLES];
    Scal *sc;
    double *partials;   // units * MAX_DOTS doubles
    // TMA engine: 1 if every stencil operand of this problem can be staged by
    // tensor copies (px % 8 == 0, 16-byte aligned vectors); tmap[TMAPS_PER_ROLE
    // * role + TMAP_HALO / TMAP_PLAIN / TMAP_HALO2] are the role's maps.
    int32_t tma;
    int32_t rr_every;   // residual replacement every rr_every outer iterations (0: never)
    int32_t bcm;        // zero-flux Neumann faces: bit f for face f (x-, x+, y-, y+, z-, z+)
    int32_t hist_cap;   // outer iterations the history buffer holds
    const CUtensorMap *tmap;
    // residual history (nullptr: not recorded): hist[2 (i-1)] = ||s_i||^2 and
    // hist[2 (i-1) + 1] = ||r_i||^2 of outer iteration i (Algorithm 1), for
    // i <= hist_cap; written by the epilogues of the reductions that produce them
    double *hist;
};

// Header of a device-side launch list: `n` entries of (problem, first unit)
// follow it as int pairs; `total` is the sum of the listed problems' units.
// `next` and `done` are the list's work counter and finished-CTA count: a
// kernel's CTAs take units by incrementing `next`, and the last CTA to finish
// sets both back to zero, so every launch on the list starts from zero (the
// host writes them as zero).
struct ListHdr {
    int32_t n;
    int32_t total;
    uint32_t next;
    uint32_t done;
};
constexpr int LIST_HDR_INTS = 4; // ints before the first (problem, first unit) entry

// Arguments common to every kernel launch.
struct KArgs {
    const Desc *descs;
    const int32_t *list; // ListHdr followed by 2*n ints
    int32_t k;           // Chebyshev step index (sweeps)
    int32_t skip;        // SKIP_* bits
    int32_t in, b, z, out, aux; // roles used by the operation
    int32_t split;       // stencil operations without dots: sub-units per work unit (0, 1: none)
};

// Tensor maps per role: the halo box (TILE_X + 2 HX) x (TILE_Y + 2), the
// plain box TILE_X x TILE_Y and the two-row halo box (TILE_X + 2 HX) x
// (TILE_Y + 4) that the paired Chebyshev sweeps read their stencil input with.
constexpr int TMAP_HALO = 0, TMAP_PLAIN = 1, TMAP_HALO2 = 2, TMAPS_PER_ROLE = 3;
constexpr int TMAPS_PER_PROBLEM = TMAPS_PER_ROLE * NROLES;
constexpr int ST_TIMEOUT = 7; // a bounded wait of the TMA ring gave up

constexpr int SKIP_STOP = 1; // skip problems whose `stop` is set
constexpr int SKIP_HALF = 2; // skip problems whose `half` is set
constexpr int SKIP_NOT_RR = 4; // skip problems whose iteration count is not a multiple of rr_every

} // namespace psolve
