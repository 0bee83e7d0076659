// psolve_engine.cu -- kernel sequencing, workspace layout, Chebyshev set-up.
#include "psolve_engine.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>

namespace psolve {

static thread_local std::string g_error;

void set_error(const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
}
void clear_error() { g_error.clear(); }
const char *last_error() { return g_error.c_str(); }

psolve_status device_info(DevInfo *out)
{
    int dev = 0;
    PS_CK(cudaGetDevice(&dev));
    int sms = 0;
    PS_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    out->dev = dev;
    out->sms = sms;
    return PSOLVE_OK;
}

// ----------------------------------------------------------------- launch --
cudaEvent_t Launcher::next_event()
{
    if (*event_next >= event_pool->size()) {
        cudaEvent_t e;
        cudaError_t st = cudaEventCreate(&e);
        if (st != cudaSuccess) {
            err = st;
            return nullptr;
        }
        event_pool->push_back(e);
    }
    return (*event_pool)[(*event_next)++];
}

// Per-kernel launch set-up, done once per device: the dynamic shared memory
// of the TMA ring (a per-device attribute of the kernel) and the resident
// CTAs per SM that size the grid.  Several host threads may race to set it
// up; each does the same idempotent calls and stores the same value.
constexpr int MAX_CONFIG_DEVICES = 64;
template <class Op>
static cudaError_t op_config(int *occ_out)
{
    static std::atomic<int> occ[MAX_CONFIG_DEVICES];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_CONFIG_DEVICES) return cudaErrorInvalidDevice;
    int o = occ[dev].load(std::memory_order_acquire);
    if (!o) {
        const int dyn = engine_dyn_smem<Op>();
        e = cudaFuncSetAttribute(k_engine<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_engine<Op>, op_threads<Op>(), dyn);
        if (e != cudaSuccess) return e;
        o = n < 1 ? 1 : n;
        occ[dev].store(o, std::memory_order_release);
    }
    *occ_out = o;
    return cudaSuccess;
}

template <class Op>
void Launcher::go(int cls, int side, KArgs a, double bytes_per_pt, double half_bytes_per_pt, int is_update)
{
    LaunchRec rec{};
    rec.cls = cls;
    rec.side = side;
    rec.iter = iter;
    rec.is_update = is_update;
    rec.rr_every = rr_every;
    rec.bytes = bytes_per_pt * npts;
    rec.bytes_half = half_bytes_per_pt * npts;
    if (dry) {
        if (recs) recs->push_back(rec);
        return;
    }
    int occ = 1;
    cudaError_t st = op_config<Op>(&occ);
    if (st != cudaSuccess) {
        if (err == cudaSuccess) err = st;
        return;
    }
    if (configure) return;
    long long g = (long long)occ * sms;
    const long long work = (Op::STENCIL && Op::ND == 0 && a.split > 1) ? units * a.split : units;
    if (work < g) g = work;
    if (g < 1) g = 1;
    a.descs = d_desc;
    a.list = d_list;
    if (timing) {
        rec.ev0 = next_event();
        rec.ev1 = next_event();
        if (err != cudaSuccess) return;
        cudaEventRecord(rec.ev0, stream);
    }
    k_engine<Op><<<(int)g, op_threads<Op>(), engine_dyn_smem<Op>(), stream>>>(a);
    st = cudaGetLastError();
    if (st != cudaSuccess && err == cudaSuccess) err = st;
    if (timing) cudaEventRecord(rec.ev1, stream);
    ++launches;
    if (recs) recs->push_back(rec);
}

// ------------------------------------------------------------ tensor maps --
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

static bool role_is_ci(int r)
{
    return r == ROLE_PH || r == ROLE_RH || r == ROLE_YA || r == ROLE_YB || r == ROLE_BC || r == ROLE_YC ||
           r == ROLE_YD;
}

void problem_encode_tmaps(Problem &P, CUtensorMap *maps, bool allow, TmapCache *cache)
{
    Desc &D = P.desc;
    if (cache) {
        cache->lo = cache->hi = 0;
        if (cache->valid && cache->allow == allow && std::memcmp(cache->vec, D.vec, sizeof D.vec) == 0) {
            D.tma = cache->tma;
            return;
        }
    }
    // a role keeps its maps when the cache holds valid maps of the same vector
    const bool keep_any = cache && cache->valid && cache->tma;
    auto finish = [&](int tma, int lo, int hi) {
        D.tma = tma;
        if (!cache) return;
        cache->valid = true;
        cache->allow = allow;
        cache->tma = tma;
        std::memcpy(cache->vec, D.vec, sizeof D.vec);
        cache->lo = lo;
        cache->hi = hi;
    };
    if (!allow || D.px % 8 != 0) return finish(0, 0, 0);
    for (int r = 0; r < NROLES; ++r)
        if (D.vec[r] && (reinterpret_cast<uintptr_t>(D.vec[r]) % 16) != 0) return finish(0, 0, 0);
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return finish(0, 0, 0);
    int lo = NROLES, hi = 0;
    for (int r = 0; r < NROLES; ++r) {
        if (keep_any && cache->vec[r] == D.vec[r]) continue;
        lo = std::min(lo, r);
        hi = r + 1;
        CUtensorMap *m = &maps[TMAPS_PER_ROLE * r];
        std::memset(m, 0, sizeof(CUtensorMap) * TMAPS_PER_ROLE);
        if (!D.vec[r]) continue;
        const bool ci = role_is_ci(r);
        const size_t es = ci ? ci_elem_bytes(P.prec) : 8;
        const CUtensorMapDataType dt = !ci || P.prec == PSOLVE_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                       : P.prec == PSOLVE_FP32      ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                                    : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
        const cuuint64_t dims[3] = {(cuuint64_t)D.nx, (cuuint64_t)D.ny, (cuuint64_t)D.nz};
        const cuuint64_t strides[2] = {(cuuint64_t)D.px * es, (cuuint64_t)D.px * D.ny * es};
        const cuuint32_t estr[3] = {1, 1, 1};
        const cuuint32_t halo[3] = {(cuuint32_t)(TILE_X + 2 * (16 / es)), (cuuint32_t)(TILE_Y + 2), 1};
        const cuuint32_t plain[3] = {(cuuint32_t)TILE_X, (cuuint32_t)TILE_Y, 1};
        const cuuint32_t halo2[3] = {(cuuint32_t)(TILE_X + 2 * (16 / es)), (cuuint32_t)(TILE_Y + 4), 1};
        for (int v = 0; v < TMAPS_PER_ROLE; ++v) {
            // no L2 promotion: the halo boxes start 16 bytes before a line, and
            // promoting their sector reads to whole lines multiplied DRAM reads
            const cuuint32_t *box = v == TMAP_HALO ? halo : (v == TMAP_PLAIN ? plain : halo2);
            CUresult e = fn(&m[v], dt, 3, D.vec[r], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (e != CUDA_SUCCESS) {
                if (cache) cache->valid = false;
                D.tma = 0;
                return;
            }
        }
    }
    if (lo >= hi) lo = hi = 0;
    finish(1, lo, hi);
}

// --------------------------------------------------- per-iteration kernels --
template <class T, bool BLK>
static void iteration_cheb(Launcher &L, const Plan &p)
{
    const bool rr = p.rr_every > 0;
    if (p.exact_bounds) prog_iteration_cheb<T, BLK, false>(L, p.degree, L.iter, rr, p.neumann, p.split, p.wide);
    else prog_iteration_cheb<T, BLK, true>(L, p.degree, L.iter, rr, p.neumann, p.split, p.wide);
}

void enqueue_iteration(Launcher &L, const Plan &plan)
{
    const bool rr = plan.rr_every > 0;
    L.rr_every = plan.rr_every;
    if (plan.precond == PSOLVE_PC_NONE) {
        prog_iteration_none(L, L.iter, rr);
        return;
    }
    const bool blk = plan.precond != PSOLVE_PC_CHEB;
    switch (plan.prec) {
    case PSOLVE_FP32:
        if (blk) iteration_cheb<float, true>(L, plan);
        else iteration_cheb<float, false>(L, plan);
        break;
    case PSOLVE_BF16:
        if (blk) iteration_cheb<__nv_bfloat16, true>(L, plan);
        else iteration_cheb<__nv_bfloat16, false>(L, plan);
        break;
    default:
        if (blk) iteration_cheb<double, true>(L, plan);
        else iteration_cheb<double, false>(L, plan);
        break;
    }
}

void enqueue_init(Launcher &L, bool use_x0) { prog_init(L, use_x0); }

void enqueue_true_residual(Launcher &L) { prog_true_residual(L); }

// Building blocks use the same kernels as the solve.
void enqueue_apply_A(Launcher &L, bool blocked)
{
    KArgs a{};
    a.in = ROLE_U;
    a.out = ROLE_V;
    if (blocked) L.go<OpApplyA<true>>(PSOLVE_K_OTHER, 0, a, 16.0);
    else L.go<OpApplyA<false>>(PSOLVE_K_OTHER, 0, a, 16.0);
}

void enqueue_dot(Launcher &L)
{
    KArgs a{};
    a.in = ROLE_U;
    a.aux = ROLE_V;
    L.go<OpDot>(PSOLVE_K_OTHER, 0, a, 16.0);
}

// M^-1 v with the solve's own kernels: sweep 1 in its first-iteration form
// reads v through ROLE_R (the caller points ROLE_R at v and sets first = 1,
// iter = 0), then the sweeps, then a widening copy of p^ into ROLE_V.
template <class T, bool BLK>
static void precond_cheb(Launcher &L, const Plan &p)
{
    const int d = p.degree;
    const bool eb = p.exact_bounds, neu = p.neumann, wide = p.wide;
    const int split = p.split;
    using TB = typename std::conditional<is_mixed<T>(), T, double>::type;
    constexpr bool MIX = is_mixed<T>();
    KArgs a{};
    a.skip = 0;
    a.in = ROLE_PCUR;
    a.out = (d <= 1) ? ROLE_PH : ROLE_YA;
    constexpr bool U = !MIX; // y_1 stored scaled (FP64, d >= 2)
    if constexpr (MIX) { // the solve's two-pass sweep 1 (OpDirUpdate, then sweep 1 on b_c)
        L.go<OpDirUpdate<T>>(PSOLVE_K_CI_FIRST, 0, a, 0.0);
        prog_sweep1<T, BLK>(L, 0, a, 0.0, neu, wide);
    } else if (U && d >= 2) {
        L.go<OpCiFirst<T, BLK, SIDE_P, U>>(PSOLVE_K_CI_FIRST, 0, a, 0.0);
    } else {
        L.go<OpCiFirst<T, BLK, SIDE_P>>(PSOLVE_K_CI_FIRST, 0, a, 0.0);
    }
    if (eb) prog_sweeps<T, TB, BLK, false>(L, d, 0, MIX ? ROLE_BC : ROLE_PCUR, ROLE_PH, 0, neu, split, wide);
    else prog_sweeps<T, TB, BLK, true>(L, d, 0, MIX ? ROLE_BC : ROLE_PCUR, ROLE_PH, 0, neu, split, wide);
    KArgs w{};
    w.in = ROLE_PH;
    w.out = ROLE_V;
    L.go<OpWiden<T>>(PSOLVE_K_OTHER, 0, w, 0.0);
}

void enqueue_precond(Launcher &L, const Plan &plan)
{
    const bool blk = plan.precond != PSOLVE_PC_CHEB;
    switch (plan.prec) {
    case PSOLVE_FP32:
        if (blk) precond_cheb<float, true>(L, plan);
        else precond_cheb<float, false>(L, plan);
        break;
    case PSOLVE_BF16:
        if (blk) precond_cheb<__nv_bfloat16, true>(L, plan);
        else precond_cheb<__nv_bfloat16, false>(L, plan);
        break;
    default:
        if (blk) precond_cheb<double, true>(L, plan);
        else precond_cheb<double, false>(L, plan);
        break;
    }
}

// The autotuner's probe: one Chebyshev sweep (k >= 3 form), one stencil with
// two dots and one update, with every role on workspace vectors and no skips.
template <class T, bool BLK>
static void tune_probe(Launcher &L, int split)
{
    using TB = typename std::conditional<is_mixed<T>(), T, double>::type;
    KArgs s{};
    s.k = 3;
    s.split = split;
    s.in = ROLE_YA;
    s.z = ROLE_YB;
    s.b = is_mixed<T>() ? ROLE_BC : ROLE_PH;
    s.out = ROLE_RH;
    L.go<OpCiSweep<T, TB, BLK, false, false, !is_mixed<T>()>>(PSOLVE_K_CI_SWEEP4, 0, s, 0.0);
    KArgs t{};
    t.in = ROLE_RH;
    L.go<OpStencil2Dot<T>>(PSOLVE_K_STENCIL_2DOT, 0, t, 0.0);
    KArgs u{};
    u.in = ROLE_PH;
    u.aux = ROLE_RH;
    L.go<OpUpdate<T>>(PSOLVE_K_UPDATE, 0, u, 0.0);
}

void enqueue_tune_probe(Launcher &L, int prec, bool blk, int split)
{
    switch (prec) {
    case PSOLVE_FP32: blk ? tune_probe<float, true>(L, split) : tune_probe<float, false>(L, split); break;
    case PSOLVE_BF16:
        blk ? tune_probe<__nv_bfloat16, true>(L, split) : tune_probe<__nv_bfloat16, false>(L, split);
        break;
    default: blk ? tune_probe<double, true>(L, split) : tune_probe<double, false>(L, split); break;
    }
}

void enqueue_flex_phase(Launcher &L, int phase)
{
    KArgs a{};
    a.skip = SKIP_STOP;
    switch (phase) {
    case FLEX_PUPDATE: L.go<OpPUpdate>(PSOLVE_K_OTHER, 0, a, L.iter == 1 ? 16.0 : 32.0); break;
    case FLEX_W:
        a.in = ROLE_PH;
        L.go<OpStencilDot<double>>(PSOLVE_K_STENCIL_DOT, 0, a, 24.0);
        break;
    case FLEX_S: L.go<OpSUpdate>(PSOLVE_K_OTHER, 0, a, 24.0); break;
    case FLEX_T:
        a.skip = SKIP_STOP | SKIP_HALF;
        a.in = ROLE_RH;
        L.go<OpStencil2Dot<double>>(PSOLVE_K_STENCIL_2DOT, 1, a, 24.0);
        break;
    default:
        a.in = ROLE_PH;
        a.aux = ROLE_RH;
        L.go<OpUpdate<double>>(PSOLVE_K_UPDATE, 0, a, 64.0, 24.0, 1);
        break;
    }
}

// One thread per grid point: (i, j, k) -> block (i / mx, j / my, k / mz),
// position inside the block; copies in the direction asked for.
// The grid side has rows of px elements (its row pitch).
__global__ void k_gather_blocks(const double *src, double *dst, int nx, int ny, int nz, long long px, int mx, int my,
                                int mz, int bx, int by, int to_blocks)
{
    const long long N = (long long)nx * ny * nz;
    const long long M = (long long)mx * my * mz;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(g % nx), j = (int)((g / nx) % ny), k = (int)(g / ((long long)nx * ny));
        const long long o = i + px * (j + (long long)ny * k);
        const int Bx = i / mx, By = j / my, Bz = k / mz;
        const long long q = Bx + (long long)bx * (By + (long long)by * Bz);
        const long long l = q * M + (i - Bx * mx) + (long long)mx * ((j - By * my) + (long long)my * (k - Bz * mz));
        if (to_blocks) dst[l] = src[o];
        else dst[o] = src[l];
    }
}

void enqueue_gather_blocks(cudaStream_t s, const double *src, double *dst, const int64_t n[3], int64_t px,
                           const int blocks[3], bool to_blocks)
{
    const long long N = n[0] * n[1] * n[2];
    const int threads = 256;
    const long long want = (N + threads - 1) / threads;
    const int grid = (int)(want < 65535 * 4 ? want : 65535 * 4);
    k_gather_blocks<<<grid, threads, 0, s>>>(src, dst, (int)n[0], (int)n[1], (int)n[2], (long long)px,
                                             (int)(n[0] / blocks[0]), (int)(n[1] / blocks[1]),
                                             (int)(n[2] / blocks[2]), blocks[0], blocks[1], to_blocks ? 1 : 0);
}

cudaError_t copy_to_pitched(const Problem &P, double *dst, const double *src, cudaStream_t s, cudaMemcpyKind kind)
{
    const size_t w = sizeof(double) * (size_t)P.n[0];
    return cudaMemcpy2DAsync(dst, sizeof(double) * (size_t)P.pitch(), src, w, w, (size_t)(P.n[1] * P.n[2]), kind,
                             s);
}

cudaError_t copy_from_pitched(const Problem &P, double *dst, const double *src, cudaStream_t s, cudaMemcpyKind kind)
{
    const size_t w = sizeof(double) * (size_t)P.n[0];
    return cudaMemcpy2DAsync(dst, w, src, sizeof(double) * (size_t)P.pitch(), w, (size_t)(P.n[1] * P.n[2]), kind,
                             s);
}

bool launch_did_work(const LaunchRec &r, int final_iter, int half_exit)
{
    if (r.side == 2) // replacement: counted on the multiples of rr_every before the exit iteration
        return r.rr_every > 0 && r.iter > 0 && r.iter % r.rr_every == 0 && r.iter < final_iter;
    if (r.iter > final_iter) return false;
    if (r.iter == final_iter && half_exit && r.side == 1) return false;
    return true;
}

double model_bytes_for(const std::vector<LaunchRec> &recs, int final_iter, int half_exit)
{
    double sum = 0.0;
    for (const LaunchRec &r : recs) {
        if (!launch_did_work(r, final_iter, half_exit)) continue;
        if (r.iter == final_iter && half_exit && r.is_update) sum += r.bytes_half;
        else sum += r.bytes;
    }
    return sum;
}

// ------------------------------------------------------------- workspace --
static int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// p^ and r^ stored divided by h (read back only by psolve_precond_apply).
static void set_hat(Desc &D, double h) { D.hat = h; }

void problem_geometry(Problem &P, int sms, int zc_choice, int copies)
{
    Desc &D = P.desc;
    D.nx = (int)P.n[0];
    D.ny = (int)P.n[1];
    D.nz = (int)P.n[2];
    D.px = (int)P.pitch();
    D.tiles_x = ceil_div(D.nx, TILE_X);
    D.tiles_y = ceil_div(D.ny, TILE_Y);
    const long long tiles = (long long)D.tiles_x * D.tiles_y;
    // Chunk length (slab depth) by a cost model: up to 3 units per SM run at
    // once, and a unit of zc planes costs about zc + 2 plane-times (its two
    // halo planes and the ring's ramp), so the solve time goes as
    // ceil(units / (3 SMs)) * (zc + 2); the smallest estimate wins, ties to
    // the deeper slab.  Over 125 grid shapes (16^3 .. 256^3, FP64 and FP32)
    // the autotuner measured this choice within 4% of the best one (geometric
    // mean).  It depends on the grid shape and the GPU only, so reductions do
    // not depend on the batch mix.  `copies` equal problems that always share
    // their launches (the blocks of BJ(BiCGS)) are counted together.
    long long zc = 1;
    double best_cost = -1.0;
    for (long long z = 1; z <= 32; z *= 2) {
        if (z > D.nz && z > 1) break;
        const long long u = (copies > 1 ? copies : 1) * tiles * ((D.nz + z - 1) / z);
        const double cost = (double)((u + 3LL * sms - 1) / (3LL * sms)) * (double)(z + 2);
        if (best_cost < 0.0 || cost <= best_cost) {
            best_cost = cost;
            zc = z;
        }
    }
    if (zc_choice > 0) zc = zc_choice < D.nz ? zc_choice : D.nz; // a tuned slab depth
    D.zc = (int)zc;
    D.nzc = ceil_div(D.nz, D.zc);
    D.units = (int)(tiles * D.nzc);
    D.bx = D.nx / P.blocks[0];
    D.by = D.ny / P.blocks[1];
    D.bz = D.nz / P.blocks[2];
    if (D.bx < 1) D.bx = 1;
    if (D.by < 1) D.by = 1;
    if (D.bz < 1) D.bz = 1;
    D.bcm = 0;
    for (int f = 0; f < 6; ++f)
        if (P.bc[f]) D.bcm |= 1 << f;
    D.cx = 1.0 / (P.h[0] * P.h[0]);
    D.cy = 1.0 / (P.h[1] * P.h[1]);
    D.cz = 1.0 / (P.h[2] * P.h[2]);
    D.cc = 2.0 * (D.cx + D.cy + D.cz);
    // w and t are stored as A u / cc (OpStencilDot)
    D.inv_cc = 1.0 / D.cc;
    D.wcx = -D.cx / D.cc;
    D.wcy = -D.cy / D.cc;
    D.wcz = -D.cz / D.cc;
    set_hat(D, 1.0);
}

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Units of the finest decomposition (one plane per unit): the partial-sum
// buffer is sized for it, so any slab depth fits the same workspace.
static long long units_max(const int64_t n[3])
{
    return (long long)((n[0] + TILE_X - 1) / TILE_X) * ((n[1] + TILE_Y - 1) / TILE_Y) * n[2];
}

size_t problem_bytes(const int64_t n[3], int prec, bool with_rt, int sms, int64_t px, bool no_stage)
{
    const int64_t p = px ? px : n[0];
    const size_t N = (size_t)(p * n[1] * n[2]);
    const size_t v64 = align_up(N * 8), vci = align_up(N * ci_elem_bytes(prec));
    // CI vectors p^, r^, y_a, y_b; mixed precision adds b_c and the paired
    // sweeps' y_c, y_d; a padded pitch adds the staging copies of b and x
    size_t b = v64 * (6 + (with_rt ? 1 : 0) + (p != n[0] && !no_stage ? 2 : 0)) + vci * (4 + (prec != PSOLVE_FP64 ? 3 : 0));
    (void)sms;
    b += align_up(sizeof(Scal)) + align_up((size_t)units_max(n) * MAX_DOTS * sizeof(double));
    return b;
}

void problem_bind(Problem &P, char *base)
{
    const size_t N = (size_t)P.nvec();
    const size_t v64 = align_up(N * 8), vci = align_up(N * ci_elem_bytes(P.prec));
    char *q = base;
    Desc &D = P.desc;
    for (int r = 0; r < NROLES; ++r) D.vec[r] = nullptr;
    const int f64[] = {ROLE_R, ROLE_P, ROLE_P2, ROLE_W, ROLE_S, ROLE_T};
    for (int r : f64) {
        D.vec[r] = q;
        q += v64;
    }
    if (P.have_rt) {
        D.vec[ROLE_RT] = q;
        q += v64;
    }
    const int fci[] = {ROLE_PH, ROLE_RH, ROLE_YA, ROLE_YB};
    for (int r : fci) {
        D.vec[r] = q;
        q += vci;
    }
    if (P.prec != PSOLVE_FP64) {
        for (int r : {ROLE_BC, ROLE_YC, ROLE_YD}) {
            D.vec[r] = q;
            q += vci;
        }
    }
    P.d_bst = P.d_xst = nullptr;
    if (P.staged()) {
        P.d_bst = reinterpret_cast<double *>(q);
        q += v64;
        P.d_xst = reinterpret_cast<double *>(q);
        q += v64;
    }
    P.d_sc = reinterpret_cast<Scal *>(q);
    q += align_up(sizeof(Scal));
    P.d_partials = reinterpret_cast<double *>(q);
    D.sc = P.d_sc;
    D.partials = P.d_partials;
}

static double mu_dirichlet(long long i, long long n)
{
    const double s = std::sin((double)i * M_PI / (2.0 * (double)(n + 1)));
    return 4.0 * s * s; // Eq. 9
}

// Extreme eigenvalues of the 1-D operator of m unknowns with face conditions
// fm (minus), fp (plus): Dirichlet on both (D, Eq. 9); one zero-flux Neumann
// face (N, Eq. 5), whose eigenvectors are cosines of (2i-1) pi j / (2m) from
// the Neumann end, so mu_i = 4 sin^2((2i-1) pi / (4m)); Neumann on both faces,
// mu_i = 4 sin^2(i pi / (2(m-1))), i = 0..m-1.  In every case min + max = 4,
// so with exact bounds theta = cc still holds.
static void mu_range(long long m, int fm, int fp, double *mn, double *mx)
{
    if (!fm && !fp) {
        *mn = mu_dirichlet(1, m);
        *mx = mu_dirichlet(m, m);
    } else if (fm != fp) {
        const double s1 = std::sin(M_PI / (4.0 * (double)m));
        const double s2 = std::sin((2.0 * (double)m - 1.0) * M_PI / (4.0 * (double)m));
        *mn = 4.0 * s1 * s1;
        *mx = 4.0 * s2 * s2;
    } else {
        *mn = 0.0;
        *mx = 4.0;
    }
}

psolve_status cheb_interval(const Problem &P, int precond, double lmin_scale, double lmax_scale,
                            double *a, double *b)
{
    // Eq. 10 / Eq. 11 over the whole grid (G, GNoComm) or the blocks (BJ).  BJ
    // blocks differ in their outer faces (a block on a Neumann face keeps it,
    // faces between blocks are Dirichlet ghosts), so the interval takes per
    // axis the smallest minimum and the largest maximum over the first, the
    // interior and the last block.
    double lo = 0.0, hi = 0.0;
    for (int d = 0; d < 3; ++d) {
        const int fm = P.bc[2 * d], fp = P.bc[2 * d + 1];
        double mn, mx;
        if (precond == PSOLVE_PC_BJ_CHEB && P.blocks[d] > 1) {
            const long long m = P.n[d] / P.blocks[d];
            double mn2, mx2;
            mu_range(m, fm, 0, &mn, &mx);
            mu_range(m, 0, fp, &mn2, &mx2);
            mn = std::min(mn, mn2);
            mx = std::max(mx, mx2);
            if (P.blocks[d] > 2) {
                mu_range(m, 0, 0, &mn2, &mx2);
                mn = std::min(mn, mn2);
                mx = std::max(mx, mx2);
            }
        } else {
            mu_range(P.n[d], fm, fp, &mn, &mx);
        }
        const double ih2 = 1.0 / (P.h[d] * P.h[d]);
        lo += mn * ih2;
        hi += mx * ih2;
    }
    *a = lmin_scale * lo;
    *b = lmax_scale * hi;
    if (!(*a > 0.0) || !(*b > *a) || !std::isfinite(*a) || !std::isfinite(*b)) {
        set_error("empty Chebyshev interval [%g, %g] (lambda in [%g, %g], scales %g, %g)", *a, *b, lo,
                  hi, lmin_scale, lmax_scale);
        return PSOLVE_E_ARG;
    }
    return PSOLVE_OK;
}

// FP32 copies of the folded coefficients, rounded to nearest as the device's
// double-to-float conversion rounds.
static void set_cheb_f32(Desc &D)
{
    for (int q = 0; q < 4; ++q) D.ci1f[q] = static_cast<float>(D.ci1[q]);
    for (int k = 0; k <= MAX_DEGREE; ++k)
        for (int q = 0; q < 6; ++q) D.cikf[k][q] = static_cast<float>(D.cik[k][q]);
    D.theta_inv_f = static_cast<float>(D.theta_inv);
}

psolve_status problem_set_cheb(Problem &P, int precond, int degree, double lmin_scale, double lmax_scale)
{
    Desc &D = P.desc;
    D.degree = degree;
    set_hat(D, 1.0);
    if (precond == PSOLVE_PC_NONE || precond == PSOLVE_PC_G_BICGS || precond == PSOLVE_PC_BJ_BICGS) {
        D.theta_inv = D.two_over_delta = D.two_sigma = 0.0; // no Chebyshev iteration
        set_cheb_f32(D);
        return PSOLVE_OK;
    }
    double a, b;
    psolve_status st = cheb_interval(P, precond, lmin_scale, lmax_scale, &a, &b);
    if (st != PSOLVE_OK) return st;
    // Eq. 15 and the rho recurrence of Algorithm 2
    const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
    D.theta_inv = 1.0 / theta;
    D.two_over_delta = 2.0 / delta;
    D.two_sigma = 2.0 * sigma;
    D.rho[0] = 1.0 / sigma;
    for (int k = 1; k <= MAX_DEGREE; ++k) D.rho[k] = 1.0 / (2.0 * sigma - D.rho[k - 1]);
    // CI sweep 1: y_1 = (2 rho_1/delta)(2u - A u / theta), A u written with
    // the neighbour-pair sums: A u = cc u - cx sx - cy sy - cz sz
    // With FP64 vectors and d >= 2, y_1 is stored divided by its x-pair
    // coefficient (> 0), s_1 below.
    const bool scaled = P.prec == PSOLVE_FP64;
    const double tod = D.two_over_delta, c1 = tod * D.rho[1];
    const double ax = c1 * D.theta_inv * D.cx;
    const double s1 = (scaled && degree >= 2) ? ax : 1.0;
    D.ci1[0] = c1 * (2.0 - D.cc * D.theta_inv) / s1;
    D.ci1[1] = ax / s1; // exactly 1 when scaled
    D.ci1[2] = c1 * D.theta_inv * D.cy / s1;
    D.ci1[3] = c1 * D.theta_inv * D.cz / s1;
    // sweeps k >= 2: w = rho_k (2 sigma y + (2/delta)(b - A y) - rho_{k-1} z)
    //   = rho_k (2 sigma - (2/delta) cc) y + rho_k (2/delta) b - rho_k rho_{k-1} z
    //     + rho_k (2/delta)(cx sx + cy sy + cz sz),  z = b/theta when k = 2,
    // with FP64 vectors stored as yhat_j = y_j / s_j, s_j = the b coefficient
    // of sweep j for 2 <= j <= d (1 otherwise), so b enters with coefficient 1;
    // p^ = y_d is then stored divided by hat = s_d
    auto b_coef = [&](int j) { return j == 2 ? D.rho[2] * tod - D.rho[2] * D.rho[1] * D.theta_inv : D.rho[j] * tod; };
    auto scale = [&](int j) {
        if (j == 1) return s1;
        return (scaled && j >= 2 && j <= degree) ? b_coef(j) : 1.0;
    };
    std::memset(D.cik, 0, sizeof D.cik);
    for (int k = 2; k <= degree && k <= MAX_DEGREE; ++k) {
        const double rk = D.rho[k], rk1 = D.rho[k - 1];
        const double sk = scale(k), q1 = scale(k - 1) / sk, q2 = scale(k - 2) / sk;
        double *c = D.cik[k];
        c[0] = rk * (D.two_sigma - tod * D.cc) * q1;
        c[1] = b_coef(k) / sk; // exactly 1 when scaled
        c[2] = -rk * rk1 * q2;
        c[3] = rk * tod * D.cx * q1;
        c[4] = rk * tod * D.cy * q1;
        c[5] = rk * tod * D.cz * q1;
    }
    if (degree >= 2) set_hat(D, scale(degree));
    set_cheb_f32(D);
    return PSOLVE_OK;
}

} // namespace psolve
