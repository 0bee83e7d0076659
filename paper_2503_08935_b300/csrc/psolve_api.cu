// psolve_api.cu -- the C ABI of libpsolve: single-grid contexts, the
// building-block entry points and the batched solve.
//
// Solve loop.  The host launches the initial-residual kernel, then replays a
// captured CUDA graph of K outer iterations (or launches them directly) and
// after each replay copies the problems' scalar blocks to pinned memory.  Two
// replays are kept in flight, so the GPU never waits for the host; kernels of
// a problem whose `stop` flag is set return at once, so iterations issued
// past convergence cost only their launch.  alpha, omega, beta and every
// convergence decision are made on the device (Algorithm 1's scalars never
// round-trip through the host inside the loop).
#include <algorithm>
#include <chrono>

#include "psolve_engine.cuh"
#include "psolve_persist.cuh"
#include "psolve_tune.cuh"

using namespace psolve;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct GraphEntry {
    Plan plan;
    int k = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t nodes = 0;
};

// State of one solve loop over a launch list of `nsc` problems whose scalar
// blocks lie contiguously at d_sc.
struct Runner {
    cudaStream_t stream = 0, cap = 0;
    const Desc *d_desc = nullptr;
    const int32_t *d_list = nullptr;
    int sms = 1;
    long long units = 1;
    Plan plan;
    int K = 1;
    bool use_graph = true;
    bool timing = false;
    double npts = 0;
    std::vector<GraphEntry> *graphs = nullptr;
    std::vector<cudaEvent_t> *events = nullptr;
    size_t event_next = 0;
    std::vector<LaunchRec> recs;
    Scal *d_sc = nullptr;
    int nsc = 1;
    Scal *h_sc[2] = {nullptr, nullptr};
    cudaEvent_t poll_ev[2] = {nullptr, nullptr};
    int64_t launches = 0;
    int iter_issued = 0;
    int last_slot = 0;

    Launcher launcher()
    {
        Launcher L;
        L.stream = stream;
        L.sms = sms;
        L.units = units;
        L.d_desc = d_desc;
        L.d_list = d_list;
        L.timing = timing;
        L.npts = npts;
        L.recs = timing ? &recs : nullptr;
        L.event_pool = events;
        L.event_next = &event_next;
        return L;
    }
};

psolve_status get_graph(Runner &R, int k, GraphEntry **out)
{
    for (GraphEntry &g : *R.graphs)
        if (g.plan == R.plan && g.k == k) {
            *out = &g;
            return PSOLVE_OK;
        }
    Launcher C;
    C.stream = R.cap;
    C.sms = R.sms;
    C.units = R.units;
    C.d_desc = R.d_desc;
    C.d_list = R.d_list;
    C.iter = 2;
    {
        // kernel attributes are set outside the capture
        Launcher cfg = C;
        cfg.configure = true;
        enqueue_iteration(cfg, R.plan);
        PS_CK(cfg.err);
    }
    PS_CK(cudaStreamBeginCapture(R.cap, cudaStreamCaptureModeThreadLocal));
    for (int j = 0; j < k; ++j) enqueue_iteration(C, R.plan);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(R.cap, &g);
    if (C.err != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        set_error("graph capture failed: %s", cudaGetErrorString(C.err != cudaSuccess ? C.err : e));
        return PSOLVE_E_CUDA;
    }
    GraphEntry ent;
    ent.plan = R.plan;
    ent.k = k;
    ent.nodes = C.launches;
    e = cudaGraphInstantiate(&ent.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        set_error("cudaGraphInstantiate: %s", cudaGetErrorString(e));
        return PSOLVE_E_CUDA;
    }
    R.graphs->push_back(ent);
    *out = &R.graphs->back();
    return PSOLVE_OK;
}

psolve_status issue(Runner &R, int slot, int k)
{
    if (R.use_graph && !R.timing) {
        GraphEntry *g = nullptr;
        psolve_status st = get_graph(R, k, &g);
        if (st != PSOLVE_OK) return st;
        PS_CK(cudaGraphLaunch(g->exec, R.stream));
        R.launches += g->nodes;
        R.iter_issued += k;
    } else {
        Launcher L = R.launcher();
        for (int j = 0; j < k; ++j) {
            L.iter = ++R.iter_issued;
            enqueue_iteration(L, R.plan);
        }
        R.launches += L.launches;
        PS_CK(L.err);
    }
    PS_CK(cudaMemcpyAsync(R.h_sc[slot], R.d_sc, sizeof(Scal) * R.nsc, cudaMemcpyDeviceToHost, R.stream));
    PS_CK(cudaEventRecord(R.poll_ev[slot], R.stream));
    return PSOLVE_OK;
}

bool all_stopped(const Scal *s, int n)
{
    for (int q = 0; q < n; ++q)
        if (!s[q].stop) return false;
    return true;
}

// Runs iterations until every problem has stopped.  maxit bounds the loop
// (the device stops each problem at its own maxit).  On return h_sc[last_slot]
// holds the final scalar blocks.
psolve_status run_loop(Runner &R, int maxit)
{
    psolve_status st = issue(R, 0, 1);
    if (st != PSOLVE_OK) return st;
    st = issue(R, 1, 1);
    if (st != PSOLVE_OK) return st;
    const long long bound = (long long)maxit + 2LL * R.K + 4;
    int slot = 0;
    for (;;) {
        PS_CK(cudaEventSynchronize(R.poll_ev[slot]));
        if (all_stopped(R.h_sc[slot], R.nsc)) break;
        if (R.iter_issued > bound) {
            set_error("device did not stop after %d issued iterations (maxit %d)", R.iter_issued, maxit);
            return PSOLVE_TIMEOUT;
        }
        st = issue(R, slot, R.K);
        if (st != PSOLVE_OK) return st;
        slot ^= 1;
    }
    R.last_slot = slot;
    PS_CK(cudaStreamSynchronize(R.stream));
    return PSOLVE_OK;
}

int auto_poll(double bytes_per_iter, int kernels_per_iter)
{
    // estimated iteration time: bytes at ~5 TB/s plus ~2 us per launch
    const double us = bytes_per_iter / 5e6 + 2.0 * kernels_per_iter;
    int k = (int)(600.0 / us);
    return std::max(1, std::min(8, k));
}

// A cached single-launch graph of the persistent solve.
struct PersistEntry {
    Plan plan;
    int maxit = 0;
    bool use_x0 = false, true_res = false;
    cudaGraphExec_t exec = nullptr;
};

// The whole solve of a launch list as one persistent kernel launch (captured
// into a CUDA graph when use_graph; cached in *cache when given).  Uploads the
// phase table from h_st (pinned; must stay untouched until the stream has
// passed the launch), then enqueues the launch; d_st->gs.err tells afterwards
// whether a barrier wait gave up.
psolve_status run_persistent(cudaStream_t s, cudaStream_t cap, const Plan &plan, int sms, long long units,
                             const Desc *d_desc, const int32_t *d_list, PersistState *d_st, PersistState *h_st,
                             int maxit, bool use_x0, bool true_res, bool use_graph, std::vector<PersistEntry> *cache)
{
    int grid = 1;
    psolve_status st = persist_configure(plan, sms, units, &grid);
    if (st != PSOLVE_OK) return st;
    persist_table(plan, use_x0, true_res, h_st);
    const size_t off = offsetof(PersistState, n_init);
    const size_t bytes = offsetof(PersistState, ph) - off +
                         sizeof(PhaseRec) * (size_t)(h_st->n_init + h_st->n_iter + h_st->n_tail);
    PS_CK(cudaMemcpyAsync(reinterpret_cast<char *>(d_st) + off, reinterpret_cast<char *>(h_st) + off, bytes,
                          cudaMemcpyHostToDevice, s));
    PersistArgs a{};
    a.descs = d_desc;
    a.list = d_list;
    a.st = d_st;
    a.iters = maxit;
    a.n_init = h_st->n_init;
    a.n_iter = h_st->n_iter;
    a.n_tail = h_st->n_tail;
    if (!use_graph) return persist_enqueue(s, plan, grid, a);
    if (cache)
        for (const PersistEntry &e : *cache)
            if (e.plan == plan && e.maxit == maxit && e.use_x0 == use_x0 && e.true_res == true_res) {
                PS_CK(cudaGraphLaunch(e.exec, s));
                return PSOLVE_OK;
            }
    PS_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    st = persist_enqueue(cap, plan, grid, a);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (st != PSOLVE_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (st == PSOLVE_OK) set_error("capture of the persistent launch: %s", cudaGetErrorString(e));
        return PSOLVE_E_CUDA;
    }
    PersistEntry ent;
    ent.plan = plan;
    ent.maxit = maxit;
    ent.use_x0 = use_x0;
    ent.true_res = true_res;
    e = cudaGraphInstantiate(&ent.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        set_error("cudaGraphInstantiate (persistent): %s", cudaGetErrorString(e));
        return PSOLVE_E_CUDA;
    }
    e = cudaGraphLaunch(ent.exec, s);
    if (cache) cache->push_back(ent);
    else {
        // one-shot graph: destroyed once the launch has completed
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaGraphExecDestroy(ent.exec);
    }
    if (e != cudaSuccess) {
        set_error("persistent graph launch: %s", cudaGetErrorString(e));
        return PSOLVE_E_CUDA;
    }
    return PSOLVE_OK;
}

void fill_timing(const std::vector<LaunchRec> &recs, int final_iter, int half_exit, psolve_result *res)
{
    for (const LaunchRec &r : recs) {
        if (!r.ev0 || !launch_did_work(r, final_iter, half_exit)) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.ev0, r.ev1) != cudaSuccess) continue;
        res->kclass_ms[r.cls] += ms;
        res->kclass_launches[r.cls] += 1;
        res->kclass_bytes[r.cls] += (r.iter == final_iter && half_exit && r.is_update) ? r.bytes_half : r.bytes;
    }
}

bool valid_h(const double h[3])
{
    for (int d = 0; d < 3; ++d)
        if (!(h[d] > 0.0) || !std::isfinite(h[d])) return false;
    return true;
}

psolve_status check_grid(const int64_t g[3])
{
    long long n = 1;
    for (int d = 0; d < 3; ++d) {
        if (g[d] < 1 || g[d] > (1LL << 30)) {
            set_error("grid size %lld on axis %d out of range", (long long)g[d], d);
            return PSOLVE_E_ARG;
        }
        n *= g[d];
        if (n >= (1LL << 31)) {
            set_error("grid has 2^31 points or more");
            return PSOLVE_E_ARG;
        }
    }
    return PSOLVE_OK;
}

psolve_status check_rr(int rr_every)
{
    if (rr_every < 0) {
        set_error("rr_every must be >= 0");
        return PSOLVE_E_ARG;
    }
    return PSOLVE_OK;
}

psolve_status check_solve_args(double rtol, int maxit, int precond, int degree)
{
    if (!(rtol >= 0.0) || !std::isfinite(rtol)) {
        set_error("rtol must be finite and >= 0");
        return PSOLVE_E_ARG;
    }
    if (maxit < 0) {
        set_error("maxit must be >= 0");
        return PSOLVE_E_ARG;
    }
    if (precond < PSOLVE_PC_NONE || precond > PSOLVE_PC_BJ_BICGS) {
        set_error("unknown preconditioner %d", precond);
        return PSOLVE_E_ARG;
    }
    if (degree < 0 || degree > MAX_DEGREE) {
        set_error("Chebyshev degree %d outside [0, %d]", degree, MAX_DEGREE);
        return PSOLVE_E_ARG;
    }
    return PSOLVE_OK;
}

psolve_status check_blocks(const Problem &P, int precond)
{
    if (precond != PSOLVE_PC_BJ_CHEB && precond != PSOLVE_PC_GNOCOMM_CHEB && precond != PSOLVE_PC_BJ_BICGS)
        return PSOLVE_OK;
    for (int d = 0; d < 3; ++d) {
        if (P.n[d] % P.blocks[d] != 0) {
            set_error("blocks[%d] = %d does not divide the grid size %lld", d, P.blocks[d], (long long)P.n[d]);
            return PSOLVE_E_ARG;
        }
        if ((P.bc[2 * d] || P.bc[2 * d + 1]) && P.n[d] / P.blocks[d] < 2) {
            set_error("axis %d has a Neumann face: its blocks need at least 2 unknowns", d);
            return PSOLVE_E_ARG;
        }
    }
    return PSOLVE_OK;
}

void fill_result(const Scal &s, const Problem &P, const Plan &plan, bool use_x0, bool true_res, double t0,
                 int64_t launches, psolve_result *res)
{
    psolve_result r;
    std::memset(&r, 0, sizeof r);
    r.status = s.status;
    r.iterations = s.iter;
    r.half_step_exit = s.half_exit;
    r.engine = P.desc.tma;
    r.slab_planes = P.desc.zc;
    r.tuned = P.tuned;
    r.rel_res_recursive = s.nb2 > 0 ? std::sqrt(s.rr / s.nb2) : 0.0;
    r.rel_res_true = !true_res ? -1.0 : (s.nb2 > 0 ? std::sqrt(s.true_rr / s.nb2) : 0.0);
    r.seconds = now_s() - t0;
    r.kernel_launches = launches;
    // algorithmic bytes of the work done (dry run of the same launch sequence)
    std::vector<LaunchRec> recs;
    Launcher D;
    D.dry = true;
    D.npts = (double)P.npts();
    D.recs = &recs;
    D.iter = 0;
    enqueue_init(D, use_x0);
    for (int it = 1; it <= s.iter; ++it) {
        D.iter = it;
        enqueue_iteration(D, plan);
    }
    if (true_res) {
        D.iter = -1;
        enqueue_true_residual(D);
    }
    r.model_bytes = model_bytes_for(recs, s.iter, s.half_exit);
    if (res) {
        // keep timing fields the caller's run filled
        for (int c = 0; c < PSOLVE_K_NCLASS; ++c) {
            r.kclass_ms[c] = res->kclass_ms[c];
            r.kclass_launches[c] = res->kclass_launches[c];
            r.kclass_bytes[c] = res->kclass_bytes[c];
        }
        *res = r;
    }
}

// Inner solver of the flexible preconditioners: one problem (G(BiCGS), the
// whole grid) or one per block (BJ(BiCGS)), each with its own Krylov
// workspace and scalars, solved together over one launch list.
struct FlexInner {
    int precond = -1;          // the flexible preconditioner the buffers were built for
    int nblk = 0;
    std::vector<Problem> probs;
    char *mem = nullptr;       // Krylov workspaces
    double *bbuf = nullptr;    // BJ: block-contiguous right-hand sides
    double *xbuf = nullptr;    // BJ: block-contiguous solutions
    Scal *d_sc = nullptr;
    Desc *d_desc = nullptr, *h_desc = nullptr;
    CUtensorMap *d_tmap = nullptr, *h_tmap = nullptr;
    int32_t *d_list = nullptr, *h_list = nullptr;
    Scal *h_sc = nullptr;      // 2 x nblk pinned
    cudaEvent_t ev[2] = {nullptr, nullptr};
    std::vector<GraphEntry> graphs;
    std::vector<cudaEvent_t> events;
    long long units = 0;

    void release()
    {
        for (GraphEntry &g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        graphs.clear();
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        events.clear();
        for (cudaEvent_t &e : ev)
            if (e) {
                cudaEventDestroy(e);
                e = nullptr;
            }
        cudaFree(mem);
        cudaFree(bbuf);
        cudaFree(xbuf);
        cudaFree(d_sc);
        cudaFree(d_desc);
        cudaFree(d_tmap);
        cudaFree(d_list);
        cudaFreeHost(h_desc);
        cudaFreeHost(h_tmap);
        cudaFreeHost(h_list);
        cudaFreeHost(h_sc);
        mem = nullptr;
        bbuf = xbuf = nullptr;
        d_sc = nullptr;
        d_desc = h_desc = nullptr;
        d_tmap = h_tmap = nullptr;
        d_list = h_list = nullptr;
        h_sc = nullptr;
        probs.clear();
        precond = -1;
        nblk = 0;
    }
};

bool is_flexible(int precond) { return precond == PSOLVE_PC_G_BICGS || precond == PSOLVE_PC_BJ_BICGS; }

} // namespace

// ====================================================================== ctx
struct psolve_ctx {
    DevInfo di;
    cudaStream_t stream = 0;
    cudaStream_t cap = 0;
    psolve_opts opts;
    Problem P;
    Desc *d_desc = nullptr;
    int32_t *d_list = nullptr;
    Desc *h_desc = nullptr;
    CUtensorMap *d_tmap = nullptr, *h_tmap = nullptr; // TMA descriptors of the workspace roles
    Scal *h_sc = nullptr; // 3 pinned slots: 2 for polling, 1 for set-up
    cudaEvent_t poll_ev[2] = {nullptr, nullptr};
    std::vector<GraphEntry> graphs;
    std::vector<PersistEntry> pgraphs;    // single-launch graphs of the persistent solve
    PersistState *d_ps = nullptr, *h_ps = nullptr; // its barrier words and phase table (device, pinned)
    std::vector<cudaEvent_t> events;
    double *d_hb = nullptr, *d_hx = nullptr; // device copies for psolve_solve_host
    bool tma_ok = true; // false: the autotuner chose the general engine
    FlexInner flex;     // G(BiCGS) / BJ(BiCGS) inner solver, built on first use
    double *d_hist = nullptr; // residual history (opts.record_history), 2 doubles per iteration
    int hist_cap = 0;         // iterations d_hist holds
    bool solved = false;      // a solve has run (its scalars are in P.d_sc)
    TmapCache tmc;            // what h_tmap / d_tmap hold (upload_desc)
    bool desc_valid = false;  // d_desc equals *h_desc
    Plan poll_plan;           // the plan poll_K was computed for (poll_K < 0: none)
    int poll_K = -1;
};

extern "C" {

void psolve_opts_default(psolve_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->lmin_scale = 1.0;
    o->lmax_scale = 1.0;
    o->blocks[0] = o->blocks[1] = o->blocks[2] = 1;
    o->cheb_prec = PSOLVE_FP64;
    o->half_step_check = 1;
    o->use_x0 = 0;
    o->poll_every = 0;
    o->use_graph = 1;
    o->timing = 0;
    o->true_residual = 1;
    o->rr_every = 0;
}

const char *psolve_last_error(void) { return last_error(); }

const char *psolve_version(void) { return "psolve 0.1 (sm_103a, 7-point FD Poisson, Bi-CGSTAB + Chebyshev)"; }

void psolve_destroy(psolve_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->di.dev);
    if (c->stream) cudaStreamSynchronize(c->stream);
    c->flex.release();
    for (GraphEntry &g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (PersistEntry &g : c->pgraphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (c->d_ps) cudaFree(c->d_ps);
    if (c->h_ps) cudaFreeHost(c->h_ps);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    for (cudaEvent_t e : c->poll_ev)
        if (e) cudaEventDestroy(e);
    if (c->P.mem) cudaFree(c->P.mem);
    if (c->d_desc) cudaFree(c->d_desc);
    if (c->d_list) cudaFree(c->d_list);
    if (c->d_hb) cudaFree(c->d_hb);
    if (c->d_hx) cudaFree(c->d_hx);
    if (c->d_hist) cudaFree(c->d_hist);
    if (c->h_desc) cudaFreeHost(c->h_desc);
    if (c->d_tmap) cudaFree(c->d_tmap);
    if (c->h_tmap) cudaFreeHost(c->h_tmap);
    if (c->h_sc) cudaFreeHost(c->h_sc);
    if (c->cap) cudaStreamDestroy(c->cap);
    delete c;
}

psolve_status psolve_create(const int64_t grid[3], const double h[3], const int32_t bc[6],
                            const psolve_opts *opts, uintptr_t stream, psolve_ctx **out)
{
    clear_error();
    if (!grid || !h || !out) {
        set_error("null argument");
        return PSOLVE_E_ARG;
    }
    psolve_status st = check_grid(grid);
    if (st != PSOLVE_OK) return st;
    if (!valid_h(h)) {
        set_error("grid spacing must be finite and > 0");
        return PSOLVE_E_ARG;
    }
    if (bc) {
        int dirichlet = 0;
        for (int f = 0; f < 6; ++f) {
            if (bc[f] != 0 && bc[f] != 1) {
                set_error("face %d: condition %d is neither 0 (Dirichlet) nor 1 (Neumann)", f, bc[f]);
                return PSOLVE_E_ARG;
            }
            if (bc[f] == 1 && grid[f / 2] < 2) {
                set_error("face %d: a Neumann face needs at least 2 unknowns on its axis", f);
                return PSOLVE_E_ARG;
            }
            dirichlet += bc[f] == 0;
        }
        if (!dirichlet) {
            set_error("every face is Neumann: the operator is singular");
            return PSOLVE_E_ARG;
        }
    }
    psolve_opts o;
    psolve_opts_default(&o);
    if (opts) o = *opts;
    for (int d = 0; d < 3; ++d)
        if (o.blocks[d] < 1 || o.blocks[d] > grid[d]) {
            set_error("blocks[%d] = %d outside [1, n]", d, o.blocks[d]);
            return PSOLVE_E_ARG;
        }
    if (o.cheb_prec < PSOLVE_FP64 || o.cheb_prec > PSOLVE_BF16) {
        set_error("unknown Chebyshev precision %d", o.cheb_prec);
        return PSOLVE_E_ARG;
    }
    if (o.slab_share < 0 || o.slab_share > 4096) {
        set_error("slab_share %d outside [0, 4096]", o.slab_share);
        return PSOLVE_E_ARG;
    }
    psolve_ctx *c = new psolve_ctx();
    c->opts = o;
    c->stream = (cudaStream_t)stream;
    st = device_info(&c->di);
    if (st != PSOLVE_OK) {
        delete c;
        return st;
    }
    Problem &P = c->P;
    for (int d = 0; d < 3; ++d) {
        P.n[d] = grid[d];
        P.h[d] = h[d];
        P.blocks[d] = o.blocks[d];
    }
    if (bc)
        for (int f = 0; f < 6; ++f) P.bc[f] = bc[f];
    P.prec = o.cheb_prec;
    P.have_rt = o.use_x0 != 0;
    // rows padded to a multiple of 8 elements when nx is not one, so that the
    // tensor copies can run on the grid (unless the general engine is forced)
    P.px = (o.engine != 1 && P.n[0] % 8 != 0) ? padded_pitch(P.n[0]) : 0;
    problem_geometry(P, c->di.sms, 0, o.slab_share > 0 ? o.slab_share : 1);
    P.mem_bytes = problem_bytes(P.n, P.prec, P.have_rt, c->di.sms, P.px);
#define CREATE_CK(call)                                                                          \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            set_error("%s: %s", #call, cudaGetErrorString(e_));                                  \
            psolve_destroy(c);                                                                   \
            return e_ == cudaErrorMemoryAllocation ? PSOLVE_E_OOM : PSOLVE_E_CUDA;               \
        }                                                                                        \
    } while (0)
    CREATE_CK(cudaMalloc(&P.mem, P.mem_bytes));
    problem_bind(P, P.mem);
    if (o.autotune) {
        TuneChoice tc;
        st = tune_problem(P, c->di.sms, c->stream, &tc);
        if (st != PSOLVE_OK) {
            psolve_destroy(c);
            return st;
        }
        problem_geometry(P, c->di.sms, tc.zc);
        c->tma_ok = tc.engine == 1;
        P.tuned = tc.from_cache ? 2 : 1;
    }
    CREATE_CK(cudaMemset(P.d_sc, 0, sizeof(Scal)));
    CREATE_CK(cudaMalloc(&c->d_desc, sizeof(Desc)));
    CREATE_CK(cudaMalloc(&c->d_list, (LIST_HDR_INTS + 2) * sizeof(int32_t)));
    CREATE_CK(cudaHostAlloc(&c->h_desc, sizeof(Desc), cudaHostAllocDefault));
    CREATE_CK(cudaHostAlloc(&c->h_sc, 3 * sizeof(Scal), cudaHostAllocDefault));
    CREATE_CK(cudaMalloc(&c->d_ps, sizeof(PersistState)));
    CREATE_CK(cudaHostAlloc(&c->h_ps, sizeof(PersistState), cudaHostAllocDefault));
    CREATE_CK(cudaMalloc(&c->d_tmap, sizeof(CUtensorMap) * TMAPS_PER_PROBLEM));
    CREATE_CK(cudaHostAlloc(&c->h_tmap, sizeof(CUtensorMap) * TMAPS_PER_PROBLEM, cudaHostAllocDefault));
    P.desc.tmap = c->d_tmap;
    const int32_t list[LIST_HDR_INTS + 2] = {1, P.desc.units, 0, 0, 0, 0};
    CREATE_CK(cudaMemcpy(c->d_list, list, sizeof list, cudaMemcpyHostToDevice));
    CREATE_CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    for (int s = 0; s < 2; ++s) CREATE_CK(cudaEventCreateWithFlags(&c->poll_ev[s], cudaEventDisableTiming));
#undef CREATE_CK
    *out = c;
    return PSOLVE_OK;
}

// Brings d_desc and d_tmap up to date with c->P.desc.  Only the tensor maps of
// vectors that changed since the last upload are encoded and copied, and the
// descriptor is copied only when it differs from the one on the device: a
// repeated solve on the same buffers (the small-grid latency case) pays for
// neither.  Every entry point synchronizes its stream before returning, so
// the pinned staging copies are never rewritten under a pending copy.
static psolve_status upload_desc(psolve_ctx *c)
{
    problem_encode_tmaps(c->P, c->h_tmap, c->opts.engine != 1 && c->tma_ok, &c->tmc);
    const TmapCache &tc = c->tmc;
    if (c->P.desc.tma && tc.hi > tc.lo) {
        const size_t first = (size_t)TMAPS_PER_ROLE * tc.lo, count = (size_t)TMAPS_PER_ROLE * (tc.hi - tc.lo);
        cudaError_t e = cudaMemcpyAsync(c->d_tmap + first, c->h_tmap + first, sizeof(CUtensorMap) * count,
                                        cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) {
            c->tmc.valid = false;
            PS_CK(e);
        }
    }
    if (!c->desc_valid || std::memcmp(c->h_desc, &c->P.desc, sizeof(Desc)) != 0) {
        *c->h_desc = c->P.desc;
        c->desc_valid = false;
        PS_CK(cudaMemcpyAsync(c->d_desc, c->h_desc, sizeof(Desc), cudaMemcpyHostToDevice, c->stream));
        c->desc_valid = true;
    }
    return PSOLVE_OK;
}

static Launcher ctx_launcher(psolve_ctx *c)
{
    Launcher L;
    L.stream = c->stream;
    L.sms = c->di.sms;
    L.units = c->P.desc.units;
    L.d_desc = c->d_desc;
    L.d_list = c->d_list;
    return L;
}

// ============================================================ flexible
// G(BiCGS) and BJ(BiCGS): the preconditioner is an inner Bi-CGSTAB solve, on
// the whole grid or on each block, so it changes from one application to the
// next; Algorithm 1 accommodates that because x is updated with the
// preconditioned vectors p^ and r^ themselves (flexible Bi-CGSTAB).  The
// outer iteration runs its phases as separate launches around the inner
// solves, and the host reads the outer scalars after the half step and after
// the update; each inner solve is the graph-replayed solve loop over its own
// problem list.

// Build the inner problems for `precond` on c's grid (once per kind).
static psolve_status flex_setup(psolve_ctx *c, int precond)
{
    FlexInner &F = c->flex;
    if (F.precond == precond) return PSOLVE_OK;
    F.release();
    const Problem &P = c->P;
    const bool bj = precond == PSOLVE_PC_BJ_BICGS;
    int nb[3] = {1, 1, 1};
    int64_t m[3] = {P.n[0], P.n[1], P.n[2]};
    if (bj)
        for (int d = 0; d < 3; ++d) {
            nb[d] = P.blocks[d];
            m[d] = P.n[d] / nb[d];
        }
    const int nblk = nb[0] * nb[1] * nb[2];
    F.probs.assign((size_t)nblk, Problem());
    size_t total = 0;
    std::vector<size_t> offs((size_t)nblk);
    for (int q = 0; q < nblk; ++q) {
        Problem &Q = F.probs[q];
        const int B[3] = {q % nb[0], (q / nb[0]) % nb[1], q / (nb[0] * nb[1])};
        for (int d = 0; d < 3; ++d) {
            Q.n[d] = m[d];
            Q.h[d] = P.h[d];
            // a block keeps the domain's condition on the faces it shares with the
            // domain, and has zero Dirichlet ghosts towards its neighbours
            Q.bc[2 * d] = B[d] == 0 ? P.bc[2 * d] : 0;
            Q.bc[2 * d + 1] = B[d] == nb[d] - 1 ? P.bc[2 * d + 1] : 0;
        }
        Q.prec = PSOLVE_FP64;
        if (!bj) { // G(BiCGS) binds the outer vectors: the same row pitch, nothing to stage
            Q.px = P.px;
            Q.no_stage = true;
        }
        problem_geometry(Q, c->di.sms, 0, nblk); // the blocks share every launch
        offs[q] = total;
        total += problem_bytes(Q.n, PSOLVE_FP64, false, c->di.sms, Q.px, Q.no_stage);
    }
    const size_t M = (size_t)(m[0] * m[1] * m[2]);
    const size_t list_bytes = sizeof(int32_t) * (LIST_HDR_INTS + 2 * (size_t)nblk);
#define FLEX_CK(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            set_error("inner solver set-up: %s: %s", #call, cudaGetErrorString(e_));       \
            F.release();                                                                   \
            return e_ == cudaErrorMemoryAllocation ? PSOLVE_E_OOM : PSOLVE_E_CUDA;         \
        }                                                                                  \
    } while (0)
    FLEX_CK(cudaMalloc(&F.mem, total));
    if (bj) {
        FLEX_CK(cudaMalloc(&F.bbuf, sizeof(double) * M * nblk));
        FLEX_CK(cudaMalloc(&F.xbuf, sizeof(double) * M * nblk));
    }
    FLEX_CK(cudaMalloc(&F.d_sc, sizeof(Scal) * nblk));
    FLEX_CK(cudaMalloc(&F.d_desc, sizeof(Desc) * nblk));
    FLEX_CK(cudaMalloc(&F.d_tmap, sizeof(CUtensorMap) * TMAPS_PER_PROBLEM * nblk));
    FLEX_CK(cudaMalloc(&F.d_list, list_bytes));
    FLEX_CK(cudaHostAlloc(&F.h_desc, sizeof(Desc) * nblk, cudaHostAllocDefault));
    FLEX_CK(cudaHostAlloc(&F.h_tmap, sizeof(CUtensorMap) * TMAPS_PER_PROBLEM * nblk, cudaHostAllocDefault));
    FLEX_CK(cudaHostAlloc(&F.h_list, list_bytes, cudaHostAllocDefault));
    FLEX_CK(cudaHostAlloc(&F.h_sc, 2 * sizeof(Scal) * nblk, cudaHostAllocDefault));
    for (int k = 0; k < 2; ++k) FLEX_CK(cudaEventCreateWithFlags(&F.ev[k], cudaEventDisableTiming));
    F.h_list[0] = nblk;
    F.h_list[2] = F.h_list[3] = 0;
    int32_t ub = 0;
    for (int q = 0; q < nblk; ++q) {
        Problem &Q = F.probs[q];
        problem_bind(Q, F.mem + offs[q]);
        Q.desc.sc = F.d_sc + q;
        Q.desc.tmap = F.d_tmap + (size_t)TMAPS_PER_PROBLEM * q;
        Q.desc.half_check = 1;
        F.h_list[LIST_HDR_INTS + 2 * q] = q;
        F.h_list[LIST_HDR_INTS + 1 + 2 * q] = ub;
        ub += Q.desc.units;
    }
    F.h_list[1] = ub;
    F.units = ub;
    FLEX_CK(cudaMemcpyAsync(F.d_list, F.h_list, list_bytes, cudaMemcpyHostToDevice, c->stream));
#undef FLEX_CK
    F.nblk = nblk;
    F.precond = precond;
    return PSOLVE_OK;
}

// out = inner Bi-CGSTAB approximation of A^-1 v (v, out: device grid vectors,
// distinct).  *inner_iters += the iteration count (the largest block count).
static psolve_status flex_inner(psolve_ctx *c, const double *v, double *out, double rtol, int maxit,
                                int64_t *inner_iters, int64_t *launches)
{
    FlexInner &F = c->flex;
    const bool bj = F.precond == PSOLVE_PC_BJ_BICGS;
    const size_t M = (size_t)(F.probs[0].npts());
    if (bj) {
        enqueue_gather_blocks(c->stream, v, F.bbuf, c->P.n, c->P.pitch(), c->P.blocks, true);
        PS_CK(cudaGetLastError());
        ++*launches;
    }
    for (int q = 0; q < F.nblk; ++q) {
        Problem &Q = F.probs[q];
        Desc &D = Q.desc;
        D.rtol = rtol;
        D.maxit = maxit;
        D.vec[ROLE_B] = bj ? (void *)(F.bbuf + q * M) : (void *)v;
        D.vec[ROLE_X] = bj ? (void *)(F.xbuf + q * M) : (void *)out;
        D.vec[ROLE_RT] = D.vec[ROLE_B]; // x0 = 0: r~ = r0 = b
        problem_encode_tmaps(Q, F.h_tmap + (size_t)TMAPS_PER_PROBLEM * q, c->opts.engine != 1);
        F.h_desc[q] = D;
    }
    PS_CK(cudaMemcpyAsync(F.d_tmap, F.h_tmap, sizeof(CUtensorMap) * TMAPS_PER_PROBLEM * F.nblk,
                          cudaMemcpyHostToDevice, c->stream));
    PS_CK(cudaMemcpyAsync(F.d_desc, F.h_desc, sizeof(Desc) * F.nblk, cudaMemcpyHostToDevice, c->stream));
    PS_CK(cudaMemsetAsync(F.d_sc, 0, sizeof(Scal) * F.nblk, c->stream));
    Runner R;
    R.stream = c->stream;
    R.cap = c->cap;
    R.d_desc = F.d_desc;
    R.d_list = F.d_list;
    R.sms = c->di.sms;
    R.units = F.units;
    R.plan.precond = PSOLVE_PC_NONE;
    R.use_graph = c->opts.use_graph != 0;
    R.npts = (double)c->P.npts();
    R.graphs = &F.graphs;
    R.events = &F.events;
    R.d_sc = F.d_sc;
    R.nsc = F.nblk;
    R.h_sc[0] = F.h_sc;
    R.h_sc[1] = F.h_sc + F.nblk;
    R.poll_ev[0] = F.ev[0];
    R.poll_ev[1] = F.ev[1];
    R.K = 4;
    Launcher L = R.launcher();
    L.iter = 0;
    enqueue_init(L, false);
    *launches += L.launches;
    PS_CK(L.err);
    psolve_status st = run_loop(R, maxit);
    *launches += R.launches;
    if (st != PSOLVE_OK) return st;
    const Scal *sc = R.h_sc[R.last_slot];
    int worst = 0;
    for (int q = 0; q < F.nblk; ++q) {
        worst = std::max(worst, sc[q].iter);
        // a breakdown or a non-finite value ends the outer solve; a solve that
        // ran out of iterations still gives a usable approximation
        if (sc[q].status != PSOLVE_OK && sc[q].status != PSOLVE_NOT_CONVERGED) {
            set_error("inner Bi-CGSTAB of problem %d stopped with status %d", q, sc[q].status);
            return (psolve_status)sc[q].status;
        }
    }
    *inner_iters += worst;
    if (bj) {
        enqueue_gather_blocks(c->stream, F.xbuf, out, c->P.n, c->P.pitch(), c->P.blocks, false);
        PS_CK(cudaGetLastError());
        ++*launches;
    }
    return PSOLVE_OK;
}

// The flexible forms keep p^ and r^ in FP64 and drive the outer phases from
// the host.
static psolve_status check_flexible(const psolve_ctx *c)
{
    if (c->P.prec != PSOLVE_FP64) {
        set_error("G(BiCGS) and BJ(BiCGS) need a context with cheb_prec = PSOLVE_FP64");
        return PSOLVE_E_ARG;
    }
    if (c->opts.persistent || c->opts.timing || c->opts.rr_every) {
        set_error("G(BiCGS) and BJ(BiCGS) run without persistent, timing and rr_every");
        return PSOLVE_E_ARG;
    }
    return PSOLVE_OK;
}

static double flex_rtol(const psolve_ctx *c, int precond)
{
    if (c->opts.inner_rtol > 0.0) return c->opts.inner_rtol;
    return precond == PSOLVE_PC_G_BICGS ? 1e-2 : 1e-6; // the experimental set-up's tolerances
}

static int flex_maxit(const psolve_ctx *c) { return c->opts.inner_maxit > 0 ? c->opts.inner_maxit : 500; }

// The outer flexible iteration on c's workspace (FP64 vectors p^ = ROLE_PH,
// r^ = ROLE_RH); D, the descriptor, is already uploaded.
static psolve_status flex_solve(psolve_ctx *c, int precond, int maxit, bool use_x0, bool tr, double t0,
                                psolve_result *res)
{
    psolve_status st = flex_setup(c, precond);
    if (st != PSOLVE_OK) return st;
    Problem &P = c->P;
    Scal *hs = c->h_sc + 2;
    int64_t launches = 0, inner_iters = 0;
    const double irtol = flex_rtol(c, precond);
    const int imaxit = flex_maxit(c);
    auto read = [&]() -> psolve_status {
        PS_CK(cudaMemcpyAsync(hs, P.d_sc, sizeof(Scal), cudaMemcpyDeviceToHost, c->stream));
        PS_CK(cudaStreamSynchronize(c->stream));
        return PSOLVE_OK;
    };
    Launcher L = ctx_launcher(c);
    L.iter = 0;
    enqueue_init(L, use_x0);
    PS_CK(L.err);
    launches += L.launches;
    st = read();
    if (st != PSOLVE_OK) return st;
    double *ph = (double *)P.desc.vec[ROLE_PH], *rh = (double *)P.desc.vec[ROLE_RH];
    L.launches = 0;
    for (int it = 1; it <= maxit && !hs->stop; ++it) {
        L.iter = it;
        enqueue_flex_phase(L, FLEX_PUPDATE);
        PS_CK(L.err);
        st = flex_inner(c, (const double *)P.desc.vec[ROLE_P], ph, irtol, imaxit, &inner_iters, &launches);
        if (st != PSOLVE_OK) return st;
        enqueue_flex_phase(L, FLEX_W);
        enqueue_flex_phase(L, FLEX_S);
        PS_CK(L.err);
        st = read();
        if (st != PSOLVE_OK) return st;
        if (hs->stop) break;
        if (!hs->half) {
            st = flex_inner(c, (const double *)P.desc.vec[ROLE_S], rh, irtol, imaxit, &inner_iters, &launches);
            if (st != PSOLVE_OK) return st;
            enqueue_flex_phase(L, FLEX_T);
        }
        enqueue_flex_phase(L, FLEX_UPDATE);
        PS_CK(L.err);
        st = read();
        if (st != PSOLVE_OK) return st;
    }
    launches += L.launches;
    if (hs->zero_x) PS_CK(cudaMemsetAsync(P.desc.vec[ROLE_X], 0, sizeof(double) * (size_t)P.nvec(), c->stream));
    if (tr) {
        Launcher T = ctx_launcher(c);
        T.iter = -1;
        enqueue_true_residual(T);
        launches += T.launches;
        PS_CK(T.err);
    }
    st = read();
    if (st != PSOLVE_OK) return st;
    Plan plan; // PSOLVE_PC_NONE; the byte model below replaces its figure
    psolve_result tmp;
    std::memset(&tmp, 0, sizeof tmp);
    fill_result(*hs, P, plan, use_x0, tr, t0, launches, &tmp);
    tmp.inner_iterations = inner_iters;
    {
        // algorithmic bytes of the outer phases (the inner solves excluded)
        std::vector<LaunchRec> recs;
        Launcher D;
        D.dry = true;
        D.npts = (double)P.npts();
        D.recs = &recs;
        D.iter = 0;
        enqueue_init(D, use_x0);
        for (int it = 1; it <= hs->iter; ++it) {
            D.iter = it;
            for (int ph = FLEX_PUPDATE; ph <= FLEX_UPDATE; ++ph) enqueue_flex_phase(D, ph);
        }
        if (tr) {
            D.iter = -1;
            enqueue_true_residual(D);
        }
        tmp.model_bytes = model_bytes_for(recs, hs->iter, hs->half_exit);
    }
    if (res) *res = tmp;
    return (psolve_status)hs->status;
}

// psolve_solve without the final copy of x: *bound is set once a context with
// a padded row pitch has staged b (and x) and runs on the copies.
static psolve_status solve_impl(psolve_ctx *c, const double *rhs, double *x, double rtol, int32_t maxit,
                                int32_t precond, int32_t degree, psolve_result *res, bool *bound)
{
    const double t0 = now_s();
    if (!c || !rhs || !x) {
        set_error("null argument");
        return PSOLVE_E_ARG;
    }
    psolve_status st = check_solve_args(rtol, maxit, precond, degree);
    if (st == PSOLVE_OK) st = check_blocks(c->P, precond);
    if (st != PSOLVE_OK) return st;
    if (c->opts.persistent && c->opts.timing) {
        set_error("timing mode times separate kernel launches; it cannot run with persistent = 1");
        return PSOLVE_E_ARG;
    }
    st = check_rr(c->opts.rr_every);
    if (st != PSOLVE_OK) return st;
    if (is_flexible(precond)) {
        st = check_flexible(c);
        if (st != PSOLVE_OK) return st;
    }
    PS_CK(cudaSetDevice(c->di.dev));
    Problem &P = c->P;
    st = problem_set_cheb(P, precond, degree, c->opts.lmin_scale, c->opts.lmax_scale);
    if (st != PSOLVE_OK) return st;
    const bool use_x0 = c->opts.use_x0 != 0;
    Desc &D = P.desc;
    D.hist = nullptr;
    D.hist_cap = 0;
    if (c->opts.record_history) {
        const int need = std::max(maxit, 1);
        if (need > c->hist_cap) {
            if (c->d_hist) cudaFree(c->d_hist);
            c->d_hist = nullptr;
            c->hist_cap = 0;
            cudaError_t e = cudaMalloc(&c->d_hist, sizeof(double) * 2 * (size_t)need);
            if (e != cudaSuccess) {
                set_error("residual history buffer: %s", cudaGetErrorString(e));
                return PSOLVE_E_OOM;
            }
            c->hist_cap = need;
        }
        // all-ones bytes are a NaN: entries a solve does not reach read as NaN
        PS_CK(cudaMemsetAsync(c->d_hist, 0xff, sizeof(double) * 2 * (size_t)c->hist_cap, c->stream));
        D.hist = c->d_hist;
        D.hist_cap = c->hist_cap;
    }
    c->solved = true;
    if (precond == PSOLVE_PC_GNOCOMM_CHEB) {
        // the paper's upper bound on useful GNoComm(CI) degrees: N_s / 2
        long long ns = P.n[0] / P.blocks[0];
        for (int d = 1; d < 3; ++d) ns = std::min<long long>(ns, P.n[d] / P.blocks[d]);
        if (2LL * degree > ns)
            set_error("warning: GNoComm(CI) degree %d exceeds half the smallest block side (%lld / 2): the "
                      "frozen block ghosts have reached every point after N_s/2 sweeps", degree, ns);
    }
    D.rtol = rtol;
    D.maxit = maxit;
    D.half_check = c->opts.half_step_check ? 1 : 0;
    D.rr_every = c->opts.rr_every;
    if (use_x0 && !P.have_rt) {
        set_error("use_x0 needs a context created with opts.use_x0 = 1");
        return PSOLVE_E_ARG;
    }
    if (P.staged()) { // the caller's rows of nx into the padded copies
        PS_CK(copy_to_pitched(P, P.d_bst, rhs, c->stream));
        if (use_x0) PS_CK(copy_to_pitched(P, P.d_xst, x, c->stream));
        rhs = P.d_bst;
        x = P.d_xst;
        *bound = true;
    }
    D.vec[ROLE_B] = (void *)rhs;
    D.vec[ROLE_X] = x;
    D.vec[ROLE_RT] = use_x0 ? P.desc.vec[ROLE_RT] : (void *)rhs;
    D.vec[ROLE_U] = D.vec[ROLE_V] = nullptr;
    st = upload_desc(c);
    if (st != PSOLVE_OK) return st;
    if (is_flexible(precond)) return flex_solve(c, precond, maxit, use_x0, c->opts.true_residual != 0, t0, res);

    Runner R;
    R.stream = c->stream;
    R.cap = c->cap;
    R.d_desc = c->d_desc;
    R.d_list = c->d_list;
    R.sms = c->di.sms;
    R.units = P.desc.units;
    R.plan.precond = precond;
    R.plan.degree = precond == PSOLVE_PC_NONE ? 0 : degree;
    R.plan.prec = precond == PSOLVE_PC_NONE ? PSOLVE_FP64 : P.prec;
    R.plan.exact_bounds = c->opts.lmin_scale == 1.0 && c->opts.lmax_scale == 1.0;
    R.plan.rr_every = c->opts.rr_every;
    R.plan.neumann = P.desc.bcm != 0;
    R.plan.split = sweep_split(R.plan.prec, P.desc.zc);
    R.plan.wide = wide_sweeps(R.plan, P.desc.tma != 0);
    R.use_graph = c->opts.use_graph != 0;
    R.timing = c->opts.timing != 0;
    R.npts = (double)P.npts();
    R.graphs = &c->graphs;
    R.events = &c->events;
    R.d_sc = P.d_sc;
    R.nsc = 1;
    R.h_sc[0] = c->h_sc;
    R.h_sc[1] = c->h_sc + 1;
    R.poll_ev[0] = c->poll_ev[0];
    R.poll_ev[1] = c->poll_ev[1];
    if (c->poll_K < 0 || !(c->poll_plan == R.plan)) {
        // the automatic poll period from one iteration's launches and bytes
        // (a dry run of the sequence); it depends on the plan alone
        std::vector<LaunchRec> recs;
        Launcher Dry;
        Dry.dry = true;
        Dry.npts = R.npts;
        Dry.recs = &recs;
        Dry.iter = 2;
        enqueue_iteration(Dry, R.plan);
        double b = 0;
        for (const LaunchRec &r : recs) b += r.bytes;
        c->poll_plan = R.plan;
        c->poll_K = auto_poll(b, (int)recs.size());
    }
    R.K = c->opts.poll_every > 0 ? c->opts.poll_every : c->poll_K;

    const bool tr = c->opts.true_residual != 0;
    if (c->opts.persistent) {
        st = run_persistent(c->stream, c->cap, R.plan, R.sms, R.units, c->d_desc, c->d_list, c->d_ps, c->h_ps,
                            maxit, use_x0, tr, R.use_graph, &c->pgraphs);
        if (st != PSOLVE_OK) return st;
        R.launches += 1;
        PS_CK(cudaMemcpyAsync(&c->h_ps->gs, &c->d_ps->gs, sizeof(GridSync), cudaMemcpyDeviceToHost, c->stream));
        PS_CK(cudaMemcpyAsync(c->h_sc + 2, P.d_sc, sizeof(Scal), cudaMemcpyDeviceToHost, c->stream));
        PS_CK(cudaStreamSynchronize(c->stream));
        if (c->h_ps->gs.err) {
            set_error("persistent solve: a %s wait gave up", c->h_ps->gs.err == 1 ? "grid barrier" : "tensor copy");
            return PSOLVE_TIMEOUT;
        }
        Scal s = c->h_sc[2];
        if (s.zero_x) {
            // b = 0 with an initial guess: x = 0, and the residual of the zeroed x
            PS_CK(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)P.nvec(), c->stream));
            if (tr) {
                Launcher T = R.launcher();
                T.iter = -1;
                enqueue_true_residual(T);
                R.launches += T.launches;
                PS_CK(T.err);
            }
            PS_CK(cudaMemcpyAsync(c->h_sc + 2, P.d_sc, sizeof(Scal), cudaMemcpyDeviceToHost, c->stream));
            PS_CK(cudaStreamSynchronize(c->stream));
            s = c->h_sc[2];
        }
        psolve_result tmp;
        std::memset(&tmp, 0, sizeof tmp);
        fill_result(s, P, R.plan, use_x0, tr, t0, R.launches, &tmp);
        if (res) *res = tmp;
        return (psolve_status)s.status;
    }

    Launcher L = R.launcher();
    L.iter = 0;
    enqueue_init(L, use_x0);
    R.launches += L.launches;
    PS_CK(L.err);
    st = run_loop(R, maxit);
    if (st != PSOLVE_OK) return st;
    Scal s = R.h_sc[R.last_slot][0];
    if (s.zero_x) PS_CK(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)P.nvec(), c->stream));
    if (tr) {
        Launcher T = R.launcher();
        T.iter = -1;
        enqueue_true_residual(T);
        R.launches += T.launches;
        PS_CK(T.err);
    }
    PS_CK(cudaMemcpyAsync(c->h_sc + 2, P.d_sc, sizeof(Scal), cudaMemcpyDeviceToHost, c->stream));
    PS_CK(cudaStreamSynchronize(c->stream));
    s = c->h_sc[2];
    psolve_result tmp;
    std::memset(&tmp, 0, sizeof tmp);
    if (R.timing) fill_timing(R.recs, s.iter, s.half_exit, &tmp);
    fill_result(s, P, R.plan, use_x0, tr, t0, R.launches, &tmp);
    if (res) *res = tmp;
    return (psolve_status)s.status;
}

psolve_status psolve_solve(psolve_ctx *c, const double *rhs, double *x, double rtol, int32_t maxit,
                           int32_t precond, int32_t degree, psolve_result *res)
{
    clear_error();
    Range range("psolve_solve");
    bool bound = false;
    const psolve_status st = solve_impl(c, rhs, x, rtol, maxit, precond, degree, res, &bound);
    if (bound) { // the solve ran on the padded copies: x back into the caller's rows
        cudaError_t e = copy_from_pitched(c->P, x, c->P.d_xst, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            set_error("copy of x from the padded layout: %s", cudaGetErrorString(e));
            return PSOLVE_E_CUDA;
        }
    }
    return st;
}

psolve_status psolve_history(psolve_ctx *c, int32_t capacity, double *rel_s, double *rel_r, int32_t *count)
{
    clear_error();
    if (!c || !count || capacity < 0) {
        set_error("bad argument");
        return PSOLVE_E_ARG;
    }
    if (!c->opts.record_history || !c->d_hist || !c->solved) {
        set_error("no residual history: create the context with opts.record_history = 1 and solve first");
        return PSOLVE_E_ARG;
    }
    PS_CK(cudaSetDevice(c->di.dev));
    Scal s;
    PS_CK(cudaMemcpyAsync(&s, c->P.d_sc, sizeof(Scal), cudaMemcpyDeviceToHost, c->stream));
    const int n = std::min(std::min((int)s.iter, c->hist_cap), (int)capacity);
    std::vector<double> raw(2 * (size_t)std::max(n, 1));
    if (n > 0)
        PS_CK(cudaMemcpyAsync(raw.data(), c->d_hist, sizeof(double) * 2 * (size_t)n, cudaMemcpyDeviceToHost,
                              c->stream));
    PS_CK(cudaStreamSynchronize(c->stream));
    // squared norms -> ||v|| / ||b||, the form Algorithm 1 tests
    const double nb = std::sqrt(s.nb2);
    for (int i = 0; i < n; ++i) {
        if (rel_s) rel_s[i] = std::sqrt(raw[2 * (size_t)i]) / nb;
        if (rel_r) rel_r[i] = std::sqrt(raw[2 * (size_t)i + 1]) / nb;
    }
    *count = s.iter;
    return PSOLVE_OK;
}

psolve_status psolve_solve_host(psolve_ctx *c, const double *rhs_host, double *x_host, double rtol,
                                int32_t maxit, int32_t precond, int32_t degree, psolve_result *res)
{
    clear_error();
    Range range("psolve_solve_host");
    const double t0 = now_s();
    if (!c || !rhs_host || !x_host) {
        set_error("null argument");
        return PSOLVE_E_ARG;
    }
    PS_CK(cudaSetDevice(c->di.dev));
    const size_t bytes = sizeof(double) * (size_t)c->P.npts();
    if (!c->d_hb) {
        cudaError_t e = cudaMalloc(&c->d_hb, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&c->d_hx, bytes);
        if (e != cudaSuccess) {
            set_error("device buffers for host solve: %s", cudaGetErrorString(e));
            return PSOLVE_E_OOM;
        }
    }
    PS_CK(cudaMemcpyAsync(c->d_hb, rhs_host, bytes, cudaMemcpyHostToDevice, c->stream));
    if (c->opts.use_x0) PS_CK(cudaMemcpyAsync(c->d_hx, x_host, bytes, cudaMemcpyHostToDevice, c->stream));
    psolve_result r;
    psolve_status st = psolve_solve(c, c->d_hb, c->d_hx, rtol, maxit, precond, degree, &r);
    if (st == PSOLVE_E_ARG || st == PSOLVE_E_CUDA || st == PSOLVE_E_OOM || st == PSOLVE_TIMEOUT) return st;
    PS_CK(cudaMemcpyAsync(x_host, c->d_hx, bytes, cudaMemcpyDeviceToHost, c->stream));
    PS_CK(cudaStreamSynchronize(c->stream));
    r.seconds = now_s() - t0;
    if (res) *res = r;
    return st;
}

psolve_status psolve_apply_A(psolve_ctx *c, const double *u, double *out, int32_t block_restricted)
{
    clear_error();
    Range range("psolve_apply_A");
    if (!c || !u || !out) {
        set_error("null argument");
        return PSOLVE_E_ARG;
    }
    if (block_restricted) {
        psolve_status st = check_blocks(c->P, PSOLVE_PC_BJ_CHEB);
        if (st != PSOLVE_OK) return st;
    }
    PS_CK(cudaSetDevice(c->di.dev));
    const Problem &P = c->P;
    if (P.staged()) { // padded rows: run on the staging copies
        PS_CK(copy_to_pitched(P, P.d_bst, u, c->stream));
        c->P.desc.vec[ROLE_U] = P.d_bst;
        c->P.desc.vec[ROLE_V] = P.d_xst;
    } else {
        c->P.desc.vec[ROLE_U] = (void *)u;
        c->P.desc.vec[ROLE_V] = out;
    }
    psolve_status st = upload_desc(c);
    if (st != PSOLVE_OK) return st;
    Launcher L = ctx_launcher(c);
    enqueue_apply_A(L, block_restricted != 0);
    PS_CK(L.err);
    if (P.staged()) PS_CK(copy_from_pitched(P, out, P.d_xst, c->stream));
    PS_CK(cudaStreamSynchronize(c->stream));
    return PSOLVE_OK;
}

psolve_status psolve_dot(psolve_ctx *c, const double *a, const double *b, double *result_host)
{
    clear_error();
    if (!c || !a || !b || !result_host) {
        set_error("null argument");
        return PSOLVE_E_ARG;
    }
    PS_CK(cudaSetDevice(c->di.dev));
    const Problem &P = c->P;
    if (P.staged()) { // padded rows: run on the staging copies
        PS_CK(copy_to_pitched(P, P.d_bst, a, c->stream));
        PS_CK(copy_to_pitched(P, P.d_xst, b, c->stream));
        a = P.d_bst;
        b = P.d_xst;
    }
    c->P.desc.vec[ROLE_U] = (void *)a;
    c->P.desc.vec[ROLE_V] = (void *)b;
    psolve_status st = upload_desc(c);
    if (st != PSOLVE_OK) return st;
    Launcher L = ctx_launcher(c);
    enqueue_dot(L);
    PS_CK(L.err);
    PS_CK(cudaMemcpyAsync(c->h_sc + 2, c->P.d_sc, sizeof(Scal), cudaMemcpyDeviceToHost, c->stream));
    PS_CK(cudaStreamSynchronize(c->stream));
    *result_host = c->h_sc[2].red[0];
    return PSOLVE_OK;
}

psolve_status psolve_precond_apply(psolve_ctx *c, const double *v, double *out, int32_t precond, int32_t degree)
{
    clear_error();
    Range range("psolve_precond_apply");
    if (!c || !v || !out) {
        set_error("null argument");
        return PSOLVE_E_ARG;
    }
    psolve_status st = check_solve_args(0.0, 0, precond, degree);
    if (st != PSOLVE_OK) return st;
    if (precond == PSOLVE_PC_NONE) {
        set_error("psolve_precond_apply needs a preconditioner");
        return PSOLVE_E_ARG;
    }
    st = check_blocks(c->P, precond);
    if (st != PSOLVE_OK) return st;
    PS_CK(cudaSetDevice(c->di.dev));
    if (is_flexible(precond)) {
        if (c->P.prec != PSOLVE_FP64) return check_flexible(c);
        if (v == out) {
            set_error("the inner solve of %s needs distinct v and out", precond == PSOLVE_PC_G_BICGS ? "G(BiCGS)" : "BJ(BiCGS)");
            return PSOLVE_E_ARG;
        }
        st = flex_setup(c, precond);
        if (st != PSOLVE_OK) return st;
        const Problem &Q = c->P;
        if (Q.staged()) PS_CK(copy_to_pitched(Q, Q.d_bst, v, c->stream));
        int64_t iters = 0, launches = 0;
        st = flex_inner(c, Q.staged() ? Q.d_bst : v, Q.staged() ? Q.d_xst : out, flex_rtol(c, precond),
                        flex_maxit(c), &iters, &launches);
        if (st != PSOLVE_OK) return st;
        if (Q.staged()) PS_CK(copy_from_pitched(Q, out, Q.d_xst, c->stream));
        PS_CK(cudaStreamSynchronize(c->stream));
        return PSOLVE_OK;
    }
    Problem &P = c->P;
    st = problem_set_cheb(P, precond, degree, c->opts.lmin_scale, c->opts.lmax_scale);
    if (st != PSOLVE_OK) return st;
    if (P.staged()) { // padded rows: run on the staging copies
        PS_CK(copy_to_pitched(P, P.d_bst, v, c->stream));
        v = P.d_bst;
    }
    double *const out_run = P.staged() ? P.d_xst : out;
    void *saved_r = P.desc.vec[ROLE_R];
    P.desc.vec[ROLE_R] = (void *)v;
    P.desc.vec[ROLE_V] = out_run;
    st = upload_desc(c);
    P.desc.vec[ROLE_R] = saved_r;
    if (st != PSOLVE_OK) return st;
    // first-iteration state: the direction update reads v as "r" and copies it
    // (this overwrites the last solve's scalars, and with them its history count)
    c->solved = false;
    Scal *init = c->h_sc + 2;
    std::memset(init, 0, sizeof(Scal));
    init->first = 1;
    PS_CK(cudaMemcpyAsync(P.d_sc, init, sizeof(Scal), cudaMemcpyHostToDevice, c->stream));
    Plan plan;
    plan.precond = precond;
    plan.degree = degree;
    plan.prec = P.prec;
    plan.exact_bounds = c->opts.lmin_scale == 1.0 && c->opts.lmax_scale == 1.0;
    plan.neumann = P.desc.bcm != 0;
    plan.split = sweep_split(plan.prec, P.desc.zc);
    plan.wide = wide_sweeps(plan, P.desc.tma != 0);
    Launcher L = ctx_launcher(c);
    enqueue_precond(L, plan);
    PS_CK(L.err);
    if (P.staged()) PS_CK(copy_from_pitched(P, out, P.d_xst, c->stream));
    PS_CK(cudaStreamSynchronize(c->stream));
    return PSOLVE_OK;
}

psolve_status psolve_cheb_interval(psolve_ctx *c, int32_t precond, double *a, double *b)
{
    clear_error();
    if (!c || !a || !b || precond < PSOLVE_PC_CHEB || precond > PSOLVE_PC_GNOCOMM_CHEB) {
        set_error("bad argument");
        return PSOLVE_E_ARG;
    }
    psolve_status st = check_blocks(c->P, precond);
    if (st != PSOLVE_OK) return st;
    return cheb_interval(c->P, precond, c->opts.lmin_scale, c->opts.lmax_scale, a, b);
}

// ==================================================================== batch
psolve_status psolve_solve_batch(int32_t count, const int64_t *grids, const double *h,
                                 const double *const *rhs, double *const *x, double rtol, int32_t maxit,
                                 int32_t precond, int32_t degree, const psolve_opts *opts, uintptr_t stream,
                                 psolve_result *results)
{
    Range range("psolve_solve_batch");
    clear_error();
    const double t0 = now_s();
    if (count < 1 || !grids || !h || !rhs || !x || !results) {
        set_error("bad argument");
        return PSOLVE_E_ARG;
    }
    psolve_status st = check_solve_args(rtol, maxit, precond, degree);
    if (st != PSOLVE_OK) return st;
    if (is_flexible(precond)) {
        set_error("batched solves take G(CI), BJ(CI), GNoComm(CI) or no preconditioner");
        return PSOLVE_E_ARG;
    }
    psolve_opts o;
    psolve_opts_default(&o);
    if (opts) o = *opts;
    if (o.use_x0) {
        set_error("batched solves start from x0 = 0");
        return PSOLVE_E_ARG;
    }
    if (o.cheb_prec < PSOLVE_FP64 || o.cheb_prec > PSOLVE_BF16) {
        set_error("unknown Chebyshev precision %d", o.cheb_prec);
        return PSOLVE_E_ARG;
    }
    if (o.slab_share < 0 || o.slab_share > 4096) {
        set_error("slab_share %d outside [0, 4096]", o.slab_share);
        return PSOLVE_E_ARG;
    }
    if (o.persistent && o.timing) {
        set_error("timing mode times separate kernel launches; it cannot run with persistent = 1");
        return PSOLVE_E_ARG;
    }
    st = check_rr(o.rr_every);
    if (st != PSOLVE_OK) return st;
    DevInfo di;
    st = device_info(&di);
    if (st != PSOLVE_OK) return st;

    std::vector<Problem> probs((size_t)count);
    size_t total_bytes = 0;
    std::vector<size_t> offs((size_t)count);
    long long total_units = 0;
    for (int q = 0; q < count; ++q) {
        Problem &P = probs[q];
        st = check_grid(grids + 3 * q);
        if (st != PSOLVE_OK) return st;
        if (!valid_h(h + 3 * q) || !rhs[q] || !x[q]) {
            set_error("problem %d: bad spacing or null vector", q);
            return PSOLVE_E_ARG;
        }
        for (int d = 0; d < 3; ++d) {
            P.n[d] = grids[3 * q + d];
            P.h[d] = h[3 * q + d];
            P.blocks[d] = o.blocks[d];
        }
        P.prec = o.cheb_prec;
        st = check_blocks(P, precond);
        if (st != PSOLVE_OK) return st;
        P.px = (o.engine != 1 && P.n[0] % 8 != 0) ? padded_pitch(P.n[0]) : 0; // as in psolve_create
        // the grids of a batch share every launch: deeper slabs than alone
        problem_geometry(P, di.sms, 0, o.slab_share > 0 ? o.slab_share : PSOLVE_SHARED_SLAB_SHARE);
        offs[q] = total_bytes;
        total_bytes += problem_bytes(P.n, P.prec, false, di.sms, P.px);
        total_units += P.desc.units;
    }
    if (total_units >= (1LL << 31)) {
        set_error("batch too large");
        return PSOLVE_E_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    char *mem = nullptr;
    Scal *d_sc = nullptr;
    Desc *d_desc = nullptr, *h_desc = nullptr;
    CUtensorMap *d_tmap = nullptr, *h_tmap = nullptr;
    int32_t *d_list = nullptr, *h_list = nullptr;
    Scal *h_sc = nullptr;
    PersistState *d_ps = nullptr, *h_ps = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    std::vector<GraphEntry> graphs;
    std::vector<cudaEvent_t> events;
    const size_t list_bytes = sizeof(int32_t) * (LIST_HDR_INTS + 2 * (size_t)count);
    auto cleanup = [&]() {
        if (s) cudaStreamSynchronize(s);
        for (GraphEntry &g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (cap) cudaStreamDestroy(cap);
        if (mem) cudaFree(mem);
        if (d_sc) cudaFree(d_sc);
        if (d_desc) cudaFree(d_desc);
        if (d_list) cudaFree(d_list);
        if (h_desc) cudaFreeHost(h_desc);
        if (d_tmap) cudaFree(d_tmap);
        if (h_tmap) cudaFreeHost(h_tmap);
        if (h_list) cudaFreeHost(h_list);
        if (h_sc) cudaFreeHost(h_sc);
        if (d_ps) cudaFree(d_ps);
        if (h_ps) cudaFreeHost(h_ps);
    };
#define BATCH_CK(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            set_error("%s: %s", #call, cudaGetErrorString(e_));                              \
            cleanup();                                                                       \
            return e_ == cudaErrorMemoryAllocation ? PSOLVE_E_OOM : PSOLVE_E_CUDA;           \
        }                                                                                    \
    } while (0)
    BATCH_CK(cudaMalloc(&mem, total_bytes));
    BATCH_CK(cudaMalloc(&d_sc, sizeof(Scal) * count));
    BATCH_CK(cudaMemsetAsync(d_sc, 0, sizeof(Scal) * count, s));
    BATCH_CK(cudaMalloc(&d_desc, sizeof(Desc) * count));
    BATCH_CK(cudaMalloc(&d_list, list_bytes));
    BATCH_CK(cudaHostAlloc(&h_desc, sizeof(Desc) * count, cudaHostAllocDefault));
    BATCH_CK(cudaMalloc(&d_tmap, sizeof(CUtensorMap) * TMAPS_PER_PROBLEM * count));
    BATCH_CK(cudaHostAlloc(&h_tmap, sizeof(CUtensorMap) * TMAPS_PER_PROBLEM * count, cudaHostAllocDefault));
    BATCH_CK(cudaHostAlloc(&h_list, list_bytes, cudaHostAllocDefault));
    BATCH_CK(cudaHostAlloc(&h_sc, 2 * sizeof(Scal) * count, cudaHostAllocDefault));
    if (o.persistent) {
        BATCH_CK(cudaMalloc(&d_ps, sizeof(PersistState)));
        BATCH_CK(cudaHostAlloc(&h_ps, sizeof(PersistState), cudaHostAllocDefault));
    }
    BATCH_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) BATCH_CK(cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming));
    h_list[0] = count;
    h_list[2] = h_list[3] = 0; // the list's work counters start at zero
    int32_t ub = 0;
    for (int q = 0; q < count; ++q) {
        Problem &P = probs[q];
        problem_bind(P, mem + offs[q]);
        bool tma_ok = true;
        if (o.autotune) {
            // per grid shape (cached), so a grid decomposes as it does alone
            TuneChoice tc;
            st = tune_problem(P, di.sms, s, &tc);
            if (st != PSOLVE_OK) {
                cleanup();
                return st;
            }
            problem_geometry(P, di.sms, tc.zc);
            tma_ok = tc.engine == 1;
            P.tuned = tc.from_cache ? 2 : 1;
        }
        P.desc.sc = d_sc + q;
        st = problem_set_cheb(P, precond, degree, o.lmin_scale, o.lmax_scale);
        if (st != PSOLVE_OK) {
            cleanup();
            return st;
        }
        P.desc.rtol = rtol;
        P.desc.maxit = maxit;
        P.desc.half_check = o.half_step_check ? 1 : 0;
        P.desc.rr_every = o.rr_every;
        const double *bq = rhs[q];
        double *xq = x[q];
        if (P.staged()) { // padded rows: the problem runs on its staging copies
            BATCH_CK(copy_to_pitched(P, P.d_bst, bq, s));
            bq = P.d_bst;
            xq = P.d_xst;
        }
        P.desc.vec[ROLE_B] = (void *)bq;
        P.desc.vec[ROLE_X] = xq;
        P.desc.vec[ROLE_RT] = (void *)bq;
        P.desc.tmap = d_tmap + (size_t)TMAPS_PER_PROBLEM * q;
        problem_encode_tmaps(P, h_tmap + (size_t)TMAPS_PER_PROBLEM * q, o.engine != 1 && tma_ok);
        h_desc[q] = P.desc;
        h_list[LIST_HDR_INTS + 2 * q] = q;
        h_list[LIST_HDR_INTS + 1 + 2 * q] = ub;
        if ((long long)ub + P.desc.units >= (1LL << 31)) {
            set_error("batch too large");
            cleanup();
            return PSOLVE_E_ARG;
        }
        ub += P.desc.units;
    }
    total_units = ub;
    h_list[1] = ub;
    BATCH_CK(cudaMemcpyAsync(d_tmap, h_tmap, sizeof(CUtensorMap) * TMAPS_PER_PROBLEM * count,
                             cudaMemcpyHostToDevice, s));
    BATCH_CK(cudaMemcpyAsync(d_desc, h_desc, sizeof(Desc) * count, cudaMemcpyHostToDevice, s));
    BATCH_CK(cudaMemcpyAsync(d_list, h_list, list_bytes, cudaMemcpyHostToDevice, s));

    Runner R;
    R.stream = s;
    R.cap = cap;
    R.d_desc = d_desc;
    R.d_list = d_list;
    R.sms = di.sms;
    R.units = total_units;
    R.plan.precond = precond;
    R.plan.degree = precond == PSOLVE_PC_NONE ? 0 : degree;
    R.plan.prec = precond == PSOLVE_PC_NONE ? PSOLVE_FP64 : o.cheb_prec;
    R.plan.exact_bounds = o.lmin_scale == 1.0 && o.lmax_scale == 1.0;
    R.plan.rr_every = o.rr_every;
    {
        int min_zc = 1 << 30;
        for (const Problem &P : probs) min_zc = std::min(min_zc, (int)P.desc.zc);
        R.plan.split = sweep_split(R.plan.prec, min_zc);
        bool all_tma = true;
        for (const Problem &P : probs) all_tma = all_tma && P.desc.tma != 0;
        R.plan.wide = wide_sweeps(R.plan, all_tma);
    }
    R.use_graph = o.use_graph != 0;
    R.timing = o.timing != 0;
    R.npts = 0;
    for (const Problem &P : probs) R.npts += (double)P.npts();
    R.graphs = &graphs;
    R.events = &events;
    R.d_sc = d_sc;
    R.nsc = count;
    R.h_sc[0] = h_sc;
    R.h_sc[1] = h_sc + count;
    R.poll_ev[0] = ev[0];
    R.poll_ev[1] = ev[1];
    R.K = o.poll_every > 0 ? o.poll_every : 4;

    const bool tr = o.true_residual != 0;
    if (o.persistent) {
        // every problem's whole solve in one cooperative launch
        st = run_persistent(s, cap, R.plan, R.sms, R.units, d_desc, d_list, d_ps, h_ps, maxit, false, tr,
                            R.use_graph, nullptr);
        if (st != PSOLVE_OK) {
            cleanup();
            return st;
        }
        R.launches += 1;
        BATCH_CK(cudaMemcpyAsync(&h_ps->gs, &d_ps->gs, sizeof(GridSync), cudaMemcpyDeviceToHost, s));
        BATCH_CK(cudaStreamSynchronize(s));
        if (h_ps->gs.err) {
            set_error("persistent batch: a %s wait gave up", h_ps->gs.err == 1 ? "grid barrier" : "tensor copy");
            cleanup();
            return PSOLVE_TIMEOUT;
        }
    } else {
        Launcher L = R.launcher();
        L.iter = 0;
        enqueue_init(L, false);
        R.launches += L.launches;
        BATCH_CK(L.err);
        st = run_loop(R, maxit);
        if (st != PSOLVE_OK) {
            cleanup();
            return st;
        }
        if (tr) {
            Launcher T = R.launcher();
            T.iter = -1;
            enqueue_true_residual(T);
            R.launches += T.launches;
            BATCH_CK(T.err);
        }
    }
    for (int q = 0; q < count; ++q)
        if (probs[q].staged()) BATCH_CK(copy_from_pitched(probs[q], x[q], probs[q].d_xst, s));
    BATCH_CK(cudaMemcpyAsync(h_sc, d_sc, sizeof(Scal) * count, cudaMemcpyDeviceToHost, s));
    BATCH_CK(cudaStreamSynchronize(s));
    psolve_status worst = PSOLVE_OK;
    for (int q = 0; q < count; ++q) {
        std::memset(&results[q], 0, sizeof(psolve_result));
        fill_result(h_sc[q], probs[q], R.plan, false, tr, t0, R.launches, &results[q]);
        if (h_sc[q].status != PSOLVE_OK && worst == PSOLVE_OK) worst = (psolve_status)h_sc[q].status;
    }
    if (R.timing) {
        psolve_result tm;
        std::memset(&tm, 0, sizeof tm);
        fill_timing(R.recs, 1 << 30, 0, &tm);
        for (int c = 0; c < PSOLVE_K_NCLASS; ++c) {
            results[0].kclass_ms[c] = tm.kclass_ms[c];
            results[0].kclass_launches[c] = tm.kclass_launches[c];
        }
    }
#undef BATCH_CK
    cleanup();
    return worst;
}

} // extern "C"
