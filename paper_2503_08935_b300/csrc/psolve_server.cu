// psolve_server.cu -- continuous-batching server: many solves of different
// sizes share every kernel launch, requests join and leave at round
// boundaries.
//
// A host worker thread repeats rounds:
//   1. admit queued requests (FIFO) while a slot and a block of the device
//      memory pool are free; set up their descriptors and launch the
//      initial-residual kernel over the newcomers only;
//   2. for each launch group (the active requests that share a
//      preconditioner: precond, degree, Chebyshev precision), replay that
//      group's captured CUDA graph of `round_iters` outer iterations over
//      the group's device-side launch list (kernels skip a problem whose
//      `stop` flag is set, so problems finish independently);
//   3. copy the active problems' scalar blocks to pinned memory, and retire
//      the stopped ones: true residual, result record, memory back to the
//      pool, slot freed.
// The initial residual and the true residual do not depend on the
// preconditioner, so they run over mixed lists of every group.
// Each problem keeps its own unit decomposition and reduction order, so a
// served result is bitwise the one psolve_solve gives for the same problem
// and options, whatever else is in the mix.
//
// Requests' rhs/x live on the caller's side of the device; the server's
// kernels run on the server's stream, so the caller must make b ready on that
// stream (use the same stream, or synchronise) before psolve_submit.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "psolve_engine.cuh"

using namespace psolve;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device block, with coalescing of free ranges.
class Pool {
  public:
    void reset(size_t bytes)
    {
        free_.clear();
        free_[0] = bytes;
        used_ = 0;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

struct Request {
    uint64_t ticket = 0;
    int group = 0;               // launch group (the request's preconditioner)
    Problem prob;
    const double *rhs = nullptr; // caller's b (device)
    double *x = nullptr;         // caller's x (device)
    double rtol = 0;
    int maxit = 0;
    double lmin_scale = 1, lmax_scale = 1;
    int half_check = 1;
    double t_submit = 0, t_admit = 0;
    size_t bytes = 0, off = 0;
};

struct Active {
    bool used = false;
    Request req;
};

constexpr int MAX_GROUPS = 32; // distinct preconditioners per server

// The requests that share one preconditioner share every launch of a round:
// one device launch list and one captured graph per group, created by the
// worker thread when the group first has an active request.  Each
// preconditioner has two launch groups: requests on the TMA ring, whose FP32
// or BF16 G(CI) sweeps run two points per thread (wide_sweeps), and the rest.
struct Group {
    Plan plan;
    int32_t *d_list = nullptr;
    int32_t *h_list = nullptr; // pinned; a list of its own per group, so the
                               // uploads of one round never share a buffer
    cudaGraphExec_t graph = nullptr;
};

} // namespace

struct psolve_server {
    DevInfo di;
    cudaStream_t stream = 0, cap = 0;
    int max_slots = 0;
    std::vector<Plan> plans; // plans[g]: launch group g (guarded by mu)
    Group groups[2 * MAX_GROUPS]; // groups[2 g + tma]: preconditioner g, problems on the TMA ring or not
    double budget = 0;
    int round_iters = 2;
    char *pool_mem = nullptr;
    size_t pool_bytes = 0;
    Pool pool;
    // device state for all slots
    Desc *d_desc = nullptr, *h_desc = nullptr;
    Scal *d_sc = nullptr, *h_sc = nullptr;
    CUtensorMap *d_tmap = nullptr, *h_tmap = nullptr;
    int32_t *d_list_new = nullptr, *d_list_fin = nullptr;
    int32_t *h_lists = nullptr; // two pinned lists back to back (new, finished)
    cudaEvent_t ev = nullptr;
    // requests
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, psolve_result> done;
    std::unordered_map<uint64_t, int> state; // 0 queued, 1 running, 2 done
    uint64_t next_ticket = 1;
    std::vector<Active> slots;
    std::atomic<bool> stop{false};
    bool failed = false;
    std::string fail_msg;
    std::thread worker;
};

namespace {

// Lists are [n, total, next, done, (slot, first unit) x n]; capacity
// max_slots entries.  Pinned host copies: a group's own, or h_lists for the
// newcomers' (which = 1) and finished requests' (which = 2) lists.
size_t list_bytes(int n) { return sizeof(int32_t) * (LIST_HDR_INTS + 2 * (size_t)n); }

cudaError_t upload_list(psolve_server *s, int32_t *h, int32_t *d, const std::vector<int> &slots)
{
    h[0] = (int32_t)slots.size();
    h[2] = h[3] = 0; // the list's work counters start at zero
    int32_t ub = 0;
    for (size_t q = 0; q < slots.size(); ++q) {
        h[LIST_HDR_INTS + 2 * q] = slots[q];
        h[LIST_HDR_INTS + 1 + 2 * q] = ub;
        ub += s->slots[slots[q]].req.prob.desc.units;
    }
    h[1] = ub;
    return cudaMemcpyAsync(d, h, list_bytes((int)slots.size()), cudaMemcpyHostToDevice, s->stream);
}

cudaError_t upload_list(psolve_server *s, int which, const std::vector<int> &slots)
{
    int32_t *h = s->h_lists + (size_t)(which - 1) * (LIST_HDR_INTS + 2 * s->max_slots);
    return upload_list(s, h, which == 1 ? s->d_list_new : s->d_list_fin, slots);
}

Launcher server_launcher(psolve_server *s, const int32_t *d_list)
{
    Launcher L;
    L.stream = s->stream;
    L.sms = s->di.sms;
    L.units = 1LL << 30; // the active set changes: size grids for a full device
    L.d_desc = s->d_desc;
    L.d_list = d_list;
    return L;
}

// The launch group of an admitted request (its descriptor's TMA flag is set
// at admission and kept).
int launch_group(const Request &r) { return 2 * r.group + (r.prob.desc.tma ? 1 : 0); }

// Device list, pinned list and captured round graph of launch group gi
// (worker thread, on first use).
cudaError_t ensure_group(psolve_server *s, int gi)
{
    Group &G = s->groups[gi];
    if (G.graph) return cudaSuccess;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        G.plan = s->plans[gi / 2];
    }
    G.plan.wide = wide_sweeps(G.plan, (gi & 1) != 0);
    cudaError_t e;
    if (!G.d_list && (e = cudaMalloc(&G.d_list, list_bytes(s->max_slots))) != cudaSuccess) return e;
    if (!G.h_list && (e = cudaHostAlloc(&G.h_list, list_bytes(s->max_slots), cudaHostAllocDefault)) != cudaSuccess)
        return e;
    Launcher C = server_launcher(s, G.d_list);
    C.stream = s->cap;
    C.iter = 2;
    Launcher cfg = C;
    cfg.configure = true;
    enqueue_iteration(cfg, G.plan);
    enqueue_init(cfg, false);
    enqueue_true_residual(cfg);
    if (cfg.err != cudaSuccess) return cfg.err;
    e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int j = 0; j < s->round_iters; ++j) enqueue_iteration(C, G.plan);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s->cap, &g);
    if (C.err != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return C.err != cudaSuccess ? C.err : e;
    }
    e = cudaGraphInstantiate(&G.graph, g, 0);
    cudaGraphDestroy(g);
    return e;
}

void finish(psolve_server *s, const Request &r, const Scal &sc, double t, const Plan &plan)
{
    psolve_result res;
    std::memset(&res, 0, sizeof res);
    res.status = sc.status;
    res.iterations = sc.iter;
    res.half_step_exit = sc.half_exit;
    res.engine = r.prob.desc.tma;
    res.slab_planes = r.prob.desc.zc;
    res.rel_res_recursive = sc.nb2 > 0 ? std::sqrt(sc.rr / sc.nb2) : 0.0;
    res.rel_res_true = sc.nb2 > 0 ? std::sqrt(sc.true_rr / sc.nb2) : 0.0;
    res.seconds = t - r.t_submit; // latency: submit -> result ready
    // algorithmic bytes of this request's work
    std::vector<LaunchRec> recs;
    Launcher D;
    D.dry = true;
    D.npts = (double)r.prob.npts();
    D.recs = &recs;
    enqueue_init(D, false);
    for (int it = 1; it <= sc.iter; ++it) {
        D.iter = it;
        enqueue_iteration(D, plan);
    }
    D.iter = -1;
    enqueue_true_residual(D);
    res.model_bytes = model_bytes_for(recs, sc.iter, sc.half_exit);
    std::lock_guard<std::mutex> lock(s->mu);
    s->done[r.ticket] = res;
    s->state[r.ticket] = 2;
}

void fail_all(psolve_server *s, int status, const char *msg)
{
    std::lock_guard<std::mutex> lock(s->mu);
    s->failed = true;
    s->fail_msg = msg;
    auto mark = [&](uint64_t t) {
        psolve_result res;
        std::memset(&res, 0, sizeof res);
        res.status = status;
        s->done[t] = res;
        s->state[t] = 2;
    };
    for (Active &a : s->slots)
        if (a.used) {
            mark(a.req.ticket);
            a.used = false;
        }
    for (Request &r : s->queue) mark(r.ticket);
    s->queue.clear();
}

#define W_CK(call)                                                                  \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            char m_[256];                                                           \
            snprintf(m_, sizeof m_, "%s: %s", #call, cudaGetErrorString(e_));       \
            fail_all(s, PSOLVE_E_CUDA, m_);                                         \
            return;                                                                 \
        }                                                                           \
    } while (0)

void worker_main(psolve_server *s)
{
    cudaSetDevice(s->di.dev);
    std::vector<int> active, fresh, fin;
    std::vector<int> by_group[2 * MAX_GROUPS];
    for (;;) {
        // ---- admission
        fresh.clear();
        {
            std::unique_lock<std::mutex> lock(s->mu);
            bool any_active = false;
            for (const Active &a : s->slots) any_active |= a.used;
            if (!any_active && s->queue.empty() && !s->stop)
                s->cv.wait_for(lock, std::chrono::milliseconds(50));
            if (s->stop) break;
            while (!s->queue.empty()) {
                int slot = -1;
                for (int q = 0; q < s->max_slots; ++q)
                    if (!s->slots[q].used) {
                        slot = q;
                        break;
                    }
                if (slot < 0) break;
                Request &r = s->queue.front();
                size_t off = 0;
                if (!s->pool.alloc(r.bytes, &off)) {
                    if (s->pool.used() == 0) { // cannot fit even in an empty pool
                        psolve_result res;
                        std::memset(&res, 0, sizeof res);
                        res.status = PSOLVE_REJECTED;
                        s->done[r.ticket] = res;
                        s->state[r.ticket] = 2;
                        s->queue.pop_front();
                        continue;
                    }
                    break; // wait for memory to free up (FIFO)
                }
                r.off = off;
                r.t_admit = now_s();
                s->state[r.ticket] = 1;
                s->slots[slot].used = true;
                s->slots[slot].req = r;
                s->queue.pop_front();
                fresh.push_back(slot);
            }
        }
        for (int slot : fresh) {
            Request &r = s->slots[slot].req;
            Problem &P = r.prob;
            problem_bind(P, s->pool_mem + r.off); // lays out the workspace; clears every role pointer
            const double *bq = r.rhs;
            double *xq = r.x;
            if (P.staged()) { // padded rows: the request runs on its staging copies
                W_CK(copy_to_pitched(P, P.d_bst, bq, s->stream));
                bq = P.d_bst;
                xq = P.d_xst;
            }
            P.desc.vec[ROLE_B] = (void *)bq;
            P.desc.vec[ROLE_X] = xq;
            P.desc.vec[ROLE_RT] = (void *)bq; // x0 = 0: r~ = r0 = b
            P.desc.sc = s->d_sc + slot;
            P.desc.tmap = s->d_tmap + (size_t)TMAPS_PER_PROBLEM * slot;
            Plan plan;
            {
                std::lock_guard<std::mutex> lock(s->mu);
                plan = s->plans[r.group];
            }
            if (problem_set_cheb(P, plan.precond, plan.degree, r.lmin_scale, r.lmax_scale) != PSOLVE_OK) {
                Scal sc{};
                sc.status = PSOLVE_E_ARG;
                sc.stop = 1;
                finish(s, r, sc, now_s(), plan);
                s->pool.release(r.off, r.bytes);
                s->slots[slot].used = false;
                continue;
            }
            problem_encode_tmaps(P, s->h_tmap + (size_t)TMAPS_PER_PROBLEM * slot, true);
            s->h_desc[slot] = P.desc;
            W_CK(cudaMemcpyAsync(s->d_tmap + (size_t)TMAPS_PER_PROBLEM * slot,
                                 s->h_tmap + (size_t)TMAPS_PER_PROBLEM * slot,
                                 sizeof(CUtensorMap) * TMAPS_PER_PROBLEM, cudaMemcpyHostToDevice, s->stream));
            W_CK(cudaMemcpyAsync(s->d_desc + slot, s->h_desc + slot, sizeof(Desc), cudaMemcpyHostToDevice,
                                 s->stream));
            W_CK(cudaMemsetAsync(s->d_sc + slot, 0, sizeof(Scal), s->stream));
        }
        fresh.erase(std::remove_if(fresh.begin(), fresh.end(), [&](int q) { return !s->slots[q].used; }),
                    fresh.end());
        if (!fresh.empty()) {
            W_CK(upload_list(s, 1, fresh));
            Launcher L = server_launcher(s, s->d_list_new);
            enqueue_init(L, false);
            W_CK(L.err);
        }
        active.clear();
        for (int q = 0; q < s->max_slots; ++q)
            if (s->slots[q].used) active.push_back(q);
        if (active.empty()) continue;

        // ---- one round over every active problem, group by group
        Range range("psolve_server round");
        for (auto &v : by_group) v.clear();
        for (int q : active) by_group[launch_group(s->slots[q].req)].push_back(q);
        for (int gi = 0; gi < 2 * MAX_GROUPS; ++gi) {
            if (by_group[gi].empty()) continue;
            W_CK(ensure_group(s, gi));
            Group &G = s->groups[gi];
            W_CK(upload_list(s, G.h_list, G.d_list, by_group[gi]));
            W_CK(cudaGraphLaunch(G.graph, s->stream));
        }
        W_CK(cudaMemcpyAsync(s->h_sc, s->d_sc, sizeof(Scal) * s->max_slots, cudaMemcpyDeviceToHost, s->stream));
        W_CK(cudaEventRecord(s->ev, s->stream));
        W_CK(cudaEventSynchronize(s->ev));

        // ---- retire the stopped ones (true residual first)
        fin.clear();
        for (int q : active)
            if (s->h_sc[q].stop) fin.push_back(q);
        if (fin.empty()) continue;
        W_CK(upload_list(s, 2, fin));
        Launcher T = server_launcher(s, s->d_list_fin);
        enqueue_true_residual(T);
        W_CK(T.err);
        for (int q : fin) {
            const Request &r = s->slots[q].req;
            if (r.prob.staged()) W_CK(copy_from_pitched(r.prob, r.x, r.prob.d_xst, s->stream));
        }
        W_CK(cudaMemcpyAsync(s->h_sc, s->d_sc, sizeof(Scal) * s->max_slots, cudaMemcpyDeviceToHost, s->stream));
        W_CK(cudaEventRecord(s->ev, s->stream));
        W_CK(cudaEventSynchronize(s->ev));
        const double t = now_s();
        for (int q : fin) {
            Active &a = s->slots[q];
            const Scal sc = s->h_sc[q];
            finish(s, a.req, sc, t, s->groups[launch_group(a.req)].plan);
            {
                std::lock_guard<std::mutex> lock(s->mu);
                s->pool.release(a.req.off, a.req.bytes);
                a.used = false;
            }
        }
        s->cv.notify_all();
    }
    // shutting down: whatever is still queued or running ends with TIMEOUT
    cudaStreamSynchronize(s->stream);
    fail_all(s, PSOLVE_TIMEOUT, "server destroyed before the request finished");
}

} // namespace

extern "C" {

psolve_status psolve_server_create(double hbm_budget_bytes, int32_t max_slots, uintptr_t stream, psolve_server **out)
{
    clear_error();
    if (!out || !(hbm_budget_bytes > 0) || max_slots < 1 || max_slots > 4096) {
        set_error("bad server argument");
        return PSOLVE_E_ARG;
    }
    psolve_server *s = new psolve_server();
    psolve_status st = device_info(&s->di);
    if (st != PSOLVE_OK) {
        delete s;
        return st;
    }
    s->stream = (cudaStream_t)stream;
    s->max_slots = max_slots;
    s->budget = hbm_budget_bytes;
    s->pool_bytes = (size_t)hbm_budget_bytes;
    s->slots.resize(max_slots);
    auto bail = [&](cudaError_t e) {
        set_error("server set-up: %s", cudaGetErrorString(e));
        psolve_server_destroy(s);
        return e == cudaErrorMemoryAllocation ? PSOLVE_E_OOM : PSOLVE_E_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&s->pool_mem, s->pool_bytes)) != cudaSuccess) return bail(e);
    s->pool.reset(s->pool_bytes);
    if ((e = cudaMalloc(&s->d_desc, sizeof(Desc) * max_slots)) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&s->d_sc, sizeof(Scal) * max_slots)) != cudaSuccess) return bail(e);
    if ((e = cudaMemset(s->d_sc, 0, sizeof(Scal) * max_slots)) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&s->d_tmap, sizeof(CUtensorMap) * TMAPS_PER_PROBLEM * max_slots)) != cudaSuccess)
        return bail(e);
    if ((e = cudaMalloc(&s->d_list_new, list_bytes(max_slots))) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&s->d_list_fin, list_bytes(max_slots))) != cudaSuccess) return bail(e);
    if ((e = cudaHostAlloc(&s->h_desc, sizeof(Desc) * max_slots, cudaHostAllocDefault)) != cudaSuccess)
        return bail(e);
    if ((e = cudaHostAlloc(&s->h_sc, sizeof(Scal) * max_slots, cudaHostAllocDefault)) != cudaSuccess)
        return bail(e);
    if ((e = cudaHostAlloc(&s->h_tmap, sizeof(CUtensorMap) * TMAPS_PER_PROBLEM * max_slots,
                           cudaHostAllocDefault)) != cudaSuccess)
        return bail(e);
    if ((e = cudaHostAlloc(&s->h_lists, 2 * list_bytes(max_slots), cudaHostAllocDefault)) != cudaSuccess)
        return bail(e);
    if ((e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
    if ((e = cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming)) != cudaSuccess) return bail(e);
    s->worker = std::thread(worker_main, s);
    *out = s;
    return PSOLVE_OK;
}

psolve_status psolve_submit(psolve_server *s, const int64_t grid[3], const double h[3], const double *rhs_dev,
                            double *x_dev, double rtol, int32_t maxit, int32_t precond, int32_t degree,
                            const psolve_opts *opts, uint64_t *ticket)
{
    clear_error();
    if (!s || !grid || !h || !rhs_dev || !x_dev || !ticket || !(rtol >= 0.0) || !std::isfinite(rtol) || maxit < 0) {
        set_error("bad argument");
        return PSOLVE_E_ARG;
    }
    if (precond < PSOLVE_PC_NONE || precond > PSOLVE_PC_GNOCOMM_CHEB || degree < 0 || degree > MAX_DEGREE) {
        set_error("served requests take PSOLVE_PC_NONE or a Chebyshev form with degree in [0, %d]", MAX_DEGREE);
        return PSOLVE_E_ARG;
    }
    long long n = 1;
    for (int d = 0; d < 3; ++d) {
        if (grid[d] < 1 || grid[d] > (1LL << 30) || !(h[d] > 0.0) || !std::isfinite(h[d])) {
            set_error("bad grid or spacing on axis %d", d);
            return PSOLVE_E_ARG;
        }
        n *= grid[d];
        if (n >= (1LL << 31)) {
            set_error("grid has 2^31 points or more");
            return PSOLVE_E_ARG;
        }
    }
    psolve_opts o;
    psolve_opts_default(&o);
    if (opts) o = *opts;
    if (o.lmin_scale != 1.0 || o.lmax_scale != 1.0) {
        set_error("served requests use the exact closed-form Chebyshev bounds (scales 1, 1)");
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
    Plan plan;
    plan.precond = precond;
    plan.degree = precond == PSOLVE_PC_NONE ? 0 : degree;
    plan.prec = precond == PSOLVE_PC_NONE ? PSOLVE_FP64 : o.cheb_prec;
    plan.exact_bounds = true; // scales 1, 1 (checked above)
    Request r;
    Problem &P = r.prob;
    for (int d = 0; d < 3; ++d) {
        P.n[d] = grid[d];
        P.h[d] = h[d];
        P.blocks[d] = o.blocks[d];
        if (o.blocks[d] < 1 || (precond >= PSOLVE_PC_BJ_CHEB && grid[d] % o.blocks[d] != 0)) {
            set_error("blocks[%d] = %d does not divide the grid", d, o.blocks[d]);
            return PSOLVE_E_ARG;
        }
    }
    P.prec = plan.prec;
    P.have_rt = false;
    // rows padded to a multiple of 8 elements when nx is not one, so that every
    // request runs on the tensor copies (b is staged at admission, x copied back
    // when the request retires)
    P.px = P.n[0] % 8 != 0 ? padded_pitch(P.n[0]) : 0;
    // deeper slabs than for a grid alone: the request shares its launches
    // with the other admitted ones (PSOLVE_SHARED_SLAB_SHARE unless asked)
    problem_geometry(P, s->di.sms, 0, o.slab_share > 0 ? o.slab_share : PSOLVE_SHARED_SLAB_SHARE);
    P.desc.rtol = rtol;
    P.desc.maxit = maxit;
    P.desc.half_check = o.half_step_check ? 1 : 0;
    r.rhs = rhs_dev;
    r.x = x_dev;
    r.rtol = rtol;
    r.maxit = maxit;
    r.lmin_scale = o.lmin_scale;
    r.lmax_scale = o.lmax_scale;
    r.bytes = problem_bytes(P.n, P.prec, false, s->di.sms, P.px);
    if ((double)r.bytes > s->budget) {
        set_error("request needs %zu bytes; the server's budget is %.0f", r.bytes, s->budget);
        return PSOLVE_REJECTED;
    }
    {
        double a, b;
        if (precond != PSOLVE_PC_NONE && cheb_interval(P, precond, o.lmin_scale, o.lmax_scale, &a, &b) != PSOLVE_OK)
            return PSOLVE_E_ARG;
    }
    r.t_submit = now_s();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->failed) {
            set_error("server failed: %s", s->fail_msg.c_str());
            return PSOLVE_E_CUDA;
        }
        int gi = -1;
        for (size_t q = 0; q < s->plans.size(); ++q)
            if (s->plans[q] == plan) gi = (int)q;
        if (gi < 0) {
            if ((int)s->plans.size() >= MAX_GROUPS) {
                set_error("the server already serves %d distinct preconditioners", MAX_GROUPS);
                return PSOLVE_E_ARG;
            }
            gi = (int)s->plans.size();
            s->plans.push_back(plan);
        }
        r.group = gi;
        r.ticket = s->next_ticket++;
        s->state[r.ticket] = 0;
        s->queue.push_back(r);
        *ticket = r.ticket;
    }
    s->cv.notify_all();
    return PSOLVE_OK;
}

psolve_status psolve_poll(psolve_server *s, uint64_t ticket, psolve_result *res)
{
    if (!s) {
        set_error("null server");
        return PSOLVE_E_ARG;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->state.find(ticket);
    if (it == s->state.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return PSOLVE_E_ARG;
    }
    if (it->second != 2) return PSOLVE_PENDING;
    psolve_result r = s->done[ticket];
    s->done.erase(ticket);
    s->state.erase(it);
    if (res) *res = r;
    return (psolve_status)r.status;
}

void psolve_server_destroy(psolve_server *s)
{
    if (!s) return;
    s->stop = true;
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->di.dev);
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (Group &G : s->groups) {
        if (G.graph) cudaGraphExecDestroy(G.graph);
        cudaFree(G.d_list);
        if (G.h_list) cudaFreeHost(G.h_list);
    }
    if (s->ev) cudaEventDestroy(s->ev);
    if (s->cap) cudaStreamDestroy(s->cap);
    cudaFree(s->pool_mem);
    cudaFree(s->d_desc);
    cudaFree(s->d_sc);
    cudaFree(s->d_tmap);
    cudaFree(s->d_list_new);
    cudaFree(s->d_list_fin);
    if (s->h_desc) cudaFreeHost(s->h_desc);
    if (s->h_sc) cudaFreeHost(s->h_sc);
    if (s->h_tmap) cudaFreeHost(s->h_tmap);
    if (s->h_lists) cudaFreeHost(s->h_lists);
    delete s;
}

} // extern "C"
