// psolve_tune.cu -- autotuner for the slab depth (z planes per work unit) and
// the stencil engine (TMA ring or general) of one grid shape.
//
// For every candidate (slab depth 1, 2, 4, 8, 16, 32 planes, at most nz;
// TMA ring when the grid allows it, and the general engine) it times a probe
// of the solve's kernel kinds on the problem's own workspace: one Chebyshev
// sweep, one stencil with two dots and one update (a timed warm-up sizes the
// measurement to about 300 us of work, at least 3 repetitions; the best of two
// trials, CUDA events on the caller's stream), and keeps the fastest.  The choice depends on the grid shape, the Chebyshev precision and
// the GPU's SM count only, so a grid gets the same decomposition (hence the
// same reduction order and bitwise the same result) alone, in a batch or in
// a later process.
//
// Cache: every decision is kept for the life of the process and, when the
// environment variable PSOLVE_TUNE_CACHE names a file, appended to it as one
// text line "psolve-tune-1 sms nx ny nz prec zc engine us" (preceded by one
// "# candidate ..." comment line per measured candidate) and read back at the
// first tuning request of a later process (the first line for a key wins).
// Lines that do not parse are ignored.
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "psolve_tune.cuh"

namespace psolve {

namespace {

struct TuneKey {
    int sms, nx, ny, nz, prec;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(sms, nx, ny, nz, prec) < std::tie(o.sms, o.nx, o.ny, o.nz, o.prec);
    }
};

std::mutex g_mu;
std::map<TuneKey, TuneChoice> g_cache;
bool g_loaded = false;

const char *cache_path()
{
    const char *p = std::getenv("PSOLVE_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

void load_locked()
{
    if (g_loaded) return;
    g_loaded = true;
    const char *path = cache_path();
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[256];
    while (std::fgets(line, sizeof line, f)) {
        TuneKey k;
        TuneChoice c;
        if (std::sscanf(line, "psolve-tune-1 %d %d %d %d %d %d %d %lf", &k.sms, &k.nx, &k.ny, &k.nz, &k.prec,
                        &c.zc, &c.engine, &c.us) != 8)
            continue;
        if (c.zc < 1 || c.zc > k.nz || (c.engine != 0 && c.engine != 1)) continue;
        c.from_cache = 1;
        g_cache.emplace(k, c); // the first line for a key wins
    }
    std::fclose(f);
}

struct Candidate {
    int zc, engine;
    double us;
};

void append_locked(const TuneKey &k, const TuneChoice &c, const std::vector<Candidate> &all)
{
    const char *path = cache_path();
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    for (const Candidate &m : all) // every measurement, as comments
        std::fprintf(f, "# candidate %d %d %d %d %d %d %d %.3f\n", k.sms, k.nx, k.ny, k.nz, k.prec, m.zc, m.engine,
                     m.us);
    std::fprintf(f, "psolve-tune-1 %d %d %d %d %d %d %d %.3f\n", k.sms, k.nx, k.ny, k.nz, k.prec, c.zc, c.engine,
                 c.us);
    std::fclose(f);
}

// Time the probe for one candidate; *us < 0 when the candidate cannot run.
psolve_status time_candidate(Problem &P, int sms, int zc, bool tma, cudaStream_t s, Desc *d_desc,
                             int32_t *d_list, CUtensorMap *d_tmap, CUtensorMap *h_tmap, cudaEvent_t ev[2],
                             double *us)
{
    *us = -1.0;
    problem_geometry(P, sms, zc);
    Desc &D = P.desc;
    // every role the probe touches on workspace vectors (b, x and r~ are the
    // caller's or not yet bound)
    D.vec[ROLE_X] = D.vec[ROLE_P2];
    D.vec[ROLE_B] = D.vec[ROLE_P];
    D.vec[ROLE_RT] = D.vec[ROLE_W];
    D.vec[ROLE_U] = D.vec[ROLE_V] = nullptr;
    D.sc = P.d_sc;
    D.partials = P.d_partials;
    D.tmap = d_tmap;
    problem_encode_tmaps(P, h_tmap, tma);
    if (tma && !D.tma) return PSOLVE_OK; // this grid cannot use the TMA ring
    if (D.tma)
        PS_CK(cudaMemcpyAsync(d_tmap, h_tmap, sizeof(CUtensorMap) * TMAPS_PER_PROBLEM, cudaMemcpyHostToDevice, s));
    PS_CK(cudaMemcpyAsync(d_desc, &D, sizeof(Desc), cudaMemcpyHostToDevice, s));
    const int32_t list[LIST_HDR_INTS + 2] = {1, D.units, 0, 0, 0, 0};
    PS_CK(cudaMemcpyAsync(d_list, list, sizeof list, cudaMemcpyHostToDevice, s));
    PS_CK(cudaMemsetAsync(P.d_sc, 0, sizeof(Scal), s));
    Launcher L;
    L.stream = s;
    L.sms = sms;
    L.units = D.units;
    L.d_desc = d_desc;
    L.d_list = d_list;
    // warm-up, timed once to size the measurement: enough repetitions for
    // about 300 us of work, and the best of two trials
    PS_CK(cudaEventRecord(ev[0], s));
    enqueue_tune_probe(L, P.prec, false, sweep_split(P.prec, D.zc));
    PS_CK(cudaEventRecord(ev[1], s));
    PS_CK(L.err);
    PS_CK(cudaEventSynchronize(ev[1]));
    float ms = 0.f;
    PS_CK(cudaEventElapsedTime(&ms, ev[0], ev[1]));
    int reps = ms > 0.f ? (int)(0.3f / ms) + 1 : 3;
    reps = reps < 3 ? 3 : (reps > 64 ? 64 : reps);
    double best = -1.0;
    for (int trial = 0; trial < 2; ++trial) {
        PS_CK(cudaEventRecord(ev[0], s));
        for (int rep = 0; rep < reps; ++rep) enqueue_tune_probe(L, P.prec, false, sweep_split(P.prec, D.zc));
        PS_CK(cudaEventRecord(ev[1], s));
        PS_CK(L.err);
        PS_CK(cudaEventSynchronize(ev[1]));
        PS_CK(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        const double t = 1e3 * ms / reps;
        if (best < 0.0 || t < best) best = t;
    }
    *us = best;
    return PSOLVE_OK;
}

} // namespace

psolve_status tune_problem(const Problem &P0, int sms, cudaStream_t s, TuneChoice *out)
{
    const TuneKey key{sms, (int)P0.n[0], (int)P0.n[1], (int)P0.n[2], P0.prec};
    std::lock_guard<std::mutex> lock(g_mu);
    load_locked();
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *out = it->second;
        return PSOLVE_OK;
    }
    Problem P = P0; // the same workspace, re-described per candidate
    Desc *d_desc = nullptr;
    int32_t *d_list = nullptr;
    CUtensorMap *d_tmap = nullptr;
    std::vector<CUtensorMap> h_tmap(TMAPS_PER_PROBLEM);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    psolve_status st = PSOLVE_OK;
    TuneChoice best;
    best.us = -1.0;
    std::vector<Candidate> all;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && st == PSOLVE_OK) {
            set_error("autotuner: %s", cudaGetErrorString(e));
            st = PSOLVE_E_CUDA;
        }
        return st == PSOLVE_OK;
    };
    if (ck(cudaMalloc(&d_desc, sizeof(Desc))) && ck(cudaMalloc(&d_list, (LIST_HDR_INTS + 2) * sizeof(int32_t))) &&
        ck(cudaMalloc(&d_tmap, sizeof(CUtensorMap) * TMAPS_PER_PROBLEM)) && ck(cudaEventCreate(&ev[0])) &&
        ck(cudaEventCreate(&ev[1]))) {
        for (int engine = 1; engine >= 0 && st == PSOLVE_OK; --engine)
            for (int zc = 1; zc <= 32 && zc <= P.n[2] && st == PSOLVE_OK; zc *= 2) {
                double us = -1.0;
                st = time_candidate(P, sms, zc, engine == 1, s, d_desc, d_list, d_tmap, h_tmap.data(), ev, &us);
                if (st == PSOLVE_OK && us >= 0.0) all.push_back(Candidate{zc, engine, us});
                if (st == PSOLVE_OK && us >= 0.0 && (best.us < 0.0 || us < best.us)) {
                    best.zc = zc;
                    best.engine = engine;
                    best.us = us;
                }
            }
        ck(cudaStreamSynchronize(s));
    }
    if (d_desc) cudaFree(d_desc);
    if (d_list) cudaFree(d_list);
    if (d_tmap) cudaFree(d_tmap);
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    if (st != PSOLVE_OK) return st;
    best.from_cache = 0;
    g_cache.emplace(key, best);
    append_locked(key, best, all);
    *out = best;
    return PSOLVE_OK;
}

} // namespace psolve
