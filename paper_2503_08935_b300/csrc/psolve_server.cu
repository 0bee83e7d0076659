// psolve_server.cu -- continuous-batching server (not built yet in this
// revision: the entry points report PSOLVE_E_ARG).
#include "psolve_engine.cuh"

using namespace psolve;

struct psolve_server {
    int unused;
};

extern "C" {

psolve_status psolve_server_create(double, int32_t, int32_t, int32_t, int32_t, uintptr_t, psolve_server **out)
{
    if (out) *out = nullptr;
    set_error("the serving loop is not available in this build");
    return PSOLVE_E_ARG;
}

psolve_status psolve_submit(psolve_server *, const int64_t *, const double *, const double *, double *, double,
                            int32_t, const psolve_opts *, uint64_t *)
{
    set_error("the serving loop is not available in this build");
    return PSOLVE_E_ARG;
}

psolve_status psolve_poll(psolve_server *, uint64_t, psolve_result *)
{
    set_error("the serving loop is not available in this build");
    return PSOLVE_E_ARG;
}

void psolve_server_destroy(psolve_server *) {}

} // extern "C"
