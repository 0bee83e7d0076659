// psolve_noalloc.cu -- psolve_dot_noalloc: the library's deterministic dot
// product for callers that must not allocate device memory.
//
// Who needs it: code that runs while another component owns all device
// memory (a framework's caching allocator or a serving process that reserved
// its HBM budget up front, where a stray cudaMalloc can fail or fragment the
// pool), and latency-critical host paths that cannot accept the device-wide
// synchronisation cudaMalloc/cudaFree may imply.  psolve_dot needs a context
// (psolve_create allocates its workspace); this entry point needs none.
//
// How: the same k_engine<OpDot> kernel as psolve_dot, with its descriptor,
// launch list, scalar block and per-unit partial sums placed in one
// file-scope __device__ array of NOALLOC_SCRATCH_BYTES bytes, which every GPU
// that loads the library keeps until the process exits.  In host code the
// array's name is only a host-side stand-in, so every call looks its device
// address up with cudaGetSymbolAddress on the current device (cheap once the
// module is loaded, and never stale after a device reset).  Every call also
// stages the descriptor from host stack memory and waits for its result, so
// no call can run inside a stream capture.  Every call shares the array: the
// scalar block (whose ticket must start at zero) is cleared on each call, and
// calls that overlap on the GPU (on different streams, or from several host
// threads) race on it.
#include "psolve_engine.cuh"

using namespace psolve;

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 4u << 20; // 4 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Scratch layout: [Desc][launch list][Scal][partials ...].
constexpr size_t OFF_DESC = 0;
constexpr size_t OFF_LIST = align256(sizeof(Desc));
constexpr size_t OFF_SCAL = OFF_LIST + align256((LIST_HDR_INTS + 2) * sizeof(int32_t));
constexpr size_t OFF_PART = OFF_SCAL + align256(sizeof(Scal));

// Device address of the scratch array on the current device.
psolve_status scratch_for_device(int dev, unsigned char **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        set_error("cudaGetSymbolAddress(scratch) on device %d: %s", dev, cudaGetErrorString(e));
        return PSOLVE_E_CUDA;
    }
    *out = static_cast<unsigned char *>(p);
    return PSOLVE_OK;
}

} // namespace

extern "C" PSOLVE_API psolve_status psolve_dot_noalloc(const int64_t grid[3], const double *a_dev,
                                                       const double *b_dev, uintptr_t stream,
                                                       double *result_host)
{
    clear_error();
    if (!grid || !a_dev || !b_dev || !result_host) {
        set_error("null argument");
        return PSOLVE_E_ARG;
    }
    long long n = 1;
    for (int d = 0; d < 3; ++d) {
        if (grid[d] < 1 || grid[d] > (1LL << 30)) {
            set_error("grid size %lld on axis %d out of range", (long long)grid[d], d);
            return PSOLVE_E_ARG;
        }
        n *= grid[d];
        if (n >= (1LL << 31)) {
            set_error("grid has 2^31 points or more");
            return PSOLVE_E_ARG;
        }
    }
    DevInfo di;
    psolve_status st = device_info(&di);
    if (st != PSOLVE_OK) return st;

    // The same unit decomposition as a context for this grid on this GPU
    // created without the autotuner (a tuned slab depth changes the units,
    // and with them the summation order).
    Problem P;
    for (int d = 0; d < 3; ++d) {
        P.n[d] = grid[d];
        P.h[d] = 1.0;
    }
    problem_geometry(P, di.sms);
    const size_t need = OFF_PART + (size_t)P.desc.units * MAX_DOTS * sizeof(double);
    if (need > NOALLOC_SCRATCH_BYTES) {
        set_error("grid of %lld points needs %zu bytes of scratch; psolve_dot_noalloc holds at most %zu "
                  "(use psolve_dot)", n, need, NOALLOC_SCRATCH_BYTES);
        return PSOLVE_E_ARG;
    }
    unsigned char *base = nullptr;
    st = scratch_for_device(di.dev, &base);
    if (st != PSOLVE_OK) return st;

    cudaStream_t s = (cudaStream_t)stream;
    Desc &D = P.desc;
    D.vec[ROLE_U] = (void *)a_dev;
    D.vec[ROLE_V] = (void *)b_dev;
    D.sc = reinterpret_cast<Scal *>(base + OFF_SCAL);
    D.partials = reinterpret_cast<double *>(base + OFF_PART);
    D.tma = 0;
    D.tmap = nullptr;
    const int32_t list[LIST_HDR_INTS + 2] = {1, D.units, 0, 0, 0, 0};
    // host staging is pageable (stack) memory; the copies complete before the
    // calls return, so the stack buffers may go out of scope afterwards
    PS_CK(cudaMemcpyAsync(base + OFF_DESC, &D, sizeof(Desc), cudaMemcpyHostToDevice, s));
    PS_CK(cudaMemcpyAsync(base + OFF_LIST, list, sizeof list, cudaMemcpyHostToDevice, s));
    PS_CK(cudaMemsetAsync(base + OFF_SCAL, 0, sizeof(Scal), s)); // the ticket starts at zero

    Launcher L;
    L.stream = s;
    L.sms = di.sms;
    L.units = D.units;
    L.d_desc = reinterpret_cast<const Desc *>(base + OFF_DESC);
    L.d_list = reinterpret_cast<const int32_t *>(base + OFF_LIST);
    enqueue_dot(L);
    PS_CK(L.err);
    double r = 0.0;
    PS_CK(cudaMemcpyAsync(&r, base + OFF_SCAL + offsetof(Scal, red), sizeof(double), cudaMemcpyDeviceToHost, s));
    PS_CK(cudaStreamSynchronize(s));
    *result_host = r;
    return PSOLVE_OK;
}
