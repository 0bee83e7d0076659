// psolve_selfcheck.cu -- psolve_selfcheck_conversions: compares the library's
// integer-pipe conversions (f2d_exact, d2f_rn in psolve_kernels.cuh) bit for
// bit with the GPU's own conversion instructions.
#include "psolve_persist_kernel.cuh"

using namespace psolve;

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_check_conversions(uint64_t seed, long long count, unsigned long long *bad)
{
    unsigned long long local = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const uint64_t z = mix64(seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull);
        // float -> double on every 32-bit pattern class (uniform bits)
        const float f = __uint_as_float((uint32_t)z);
        const double a = f2d_exact(f), b = (double)f;
        if (!(isnan(a) && isnan(b)) && __double_as_longlong(a) != __double_as_longlong(b)) ++local;
        // double -> float: uniform bits, and with the 29 dropped bits forced to
        // a tie (0x10000000) or one either side of it, on every fourth sample
        uint64_t bits = mix64(z);
        const int kind = (int)(z >> 62);
        if (kind == 1) bits = (bits & ~0x1fffffffull) | 0x10000000ull;
        if (kind == 2) bits = (bits & ~0x1fffffffull) | 0x0fffffffull;
        if (kind == 3) bits = (bits & ~0x1fffffffull) | 0x10000001ull;
        if ((i & 3) == 1) bits = (bits & 0x800fffffffffffffull) | ((uint64_t)(897 + (z % 254)) << 52); // normal
        if ((i & 3) == 3) { // results in or near the float subnormal range, with exact ties at the rounding bit
            const uint64_t e = 860 + (z % 40);  // 860..899
            bits = (bits & 0x800fffffffffffffull) | (e << 52);
            const int64_t sh = 926 - (int64_t)e;
            if (kind == 1 && sh >= 30 && sh <= 52)
                bits = (bits & ~((1ull << sh) - 1ull)) | (1ull << (sh - 1));
        }
        const double d = __longlong_as_double((long long)bits);
        const float x = d2f_rn(d), y = __double2float_rn(d);
        if (!(isnan(x) && isnan(y)) && __float_as_uint(x) != __float_as_uint(y)) ++local;
    }
    if (local) atomicAdd(bad, local);
}

} // namespace

extern "C" PSOLVE_API psolve_status psolve_selfcheck_conversions(uint64_t seed, int64_t count,
                                                                 int64_t *mismatches)
{
    clear_error();
    if (!mismatches || count < 0) {
        set_error("bad argument");
        return PSOLVE_E_ARG;
    }
    unsigned long long *d_bad = nullptr;
    PS_CK(cudaMalloc(&d_bad, sizeof *d_bad));
    cudaError_t e = cudaMemset(d_bad, 0, sizeof *d_bad);
    if (e == cudaSuccess) {
        k_check_conversions<<<1184, 256>>>(seed, (long long)count, d_bad);
        e = cudaGetLastError();
    }
    unsigned long long bad = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost);
    cudaFree(d_bad);
    if (e != cudaSuccess) {
        set_error("conversion self-check: %s", cudaGetErrorString(e));
        return PSOLVE_E_CUDA;
    }
    *mismatches = (int64_t)bad;
    return PSOLVE_OK;
}

namespace {

// One thread initialises an mbarrier that nothing will ever complete and waits
// on it with the bounded wait the TMA ring uses, here with a short limit.
__global__ void k_check_wait_timeout(long long limit, int *status)
{
    __shared__ alignas(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) *status = mbar_wait(&bar, 0, limit) ? PSOLVE_OK : PSOLVE_TIMEOUT;
}

} // namespace

extern "C" PSOLVE_API psolve_status psolve_selfcheck_wait_timeout(int64_t limit_cycles, int32_t *status)
{
    clear_error();
    if (!status || limit_cycles < 0 || limit_cycles > (1LL << 34)) {
        set_error("bad argument");
        return PSOLVE_E_ARG;
    }
    int *d = nullptr;
    PS_CK(cudaMalloc(&d, sizeof(int)));
    cudaError_t e = cudaMemset(d, 0xff, sizeof(int));
    if (e == cudaSuccess) {
        k_check_wait_timeout<<<1, 32>>>((long long)limit_cycles, d);
        e = cudaGetLastError();
    }
    int h = -1;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        set_error("wait self-check: %s", cudaGetErrorString(e));
        return PSOLVE_E_CUDA;
    }
    *status = h;
    return PSOLVE_OK;
}

namespace {

// Every CTA but `absent` meets at one grid barrier with a wait limit of
// limit_ns; CTA `absent` (or none, when absent < 0) never arrives.
__global__ void k_check_grid_timeout(GridSync *gs, int absent, unsigned long long limit_ns, int *passed,
                                     int *gave_up)
{
    __shared__ int s_flag;
    if ((int)blockIdx.x == absent) return;
    uint32_t target = 0;
    const bool ok = grid_sync(gs, target, &s_flag, limit_ns);
    if (threadIdx.x == 0) atomicAdd(ok ? passed : gave_up, 1);
}

} // namespace

extern "C" PSOLVE_API psolve_status psolve_selfcheck_grid_timeout(int64_t limit_ns, int32_t absent_cta,
                                                                  int32_t *ctas, int32_t *passed,
                                                                  int32_t *gave_up, int32_t *error_word)
{
    clear_error();
    if (!ctas || !passed || !gave_up || !error_word || limit_ns < 1000 || limit_ns > 2000000000LL) {
        set_error("bad argument");
        return PSOLVE_E_ARG;
    }
    DevInfo di;
    psolve_status st = device_info(&di);
    if (st != PSOLVE_OK) return st;
    const int grid = 2 * di.sms; // 2 small CTAs per SM: co-resident, and the launch is cooperative anyway
    if (absent_cta >= grid) {
        set_error("absent_cta %d outside the %d CTAs of the check", absent_cta, grid);
        return PSOLVE_E_ARG;
    }
    GridSync *d_gs = nullptr;
    int *d_cnt = nullptr;
    PS_CK(cudaMalloc(&d_gs, sizeof(GridSync)));
    cudaError_t e = cudaMalloc(&d_cnt, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d_gs, 0, sizeof(GridSync));
    if (e == cudaSuccess) e = cudaMemset(d_cnt, 0, 2 * sizeof(int));
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(32);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, k_check_grid_timeout, d_gs, (int)absent_cta, (unsigned long long)limit_ns,
                               d_cnt, d_cnt + 1);
    }
    int h[2] = {0, 0};
    GridSync g{};
    if (e == cudaSuccess) e = cudaMemcpy(h, d_cnt, sizeof h, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&g, d_gs, sizeof g, cudaMemcpyDeviceToHost);
    cudaFree(d_gs);
    if (d_cnt) cudaFree(d_cnt);
    if (e != cudaSuccess) {
        set_error("grid barrier self-check: %s", cudaGetErrorString(e));
        return PSOLVE_E_CUDA;
    }
    *ctas = grid;
    *passed = h[0];
    *gave_up = h[1];
    *error_word = g.err;
    return PSOLVE_OK;
}
