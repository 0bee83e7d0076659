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

namespace {

// FP64 instruction throughput: every thread runs FP64_CHAINS independent
// chains of `iters` dependent FP64 instructions (kind 0: fused multiply-add,
// kind 1: add), so the FP64 pipe, not latency, limits the loop.  Thread 0 of
// CTA 0 records the SM clock and the global timer around its loop, which
// gives the SM clock the run saw.  The chains' sum is stored only when it
// equals an impossible value, which keeps them live without a store per
// thread.
constexpr int FP64_CHAINS = 8;

template <int KIND>
__global__ void __launch_bounds__(256) k_fp64_rate(long long iters, double a, double c, double *sink,
                                                   long long *clk)
{
    double v[FP64_CHAINS];
#pragma unroll
    for (int q = 0; q < FP64_CHAINS; ++q) v[q] = 1e-3 * (double)(threadIdx.x + 8 * q + 1);
    long long c0 = 0, t0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c0 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    }
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < FP64_CHAINS; ++q) v[q] = KIND == 0 ? fma(v[q], a, c) : v[q] + c;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long t1;
        const long long c1 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        clk[0] = c1 - c0;
        clk[1] = t1 - t0;
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < FP64_CHAINS; ++q) s += v[q];
    if (s == -1.25e300) sink[0] = s;
}

} // namespace

extern "C" PSOLVE_API psolve_status psolve_measure_fp64_rate(int32_t kind, int64_t iters, uintptr_t stream,
                                                             double *instr_per_s, double *ms_out,
                                                             double *sm_mhz)
{
    clear_error();
    if (!instr_per_s || (kind != 0 && kind != 1) || iters < 1 || iters > (1LL << 24)) {
        set_error("bad argument");
        return PSOLVE_E_ARG;
    }
    DevInfo di;
    psolve_status st = device_info(&di);
    if (st != PSOLVE_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = 8 * di.sms; // 8 CTAs of 256 threads: every SM full
    double *d_sink = nullptr;
    long long *d_clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PS_CK(cudaMalloc(&d_sink, sizeof(double) + 2 * sizeof(long long)));
    d_clk = reinterpret_cast<long long *>(d_sink + 1);
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // the multiplier is below 1 and the addend small, so the chains stay finite
    const double a = 0.999999, c = 1e-7;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) { // the first run warms up
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            if (kind == 0) k_fp64_rate<0><<<grid, 256, 0, s>>>((long long)iters, a, c, d_sink, d_clk);
            else k_fp64_rate<1><<<grid, 256, 0, s>>>((long long)iters, a, c, d_sink, d_clk);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    long long clk[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(clk, d_clk, sizeof clk, cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_sink);
    if (e != cudaSuccess) {
        set_error("FP64 rate measurement: %s", cudaGetErrorString(e));
        return PSOLVE_E_CUDA;
    }
    const double instr = (double)grid * 256.0 * FP64_CHAINS * (double)iters;
    *instr_per_s = instr / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    if (sm_mhz) *sm_mhz = clk[1] > 0 ? (double)clk[0] / (double)clk[1] * 1e3 : 0.0;
    return PSOLVE_OK;
}
