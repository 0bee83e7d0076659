// psolve_selfcheck.cu -- psolve_selfcheck_conversions: compares the library's
// integer-pipe conversions (f2d_exact, d2f_rn in psolve_kernels.cuh) bit for
// bit with the GPU's own conversion instructions.
#include "psolve_engine.cuh"

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
        if (i & 1) bits = (bits & 0x800fffffffffffffull) | ((uint64_t)(897 + (z % 254)) << 52); // float range
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
