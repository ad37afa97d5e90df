// Exhaustive check of the integer-pipe FP32 <-> FP64 conversions of the library against the
// hardware conversions (test infrastructure: built and run by tests/test_gpu_conversions.py).
//   f32_to_f64: every one of the 2^32 float bit patterns.
//   f64_to_f32: doubles around every float exponent (normal, subnormal, overflow), exact ties,
//               and random bit patterns.
// Prints the mismatch counts; exit status 0 when both are zero.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#include "gbmd_internal.cuh"

using gbmd::f32_to_f64;
using gbmd::f64_to_f32;

__device__ __forceinline__ bool same_double(double a, double b)
{
    return __double_as_longlong(a) == __double_as_longlong(b);
}

__global__ void k_f2d(uint64_t base, uint64_t count, unsigned long long* bad)
{
    unsigned long long local = 0;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += uint64_t(gridDim.x) * blockDim.x) {
        const float f = __uint_as_float(uint32_t(base + i));
        if (!same_double(double(f), f32_to_f64(f))) ++local;
    }
    if (local) atomicAdd(bad, local);
}

__device__ __forceinline__ uint64_t mix(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_d2f(uint64_t count, unsigned long long* bad)
{
    unsigned long long local = 0;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t r = mix(i);
        uint64_t bits;
        switch (i & 3u) {
        case 0:                          // exponent near the float range: normal, subnormal, overflow
            bits = (r & 0x800FFFFFFFFFFFFFull) | (uint64_t(860 + (r >> 52) % 320) << 52);
            break;
        case 1:                          // exact ties and one ulp around them at the subnormal/normal edge
            bits = (r & 0x800FFFFFE0000000ull) | 0x0000000010000000ull | (uint64_t(860 + (r >> 52) % 320) << 52);
            bits += (r >> 40) % 3 - 1;
            break;
        default:                         // any bit pattern (zeros, subnormals, NaN, inf included)
            bits = r;
        }
        const double x = __longlong_as_double((long long)bits);
        if (__float_as_uint(__double2float_rn(x)) != __float_as_uint(f64_to_f32(x))) ++local;
    }
    if (local) atomicAdd(bad, local);
}

int main()
{
    unsigned long long* bad;
    if (cudaMalloc(&bad, 2 * sizeof(unsigned long long)) != cudaSuccess) return 2;
    cudaMemset(bad, 0, 2 * sizeof(unsigned long long));
    k_f2d<<<4096, 256>>>(0ull, 1ull << 32, bad);
    k_d2f<<<4096, 256>>>(1ull << 28, bad + 1);
    unsigned long long h[2] = {0, 0};
    cudaMemcpy(h, bad, sizeof(h), cudaMemcpyDeviceToHost);
    const cudaError_t e = cudaGetLastError();
    printf("f32_to_f64 mismatches %llu of 4294967296; f64_to_f32 mismatches %llu of %llu; %s\n", h[0], h[1],
           1ull << 28, cudaGetErrorString(e));
    cudaFree(bad);
    return (e != cudaSuccess || h[0] || h[1]) ? 1 : 0;
}
