// Counter-based random numbers for the thermal noise of Eq. b (Sec. 3.1.2):
// Philox4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11).  Counter (site m, time step n), key =
// the seed; every (m, n) gets its own four 32-bit outputs, so a site's noise
// does not depend on how the grid is tiled or on which kernel draws it.
#pragma once
#include <stdint.h>

namespace tdgl {

__host__ __device__ __forceinline__ void philox_mulhilo(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo)
{
#ifdef __CUDA_ARCH__
    hi = __umulhi(a, b);
    lo = a * b;
#else
    const uint64_t p = (uint64_t)a * b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
#endif
}

__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                       uint32_t k1, uint32_t out[4])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;   // Weyl sequence of the key
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0, lo0, hi1, lo1;
        philox_mulhilo(0xD2511F53u, c0, hi0, lo0);
        philox_mulhilo(0xCD9E8D57u, c2, hi1, lo1);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// (v1, v2), each uniform on [-1, 1): v = (x >> 8) 2^-23 - 1, exact in FP32.
__host__ __device__ __forceinline__ float2 noise_uv(unsigned long long seed, long long m, unsigned long long n)
{
    uint32_t x[4];
    philox4x32_10((uint32_t)m, (uint32_t)((unsigned long long)m >> 32), (uint32_t)n, (uint32_t)(n >> 32), (uint32_t)seed,
                  (uint32_t)(seed >> 32), x);
    return make_float2((float)(x[0] >> 8) * 1.1920928955078125e-07f - 1.f,
                       (float)(x[1] >> 8) * 1.1920928955078125e-07f - 1.f);
}

}  // namespace tdgl
