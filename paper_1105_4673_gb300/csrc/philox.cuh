// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11), for host and device.
// Each round multiplies words 0 and 2 by the two Philox constants, keeps the
// low halves, and xors the high halves into words 1 and 3 together with the
// round key; the key is bumped by the golden-ratio Weyl increments between
// rounds.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define FSKMC_HD __host__ __device__ __forceinline__
#else
#define FSKMC_HD inline
#endif

namespace fskmc {

struct u32x4 {
    uint32_t x, y, z, w;
};

FSKMC_HD void mul_hilo(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo)
{
#if defined(__CUDA_ARCH__)
    lo = a * b;
    hi = __umulhi(a, b);
#else
    uint64_t p = (uint64_t)a * (uint64_t)b;
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
#endif
}

FSKMC_HD u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mul_hilo(0xD2511F53u, c.x, hi0, lo0);
        mul_hilo(0xCD9E8D57u, c.z, hi1, lo1);
        c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Counter layout of every draw in the library: (a, b, c, replica | tag<<24).
enum : uint32_t { TAG_EVENT = 0u, TAG_SSA = 1u, TAG_INIT = 2u, TAG_SCHED = 3u };

FSKMC_HD u32x4 draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    return philox4x32_10(u32x4{a, b, c, d}, (uint32_t)seed, (uint32_t)(seed >> 32));
}

}  // namespace fskmc
