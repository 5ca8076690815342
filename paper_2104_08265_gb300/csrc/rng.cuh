// Counter-based random numbers shared by the rasterization (fluctuation) and the noise of
// Eq. 1: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller normals (Box and
// Muller 1958).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace wcsim {

// Philox4x32-10: 10 rounds of the multiply-xor bijection with a Weyl-sequence key schedule.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// sqrt(x) for x >= 0 from the hardware reciprocal square root (a few ulp, 0 at 0).
__device__ __forceinline__ float sqrt_fast(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

// Two standard normals from two Philox words: u = (x + 1/2) 2^-32,
// z0, z1 = sqrt(-2 ln u0) (cos, sin)(2 pi u1).  Hardware log2 / sin / cos (absolute error
// ~1e-6 in z); the angle is taken as 2 pi (u1 - 1/2) in [-pi, pi], where the hardware sine
// and cosine are accurate, and the half turn is undone by negating both.
__device__ __forceinline__ void box_muller2(uint32_t x0, uint32_t x1, float& z0, float& z1)
{
    const float sc = 2.3283064365386963e-10f, off = 1.1641532182693481e-10f;
    const float two_pi = 6.28318530717958648f, ln2x2 = -1.38629436111989061f;   // -2 ln 2
    const float u0 = fmaf((float)x0, sc, off), u1 = fmaf((float)x1, sc, off);
    const float r = sqrt_fast(ln2x2 * __log2f(u0));
    float sn, cs;
    __sincosf(two_pi * (u1 - 0.5f), &sn, &cs);
    z0 = -r * cs;
    z1 = -r * sn;
}

// Four standard normals from one Philox block: two Box-Muller pairs, (x.x, x.y) and
// (x.z, x.w).
__device__ __forceinline__ void box_muller4(uint4 x, float z[4])
{
    box_muller2(x.x, x.y, z[0], z[1]);
    box_muller2(x.z, x.w, z[2], z[3]);
}

// Counter tag of the noise stream (word 2 of the Philox counter; the fluctuation stream has
// a depo id there and is keyed by another seed).
constexpr uint32_t kNoiseTag = 0x4E4F4953u;

// The unit-mean-square complex Gaussian xi_w(k) of Eq. 1's noise: counter (k div 2, w, tag,
// plane id), key = noise seed; the block's first normal pair serves k = 2 (k div 2), the
// second k + 1; (z_re + i z_im) / sqrt 2, or z_re alone at k = 0 and at k = n / 2.
__device__ __forceinline__ float2 noise_xi(uint32_t w, int k, int n, uint32_t plane_id,
                                           uint64_t seed)
{
    const uint4 x = philox(make_uint4((uint32_t)(k >> 1), w, kNoiseTag, plane_id),
                           (uint32_t)seed, (uint32_t)(seed >> 32));
    float zr, zi;
    if (k & 1) box_muller2(x.z, x.w, zr, zi);
    else box_muller2(x.x, x.y, zr, zi);
    if (k == 0 || 2 * k == n) return make_float2(zr, 0.0f);
    const float h = 0.707106781186547524f;
    return make_float2(zr * h, zi * h);
}

}  // namespace wcsim
