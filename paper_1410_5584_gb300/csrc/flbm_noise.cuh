// flbm_noise.cuh -- counter-based Gaussian noise on the device.
//
// Philox4x32-10 (J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11): a 10-round bijection of a
// 128-bit counter under a 64-bit key; each round multiplies two words by fixed
// odd constants, swaps halves and mixes in the key, which is advanced by the
// Weyl constants between rounds.  Gaussians come from the Box-Muller transform
// (the paper's generator, Sec. VI A) on pairs of output words.
#pragma once
#include <cstdint>

#include "flbm_lattice.cuh"

namespace flbm {

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1)
{
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        // one 32x32 -> 64-bit product gives both halves
        const uint64_t p0 = (uint64_t)M0 * x.x;
        const uint64_t p1 = (uint64_t)M1 * x.z;
        x = make_uint4((uint32_t)(p1 >> 32) ^ x.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ x.w ^ k1, (uint32_t)p0);
        k0 += W0;
        k1 += W1;
    }
    return x;
}

// Box-Muller on one pair of words: u1 = ((a >> 8) + 1) 2^-24 in (0, 1] and
// u2 = (b >> 8) 2^-24 in [0, 1) are exact in float; g0 = r cos(2 pi u2),
// g1 = r sin(2 pi u2), r = sqrt(-2 ln u1).
// The angle is folded exactly into [-pi, pi) (u2 - 1 for u2 >= 1/2, the same
// sine and cosine), where the hardware sine/cosine have an absolute error of
// about 2^-21; r = x rsqrt(x).
//
// ln u1: for u1 <= 31/32 the hardware log2 (absolute error <= 2^-22 on
// [1/2, 2], 2 ulp below) is accurate to ~5e-6 relative since |ln u1| >= 0.0317;
// nearer 1, where an absolute error would swamp the small radius, the Mercator
// series ln(1 - v) = -(v + v^2/2 + ... + v^5/5) with v = 1 - u1 <= 1/32 (exact by
// Sterbenz's lemma) is used, truncation error below 1e-8 relative.
__device__ __forceinline__ float log_unit_interval(float u1)
{
    const float v = 1.0f - u1;
    float ps = fmaf(v, 0.2f, 0.25f);
    ps = fmaf(v, ps, 0.333333333333333333f);
    ps = fmaf(v, ps, 0.5f);
    ps = fmaf(v, ps, 1.0f);
    const float near1 = -v * ps;
    const float far = __log2f(u1) * 0.693147180559945309f;
    return u1 > 0.96875f ? near1 : far;
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float &g0, float &g1)
{
    const float u1 = fmaf((float)(a >> 8), 0x1.0p-24f, 0x1.0p-24f); // ((a >> 8) + 1) 2^-24, exact
    const float u2 = (float)(b >> 8) * 0x1.0p-24f;
    const float r2 = -2.0f * log_unit_interval(u1);
    // r = sqrt(r2); the tiny offset makes r2 = 0 (u1 = 1) give 0 instead of 0 * inf
    // and is far below the rounding of the smallest nonzero r2 (~1.2e-7)
    const float r = r2 * rsqrtf(r2 + 1e-30f);
    const float t = u2 < 0.5f ? u2 : u2 - 1.0f;
    float s, c;
    __sincosf(6.28318530717958647692f * t, &s, &c);
    g0 = r * c;
    g1 = r * s;
}

// Does species S use the Gaussian of mode a?  Non-conserved modes a > D of
// each species have their own draws; the momenta (1..D) are drawn once, for
// species 0, and used with the opposite sign for species 1 (Sec. IV A).
template <class L, int S>
__host__ __device__ constexpr bool uses_mode(int a)
{
    return a < L::Q && (a > L::D || (S == 0 && a >= 1 && a <= L::D));
}

// Fill g[a] with the standard Gaussian of mode a for every mode species S uses:
// counter (site, step, S, a/4), lane a mod 4.  Only the needed Philox blocks
// and Box-Muller pairs are evaluated (decided at compile time).
template <class L, int S>
__device__ __forceinline__ void draw_gaussians(uint32_t site, uint32_t step, uint32_t k0, uint32_t k1,
                                               float (&g)[L::Q])
{
    static_for<(L::Q + 3) / 4>([&](auto sc) {
        constexpr int slot = decltype(sc)::value;
        constexpr bool u0 = uses_mode<L, S>(4 * slot), u1 = uses_mode<L, S>(4 * slot + 1);
        constexpr bool u2 = uses_mode<L, S>(4 * slot + 2), u3 = uses_mode<L, S>(4 * slot + 3);
        if constexpr (u0 || u1 || u2 || u3) {
            const uint4 x = philox4x32_10(make_uint4(site, step, (uint32_t)S, (uint32_t)slot), k0, k1);
            if constexpr (u0 || u1) {
                float g0, g1;
                box_muller(x.x, x.y, g0, g1);
                if constexpr (u0) g[4 * slot] = g0;
                if constexpr (u1) g[4 * slot + 1] = g1;
            }
            if constexpr (u2 || u3) {
                float g2, g3;
                box_muller(x.z, x.w, g2, g3);
                if constexpr (u2) g[4 * slot + 2] = g2;
                if constexpr (u3) g[4 * slot + 3] = g3;
            }
        }
    });
}

} // namespace flbm
