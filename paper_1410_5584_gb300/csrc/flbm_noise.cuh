// flbm_noise.cuh -- counter-based Gaussian noise on the device.
//
// Philox4x32-10 (J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11): a 10-round bijection of a
// 128-bit counter under a 64-bit key; each round multiplies two words by fixed
// odd constants, swaps halves and mixes in the key, which is advanced by the
// Weyl constants between rounds.  Gaussians come from the Box-Muller transform
// (the paper's generator, Sec. VI A) on pairs of 21-bit uniforms, six of which
// are cut from the four output words of a block.
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

// Hardware approximations (PTX lg2/sqrt/sin/cos .approx.ftz).  Every argument
// they get below is zero or a normal number, so flushing subnormals changes no
// result and spares the subnormal handling of the non-ftz forms.
__device__ __forceinline__ float lg2_hw(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_hw(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void sincos_hw(float x, float &s, float &c)
{
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(x));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(x));
}

// -2 ln u1 for u1 in (0, 1].  For u1 <= 31/32 the hardware log2 (absolute error
// <= 2^-22 on [1/2, 2], 2 ulp below) is accurate to ~5e-6 relative since
// |ln u1| >= 0.0317; nearer 1, where an absolute error would swamp the small
// radius, the Mercator series -2 ln(1 - v) = 2 (v + v^2/2 + ... + v^5/5) with
// v = 1 - u1 <= 1/32 (exact by Sterbenz's lemma) is used, truncation error
// below 1e-8 relative.
__device__ __forceinline__ float minus_two_log_unit_interval(float u1)
{
    const float v = 1.0f - u1;
    float ps = fmaf(v, 0.4f, 0.5f);
    ps = fmaf(v, ps, 0.666666667f);
    ps = fmaf(v, ps, 1.0f);
    ps = fmaf(v, ps, 2.0f);
    const float near1 = v * ps;
    const float far = lg2_hw(u1) * -1.38629436111989061883f; // -2 ln 2
    return u1 > 0.96875f ? near1 : far;
}

// Box-Muller on one pair of 21-bit uniforms held in the top bits of two words,
// scaled: g0 = scale r cos(2 pi u2), g1 = scale r sin(2 pi u2),
// r = sqrt(-2 ln u1), with u1 = ((a >> 11) + 1) 2^-21 in (0, 1] and
// u2 = (b >> 11) 2^-21 in [0, 1), both exact in float.  The angle is taken in
// [-pi, pi), where the hardware sine and cosine have an absolute error of about
// 2^-21: reading b as signed and shifting arithmetically gives u2 for u2 < 1/2
// and u2 - 1 above (the same sine and cosine).
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float scale, float &g0, float &g1)
{
    const float u1 = fmaf((float)(a >> 11), 0x1.0p-21f, 0x1.0p-21f); // ((a >> 11) + 1) 2^-21, exact
    const float r = scale * sqrt_hw(minus_two_log_unit_interval(u1)); // u1 = 1 gives r = 0
    // 2 pi t with t = (signed b >> 11) 2^-21: one rounding, as 2 pi 2^-21 is the
    // float 2 pi times a power of two
    const float ang = (float)((int32_t)b >> 11) * (6.28318530717958647692f * 0x1.0p-21f);
    float s, c;
    sincos_hw(ang, s, c);
    g0 = r * c;
    g1 = r * s;
}

// The fifth and sixth uniforms of a Philox block, packed from the low bits of
// its words into the top 21 bits of one word, as box_muller reads them:
// ((hi mod 2^11) 2^10 + (lo mod 2^10)) 2^11.
__device__ __forceinline__ uint32_t low_bits_word(uint32_t hi, uint32_t lo)
{
    return (hi << 21) | ((lo & 0x3FFu) << 11);
}

// Does species S use the Gaussian of mode a?  Non-conserved modes a > D of
// each species have their own draws; the momenta (1..D) are drawn once, for
// species 0, and used with the opposite sign for species 1 (Sec. IV A).
template <class L, int S>
__host__ __device__ constexpr bool uses_mode(int a)
{
    return a < L::Q && (a > L::D || (S == 0 && a >= 1 && a <= L::D));
}

// Scale kind of mode a: 1 for a momentum mode (scaled by scale_j), 0 otherwise.
template <class L> __host__ __device__ constexpr int scale_kind(int a) { return a >= 1 && a <= L::D ? 1 : 0; }

// One Box-Muller pair for modes (a0, a0 + 1) of species S.  When both modes are
// used with different scales (D2Q9: momentum mode 2 beside mode 3) the radius
// stays unscaled and each output takes its own scale.
template <class L, int S, int a0>
__device__ __forceinline__ void gaussian_pair(uint32_t wa, uint32_t wb, float scale_j, float scale, float (&g)[L::Q])
{
    constexpr bool use0 = uses_mode<L, S>(a0), use1 = uses_mode<L, S>(a0 + 1);
    if constexpr (use0 || use1) {
        constexpr int k0 = scale_kind<L>(a0), k1 = scale_kind<L>(a0 + 1);
        constexpr bool mixed = use0 && use1 && k0 != k1;
        constexpr int kind = use0 ? k0 : k1;
        float g0, g1;
        if constexpr (mixed) {
            box_muller(wa, wb, 1.0f, g0, g1);
            g0 *= k0 ? scale_j : scale;
            g1 *= k1 ? scale_j : scale;
        } else {
            box_muller(wa, wb, kind ? scale_j : scale, g0, g1);
        }
        if constexpr (use0) g[a0] = g0;
        if constexpr (use1) g[a0 + 1] = g1;
    }
}

// Philox blocks per species: mode a >= 1 is Gaussian n = a - 1 of its
// species, and block b holds Gaussians 6 b .. 6 b + 5.
template <class L> constexpr int kNoiseBlocks = (L::Q + 4) / 6;

// Fill g[a] with the Gaussian of mode a, times its scale, for every mode
// species S uses in the Philox blocks [BLK_LO, BLK_HI) (all by default).  Block
// b has counter (site, step, S, b); its words x0 .. x3 give six 21-bit
// uniforms, the top 21 bits of each word and two packed from the low bits, and
// three Box-Muller pairs: modes (6b+1, 6b+2) on (x0, x1), (6b+3, 6b+4) on
// (x2, x3) and (6b+5, 6b+6) on the packed two.  The momentum modes (species 0
// only) are scaled by scale_j, the others by scale.  Only the needed Philox
// blocks and Box-Muller pairs are evaluated (decided at compile time).
template <class L, int S, int BLK_LO = 0, int BLK_HI = kNoiseBlocks<L>>
__device__ __forceinline__ void draw_gaussians(uint32_t site, uint32_t step, uint32_t k0, uint32_t k1,
                                               float scale_j, float scale, float (&g)[L::Q])
{
    static_for<kNoiseBlocks<L>>([&](auto bc) {
        constexpr int b = decltype(bc)::value;
        constexpr int a = 6 * b + 1; // first mode of the block
        constexpr bool any = uses_mode<L, S>(a) || uses_mode<L, S>(a + 1) || uses_mode<L, S>(a + 2) ||
                             uses_mode<L, S>(a + 3) || uses_mode<L, S>(a + 4) || uses_mode<L, S>(a + 5);
        if constexpr (any && b >= BLK_LO && b < BLK_HI) {
            const uint4 x = philox4x32_10(make_uint4(site, step, (uint32_t)S, (uint32_t)b), k0, k1);
            gaussian_pair<L, S, a>(x.x, x.y, scale_j, scale, g);
            gaussian_pair<L, S, a + 2>(x.z, x.w, scale_j, scale, g);
            gaussian_pair<L, S, a + 4>(low_bits_word(x.x, x.y), low_bits_word(x.z, x.w), scale_j, scale, g);
        }
    });
}

} // namespace flbm
