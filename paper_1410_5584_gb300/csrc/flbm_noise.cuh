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

// -2 ln u1 for u1 in (0, 1].  Away from 1 the hardware log2 is used: its
// absolute error (about 2^-22) puts an error of at most 3.3e-7 on -2 ln u1, so
// at most 1.3e-6 on the radius r = sqrt(-2 ln u1) >= 0.125 there.  For
// u1 > 1 - 2^-7, where that absolute error would swamp the small radius, the
// Mercator series -2 ln(1 - v) = 2 v + v^2 + (2/3) v^3 + ..., v = 1 - u1 (exact
// by Sterbenz's lemma), is cut after two terms: v (2 + v) leaves out at most
// (2/3) v^3 <= 3.2e-7, again at most 1.3e-6 on r.  Either way a Gaussian is
// within about 1.3e-6 of its exact value.
__device__ __forceinline__ float minus_two_log_unit_interval(float u1)
{
    const float v = 1.0f - u1;
    const float near1 = v * (2.0f + v);
    const float far = lg2_hw(u1) * -1.38629436111989061883f; // -2 ln 2
    return v < 0x1.0p-7f ? near1 : far;
}

// Box-Muller on one pair of 21-bit uniforms, scaled: g0 = scale r cos(2 pi u2),
// g1 = scale r sin(2 pi u2), r = sqrt(-2 ln u1), with u1 = (U1 + 1) 2^-21 in
// (0, 1] and u2 = U2 2^-21 in [0, 1), both exact in float.  T2 is U2 read as a
// signed 21-bit number (U2 for U2 < 2^20, U2 - 2^21 above), so that the angle
// is taken in [-pi, pi), where the hardware sine and cosine have an absolute
// error of about 2^-21; the two readings give the same sine and cosine.
__device__ __forceinline__ void box_muller(uint32_t U1, int32_t T2, float scale, float &g0, float &g1)
{
    const float u1 = fmaf((float)U1, 0x1.0p-21f, 0x1.0p-21f); // (U1 + 1) 2^-21, exact
    const float r = scale * sqrt_hw(minus_two_log_unit_interval(u1)); // u1 = 1 gives r = 0
    // 2 pi T2 2^-21: one rounding, as 2 pi 2^-21 is the float 2 pi times a power of two
    const float ang = (float)T2 * (6.28318530717958647692f * 0x1.0p-21f);
    float s, c;
    sincos_hw(ang, s, c);
    g0 = r * c;
    g1 = r * s;
}

// The six 21-bit uniforms of a Philox block x0 .. x3: U_k = x_k >> 11 for
// k = 0 .. 3, U4 = (x0 mod 2^11) 2^10 + (x1 mod 2^10) and
// U5 = (x2 mod 2^11) 2^10 + (x3 mod 2^10).  The angle uniforms (U1, U3, U5)
// are taken signed (see box_muller).
__device__ __forceinline__ uint32_t uniform_hi(uint32_t x) { return x >> 11; }
__device__ __forceinline__ int32_t uniform_hi_signed(uint32_t x) { return (int32_t)x >> 11; }
__device__ __forceinline__ uint32_t uniform_lo(uint32_t hi, uint32_t lo)
{
    return ((hi << 10) & 0x1FFC00u) | (lo & 0x3FFu);
}
__device__ __forceinline__ int32_t uniform_lo_signed(uint32_t hi, uint32_t lo)
{
    // bit 10 of hi is the sign bit of the 21-bit value
    return ((int32_t)(hi << 21) >> 11) | (int32_t)(lo & 0x3FFu);
}

// Gaussians n = 0 .. Q-1 of species slot `slot` at (site, step), block b
// holding n = 6 b .. 6 b + 5 in the layout of draw_gaussians below.  The
// population-space noise (FLBM_OPT_GHOST_NOISE) draws Gaussian n = i for
// population i in slots 2 and 3, which the mode draws (slots 0, 1) never use.
template <int Q>
__device__ __forceinline__ void population_gaussians(uint32_t site, uint32_t step, uint32_t slot, uint32_t k0,
                                                     uint32_t k1, float (&eta)[Q])
{
    static_for<(Q + 5) / 6>([&](auto bc) {
        constexpr int b = decltype(bc)::value;
        const uint4 x = philox4x32_10(make_uint4(site, step, slot, (uint32_t)b), k0, k1);
        float g[6];
        box_muller(uniform_hi(x.x), uniform_hi_signed(x.y), 1.0f, g[0], g[1]);
        box_muller(uniform_hi(x.z), uniform_hi_signed(x.w), 1.0f, g[2], g[3]);
        box_muller(uniform_lo(x.x, x.y), uniform_lo_signed(x.z, x.w), 1.0f, g[4], g[5]);
        static_for<6>([&](auto lc) {
            constexpr int l = decltype(lc)::value;
            if constexpr (6 * b + l < Q) eta[6 * b + l] = g[l];
        });
    });
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
__device__ __forceinline__ void gaussian_pair(uint32_t wa, int32_t wb, float scale_j, float scale, float (&g)[L::Q])
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
            gaussian_pair<L, S, a>(uniform_hi(x.x), uniform_hi_signed(x.y), scale_j, scale, g);
            gaussian_pair<L, S, a + 2>(uniform_hi(x.z), uniform_hi_signed(x.w), scale_j, scale, g);
            gaussian_pair<L, S, a + 4>(uniform_lo(x.x, x.y), uniform_lo_signed(x.z, x.w), scale_j, scale, g);
        }
    });
}

} // namespace flbm
