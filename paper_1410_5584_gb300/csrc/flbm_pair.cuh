// flbm_pair.cuh -- two floats handled by one instruction: the packed FP32
// arithmetic of sm_100 and later (add, sub, mul, fma on .f32x2 operands).
// The collide uses it where both species run the same arithmetic on their
// own values (one lane per species).  Each lane is rounded exactly as the
// scalar instruction would round it.
#pragma once
#include <cstdint>

namespace flbm {

struct F2 {
    unsigned long long v;
    F2() = default;
    __device__ __forceinline__ explicit F2(unsigned long long bits) : v(bits) {}
    __device__ __forceinline__ F2(float lo, float hi)
    {
        asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(lo), "f"(hi));
    }
    // the same value in both lanes; built from the bit patterns so that a
    // constant argument gives a compile-time constant
    __device__ __forceinline__ explicit F2(int k) : v(splat((float)k)) {}
    __device__ __forceinline__ static unsigned long long splat(float x)
    {
        const unsigned long long b = __float_as_uint(x);
        return (b << 32) | b;
    }
    __device__ __forceinline__ float lo() const
    {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
        (void)b;
        return a;
    }
    __device__ __forceinline__ float hi() const
    {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
        (void)a;
        return b;
    }
};

__device__ __forceinline__ F2 splat2(float x) { return F2(F2::splat(x)); }
// a float2 of the kernel parameters (or any 8-byte aligned pair) as one packed value
__device__ __forceinline__ F2 pair2(const float2 &x) { return F2(*reinterpret_cast<const unsigned long long *>(&x)); }
__device__ __forceinline__ F2 neg2(F2 a) { return F2(a.v ^ 0x8000000080000000ull); }

__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c)
{
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b)
{
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b)
{
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    F2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}

// A product whose rounding is deferred, so that "c + k * x" and "c - k * x"
// (the forms of the factored transforms, with k a small integer constant)
// become one fused multiply-add, as the scalar compiler contracts them.
struct P2 {
    F2 a, b;
};
__device__ __forceinline__ P2 operator*(F2 a, F2 b) { return {a, b}; }
__device__ __forceinline__ F2 operator+(F2 c, P2 p) { return fma2(p.a, p.b, c); }
__device__ __forceinline__ F2 operator+(P2 p, F2 c) { return fma2(p.a, p.b, c); }
__device__ __forceinline__ F2 operator-(F2 c, P2 p) { return fma2(neg2(p.a), p.b, c); }
__device__ __forceinline__ F2 operator-(P2 p, F2 c) { return mul2(p.a, p.b) - c; }

} // namespace flbm
