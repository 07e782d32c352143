// rng.cuh -- the estimator's normal variates on the device.
//
// The paper asks for the Brownian increments dW = sqrt(dt) N(0,1) (Sec. 4) and
// fixes no generator. They come from the counter-based Philox4x32-10 of
// Salmon, Moraes, Dror and Shaw ("Parallel random numbers: as easy as 1, 2, 3",
// SC'11): ten rounds, each two 32x32->64 multiplies whose high halves are
// xored with the other counter words and the round key, the key bumped by the
// Weyl constants between rounds. A 4-word block feeds two Box--Muller pairs.
//
// Uniforms from a word w with m = w & 0x7FFFFF (exact in single precision):
//   u1 = 1 - m 2^-23 in (0, 1],  u2 = m 2^-23 in [0, 1),  ub = (m + 1) 2^-23 in (0, 1].
#pragma once

#include <stdint.h>

namespace sdd {

// Rounds R0 .. R1-1 of Philox4x32-10 on counter state c; round r uses the key
// (k0 + r W0, k1 + r W1). Splitting the ten rounds lets a caller place them
// in the shadow of memory loads.
template <int R0, int R1>
__host__ __device__ __forceinline__ void philox_rounds(uint4& c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = R0; r < R1; ++r) {
        const uint32_t kr0 = k0 + (uint32_t)r * 0x9E3779B9u;
        const uint32_t kr1 = k1 + (uint32_t)r * 0xBB67AE85u;
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ kr0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ kr1,
                       (uint32_t)p0);
    }
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
    philox_rounds<0, 10>(c, k0, k1);
    return c;
}

// The same rounds with the round keys precomputed: rk[2r], rk[2r + 1] are
// (k0 + r W0, k1 + r W1). Passed as kernel parameters, they are read straight
// from the constant bank by the xor instructions.
struct PhiloxKeys {
    uint32_t rk[20];
};

__host__ __device__ inline PhiloxKeys philox_keys(uint64_t seed)
{
    PhiloxKeys k;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        k.rk[2 * r] = k0;
        k.rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return k;
}

template <int R0, int R1>
__device__ __forceinline__ void philox_rounds_rk(uint4& c, const PhiloxKeys& K)
{
#pragma unroll
    for (int r = R0; r < R1; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ K.rk[2 * r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ K.rk[2 * r + 1], (uint32_t)p0);
    }
}

__device__ __forceinline__ float sqrt_approx(float v)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Box--Muller pair scaled by sigma: (sigma R cos 2 pi u2, sigma R sin 2 pi u2),
// R = sqrt(-2 ln u1). `scale` = -2 sigma^2 ln 2, so that
// sigma R = sqrt(scale * log2(u1)). The angle is taken as 2 pi (u2 - 1/2),
// which keeps the argument of the fast sine and cosine in [-pi, pi); then
// cos(2 pi u2) = -cos(2 pi (u2 - 1/2)) and likewise for the sine.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float scale, float& z0, float& z1)
{
    const float u1 = 2.0f - __uint_as_float(0x3F800000u | (a & 0x7FFFFFu));
    const float v = __uint_as_float(0x3F800000u | (b & 0x7FFFFFu)) - 1.5f;
    const float r = sqrt_approx(scale * __log2f(u1));
    float s, c;
    __sincosf(6.28318530717958647692f * v, &s, &c);
    z0 = -r * c;
    z1 = -r * s;
}

// Both Box--Muller pairs of one Philox block (words 0,1 -> zA, words 2,3 -> zB),
// the arithmetic of the two pairs done with paired single-precision
// instructions. Same values as two calls of box_muller.
__device__ __forceinline__ void box_muller2(uint4 r, float scale, float2& zA, float2& zB)
{
    const float2 f1 = make_float2(__uint_as_float(0x3F800000u | (r.x & 0x7FFFFFu)),
                                  __uint_as_float(0x3F800000u | (r.z & 0x7FFFFFu)));
    const float2 f2 = make_float2(__uint_as_float(0x3F800000u | (r.y & 0x7FFFFFu)),
                                  __uint_as_float(0x3F800000u | (r.w & 0x7FFFFFu)));
    const float2 u1 = __ffma2_rn(f1, make_float2(-1.0f, -1.0f), make_float2(2.0f, 2.0f));   // exact
    const float2 v = __fadd2_rn(f2, make_float2(-1.5f, -1.5f));                            // exact
    const float2 l = __fmul2_rn(make_float2(__log2f(u1.x), __log2f(u1.y)), make_float2(scale, scale));
    const float ra = sqrt_approx(l.x), rb = sqrt_approx(l.y);
    const float2 ang = __fmul2_rn(v, make_float2(6.28318530717958647692f, 6.28318530717958647692f));
    float sa, ca, sb, cb;
    __sincosf(ang.x, &sa, &ca);
    __sincosf(ang.y, &sb, &cb);
    zA = __fmul2_rn(make_float2(-ra, -ra), make_float2(ca, sa));
    zB = __fmul2_rn(make_float2(-rb, -rb), make_float2(cb, sb));
}

__device__ __forceinline__ float uniform_pos(uint32_t w)
{
    // (1 + m 2^-23) - (1 - 2^-23) = (m + 1) 2^-23, exact
    return __uint_as_float(0x3F800000u | (w & 0x7FFFFFu)) - 0.99999988079071044921875f;
}

}  // namespace sdd
