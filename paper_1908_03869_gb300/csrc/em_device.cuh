// Device building blocks of the Euler-Maruyama path (sm_103a).
//
//   * Philox4x32-10 (Salmon et al., SC'11) with the round keys precomputed on
//     the host and passed in the kernel's parameter space, so every round's
//     key operand is a constant-bank read shared by all threads.
//   * Uniforms u = (w + 1/2) 2^-32 (reading of Eq. 3's "uniform over [0,1]"),
//     converted in FP32 with a single correctly rounded operation.
//   * Box-Muller (Eq. 3) in FP32 (SFU approximations) and FP64.
//   * Two-constant Cody-Waite reduction of a phase to [-pi, pi] before the SFU
//     sine/cosine (W. J. Cody, W. Waite, "Software Manual for the Elementary
//     Functions", 1980: x - q C1 - q C2 with C1 + C2 ~ 2 pi).
//   * Butterfly sums over the G lanes that share an orbit.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sdeb {

// ---------------------------------------------------------------------------
// Philox4x32-10
// ---------------------------------------------------------------------------

struct PhiloxKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

struct U32x4 {
    uint32_t x, y, z, w;
};

// One round: multiply words 0 and 2 by the two round multipliers, keep the
// 64-bit products' halves, mix the high halves with words 1 and 3 and the key.
__device__ __forceinline__ void philox_round(uint32_t &c0, uint32_t &c1, uint32_t &c2,
                                             uint32_t &c3, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
}

__device__ __forceinline__ U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               const PhiloxKeys &keys) {
#pragma unroll
    for (int r = 0; r < 10; ++r) philox_round(c0, c1, c2, c3, keys.k0[r], keys.k1[r]);
    return U32x4{c0, c1, c2, c3};
}

// Host-side key schedule: round r uses (k0 + r W0, k1 + r W1), W0/W1 the two
// Weyl increments (32-bit fractions of the golden ratio and of sqrt(3) - 1).
inline PhiloxKeys philox_key_schedule(uint64_t seed) {
    PhiloxKeys k;
    uint32_t a = (uint32_t)(seed & 0xffffffffu), b = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        k.k0[r] = a;
        k.k1[r] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return k;
}

// ---------------------------------------------------------------------------
// Uniforms
// ---------------------------------------------------------------------------

// Exact float of a 16-bit value: place it in the mantissa of 2^23 and subtract.
__device__ __forceinline__ float u16_to_f32(uint32_t v16) {
    return __uint_as_float(0x4b000000u | v16) - 8388608.0f;
}

// u = (w + 1/2) 2^-32 rounded once to FP32: the inner fma is exact
// ((lo + 1/2) 2^-32 needs 17 bits), the outer one rounds the exact value.
__device__ __forceinline__ float uniform_f32(uint32_t w) {
    float hi = u16_to_f32(w >> 16);
    float lo = u16_to_f32(w & 0xffffu);
    return __fmaf_rn(hi, 0x1p-16f, __fmaf_rn(lo, 0x1p-32f, 0x1p-33f));
}

// a = u - 1/2 = (w - 2^31 + 1/2) 2^-32 in (-1/2, 1/2), rounded once: the
// signed high half is converted through the 1.5 * 2^23 bias.
__device__ __forceinline__ float centered_uniform_f32(uint32_t w) {
    int32_t s = (int32_t)(w ^ 0x80000000u);
    int32_t hi = s >> 16;  // arithmetic shift, in [-2^15, 2^15)
    float fhi = __int_as_float(0x4b400000 + hi) - 12582912.0f;
    float flo = u16_to_f32((uint32_t)s & 0xffffu);
    return __fmaf_rn(fhi, 0x1p-16f, __fmaf_rn(flo, 0x1p-32f, 0x1p-33f));
}

__device__ __forceinline__ double uniform_f64(uint32_t w) {
    return ((double)w + 0.5) * 0x1p-32;
}

// ---------------------------------------------------------------------------
// Box-Muller, Eq. 3: n_cos = sqrt(-2 ln U1) cos(2 pi U2), n_sin = ... sin(...)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float sqrt_approx_f32(float y) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(y));
    return r;
}

__device__ __forceinline__ float lg2_approx_f32(float y) {
    float r;
    asm("lg2.approx.f32 %0, %1;" : "=f"(r) : "f"(y));
    return r;
}

// FP32.  y = -2 ln U1 comes from the SFU log2 except when U1 is within 2^-4
// of 1, where the absolute error of an SFU logarithm would dominate: there
// t = 1 - U1 = (~w + 1/2) 2^-32 is formed exactly (~w < 2^28) and
// -2 ln(1 - t) = 2 t (1 + t/2 + t^2/3 + ... + t^6/7) + O(t^8), the dropped
// terms below 2^-25 relative for t <= 2^-4.  The angle uses the centred
// uniform so the SFU sees an argument in (-pi, pi):
// cos(2 pi U2) = -cos(2 pi (U2 - 1/2)), likewise for sin.
__device__ __forceinline__ void box_muller_f32(uint32_t w_first, uint32_t w_second, float &n_cos,
                                               float &n_sin) {
    const float kMinus2Ln2 = -1.38629436111989061883f;  // -2 ln 2
    float u1 = uniform_f32(w_first);
    const uint32_t comp = ~w_first;  // 2^32 - 1 - w
    float t = uniform_f32(comp);     // 1 - U1, exact to rounding
    float poly = __fmaf_rn(t, 1.0f / 7.0f, 1.0f / 6.0f);
    poly = __fmaf_rn(poly, t, 1.0f / 5.0f);
    poly = __fmaf_rn(poly, t, 1.0f / 4.0f);
    poly = __fmaf_rn(poly, t, 1.0f / 3.0f);
    poly = __fmaf_rn(poly, t, 1.0f / 2.0f);
    poly = __fmaf_rn(poly, t, 1.0f);
    float y_series = 2.0f * t * poly;
    float y_log = kMinus2Ln2 * lg2_approx_f32(u1);
    float y = (comp < 0x10000000u) ? y_series : y_log;
    float radius = sqrt_approx_f32(y);
    float a = centered_uniform_f32(w_second);
    float ang = 6.28318530717958647692f * a;
    float s, c;
    __sincosf(ang, &s, &c);
    n_cos = -radius * c;
    n_sin = -radius * s;
}

__device__ __forceinline__ void box_muller_f64(uint32_t w_first, uint32_t w_second, double &n_cos,
                                               double &n_sin) {
    double u1 = uniform_f64(w_first);
    double u2 = uniform_f64(w_second);
    double radius = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    n_cos = radius * c;
    n_sin = radius * s;
}

template <typename Real>
__device__ __forceinline__ void box_muller(uint32_t w_first, uint32_t w_second, Real &n_cos,
                                           Real &n_sin);
template <>
__device__ __forceinline__ void box_muller<float>(uint32_t a, uint32_t b, float &c, float &s) {
    box_muller_f32(a, b, c, s);
}
template <>
__device__ __forceinline__ void box_muller<double>(uint32_t a, uint32_t b, double &c, double &s) {
    box_muller_f64(a, b, c, s);
}

// ---------------------------------------------------------------------------
// Phase sine / cosine
// ---------------------------------------------------------------------------

// FP32: the phase is x - c (state minus its Kahan compensation word).
// q = nearest integer to x / (2 pi) (by the 1.5 * 2^23 rounding bias, valid
// for |x| < 2^22), r1 = x - q C1 is exact in one fma (C1 = 2 pi rounded to
// float; for q != 0 both x and q C1 have their lowest bit at or above 2^-22
// while |r1| < 4), then r = r1 - q C2 - c.
__device__ __forceinline__ void sincos_phase(float x, float c_comp, float &s, float &c) {
    const float kInv2Pi = 0x1.45f306p-3f;
    const float kC1 = 0x1.921fb6p+2f;
    const float kC2 = -0x1.777a5cp-23f;
    float q = __fmaf_rn(x, kInv2Pi, 12582912.0f) - 12582912.0f;
    float r = __fmaf_rn(-q, kC1, x);
    r = __fmaf_rn(-q, kC2, r) - c_comp;
    __sincosf(r, &s, &c);
}

__device__ __forceinline__ void sincos_phase(float x, float &s, float &c) { sincos_phase(x, 0.0f, s, c); }

__device__ __forceinline__ void sincos_phase(double x, double c_comp, double &s, double &c) {
    sincos(x - c_comp, &s, &c);
}

__device__ __forceinline__ void sincos_phase(double x, double &s, double &c) { sincos(x, &s, &c); }

// ---------------------------------------------------------------------------
// Sums over the G consecutive lanes of one orbit.  With a butterfly every
// lane of the group ends with the bit-identical total (a + b == b + a).
// ---------------------------------------------------------------------------

template <int G, typename Real>
__device__ __forceinline__ Real group_sum(Real v) {
#pragma unroll
    for (int off = 1; off < G; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// ---------------------------------------------------------------------------
// State update: Kahan-compensated in FP32, plain in FP64.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void accumulate(float &x, float &comp, float inc) {
    float y = __fsub_rn(inc, comp);
    float t = __fadd_rn(x, y);
    comp = __fsub_rn(__fsub_rn(t, x), y);
    x = t;
}

__device__ __forceinline__ void accumulate(double &x, double & /*comp*/, double inc) {
    x = __dadd_rn(x, inc);
}

}  // namespace sdeb
