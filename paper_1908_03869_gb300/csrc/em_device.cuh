// Device building blocks of the Euler-Maruyama path (sm_103a).
//
//   * Philox4x32-10 (Salmon et al., SC'11) with the round keys precomputed on
//     the host and passed in the kernel's parameter space, so every round's
//     key operand is a constant-bank read shared by all threads.
//   * Uniforms u = (w + 1/2) 2^-32 (reading of Eq. 3's "uniform over [0,1]"),
//     in FP32 within one ulp of the exact value.
//   * Box-Muller (Eq. 3) in FP32 (SFU approximations) and FP64.
//   * Two-constant Cody-Waite reduction of a phase to [-pi, pi] before the SFU
//     sine/cosine (W. J. Cody, W. Waite, "Software Manual for the Elementary
//     Functions", 1980: x - q C1 - q C2 with C1 + C2 ~ 2 pi).
//   * Butterfly sums over the G lanes that share an orbit.
#pragma once

#ifdef __CUDACC_RTC__
// Compiled at run time (NVRTC) for user-defined models: no host headers.
typedef unsigned char uint8_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
#else
#include <cstdint>
#include <cuda_runtime.h>
#endif

#ifndef __CUDACC_RTC__
#include "check.cuh"  // the run-time compiled path gets it ahead of this header
#endif

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
// The 32 x 32 -> 64 products are written as 64-bit multiplies so each maps
// to a single wide integer multiply-add.
__device__ __forceinline__ void philox_round(uint32_t &c0, uint32_t &c1, uint32_t &c2,
                                             uint32_t &c3, uint32_t k0, uint32_t k1) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
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

// Counters (c0, c1, c2, 0) whose words c1 and c2 stay fixed while c0 runs
// (the noise counter (k, block, orbit, 0) of one lane): the first round's
// product of c2 and its mix with c1 and the round key depend only on the fixed
// words, so they are formed once (philox_round1_fixed), and each counter then
// costs one product and one xor for round 1 (c3 = 0 drops out of the mix).
struct PhiloxRound1 {
    uint32_t n0;   // hi(M1 c2) ^ c1 ^ key0 of round 1: word 0 after round 1
    uint32_t lo1;  // lo(M1 c2): word 1 after round 1
};

__device__ __forceinline__ PhiloxRound1 philox_round1_fixed(uint32_t c1, uint32_t c2, const PhiloxKeys &keys) {
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    return PhiloxRound1{(uint32_t)(p1 >> 32) ^ c1 ^ keys.k0[0], (uint32_t)p1};
}

__device__ __forceinline__ U32x4 philox4x32_10_fixed(uint32_t c0, const PhiloxRound1 &f, const PhiloxKeys &keys) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint32_t x0 = f.n0, x1 = f.lo1, x2 = (uint32_t)(p0 >> 32) ^ keys.k1[0], x3 = (uint32_t)p0;
#pragma unroll
    for (int r = 1; r < 10; ++r) philox_round(x0, x1, x2, x3, keys.k0[r], keys.k1[r]);
    return U32x4{x0, x1, x2, x3};
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

// u = (w + 1/2) 2^-32 in FP32: the integer converts once (round to
// nearest, 24 bits) and the affine map rounds again, so u is within one ulp
// of the exact value and never 0 or 1 beyond that ulp (w = 2^32 - 1 gives
// u = 1.0f; callers that take a logarithm use the complement word there).
__device__ __forceinline__ float uniform_f32(uint32_t w) {
    return __fmaf_rn(__uint2float_rn(w), 0x1p-32f, 0x1p-33f);
}

// a = u - 1/2 = (w - 2^31 + 1/2) 2^-32 in [-1/2, 1/2] from the signed word.
__device__ __forceinline__ float centered_uniform_f32(uint32_t w) {
    return __fmaf_rn(__int2float_rn((int32_t)(w ^ 0x80000000u)), 0x1p-32f, 0x1p-33f);
}

__device__ __forceinline__ double uniform_f64(uint32_t w) {
    return ((double)w + 0.5) * 0x1p-32;
}

// ---------------------------------------------------------------------------
// Box-Muller, Eq. 3: n_cos = sqrt(-2 ln U1) cos(2 pi U2), n_sin = ... sin(...)
// ---------------------------------------------------------------------------

// SFU approximations in their flush-to-zero forms: every argument they get
// here is a normal number or zero (uniforms >= 2^-33, radii of those, phases
// reduced to [-pi, pi]), where the .ftz and plain forms return the same
// value, and the .ftz forms skip the subnormal rescaling around the SFU.
__device__ __forceinline__ float sqrt_approx_f32(float y) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
    return r;
}

__device__ __forceinline__ float lg2_approx_f32(float y) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
    return r;
}

// Reciprocal for the Newton solves of the implicit schemes: in FP32 the SFU's
// rcp.approx.ftz (an inexact Jacobian solve only perturbs a Newton
// correction at the level of its own rounding), in FP64 the quotient.
__device__ __forceinline__ float recip_fast(float y) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
    return r;
}
__device__ __forceinline__ double recip_fast(double y) { return 1.0 / y; }

__device__ __forceinline__ void sincos_approx_f32(float x, float &s, float &c) {
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(x));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(x));
}

// FP32, in polar form, with the amplitude in units of sqrt(2 ln 2): the pair
// is (a c, a s) with a = kBmAmpUnitF32 * amp, amp = -sqrt(y'),
// y' = -2 ln(U1) / (2 ln 2) = -log2 U1.  Leaving the constant factor to the
// caller (which folds it into the noise strength) saves a multiply per pair.
// y' comes from the SFU log2 except when U1 is within 2^-6 of 1, where the
// absolute error of an SFU logarithm would dominate: there t = 1 - U1 =
// (~w + 1/2) 2^-32 comes from the complement word and
// -log2(1 - t) = t (2 + t + 2t^2/3 + t^3/2) / (2 ln 2) + O(t^5), the dropped
// terms below t^4/5 <= 2^-24/5 relative for t <= 2^-6 (the coefficients are
// pre-divided by 2 ln 2).  The angle is 2 pi (U2 - 1/2) = 2 pi w 2^-32 - pi
// (1 - 2^-32) in one fused multiply-add of the converted word, an argument in
// [-pi, pi] for the SFU: cos(2 pi U2) = -cos(2 pi (U2 - 1/2)), likewise for
// sin, hence the negative amplitude.
constexpr float kBmAmpUnitF32 = 1.17741002251547469f;  // sqrt(2 ln 2)

__device__ __forceinline__ void box_muller_polar_f32(uint32_t w_first, uint32_t w_second, float &amp, float &c,
                                                     float &s) {
    // For w >= 2^31 the signed reading of w is w - 2^32 = -(comp + 1), comp =
    // 2^32 - 1 - w the complement word, so t = 1 - U1 = (comp + 1/2) 2^-32 is
    // one fma of it; t is only used when comp < 2^26.
    const float t = __fmaf_rn(__int2float_rn((int32_t)w_first), -0x1p-32f, -0x1p-33f);
    float poly = __fmaf_rn(t, 0.360673760222240845f, 0.480898346962987793f);  // 1/(4 ln 2), 1/(3 ln 2)
    poly = __fmaf_rn(poly, t, 0.721347520444481703f);                         // 1/(2 ln 2)
    poly = __fmaf_rn(poly, t, 1.44269504088896341f);                          // 1/ln 2
    const float y_series = t * poly;
    const float y_log = -lg2_approx_f32(uniform_f32(w_first));
    const float y = (w_first > 0xFBFFFFFFu) ? y_series : y_log;  // comp < 2^26
    amp = -sqrt_approx_f32(y);
    // 2 pi 2^-32 (an exact scaling of float(2 pi)) and -float(pi): the word's
    // conversion rounds at most 2^8, the constant 8.7e-8 and the sum once,
    // below 6e-7 rad in all
    const float ang = __fmaf_rn(__uint2float_rn(w_second), 0x1.921fb6p-30f, -0x1.921fb6p+1f);
    sincos_approx_f32(ang, s, c);
}

__device__ __forceinline__ void box_muller_f32(uint32_t w_first, uint32_t w_second, float &n_cos,
                                               float &n_sin) {
    float amp, c, s;
    box_muller_polar_f32(w_first, w_second, amp, c, s);
    const float a = amp * kBmAmpUnitF32;
    n_cos = a * c;
    n_sin = a * s;
}

// FP64, polar form: amp = radius, (c, s) = (cos, sin)(2 pi U2).
__device__ __forceinline__ void box_muller_polar_f64(uint32_t w_first, uint32_t w_second, double &amp,
                                                     double &c, double &s) {
    const double u1 = uniform_f64(w_first);
    const double u2 = uniform_f64(w_second);
    amp = sqrt(-2.0 * log(u1));
    sincospi(2.0 * u2, &s, &c);
}

__device__ __forceinline__ void box_muller_f64(uint32_t w_first, uint32_t w_second, double &n_cos,
                                               double &n_sin) {
    double amp, c, s;
    box_muller_polar_f64(w_first, w_second, amp, c, s);
    n_cos = amp * c;
    n_sin = amp * s;
}

// The factor box_muller_polar leaves out of the amplitude (FP32: sqrt(2 ln 2);
// FP64: 1, the amplitude is the radius).
template <typename Real>
__device__ __forceinline__ constexpr Real bm_amp_unit() { return sizeof(Real) == 4 ? Real(kBmAmpUnitF32) : Real(1); }

template <typename Real>
__device__ __forceinline__ void box_muller_polar(uint32_t w_first, uint32_t w_second, Real &amp, Real &c, Real &s);
template <>
__device__ __forceinline__ void box_muller_polar<float>(uint32_t a, uint32_t b, float &amp, float &c, float &s) {
    box_muller_polar_f32(a, b, amp, c, s);
}
template <>
__device__ __forceinline__ void box_muller_polar<double>(uint32_t a, uint32_t b, double &amp, double &c,
                                                         double &s) {
    box_muller_polar_f64(a, b, amp, c, s);
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

// FP32: the phase is x - c (state minus its Kahan compensation word),
// reduced to [-pi, pi] before the SFU.  q = nearest integer to x / (2 pi)
// (by the 1.5 * 2^23 rounding bias, valid for |x| < 2^22), r1 = x - q C1 is
// exact in one fma (C1 = 2 pi rounded to float; for q != 0 both x and q C1
// have their lowest bit at or above 2^-22 while |r1| < 4), then
// r = r1 - q C2 - c.
__device__ __forceinline__ float reduce_phase(float x, float c_comp) {
    const float kInv2Pi = 0x1.45f306p-3f;
    const float kC1 = 0x1.921fb6p+2f;
    const float kC2 = -0x1.777a5cp-23f;
    float q = __fmaf_rn(x, kInv2Pi, 12582912.0f) - 12582912.0f;
    float r = __fmaf_rn(-q, kC1, x);
    return __fsub_rn(__fmaf_rn(-q, kC2, r), c_comp);
}

// FP64 keeps the phase unreduced; sin/cos are CUDA's double functions.
__device__ __forceinline__ double reduce_phase(double x, double c_comp) { return x - c_comp; }

__device__ __forceinline__ void sincos_reduced(float r, float &s, float &c) { sincos_approx_f32(r, s, c); }
__device__ __forceinline__ void sincos_reduced(double r, double &s, double &c) { sincos(r, &s, &c); }

__device__ __forceinline__ void sincos_phase(float x, float c_comp, float &s, float &c) {
    sincos_reduced(reduce_phase(x, c_comp), s, c);
}

__device__ __forceinline__ void sincos_phase(float x, float &s, float &c) { sincos_phase(x, 0.0f, s, c); }

__device__ __forceinline__ void sincos_phase(double x, double c_comp, double &s, double &c) {
    sincos_reduced(reduce_phase(x, c_comp), s, c);
}

__device__ __forceinline__ void sincos_phase(double x, double &s, double &c) { sincos(x, &s, &c); }

// ---------------------------------------------------------------------------
// Explicitly rounded arithmetic: the model increments use these so the
// compiler has no contraction choice left and every kernel that steps the
// same model (forward, adjoint replay) produces identical bits.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float fma_r(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_r(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_r(double a, double b) { return __dmul_rn(a, b); }

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

// Kahan compensation applied every kCompPeriod steps (the FP32 phase
// models).  The state is the pair (x, c) with value x - c, as above; within
// a period each increment only enters c (c -= inc, one rounding at the
// magnitude of a few increments, far below x's), and at the end of each
// period renormalize() moves c into x: t = x - c rounded, and c becomes that
// rounding's error, (t - x) + c, so the value t - c is unchanged.  Periods
// end at global step multiples of kCompPeriod, so a run resumed from a
// stored (x, c) at any step, or replayed from a checkpoint, takes the same
// roundings.
constexpr uint32_t kCompPeriod = 16;

__device__ __forceinline__ void accumulate_delayed(float &, float &comp, float inc) { comp = __fsub_rn(comp, inc); }

__device__ __forceinline__ void renormalize(float &x, float &comp) {
    const float t = __fsub_rn(x, comp);
    comp = __fadd_rn(__fsub_rn(t, x), comp);
    x = t;
}

template <typename Real>
__device__ __forceinline__ Real state_value(Real x, Real comp) { return x - comp; }

}  // namespace sdeb
