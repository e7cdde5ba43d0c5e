// pamc_device.cuh -- device-side building blocks shared by the kernels:
// the Philox4x32-10 counter-based generator, the deterministic binary64 exp
// used for every acceptance threshold and resampling weight, and the
// threshold formulas of Eq. 4 (heat-bath), Metropolis and the cascaded
// three-state sampler of Suppl. S3.
//
// Every floating-point operation below is an explicit correctly rounded
// intrinsic (__dmul_rn, __dadd_rn, __ddiv_rn, __fma_rn), so no compiler
// contraction can change a bit: the values are a function of the inputs only.
#pragma once
#include <cstdint>

namespace pamc {

enum : uint32_t { kTagInit = 1, kTagPerm = 2, kTagFlip = 3, kTagResample = 4, kTagNcm = 5 };

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (c0,c1,c2,c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0))
// with the key advanced by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t a = 0xD2511F53u * c0, ah = __umulhi(0xD2511F53u, c0);
        const uint32_t b = 0xCD9E8D57u * c2, bh = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = bh ^ c1 ^ k0, n2 = ah ^ c3 ^ k1;
        c0 = n0; c1 = b; c2 = n2; c3 = a;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

// The ten round keys of a seed, passed to kernels by value so that the rounds
// read them as constants instead of recomputing the key schedule per call.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

inline __host__ __device__ PhiloxKeys make_philox_keys(uint64_t seed) {
    PhiloxKeys K;
    uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        K.k0[i] = a;
        K.k1[i] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return K;
}

__device__ __forceinline__ u32x4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           const PhiloxKeys &K) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ K.k0[i];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ K.k1[i];
        c0 = n0; c1 = (uint32_t)p1; c2 = n2; c3 = (uint32_t)p0;
    }
    return {c0, c1, c2, c3};
}

// ---------------------------------------------------------------------------
// Deterministic exp: x = k ln2 + r (Cody & Waite, with ln2 split into a
// 32-significant-bit head and a tail), e^r by the degree-13 Taylor series in
// Horner form with fused multiply-adds, result scaled by 2^k.  Constants are
// ln 2 and 1/i! rounded to binary64.  Flushes to 0 below -707, +inf above 709.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double det_exp(double x) {
    if (x != x) return x;
    if (x > 709.0) return __longlong_as_double(0x7ff0000000000000ll);
    if (x < -707.0) return 0.0;
    const double kd = floor(__dadd_rn(__dmul_rn(x, 0x1.71547652b82fep+0), 0.5));
    double r = __fma_rn(-kd, 0x1.62e42fee00000p-1, x);
    r = __fma_rn(-kd, 0x1.a39ef35793c76p-33, r);
    double p = 0x1.6124613a86d09p-33;            // 1/13!
    p = __fma_rn(p, r, 0x1.1eed8eff8d898p-29);   // 1/12!
    p = __fma_rn(p, r, 0x1.ae64567f544e4p-26);   // 1/11!
    p = __fma_rn(p, r, 0x1.27e4fb7789f5cp-22);   // 1/10!
    p = __fma_rn(p, r, 0x1.71de3a556c734p-19);   // 1/9!
    p = __fma_rn(p, r, 0x1.a01a01a01a01ap-16);   // 1/8!
    p = __fma_rn(p, r, 0x1.a01a01a01a01ap-13);   // 1/7!
    p = __fma_rn(p, r, 0x1.6c16c16c16c17p-10);   // 1/6!
    p = __fma_rn(p, r, 0x1.1111111111111p-7);    // 1/5!
    p = __fma_rn(p, r, 0x1.5555555555555p-5);    // 1/4!
    p = __fma_rn(p, r, 0x1.5555555555555p-3);    // 1/3!
    p = __fma_rn(p, r, 0.5);                     // 1/2!
    p = __fma_rn(p, r, 1.0);                     // 1/1!
    p = __fma_rn(p, r, 1.0);                     // 1/0!
    return ldexp(p, (int)kd);
}

// round half up for x >= 0: floor plus a test of the (exact) fraction
__device__ __forceinline__ uint64_t round_nonneg(double x) {
    const double f = floor(x);
    const double fr = __dsub_rn(x, f);
    uint64_t v = (uint64_t)f;
    if (fr >= 0.5) v += 1;
    return v;
}

constexpr double kTwo32 = 4294967296.0;

// Eq. 4: s <- +1 iff u < T(h), T(h) = round(2^32 / (1 + e^{-2 beta h}))
__device__ __forceinline__ uint64_t thr_heatbath(double beta, int64_t h) {
    const double x = __dmul_rn(__dmul_rn(-2.0, beta), (double)h);
    const double e = det_exp(x);
    const double p = __ddiv_rn(1.0, __dadd_rn(1.0, e));
    return round_nonneg(__dmul_rn(p, kTwo32));
}

// Metropolis: flip iff u < T_M(dE), T_M = 2^32 for dE <= 0
__device__ __forceinline__ uint64_t thr_metropolis(double beta, int64_t dE) {
    if (dE <= 0) return 1ull << 32;
    const double e = det_exp(-__dmul_rn(beta, (double)dE));
    return round_nonneg(__dmul_rn(e, kTwo32));
}

// Suppl. S3 first p-bit: P(label 0) = 1/(1 + e^{beta a} + e^{beta b})
__device__ __forceinline__ uint64_t thr_potts_b1_from(double ea, double eb) {
    const double den = __dadd_rn(__dadd_rn(1.0, ea), eb);
    return round_nonneg(__dmul_rn(__ddiv_rn(1.0, den), kTwo32));
}

// Suppl. S3 second p-bit: P(label 1 | not 0) = 1/(1 + e^{beta c})
__device__ __forceinline__ uint64_t thr_potts_b2(double beta, int64_t c) {
    const double e = det_exp(__dmul_rn(beta, (double)c));
    return round_nonneg(__dmul_rn(__ddiv_rn(1.0, __dadd_rn(1.0, e)), kTwo32));
}

}  // namespace pamc
