// Device-side building blocks of the ProbMinHash kernels: the counter-based
// random stream, the canonical FP64 point values of the four algorithm
// families and their FP32 approximations with error bounds.
//
// Families (Sec. Sequence Generation): F1 = ProbMinHash1/1a (with replacement,
// uncorrelated), F2 = ProbMinHash2 (without replacement, uncorrelated),
// F3 = ProbMinHash3/3a (with replacement, correlated), F4 = ProbMinHash4
// (without replacement, correlated).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pmh {

constexpr uint64_t kPhi = 0x9E3779B97F4A7C15ull;   // 2^64 / golden ratio (SplitMix64 increment)
constexpr uint64_t kEmptyKey = ~0ull;
constexpr uint32_t kFull = 0xFFFFFFFFu;

// Relative error bound of every FP32 point value against its canonical FP64
// value: |x32 - x64| <= kEta * x32.  The sources (each in units u = 2^-24):
// 1/w from a truncated mantissa and a correctly rounded reciprocal (3u),
// Exp(1) via the reduced-range log1p below with a rounded U or 1 - U (6u),
// Exp(lambda;0,1) via log1pf with |U*expm1(-lambda)| <= 1/2 (12u), the table
// entries and their products (<= 4u), the FP32 sums of the uncorrelated
// families (a lane-sequential running sum of at most 32 positive terms, <= 31u;
// in deep mode a warp scan plus an error-free carry, <= 7u), the final
// product (u) and the FP64 value's own rounding (< u).  The worst family
// totals below 48u; kEta = 64u covers it.
constexpr float kEta = 0x1p-18f;

__host__ __device__ inline int family_of(int variant) {
    // PMH_V1 = 0, V1A = 1 -> F1; V2 = 2 -> F2; V3 = 3, V3A = 4 -> F3; V4 = 5 -> F4;
    // binary-weight V3U = 6, V3AU = 7 -> F3; V4U = 8 -> F4
    switch (variant) {
        case 0: case 1: return 1;
        case 2: return 2;
        case 3: case 4: case 6: case 7: return 3;
        default: return 4;
    }
}
// Binary-weight specialisations (Sec. Conventional Jaccard Similarity): every
// element with w > 0 counts with weight 1, ProbMinHash3/3a/4 draw Uniform([0,1))
// instead of their truncated exponentials, and gamma_i = i.
__host__ __device__ inline bool variant_unweighted(int variant) { return variant >= 6 && variant <= 8; }

// Per-m constants of Sec. ProbMinHash2/3/4, computed on the host in FP64
// (arrays indexed as in the paper, length m+1).
struct Tables {
    uint32_t m;
    const double *beta;     // beta_i = m/(m-i+1)
    const double *gamma;    // gamma_i = log1p(i/(m-i))/lambda_1, i < m
    const double *dgamma;   // gamma_i - gamma_{i-1}
    const double *c4;       // expm1(-lambda_i), lambda_i = log1p(1/(m-i))
    const double *inv4;     // 1/lambda_i
    const float *beta32, *gamma32, *dgamma32, *c4_32, *inv4_32;
    const float4 *p4;       // ProbMinHash4 point i: {gamma_{i-1}, dgamma_i, c4_i, inv4_i} in FP32, one 16-byte load (i = m: {gamma_{m-1}, 0, 0, 0})
    double c3, inv3, delta; // ProbMinHash3: expm1(-lambda), 1/lambda; ProbMinHash4: delta = 1/lambda_1
    float c3_32, inv3_32, delta32;
    float te_lo;            // (1-e^{-lambda_1})/lambda_1 rounded down: Exp(lambda_1;0,1) >= U * te_lo
    float lambda1_32;       // lambda_1 = log(1 + 1/(m-1))
    // Rejection sampler for Exp(lambda_i;0,1) (Sec. Truncated Exponential Sampling), i = 1..m-1
    // (ProbMinHash3 uses i = 1): c1 = (e^l - 1)/l, c3 = (1 - e^-l)/l, the rate l itself; k1 = the
    // smallest 53-bit k with fl(k 2^-53 c1) >= 1 (the first draw c1 U lands below 1 iff U's 53-bit
    // integer is below k1); k2 = ceil(c2 2^53), c2 = log(2/(1+e^-l))/l (U < c2 iff k < k2)
    const uint64_t *rej_k1, *rej_k2;
    const double *rej_c1, *rej_c3, *rej_lam;
    const float *rej_c1_32;
    float rej_u1_32;        // filter: a 23-bit uniform below this has k < k1 at point 1 (else TE may be ~0)
};

// ------------------------------------------------------------------ stream
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output j+1 of a generator
// seeded with `key` is mix(key + (j+1)*phi).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t value_word(uint64_t key, uint64_t i) {   // word 2i-2
    return mix64(key + (2 * i - 1) * kPhi);
}
__device__ __forceinline__ uint64_t label_word(uint64_t key, uint64_t i) {   // word 2i-1
    return mix64(key + (2 * i) * kPhi);
}
// floor(w * r / 2^64)
__device__ __forceinline__ uint32_t uniform_int(uint64_t w, uint32_t r) {
    return (uint32_t)__umul64hi(w, (uint64_t)r);
}

// ----------------------------------------------------------- FP64 (canonical)
// Fixed evaluation order t = b*c, s = a + t, x = w_inv*s with every operation
// rounded on its own (the _rn intrinsics are never contracted into FMAs).
__device__ __forceinline__ double unif53(uint64_t w) { return __dmul_rn((double)(w >> 11), 0x1p-53); }
__device__ __forceinline__ double exp1_64(uint64_t w) { return -log1p(-unif53(w)); }
__device__ __forceinline__ double texp_64(uint64_t w, double c, double inv) {
    double a = __dmul_rn(unif53(w), c);
    double l = log1p(a);
    return __dmul_rn(-l, inv);
}
// F1 term: w_inv * E
__device__ __forceinline__ double term1_64(uint64_t vw, double w_inv) { return __dmul_rn(w_inv, exp1_64(vw)); }
// F2 term: w_inv * (beta_i * E)
__device__ __forceinline__ double term2_64(const Tables &T, uint64_t vw, uint32_t i, double w_inv) {
    return __dmul_rn(w_inv, __dmul_rn(T.beta[i], exp1_64(vw)));
}
// F3 point: w_inv * ((i-1) + TE_lambda)
__device__ __forceinline__ double point3_64(const Tables &T, uint64_t vw, uint64_t i, double w_inv) {
    double s = __dadd_rn((double)(i - 1), texp_64(vw, T.c3, T.inv3));
    return __dmul_rn(w_inv, s);
}
// F4 point: w_inv * (gamma_{i-1} + dgamma_i * TE_{lambda_i}); i = m: w_inv * (gamma_{m-1} + delta * E)
__device__ __forceinline__ double point4_64(const Tables &T, uint64_t vw, uint32_t i, double w_inv) {
    double s;
    if (i < T.m) {
        double t = __dmul_rn(T.dgamma[i], texp_64(vw, T.c4[i], T.inv4[i]));
        s = __dadd_rn(T.gamma[i - 1], t);
    } else {
        double t = __dmul_rn(T.delta, exp1_64(vw));
        s = __dadd_rn(T.gamma[T.m - 1], t);
    }
    return __dmul_rn(w_inv, s);
}
// Binary-weight F3/F4 point: w_inv * ((i-1) + U), for every i (gamma_i = i)
__device__ __forceinline__ double point_unw_64(uint64_t vw, uint64_t i, double w_inv) {
    return __dmul_rn(w_inv, __dadd_rn((double)(i - 1), unif53(vw)));
}
__device__ __forceinline__ double lower3_64(uint64_t i, double w_inv) { return __dmul_rn(w_inv, (double)(i - 1)); }
__device__ __forceinline__ double lower4_64(const Tables &T, uint32_t i, double w_inv) {
    return __dmul_rn(w_inv, T.gamma[i - 1]);
}

// ------------------------------------------------ Exp(lambda;0,1) by rejection
// Algorithm "Fast generation of random values from Exp(lambda;0,1)" (Sec.
// Truncated Exponential Sampling), point i of an element with stream key
// `key`, table index ti (the rate lambda_ti).  The first uniform is the value
// word vw: c1 U below 1 is returned as it is (the rectangle under e^-lambda).
// Otherwise the rejection loop draws from the region between e^-lambda and
// the density; its uniforms are stream words 2^40 + 256 (i-1) + j (attempt t:
// j = 2t for x, 2t+1 for y), and after 64 rejected attempts (probability below
// 2^-190) the inversion of vw is returned.  The loop's uniforms are exact in
// FP64 and so are 1 - x and 1 - y; the comparisons are evaluated in FP64 with
// every operation rounded on its own, so both precisions return the same value.
constexpr int kTeRejMax = 64;
__device__ __forceinline__ uint64_t te_aux_word(uint64_t key, uint64_t i, uint32_t j) {
    return mix64(key + ((1ull << 40) + ((i - 1) << 8) + (uint64_t)j + 1ull) * kPhi);
}
static __device__ __noinline__ double texp_rej_loop(const Tables &T, uint32_t ti, uint64_t key, uint64_t i, uint64_t vw) {
    const double c1 = T.rej_c1[ti], c3 = T.rej_c3[ti], lam = T.rej_lam[ti];
    const uint64_t k2 = T.rej_k2[ti];
    for (int t = 0; t < kTeRejMax; ++t) {
        const uint64_t kx = te_aux_word(key, i, 2u * t) >> 11;
        double x = __dmul_rn((double)kx, 0x1p-53);
        if (kx < k2) return x;                                        // below c2: under the density
        double y = __dmul_rn(0.5, unif53(te_aux_word(key, i, 2u * t + 1u)));
        if (y > __dsub_rn(1.0, x)) { x = __dsub_rn(1.0, x); y = __dsub_rn(1.0, y); }   // reflection
        if (x <= __dmul_rn(c3, __dsub_rn(1.0, y))) return x;          // below the tangent at 0
        const double yc = __dmul_rn(y, c1);
        if (yc <= __dsub_rn(1.0, x)) return x;                        // below the tangent at 1
        if (__dmul_rn(yc, lam) <= expm1(__dmul_rn(lam, __dsub_rn(1.0, x)))) return x;   // below the density
    }
    return texp_64(vw, T.c4[ti], T.inv4[ti]);
}
__device__ __forceinline__ double texp_rej_64(const Tables &T, uint32_t ti, uint64_t key, uint64_t i, uint64_t vw) {
    if ((vw >> 11) < T.rej_k1[ti]) return __dmul_rn(unif53(vw), T.rej_c1[ti]);
    return texp_rej_loop(T, ti, key, i, vw);
}
// F3 / F4 points with the rejection sampler (same order of operations as point3_64 / point4_64)
__device__ __forceinline__ double point3r_64(const Tables &T, uint64_t key, uint64_t vw, uint64_t i, double w_inv) {
    const double s = __dadd_rn((double)(i - 1), texp_rej_64(T, 1, key, i, vw));
    return __dmul_rn(w_inv, s);
}
__device__ __forceinline__ double point4r_64(const Tables &T, uint64_t key, uint64_t vw, uint32_t i, double w_inv) {
    if (i >= T.m) return point4_64(T, vw, i, w_inv);   // the last point uses delta * Exp(1)
    const double t = __dmul_rn(T.dgamma[i], texp_rej_64(T, i, key, i, vw));
    return __dmul_rn(w_inv, __dadd_rn(T.gamma[i - 1], t));
}

// ------------------------------------------------------------ FP32 (filter)
// k * 2^-53 as a float for a 53-bit integer k, built from integer operations
// (normalise, truncate the mantissa to 23 bits): relative error < 2^-23, and
// exactly 0 for k = 0.  Keeps the FP32 path off the FP64 / conversion pipes.
__device__ __forceinline__ float u53_to_float(uint64_t k) {
    if (k == 0) return 0.0f;
    const int lz = __clzll((long long)k);          // 11..63
    const uint64_t nrm = k << lz;                   // leading one at bit 63
    const uint32_t mant = (uint32_t)(nrm >> 40) & 0x7FFFFFu;
    const uint32_t ex = (uint32_t)(63 - lz - 53 + 127);
    return __uint_as_float((ex << 23) | mant);
}
// log1p(f) for f in [sqrt(1/2) - 1, sqrt(2) - 1] as f + f^2 r(f), r a degree-8
// polynomial fitted to (log1p(f) - f) / f^2 by weighted least squares on
// Chebyshev nodes of that interval (weights: relative error of the result;
// csrc/fit_log1p.py).  FP32 Horner evaluation: at most 1.35 ulp from log1p(f)
// over the interval (checked against FP64 on 2e6 points).
__device__ __forceinline__ float log1p_reduced(float f) {
    float r = -0.07473210990428925f;
    r = __fmaf_rn(r, f, 0.128195121884346f);
    r = __fmaf_rn(r, f, -0.1326199471950531f);
    r = __fmaf_rn(r, f, 0.14196686446666718f);
    r = __fmaf_rn(r, f, -0.16608595848083496f);
    r = __fmaf_rn(r, f, 0.200011745095253f);
    r = __fmaf_rn(r, f, -0.2500157654285431f);
    r = __fmaf_rn(r, f, 0.3333333730697632f);
    r = __fmaf_rn(r, f, -0.49999988079071045f);
    return __fmaf_rn(__fmul_rn(f, f), r, f);
}

// Exp(1) = -ln(1 - U), U = (w >> 11) 2^-53, without branches: the lanes of a
// warp evaluate different points, and a two-way branch would run both ways.
// 1 - U = 2^e (1 + f) with f in [sqrt(1/2) - 1, sqrt(2) - 1):
//   U < 1 - sqrt(1/2): e = 0, f = -U (U converted once to FP32);
//   otherwise V = 1 - U is formed exactly in integers, converted once, and its
//   exponent and mantissa give e and f (exactly).
// -ln(1 - U) = -(e ln2 + log1p(f)), with ln2 split so that e * ln2_hi is exact.
// Error: at most ~2.1 ulp of the result for the first case (conversion of U
// 0.7, log1p 1.35) and ~4 ulp for the second (conversion of V 1.45, log1p
// 1.4, two roundings 1.0), measured against FP64 by tests/test_math_gpu.py.
__device__ __forceinline__ float exp1_32(uint64_t w) {
    const uint64_t k = w >> 11;
    const bool small = k < 2638147582215219ull;                // U < 1 - sqrt(1/2)
    const float x = u53_to_float(small ? k : (1ull << 53) - k);
    const uint32_t b = __float_as_uint(x);
    int e = (int)(b >> 23) - 127;
    uint32_t mb = (b & 0x7FFFFFu) | 0x3F800000u;                // mantissa in [1, 2)
    const bool high = mb >= 0x3FB504F3u;                       // >= sqrt(2): halve it
    mb -= high ? 0x00800000u : 0u;
    e += high ? 1 : 0;
    const float f = small ? -x : __fsub_rn(__uint_as_float(mb), 1.0f);
    const float ef = small ? 0.0f : (float)e;
    const float lp = log1p_reduced(f);
    return -__fmaf_rn(ef, 0x1.62e4p-1f, __fmaf_rn(ef, 0x1.7f7d1cp-20f, lp));
}
// Exp(lambda;0,1) = -log1p(U c) / lambda, c = expm1(-lambda) in [-1/2, 0).  The
// argument U c lies in (c, 0].  When it is at least sqrt(1/2) - 1 (always when
// lambda <= ln sqrt(2): ProbMinHash3 with m >= 4, and every point of ProbMinHash4
// but the two before the last) the reduced-range log1p applies directly, so the
// lanes of a warp do not split; otherwise log1pf.
__device__ __forceinline__ float texp_32(uint64_t w, float c, float inv) {
    const float x = __fmul_rn(u53_to_float(w >> 11), c);
    const float l = x >= -0.29289321f ? log1p_reduced(x) : log1pf(x);
    return __fmul_rn(-l, inv);
}
// FP32 candidate of the rejection sampler: the first draw c1 U (u53_to_float of U
// within 2u, c1 rounded to FP32 within u/2, one product rounding: below 4u of the
// FP64 value), or the FP64 loop's value rounded once.
__device__ __forceinline__ float texp_rej_32(const Tables &T, uint32_t ti, uint64_t key, uint64_t i, uint64_t vw) {
    const uint64_t k = vw >> 11;
    if (k < T.rej_k1[ti]) return __fmul_rn(u53_to_float(k), T.rej_c1_32[ti]);
    return __double2float_rn(texp_rej_loop(T, ti, key, i, vw));
}
// A positive, finite weight (the item's weights are validated before use):
// the sign bit is clear and the bits are not all zero (rejects +-0).
__device__ __forceinline__ bool weight_positive(double w) { return __double_as_longlong(w) > 0; }
// A lower bound of U with 23-bit resolution: 1.f - 1 for the float 1.f whose
// mantissa is the word's top 23 bits (the subtraction is exact).
__device__ __forceinline__ float unif_lo(uint64_t w) {
    return __fsub_rn(__uint_as_float(0x3F800000u | (uint32_t)(w >> 41)), 1.0f);
}

// 1/w scaled by 2^sigma as a float, from the double's bits (mantissa
// truncated to 23 bits: relative error <= 2^-23, then a correctly rounded
// reciprocal).  Weights too small for the float range give 2^100: every point
// of such an element is then far beyond any bound (E >= 2^-53 unless E = 0,
// and E = 0 gives x = 0 exactly in both precisions).
// The float whose reciprocal winv_scaled takes: w * 2^-sigma with the mantissa
// truncated to 23 bits (exponent clamped at 254), or 0 when it is below the
// normal float range.  winv_from_ws(ws_scaled(w, s)) == winv_scaled(w, s).
__device__ __forceinline__ float ws_scaled(double w, int sigma) {
    uint64_t b = (uint64_t)__double_as_longlong(w);
    int e = (int)((b >> 52) & 0x7FF);
    int ef = e - 1023 - sigma + 127;
    if (e == 0 || ef <= 0) return 0.0f;
    if (ef >= 254) ef = 254;
    return __uint_as_float(((uint32_t)ef << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu));
}
__device__ __forceinline__ float winv_from_ws(float ws) { return ws == 0.0f ? 0x1p100f : __frcp_rn(ws); }
__device__ __forceinline__ float winv_scaled(double w, int sigma) {
    uint64_t b = (uint64_t)__double_as_longlong(w);
    int e = (int)((b >> 52) & 0x7FF);
    int ef = e - 1023 - sigma + 127;
    if (e == 0 || ef <= 0) return 0x1p100f;
    if (ef >= 254) ef = 254;
    uint32_t fb = ((uint32_t)ef << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu);
    return __frcp_rn(__uint_as_float(fb));
}

}  // namespace pmh
