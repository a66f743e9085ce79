// FP64 softplus triple (z, z', z'') evaluated mostly on the FP32 and integer pipes.
//
// GB300 executes FP64 at 1/63 of the FP32 rate and bills each warp-level FP64
// instruction 16 SM clocks, while an FP64-bound kernel leaves most of its issue slots
// and the FP32/integer pipes idle. So the activation of the FP64 path keeps only the
// final rounding of each output to double (one FP64 add per output, four per neuron) on
// the FP64 pipe; everything else runs in double-float arithmetic: an unevaluated sum
// hi + lo of two FP32 numbers, about 48 significant bits (T. J. Dekker, Numer. Math. 18,
// 1971, and D. E. Knuth, TAOCP vol. 2: the exact sum and product transforms used below;
// the product's error term comes from one FP32 FMA).
//
// With x = -|y| (clamped at -700) and e = exp(x):
//   z  = max(y, 0) + log1p(e)
//   s  = z'  = 1/(1+e) for y >= 0, e/(1+e) for y < 0
//   t  = z'' = e/(1+e)^2
// Steps (table-driven, after P. T. P. Tang, ACM TOMS 15(2) 1989 and 16(4) 1990):
//   x = (128 m + j) ln2/128 + r, |r| <= ln2/256 (k = 128 m + j from an FP32 product;
//       r from |y| cut exactly into three floats and ln2/128 split in three, k C1 exact),
//   e = 2^m * T_j * (1 + expm1(r)), T_j = 2^(j/128) as a float pair, expm1 to degree 5;
//   k' = round(256 e), F = 1 + k'/256, rr = (e - k'/256)/F (the difference is exact),
//   log1p(e) = log F + log1p(rr),  1/(1+e) = (1/F) / (1 + rr),  |rr| <= 1/512,
//   the series to rr^7 with the terms from rr^3 on in FP32.
// Points with e < 2^-60 (|y| > 41.6) take z = e (or y), s = e (or 1), t = e directly from
// e in FP64: there 1 + e rounds to 1, and the float pairs of smaller e would lose their
// low parts to the FP32 exponent range.
// Accuracy (swept on the CPU against extended precision by the tests, 1.6 M arguments up
// to |y| = 800): |z - z_ref| <= 5.1e-15, s within 1.8e-14 and t within 3.2e-14 relative;
// float pairs carry about 2^-48 per operation, and the chains here are a few deep.
//
// The header compiles for the host as well (the same FP32 operations, no contraction),
// so the tests can sweep the exact device arithmetic on the CPU.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define ACTDF_FN __host__ __device__ __forceinline__
#else
#define ACTDF_FN inline
#endif

namespace commet {
namespace actdf {

// table sizes: 2^(j/128) for j in [0, 128); (log F, 1/F) for F = 1 + k/256, k in [0, 256]
constexpr int kExpN = 128;
constexpr int kLogN = 256;
// table layout in 8-byte slots, each one float pair (hi, lo):
// [0, 128) T_j; then per k: (log F_k) at 128 + 2k, (1/F_k) at 128 + 2k + 1
constexpr int kSlots = kExpN + 2 * (kLogN + 1);

struct f2 {
    float h, l;
};

// --------------------------------------------------------------- primitives
ACTDF_FN float fadd(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
ACTDF_FN float fsub(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
ACTDF_FN float fmul(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
ACTDF_FN float ffma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
    return __fmaf_rn(a, b, c);
#else
    return std::fmaf(a, b, c);
#endif
}
ACTDF_FN int32_t f_as_i(float f) {
#if defined(__CUDA_ARCH__)
    return __float_as_int(f);
#else
    int32_t i;
    std::memcpy(&i, &f, 4);
    return i;
#endif
}
ACTDF_FN float i_as_f(int32_t i) {
#if defined(__CUDA_ARCH__)
    return __int_as_float(i);
#else
    float f;
    std::memcpy(&f, &i, 4);
    return f;
#endif
}
ACTDF_FN int32_t d_hi(double d) {
#if defined(__CUDA_ARCH__)
    return __double2hiint(d);
#else
    uint64_t u;
    std::memcpy(&u, &d, 8);
    return (int32_t)(uint32_t)(u >> 32);
#endif
}
ACTDF_FN int32_t d_lo(double d) {
#if defined(__CUDA_ARCH__)
    return __double2loint(d);
#else
    uint64_t u;
    std::memcpy(&u, &d, 8);
    return (int32_t)(uint32_t)u;
#endif
}
ACTDF_FN double hilo(int32_t hi, int32_t lo) {
#if defined(__CUDA_ARCH__)
    return __hiloint2double(hi, lo);
#else
    const uint64_t u = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo;
    double d;
    std::memcpy(&d, &u, 8);
    return d;
#endif
}
ACTDF_FN double dadd(double a, double b) {
#if defined(__CUDA_ARCH__)
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}

// s + e = a + b exactly, given |a| >= |b| or a = 0
ACTDF_FN f2 fast_two_sum(float a, float b) {
    const float s = fadd(a, b);
    return {s, fsub(b, fsub(s, a))};
}
// (a.h + a.l) * (b.h + b.l) to about 2^-47, not renormalised
ACTDF_FN f2 df_mul(f2 a, f2 b) {
    const float p = fmul(a.h, b.h);
    float e = ffma(a.h, b.h, -p);
    e = ffma(a.h, b.l, e);
    e = ffma(a.l, b.h, e);
    return {p, e};
}

// FP32 value of a normal float pattern as an exact double, built with integer
// operations; zero and subnormal floats (below 2^-126) give zero
ACTDF_FN double f_to_d(float f) {
    const int32_t b = f_as_i(f);
    const int32_t mag = b & 0x7fffffff;
    const int32_t hi = (int32_t)(((uint32_t)mag >> 3) + 0x38000000u) | (b & (int32_t)0x80000000);
    const int32_t lo = (int32_t)((uint32_t)b << 29);
    return (mag >= 0x00800000) ? hilo(hi, lo) : 0.0;
}
// round hi + lo to double: the one FP64 operation per output
ACTDF_FN double df_to_d(f2 a) { return dadd(f_to_d(a.h), f_to_d(a.l)); }

// s + e = a + b exactly, any order of magnitude (Knuth)
ACTDF_FN f2 two_sum(float a, float b) {
    const float s = fadd(a, b);
    const float bb = fsub(s, a);
    return {s, fadd(fsub(a, fsub(s, bb)), fsub(b, bb))};
}

// ln2/128 = C1 + C2 + C3 + O(1e-20): C1 with 7 significant bits (k C1 exact in FP32 for
// k < 2^17, all k here), C2 and C3 floats; 128/ln2 for the FP32 product that picks k
constexpr float kC1 = 0x1.64p-8f;
constexpr float kC2 = -0x1.1bd01p-16f;
constexpr float kC3 = -0x1.718432p-42f;
constexpr float kInvC = 0x1.715476p+7f;
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: adding it rounds to an integer in the low bits

// softplus triple of y; tab = the kSlots float pairs (see make_table below)
ACTDF_FN void softplus3(double y, double &z, double &s, double &t, const f2 *tab) {
    const int32_t yH = d_hi(y), yL = d_lo(y);
    const bool neg = yH < 0;
    // |y| clamped at 700 (0x4085E000 is the high word of 700.0)
    int32_t aH = yH & 0x7fffffff, aL = yL;
    if (aH >= 0x4085E000) {
        aH = 0x4085E000;
        aL = 0;
    }
    // |y| = a1 + a2 + a3 exactly: its 53-bit mantissa cut into 24, 23 and 6 bits, each an
    // exact float (built with integer operations; a part below 2^-126 is zero, which
    // changes r by less than 2^-100)
    const int32_t E = aH >> 20;
    const float a1 = (E >= 897) ? i_as_f((int32_t)(((uint32_t)(aH - 0x38000000) << 3) | ((uint32_t)aL >> 29))) : 0.0f;
    const float a2 = (E >= 943) ? fmul(fsub(i_as_f(0x4B000000 | (int32_t)(((uint32_t)aL >> 6) & 0x7fffffu)), 8388608.0f),
                                       i_as_f((E - 942) << 23))
                                : 0.0f;
    const float a3 = (E >= 949) ? fmul(fsub(i_as_f(0x4B000000 | (aL & 63)), 8388608.0f), i_as_f((E - 948) << 23)) : 0.0f;
    // kn = round(|y| 128/ln2) >= 0 and r = kn ln2/128 - |y|, so that -|y| = k ln2/128 + r
    // with k = -kn: kn C1 - a1 is exact, kn C2 exact as a float pair, the sums exact up to
    // the last one (|r| <= ln2/256 + 2^-14, about 2^-50 absolute in the end)
    const float knm = ffma(a1, kInvC, kMagic);
    const int32_t k = 0x4B400000 - f_as_i(knm);  // k = -kn <= 0
    const float knf = fsub(knm, kMagic);
    const float t1 = ffma(knf, kC1, -a1);
    const float ph = fmul(knf, kC2), pe = ffma(knf, kC2, -ph);
    const f2 u1 = two_sum(t1, ph);
    const f2 u2 = two_sum(u1.h, -a2);
    const float rest = fsub(fadd(fadd(fadd(u1.l, u2.l), pe), fmul(knf, kC3)), a3);
    const f2 rr2 = fast_two_sum(u2.h, rest);
    const int32_t j = k & (kExpN - 1);
    const int32_t m = k >> 7;
    const float rh = rr2.h, rl = rr2.l;
    // expm1(r) = r + r^2/2 + r^3/6 + r^4/24 + r^5/120
    const float sqh = fmul(rh, rh);
    float sql = ffma(rh, rh, -sqh);
    sql = ffma(fadd(rh, rh), rl, sql);
    const float h2 = fmul(0.5f, sqh), l2 = fmul(0.5f, sql);
    const float tail = fmul(fmul(sqh, rh), ffma(rh, ffma(rh, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f));
    const f2 p0 = fast_two_sum(rh, h2);
    const float pl = fadd(fadd(fadd(l2, p0.l), rl), tail);
    // E' = T_j (1 + p) in [1, 2)
    const f2 T = tab[j];
    const float a = fmul(T.h, p0.h);
    const float ae = ffma(T.h, p0.h, -a);
    const f2 b = fast_two_sum(T.h, a);
    // low parts added from the smallest up: T.l p, T.h pl, then ae (~2^-33), T.l and b.l (~2^-25)
    const float lo = fadd(fadd(fadd(ffma(T.h, pl, fmul(T.l, p0.h)), ae), T.l), b.l);
    const f2 Ep = fast_two_sum(b.h, lo);

    if (m < -60) {
        // e < 2^-60: 1 + e rounds to 1 in every output
        const double Ed = df_to_d(Ep);
        const double e = hilo(d_hi(Ed) + (m << 20), d_lo(Ed));
        z = neg ? e : y;
        s = neg ? e : 1.0;
        t = e;
        return;
    }
    const float sc = i_as_f((m + 127) << 23);
    const f2 e{fmul(Ep.h, sc), fmul(Ep.l, sc)};
    // k' = round(256 e) in [0, 256]; d = e - k'/256 exactly
    const float kk_f = ffma(e.h, 256.0f, kMagic);
    const int32_t kk = f_as_i(kk_f) - 0x4B400000;
    const float dh = ffma(fsub(kk_f, kMagic), -1.0f / 256.0f, e.h);
    const f2 lF = tab[kExpN + 2 * kk], iF = tab[kExpN + 2 * kk + 1];
    // rr = d / F, renormalised: e's low part is large relative to the small d
    const f2 q0 = df_mul(f2{dh, e.l}, iF);
    const f2 q = fast_two_sum(q0.h, q0.l);
    const float r2 = fmul(q.h, q.h);
    float r2e = ffma(q.h, q.h, -r2);
    r2e = ffma(fadd(q.h, q.h), q.l, r2e);
    const float c3 = fmul(r2, q.h);  // rr^3
    // log1p(rr) = rr - rr^2/2 + rr^3 (1/3 - rr/4 + rr^2/5 - rr^3/6 + rr^4/7)
    const float g = fmul(c3, ffma(q.h, ffma(q.h, ffma(q.h, ffma(q.h, 1.0f / 7.0f, -1.0f / 6.0f), 0.2f), -0.25f),
                                  1.0f / 3.0f));
    const f2 s1 = fast_two_sum(q.h, fmul(-0.5f, r2));
    const f2 s2 = fast_two_sum(lF.h, s1.h);
    const float llo = fadd(fadd(fadd(fadd(ffma(-0.5f, r2e, q.l), s1.l), g), lF.l), s2.l);
    const f2 Lg = fast_two_sum(s2.h, llo);
    // 1/(1 + rr) = 1 - rr + rr^2 - rr^3 (1 - rr + rr^2)
    const f2 v1 = fast_two_sum(1.0f, -q.h);
    const f2 v2 = fast_two_sum(v1.h, r2);
    const float vw = fmul(c3, ffma(q.h, q.h, fsub(1.0f, q.h)));
    const float vlo = fadd(fadd(fsub(fsub(r2e, q.l), vw), v2.l), v1.l);
    const f2 V = fast_two_sum(v2.h, vlo);
    const f2 w0 = df_mul(iF, V);
    const f2 w = fast_two_sum(w0.h, w0.l);  // 1/(1+e)
    const f2 ew0 = df_mul(e, w);
    const f2 ew = fast_two_sum(ew0.h, ew0.l);  // e/(1+e)
    const f2 tt0 = df_mul(ew, w);              // e/(1+e)^2
    const double L = df_to_d(Lg);
    const double ypos = neg ? 0.0 : y;
    z = dadd(ypos, L);
    s = df_to_d(neg ? ew : w);
    t = df_to_d(tt0);
}

// (host only) the kSlots float pairs from extended precision: T_j = 2^(j/128); log F_k and 1/F_k,
// F_k = 1 + k/256; each value v stored as hi = (float)v, lo = (float)(v - hi)
inline void make_table(f2 *tab) {
    auto pair = [](long double v) {
        const float h = (float)v;
        return f2{h, (float)(v - (long double)h)};
    };
    for (int j = 0; j < kExpN; ++j) tab[j] = pair(exp2l((long double)j / kExpN));
    for (int k = 0; k <= kLogN; ++k) {
        const long double F = 1.0L + (long double)k / kLogN;
        tab[kExpN + 2 * k] = pair(logl(F));
        tab[kExpN + 2 * k + 1] = pair(1.0L / F);
    }
}

}  // namespace actdf
}  // namespace commet
