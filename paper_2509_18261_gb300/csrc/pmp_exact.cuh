// pmp_exact.cuh -- correctly rounded binary64 square root and quotient from
// integer and FP32 instructions, and comparisons decided on the bit patterns.
//
// GB300 executes FP64 at 2 lanes per clock per SM, integer and FP32 work at
// 64-128; a binary64 square root or division compiled to the FP64 unit is a
// sequence of FP64 instructions.  These two functions compute the same
// correctly rounded results (round to nearest even) from the operands' integer
// significands by digit recurrence -- the restoring long division and
// digit-by-digit square root of e.g. Ercegovac & Lang, "Digital Arithmetic"
// (2004), ch. 5 and 6 -- in radix 2^15 to 2^18:
//   - each digit is estimated in FP32 from the top bits of the partial
//     remainder (error below one unit of the digit, bounds in the comments);
//   - the partial remainder is updated exactly in 64-bit integers (modulo
//     2^64 where an intermediate term is wider: the true remainder is known to
//     be below 2^57, so the wrapped difference is exact);
//   - a digit one too large or too small is corrected from the remainder.
// The recurrence yields the result truncated to 54 bits.  A binary64 square
// root or quotient is never exactly halfway between two doubles (its odd
// part would need more than 53 bits), so adding one in the 54th bit and
// truncating to 53 rounds to nearest.
//
// Normal operands with a normal result take this path, and so do the zeros
// that the kernels meet (sqrt(+0), +-0 / normal); the rest (subnormal,
// infinite, NaN, negative sqrt, overflow, underflow) use the compiler's sqrt /
// division.  The functions are __host__ __device__: the host
// build is checked against the C library's correctly rounded results, the
// device build against the GPU's.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define PMP_EXACT_FN __host__ __device__ __forceinline__
#else
#define PMP_EXACT_FN inline
#endif

namespace pmp {
namespace exact {

constexpr uint64_t kMant = (1ULL << 52) - 1;
constexpr uint64_t kHidden = 1ULL << 52;
constexpr uint64_t kSign = 1ULL << 63;

PMP_EXACT_FN uint64_t bits_of(double x)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    std::memcpy(&u, &x, sizeof u);
    return u;
#endif
}

PMP_EXACT_FN double double_of(uint64_t u)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double x;
    std::memcpy(&x, &u, sizeof x);
    return x;
#endif
}

// x > 0.0 without an FP64 comparison: bit patterns 1 .. 0x7ff0...0 are the
// positive subnormals, normals and +inf.
PMP_EXACT_FN bool positive(double x) { return bits_of(x) - 1ULL < 0x7ff0000000000000ULL; }

// Comparisons with 0 and 1 decided on the bit patterns, with the IEEE 754
// result for every operand (signed zeros, infinities and NaN included): an
// FP64 comparison occupies the FP64 pipe like an addition.
// x >= 0: +-0, positive finite, +inf
PMP_EXACT_FN bool ge0(double x)
{
    const uint64_t u = bits_of(x);
    return u <= 0x7ff0000000000000ULL || u == kSign;
}
// x < 0: negative non-zero, -inf
PMP_EXACT_FN bool lt0(double x)
{
    const uint64_t u = bits_of(x);
    return u > kSign && u <= 0xfff0000000000000ULL;
}
// x != 0 (NaN included)
PMP_EXACT_FN bool ne0(double x) { return (bits_of(x) << 1) != 0; }
// x > 1
PMP_EXACT_FN bool gt1(double x)
{
    const uint64_t u = bits_of(x);
    return u > 0x3ff0000000000000ULL && u <= 0x7ff0000000000000ULL;
}
// x < 1: [+0, 1) or negative (-0 and -inf included)
PMP_EXACT_FN bool lt1(double x)
{
    const uint64_t u = bits_of(x);
    return u < 0x3ff0000000000000ULL || (u >= kSign && u <= 0xfff0000000000000ULL);
}

// m / 2 for an odd integer m (|m| < 2^31), i.e. the double (m - 1) / 2 + 0.5
// that a cell centre c + 1/2 is, built from its bits without an FP64
// conversion or addition (exact: the value has at most 32 significant bits).
PMP_EXACT_FN double half_odd(int m)
{
    const uint32_t a = m < 0 ? (uint32_t)(-(int64_t)m) : (uint32_t)m;  // odd, >= 1
#if defined(__CUDA_ARCH__)
    const int e = 31 - __clz(a);
#else
    const int e = 31 - __builtin_clz(a);
#endif
    // a = 1.f 2^e, so m / 2 = 1.f 2^(e - 1): biased exponent 1022 + e
    const uint64_t mant = ((uint64_t)a << (52 - e)) & kMant;
    return double_of((m < 0 ? kSign : 0) | ((uint64_t)(1022 + e) << 52) | mant);
}

// One digit of the division recurrence: with 0 <= R < mb on entry,
// d = floor(R 2^s / mb), R <- R 2^s - d mb, Q <- Q 2^s + d.  The FP32
// estimate R 2^s / mb (R and mb truncated to 32 bits, rb = RN(1 / (mb >> 21)))
// is within 2^-4 of the exact quotient (d < 2^18, four FP32 roundings of
// 2^-24 each, truncation below 2^-13), so its truncation is the digit or one
// off; the remainder's sign or size tells which.
PMP_EXACT_FN void div_digit(uint64_t &R, uint64_t &Q, uint64_t mb, float rbs, int s)
{
    const uint32_t d = (uint32_t)((float)(uint32_t)(R >> 21) * rbs);
    R = (R << s) - (uint64_t)d * mb;  // true value in (-mb, 2 mb)
    Q = (Q << s) + d;
    if ((int64_t)R < 0) {
        R += mb;
        Q -= 1;
    } else if (R >= mb) {
        R -= mb;
        Q += 1;
    }
}

// 2^s as a float, 0 <= s < 127.
PMP_EXACT_FN float pow2f(int s)
{
    const uint32_t u = (uint32_t)(127 + s) << 23;
    float f;
#if defined(__CUDA_ARCH__)
    f = __uint_as_float(u);
#else
    std::memcpy(&f, &u, sizeof f);
#endif
    return f;
}

// a / b rounded to nearest even.
PMP_EXACT_FN double div_rn(double a, double b)
{
    const uint64_t ua = bits_of(a), ub = bits_of(b);
    const uint32_t ea = (uint32_t)(ua >> 52) & 0x7ffu, eb = (uint32_t)(ub >> 52) & 0x7ffu;
    const uint64_t ma = (ua & kMant) | kHidden, mb = (ub & kMant) | kHidden;  // [2^52, 2^53)
    const uint32_t lt = ma < mb ? 1u : 0u;
    // a / b = (ma / mb) 2^(ea - eb); Q = floor(ma 2^(53 + lt) / mb) lies in
    // [2^53, 2^54), and the rounded quotient is ((Q + 1) >> 1) 2^(be - 1075).
    const int be = (int)ea - (int)eb + 1023 - (int)lt;
    if (ea - 1u >= 2046u || eb - 1u >= 2046u || be < 1 || be > 2045) {
        if ((ua << 1) == 0 && eb - 1u < 2046u) return double_of((ua ^ ub) & kSign);  // +-0 / normal
        return a / b;
    }
    const float rb = 1.0f / (float)(uint32_t)(mb >> 21);  // mb >> 21 in [2^31, 2^32)
    uint64_t R = lt ? ma : ma - mb;  // the integer digit floor(ma / mb) is 1 - lt
    uint64_t Q = lt ? 0u : 1u;
    div_digit(R, Q, mb, rb * pow2f(18), 18);
    div_digit(R, Q, mb, rb * pow2f(18), 18);
    const int s3 = 17 + (int)lt;
    div_digit(R, Q, mb, rb * pow2f(s3), s3);
    const uint64_t r53 = (Q + 1) >> 1;  // in [2^52, 2^53]; 2^53 carries into the exponent
    return double_of(((ua ^ ub) & kSign) | (((uint64_t)be << 52) + (r53 - kHidden)));
}

// Digit correction of the square-root recurrence: with R = T - Y^2 for the
// current partial root Y, bring Y to floor(sqrt(T)) when it is one off.
PMP_EXACT_FN void sqrt_fix(uint64_t &Y, int64_t &R)
{
    if (R < 0) {
        R += (int64_t)(2 * Y) - 1;  // (Y - 1)^2 = Y^2 - 2Y + 1
        Y -= 1;
    } else if (R > (int64_t)(2 * Y)) {
        R -= (int64_t)(2 * Y) + 1;  // (Y + 1)^2 = Y^2 + 2Y + 1
        Y += 1;
    }
}

// sqrt(x) rounded to nearest even.
PMP_EXACT_FN double sqrt_rn(double x)
{
    const uint64_t ux = bits_of(x);
    const uint32_t bx = (uint32_t)(ux >> 52);  // sign and biased exponent
    if (bx - 1u >= 2046u) return ux == 0 ? x : std::sqrt(x);  // sqrt(+0) = +0
    const int e = (int)bx - 1023;
    const uint32_t odd = (uint32_t)e & 1u;
    const uint64_t M = ((ux & kMant) | kHidden) << odd;  // [2^52, 2^54); x = M 2^(e - odd - 52)
    const int eh = (e - (int)odd) / 2;                   // exact: e - odd is even
    // Y = floor(sqrt(N)), N = M 2^54, is found in three stages on the
    // leading bits of N: T0 = N >> 62 (23-bit root), T1 = N >> 32 (+15
    // bits), T2 = N (+16 bits).  sqrt(x) = sqrt(N) 2^(eh - 53) and its
    // rounding is ((Y + 1) >> 1) 2^(eh - 52).
    //
    // Stage 0: T0 = M >> 8 in [2^44, 2^46).  The FP32 root of T0 (T0
    // truncated to 30 bits, two roundings) is within 0.77 of sqrt(T0) < 2^23.
    const uint64_t T0 = M >> 8;
    uint64_t Y = (uint64_t)(uint32_t)std::sqrt((float)(uint32_t)(M >> 24) * 65536.0f);
    int64_t R = (int64_t)(T0 - Y * Y);
    sqrt_fix(Y, R);
    // Stage 1: T1 = T0 2^30 + (M mod 2^8) 2^22.  The next digit is within
    // 2^-6 of R 2^14 / Y (the digit is below 2^15, inv = RN(1 / Y)).
    const float inv = 1.0f / (float)(uint32_t)Y;  // Y < 2^23: exact conversion
    uint32_t d = (uint32_t)((float)(uint32_t)R * (inv * 16384.0f));
    R = (int64_t)(((uint64_t)R << 30) + ((M & 0xffu) << 22) - (uint64_t)d * ((Y << 16) + d));
    Y = (Y << 15) + d;
    sqrt_fix(Y, R);
    // Stage 2: T2 = T1 2^32.  The digit (below 2^16) is within 2^-5 of
    // R 2^15 / Y ~ R inv (Y / 2^15 differs from the stage-0 root by less than
    // one part in 2^22).  R 2^32 and d (Y 2^17 + d) exceed 64 bits; their
    // wrapped difference is the true remainder, below 2^56.
    d = (uint32_t)((float)(uint32_t)((uint64_t)R >> 8) * (inv * 256.0f));
    R = (int64_t)(((uint64_t)R << 32) - (uint64_t)d * ((Y << 17) + d));
    Y = (Y << 16) + d;
    sqrt_fix(Y, R);
    const uint64_t r53 = (Y + 1) >> 1;  // in [2^52, 2^53]; 2^53 carries into the exponent
    return double_of(((uint64_t)(eh + 1023) << 52) + (r53 - kHidden));
}

}  // namespace exact
}  // namespace pmp
