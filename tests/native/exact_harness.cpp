// Host check of the library's integer / FP32 binary64 square root and
// quotient (pmp_exact.cuh) against the C library's correctly rounded sqrt and
// the host's IEEE division, bit for bit.  Inputs: random operands over the
// whole normal range, squares and quotients perturbed by a few units in the
// last place (the cases closest to a rounding boundary), significands at
// their extremes, and the exponent limits of the fast path.
#include <cstdint>
#include <cstring>

#include "pmp_exact.cuh"

namespace {

uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

double from_bits(uint64_t u)
{
    double x;
    std::memcpy(&x, &u, sizeof x);
    return x;
}

uint64_t to_bits(double x)
{
    uint64_t u;
    std::memcpy(&u, &x, sizeof u);
    return u;
}

// A random double with biased exponent in [lo, hi] and a significand that is
// uniform, all ones, or the hidden bit alone.
double rnd(uint64_t &s, uint32_t lo, uint32_t hi, int sign)
{
    const uint64_t r = splitmix(s);
    uint64_t m = r & pmp::exact::kMant;
    const uint32_t pick = (uint32_t)(splitmix(s) % 16);
    if (pick == 0) m = pmp::exact::kMant;
    if (pick == 1) m = 0;
    if (pick == 2) m = (splitmix(s) & 0xff) ;
    if (pick == 3) m = pmp::exact::kMant - (splitmix(s) & 0xff);
    const uint64_t e = lo + splitmix(s) % (uint64_t)(hi - lo + 1);
    return from_bits((sign ? pmp::exact::kSign : 0) | (e << 52) | m);
}

double nudge(double x, int64_t k) { return from_bits((uint64_t)((int64_t)to_bits(x) + k)); }

}  // namespace

extern "C" {

// Runs n checks of each kind from the seed; counts[0..3] = square roots
// checked, square roots wrong, quotients checked, quotients wrong.  The first
// mismatching operands go to bad[0..2] (x, a, b).
void exact_check(uint64_t seed, long long n, long long *counts, double *bad)
{
    uint64_t s = seed;
    long long ns = 0, bs = 0, nd = 0, bd = 0;
    auto chk_sqrt = [&](double x) {
        ++ns;
        if (to_bits(pmp::exact::sqrt_rn(x)) != to_bits(std::sqrt(x))) {
            if (bs++ == 0) bad[0] = x;
        }
    };
    auto chk_div = [&](double a, double b) {
        ++nd;
        if (to_bits(pmp::exact::div_rn(a, b)) != to_bits(a / b)) {
            if (bd++ == 0) {
                bad[1] = a;
                bad[2] = b;
            }
        }
    };
    for (long long i = 0; i < n; ++i) {
        const uint32_t kind = (uint32_t)(splitmix(s) % 8);
        // square roots
        if (kind < 3) {
            chk_sqrt(rnd(s, 1, 2046, 0));
        } else if (kind < 6) {
            const double y = rnd(s, 600, 1400, 0);
            const double x = y * y;
            chk_sqrt(nudge(x, (int64_t)(splitmix(s) % 7) - 3));
        } else if (kind == 6) {
            // exact squares: a root of at most 26 significant bits
            const double y = from_bits((to_bits(rnd(s, 700, 1300, 0)) >> 27) << 27);
            chk_sqrt(y * y);
        } else {
            const uint32_t e = (uint32_t)(splitmix(s) % 2) ? 1u + (uint32_t)(splitmix(s) % 3) : 2046u - (uint32_t)(splitmix(s) % 3);
            chk_sqrt(rnd(s, e, e, 0));
        }
        // quotients
        const int sa = (int)(splitmix(s) & 1), sb = (int)(splitmix(s) & 1);
        if (kind < 3) {
            chk_div(rnd(s, 1, 2046, sa), rnd(s, 1, 2046, sb));
        } else if (kind < 6) {
            const double b = rnd(s, 700, 1300, sb), q = rnd(s, 700, 1300, sa);
            chk_div(nudge(b * q, (int64_t)(splitmix(s) % 7) - 3), b);
        } else if (kind == 6) {
            // exact quotients: b of at most 30 and q of at most 23 significant bits
            const double b = from_bits((to_bits(rnd(s, 700, 1300, sb)) >> 23) << 23);
            const double q = from_bits((to_bits(rnd(s, 700, 1300, sa)) >> 30) << 30);
            chk_div(b * q, b);
        } else {
            // exponents at the edges of the normal result range
            const double a = rnd(s, 1, 2046, sa);
            const uint32_t ea = (uint32_t)(to_bits(a) >> 52) & 0x7ffu;
            const int lo = (int)ea - 1023 - 2, hi = (int)ea + 1023 - 2045 + 2;
            const int t = (splitmix(s) & 1) ? lo + (int)(splitmix(s) % 5) : hi - (int)(splitmix(s) % 5);
            const int eb = t < 1 ? 1 : (t > 2046 ? 2046 : t);
            chk_div(a, rnd(s, (uint32_t)eb, (uint32_t)eb, sb));
        }
    }
    counts[0] = ns;
    counts[1] = bs;
    counts[2] = nd;
    counts[3] = bd;
}

}  // extern "C"

extern "C" {

// Checks the bit-pattern comparisons of pmp_exact.cuh (x > 0, x >= 0, x < 0,
// x != 0, x > 1, x < 1) against the host's IEEE comparisons: the special
// values (signed zeros, infinities, NaNs of both signs, the smallest
// subnormals, 1 and its neighbours), then n random bit patterns and n
// random doubles near 0 and 1.  Returns the number of disagreements; the
// first disagreeing operand goes to *bad.
long long exact_check_compare(uint64_t seed, long long n, double *bad)
{
    long long wrong = 0;
    auto chk = [&](double x) {
        const bool ok = pmp::exact::positive(x) == (x > 0.0) && pmp::exact::ge0(x) == (x >= 0.0) &&
                        pmp::exact::lt0(x) == (x < 0.0) && pmp::exact::ne0(x) == (x != 0.0) &&
                        pmp::exact::gt1(x) == (x > 1.0) && pmp::exact::lt1(x) == (x < 1.0);
        if (!ok && wrong++ == 0) *bad = x;
    };
    const uint64_t special[] = {0x0ULL, 0x8000000000000000ULL, 0x1ULL, 0x8000000000000001ULL,
                                0x000fffffffffffffULL, 0x0010000000000000ULL, 0x7fefffffffffffffULL,
                                0x7ff0000000000000ULL, 0xfff0000000000000ULL, 0x7ff0000000000001ULL,
                                0x7ff8000000000000ULL, 0x7fffffffffffffffULL, 0xfff0000000000001ULL,
                                0xfff8000000000000ULL, 0xffffffffffffffffULL, 0x3ff0000000000000ULL,
                                0x3fefffffffffffffULL, 0x3ff0000000000001ULL, 0xbff0000000000000ULL,
                                0xbfefffffffffffffULL, 0xbff0000000000001ULL};
    for (uint64_t u : special) chk(from_bits(u));
    uint64_t s = seed;
    for (long long i = 0; i < n; ++i) {
        chk(from_bits(splitmix(s)));
        const uint64_t r = splitmix(s);
        const double near = (double)(int64_t)(r % 2001) / 1000.0 - 1.0;  // [-1, 1] in steps of 1e-3
        chk(near);
        chk(near + 1.0);
        chk(nudge(1.0, (int64_t)(r % 7) - 3));
    }
    return wrong;
}

}  // extern "C"

extern "C" {

// half_odd(2c + 1) against the host's (double)c + 0.5 for every c in
// [lo, hi]; returns the number of disagreements, the first c in *bad.
long long exact_check_half_odd(long long lo, long long hi, long long *bad)
{
    long long wrong = 0;
    for (long long c = lo; c <= hi; ++c) {
        const double want = (double)c + 0.5;
        if (to_bits(pmp::exact::half_odd((int)(2 * c + 1))) != to_bits(want) && wrong++ == 0) *bad = c;
    }
    return wrong;
}

}  // extern "C"
