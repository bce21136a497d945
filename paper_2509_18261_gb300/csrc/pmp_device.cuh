// pmp_device.cuh -- device-side building blocks of the PMP library (sm_103a).
//
// Everything here is FP64 and is compiled with -fmad=false: each product and
// sum is rounded on its own, in the order written, except where the code calls
// fma() (one rounding), so that one quantity has one value whichever kernel
// computes it (gather, deposit, sorted segment sum, Step 4).  That fixed order
// is the contract that makes the sorted deposit deterministic.  Products that
// feed a running sum or another term are fused where the oracle fuses them:
// the supernova gather sums, the sum of kernel weights, the momentum and
// energy rows of Eq. du and the Step-4 sums (a DFMA costs the FP64 pipe what a
// DADD or DMUL costs).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pmp.h"
#include "pmp_exact.cuh"

namespace pmp {

constexpr int NF = 5;
constexpr double kEpsMachine = 2.220446049250313e-16;  // 2^-52, the FP64 machine epsilon
constexpr double kPi = 3.141592653589793;
constexpr int kMaxR = 6;
constexpr int kMaxS = 8;

// Geometry of one mesh as the kernels see it.
struct Box {
    int n0, n1, n2, g;
    int per0, per1, per2, pad_;
    long long px, pxy;  // padded row length and padded plane size
    long long fs;       // field stride (doubles)
    long long ncells;   // padded cell count

    __host__ __device__ __forceinline__ long long at(int i, int j, int k) const
    {
        return (long long)(k + g) * pxy + (long long)(j + g) * px + (long long)(i + g);
    }
};

// Parameters with the derived constants each formula uses, all computed on
// the host in the same order as the formulas below state them.
struct KParams {
    double rK, r2;   // r_K, r_K * r_K
    double dt, G;
    double gg;       // gamma * (gamma - 1)
    double lam2;     // lambda_bh * lambda_bh
    double ctr;      // ((J * J) * pi) / (G * (dx * dx)): rho_Tr = ctr c_s^2
    double cap, rho_min;
    double A_sf, A_p, mu_H, RM_ej, RM_st, eps_K;
    double V, dx;    // V = (dx * dx) * dx
    double four_pi;  // 4 * pi
    double frac[8];  // (a + 1/2) / S, a < S: sub-point positions inside a cell
    int S, S3, R, kind;
    int Slog;        // log2(S) when S is a power of two, else -1
    float fracf[8];  // frac[] rounded to FP32
    float band_lo, band_hi;  // r2 (1 -/+ 2^-14) rounded outward to FP32
    float cap_lo, rho_min_hi;  // cap rounded down, rho_min rounded up to FP32
};

struct Parts {
    long long count;
    const double *x, *y, *z;
    double *m, *px, *py, *pz;
    const double *e;
};

// Device status words of a context.
struct DevStatus {
    int code;
    int pad_;
    long long index;
    unsigned long long n_limited;
    unsigned long long n_noroot;
};

__device__ __forceinline__ void report(DevStatus *st, int code, long long index)
{
    if (atomicCAS(&st->code, 0, code) == 0) st->index = index;
}

__device__ __forceinline__ int wrapi(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
// exp and log (the library's own; see pmp.h)
// ---------------------------------------------------------------------------

// ln 2 = 0.6931471805599453094172321...: kLn2Hi holds its leading 32
// significant bits (so k * kLn2Hi is exact for |k| < 2^21), kLn2Lo the rest
// rounded to double.  This two-part split of ln 2 (and 1/ln 2) is the one
// Cody & Waite's reduction uses; the published fdlibm library prints the
// same digits.  The log arrangement f - (hf - s (hf + R)) below also follows
// fdlibm's published e_log; the polynomials are this library's own.
constexpr double kLn2Hi = 6.93147180369123816490e-01;
constexpr double kLn2Lo = 1.90821492927058770002e-10;
constexpr double kInvLn2 = 1.44269504088896338700e+00;

__host__ __device__ constexpr double fact_d(int j) { return j <= 1 ? 1.0 : (double)j * fact_d(j - 1); }

// 2^k for -1022 <= k <= 1023 (exact).
__device__ __forceinline__ double two_to(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// exp(x) by Cody & Waite reduction x = k ln2 + r (|r| <= ln2 / 2), the
// degree-13 Taylor polynomial of e^r in Horner form (coefficients 1/j!,
// correctly rounded; j! is exact), and scaling by 2^k.
__device__ __forceinline__ double pmp_exp(double x)
{
    if (x != x) return x;
    if (x > 709.79) return __longlong_as_double(0x7ff0000000000000LL);
    if (x < -745.2) return 0.0;
    const double kd = floor(x * kInvLn2 + 0.5);
    const int k = (int)kd;
    const double r = (x - kd * kLn2Hi) - kd * kLn2Lo;
    constexpr double c13 = 1.0 / fact_d(13), c12 = 1.0 / fact_d(12), c11 = 1.0 / fact_d(11),
                     c10 = 1.0 / fact_d(10), c9 = 1.0 / fact_d(9), c8 = 1.0 / fact_d(8), c7 = 1.0 / fact_d(7),
                     c6 = 1.0 / fact_d(6), c5 = 1.0 / fact_d(5), c4 = 1.0 / fact_d(4), c3 = 1.0 / fact_d(3),
                     c2 = 1.0 / fact_d(2);
    double p = c13;
    p = p * r + c12;
    p = p * r + c11;
    p = p * r + c10;
    p = p * r + c9;
    p = p * r + c8;
    p = p * r + c7;
    p = p * r + c6;
    p = p * r + c5;
    p = p * r + c4;
    p = p * r + c3;
    p = p * r + c2;
    p = p * r + 1.0;
    p = p * r + 1.0;
    if (k < -1000) return (p * two_to(k + 200)) * two_to(-200);
    if (k > 1000) return (p * two_to(k - 200)) * two_to(200);
    return p * two_to(k);
}

// log(x), x > 0: x = 2^e (1 + f), 1 + f in [sqrt(1/2), sqrt(2)); with
// s = f / (2 + f), z = s^2, R = sum_{j=1..11} 2 z^j / (2j + 1) and hf = f^2/2,
// log(1 + f) = 2 atanh(s) = f - (hf - s (hf + R)); log x = e ln2 + log(1 + f)
// with the small terms added first.
__device__ __forceinline__ double pmp_log(double x)
{
    if (x != x || x < 0.0) return __longlong_as_double(0x7ff8000000000000LL);
    if (x == 0.0) return __longlong_as_double(0xfff0000000000000LL);
    if (isinf(x)) return x;
    int e;
    double m = frexp(x, &e);  // exact: x = m 2^e, m in [0.5, 1)
    m = m * 2.0;
    e = e - 1;
    if (m > 1.4142135623730951) {
        m = m * 0.5;
        e = e + 1;
    }
    const double f = m - 1.0;
    const double s = f / (2.0 + f);
    const double z = s * s;
    double R = 2.0 / 23.0;
    R = R * z + 2.0 / 21.0;
    R = R * z + 2.0 / 19.0;
    R = R * z + 2.0 / 17.0;
    R = R * z + 2.0 / 15.0;
    R = R * z + 2.0 / 13.0;
    R = R * z + 2.0 / 11.0;
    R = R * z + 2.0 / 9.0;
    R = R * z + 2.0 / 7.0;
    R = R * z + 2.0 / 5.0;
    R = R * z + 2.0 / 3.0;
    R = R * z;
    const double hf = 0.5 * (f * f);
    const double ed = (double)e;
    return ed * kLn2Hi - ((hf - (s * (hf + R) + ed * kLn2Lo)) - f);
}

__device__ __forceinline__ double pmp_pow(double x, double a) { return pmp_exp(a * pmp_log(x)); }

// FP64 -> FP32 by truncating the significand, with integer operations only
// (the FP64 pipe of this GPU is scarce).  |result - v| <= 2^-23 |v| for
// 2^-126 <= |v| < 2^128; returns exactly 0 for +-0 and NaN outside that range.
__device__ __forceinline__ float f32_trunc(double v)
{
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e <= 0 || e >= 255) return ((hi & 0x7fffffffu) | lo) == 0u ? 0.0f : __int_as_float(0x7fc00000);
    return __uint_as_float((hi & 0x80000000u) | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// ---------------------------------------------------------------------------
// per-cell formulas
// ---------------------------------------------------------------------------

__device__ __forceinline__ void load_cell(const double *__restrict__ u, const Box &B, long long c, double U[NF])
{
#pragma unroll
    for (int f = 0; f < NF; ++f) U[f] = __ldg(u + (long long)f * B.fs + c);
}

// Every quotient by rho in the sink formulas is a product with the one
// reciprocal inv = 1/rho of the cell (one division per cell instead of five).
// Ideal-gas c_s^2 = gamma (gamma - 1) e_int / rho, e_int = E - |p|^2 / (2 rho)
// clamped at 0, evaluated as e_int = E - |p|^2 (inv/2) and c_s^2 =
// (gamma (gamma - 1) e_int) inv; c_s; and rho_Tr = J^2 pi c_s^2 / (G dx^2)
// (Eq. truelove).
__device__ __forceinline__ double sink_cs2(const KParams &P, const double U[NF], double inv)
{
    const double ke2 = (U[1] * U[1] + U[2] * U[2]) + U[3] * U[3];
    double eint = U[4] - ke2 * (0.5 * inv);
    if (exact::lt0(eint)) eint = 0.0;  // eint < 0, decided on the bits
    return (P.gg * eint) * inv;
}

__device__ __forceinline__ void sink_cell(const KParams &P, const double U[NF], double inv, double &cs,
                                          double &rho_tr)
{
    const double cs2 = sink_cs2(P, U, inv);
    cs = exact::sqrt_rn(cs2);
    rho_tr = P.ctr * cs2;
}

__device__ __forceinline__ double sink_rho_tr(const KParams &P, const double U[NF])
{
    return P.ctr * sink_cs2(P, U, exact::div_rn(1.0, U[0]));
}

// Accretion limiter of Sec. 3.1.1 composed with the density floor, on the
// removal a = -drho: a_lim = max(0, min(max(min(a, cap rho), rho - rho_Tr),
// rho - rho_min)), eta = a_lim / a if a_lim < a else 1.  When a <= cap rho and
// a <= rho - rho_min, a_lim >= a follows from the definition, so eta = 1
// without computing rho_Tr.
__device__ __forceinline__ double sink_eta(const KParams &P, const double U[NF], const double D[NF])
{
    const double a = -D[0];
    if (!(a > 0.0)) return 1.0;
    const double rho = U[0];
    const double capr = P.cap * rho;
    const double fl = rho - P.rho_min;
    if (a <= capr && a <= fl) return 1.0;
    const double rtr = sink_rho_tr(P, U);
    double al = a < capr ? a : capr;
    const double t = rho - rtr;
    al = al > t ? al : t;
    al = al < fl ? al : fl;
    if (al < 0.0) al = 0.0;
    return al < a ? exact::div_rn(al, a) : 1.0;
}

// Supernova momentum limiter (Eq. lambda) with T the pre-deposit temperature:
// lambda = 1 if the constraint holds at 1; otherwise the largest root in
// [0, 1] of |dp|^2 l^2 + 2 (p . dp) l + |p|^2 - 2 rho' (E' - e_int0 rho'/rho),
// from the cancellation-free quadratic formula (Press et al., Numerical
// Recipes, Sec. 5.6); 0 if there is none (noroot set).  sn_lambda_dp is the
// limiter for a change whose momentum is not zero (no test for Delta p = 0),
// and returns rho' = U_0 + D_0 and E' = U_4 + D_4 for the update.
__device__ __forceinline__ double sn_lambda_dp(const double U[NF], const double D[NF], int &noroot, double &rho1,
                                               double &E1)
{
    noroot = 0;
    rho1 = U[0] + D[0];
    E1 = U[4] + D[4];
    const double p2 = (U[1] * U[1] + U[2] * U[2]) + U[3] * U[3];
    const double eint0 = U[4] - exact::div_rn(p2, 2.0 * U[0]);
    const double pn0 = U[1] + D[1], pn1 = U[2] + D[2], pn2 = U[3] + D[3];
    const double pnn = (pn0 * pn0 + pn1 * pn1) + pn2 * pn2;
    const double therm = exact::div_rn(eint0 * rho1, U[0]);
    const double lhs = therm + exact::div_rn(pnn, 2.0 * rho1);
    if (lhs <= E1) return 1.0;
    const double A = (D[1] * D[1] + D[2] * D[2]) + D[3] * D[3];
    if (!exact::positive(A)) return 1.0;  // !(A > 0)
    const double B = (U[1] * D[1] + U[2] * D[2]) + U[3] * D[3];
    const double C = p2 - (2.0 * rho1) * (E1 - therm);
    const double disc = B * B - A * C;
    if (!exact::ge0(disc)) {
        noroot = 1;
        return 0.0;
    }
    const double sq = exact::sqrt_rn(disc);
    double hi, lo;
    if (exact::ge0(B)) {
        const double Q = -(B + sq);
        hi = exact::ne0(Q) ? exact::div_rn(C, Q) : 0.0;
        lo = exact::div_rn(Q, A);
    } else {
        const double Q = sq - B;
        hi = exact::div_rn(Q, A);
        lo = exact::div_rn(C, Q);
    }
    if (exact::lt0(hi) || exact::gt1(lo)) {
        noroot = 1;
        return 0.0;
    }
    return exact::lt1(hi) ? hi : 1.0;
}

__device__ __forceinline__ double sn_lambda(const double U[NF], const double D[NF], int &noroot)
{
    noroot = 0;
    if (((exact::bits_of(D[1]) | exact::bits_of(D[2]) | exact::bits_of(D[3])) << 1) == 0) return 1.0;  // Delta p = 0
    double rho1, E1;
    return sn_lambda_dp(U, D, noroot, rho1, E1);
}

// ---------------------------------------------------------------------------
// kernel geometry of one particle
// ---------------------------------------------------------------------------

// Per-axis data of a particle's kernel: for offset o in [-R, R] the unwrapped
// cell c = host + o, its owning valid index, whether it is inside the domain
// (always on a periodic axis), and the centre offset d = (c + 1/2) - x.
template <int R>
struct Axis {
    static constexpr int W = 2 * R + 1;
    int c[W];
    int w[W];
    bool in[W];
    double d[W];
    double sq[W];

    __device__ __forceinline__ void init(double x, int n, int per)
    {
        const int h = (int)floor(x);
#pragma unroll
        for (int o = 0; o < W; ++o) {
            const int ci = h + o - R;
            c[o] = ci;
            w[o] = wrapi(ci, n);
            in[o] = per || (ci >= 0 && ci < n);
            d[o] = ((double)ci + 0.5) - x;
            sq[o] = d[o] * d[o];
        }
    }
};

// Sub-points per axis of a cell for the covered fraction: ((c + (a + 1/2)/S) - x)^2.
__device__ __forceinline__ void sub_squares(int S, int c, double x, double out[kMaxS])
{
    for (int a = 0; a < S; ++a) {
        const double t = ((double)c + ((double)a + 0.5) / (double)S) - x;
        out[a] = t * t;
    }
}

// Number of the S^3 sub-points of cell (ci, cj, ck) strictly inside r_K.  A
// cell whose farthest corner is inside has all S^3 (each sub-point offset is
// bounded by the corner offset, and rounding is monotone).
__device__ __forceinline__ int covered_count(const KParams &P, int ci, int cj, int ck, double x, double y, double z)
{
    const int S = P.S;
    {
        const double ax0 = fabs((double)ci - x), ax1 = fabs(((double)ci + 1.0) - x);
        const double ay0 = fabs((double)cj - y), ay1 = fabs(((double)cj + 1.0) - y);
        const double az0 = fabs((double)ck - z), az1 = fabs(((double)ck + 1.0) - z);
        const double fx = ax0 > ax1 ? ax0 : ax1, fy = ay0 > ay1 ? ay0 : ay1, fz = az0 > az1 ? az0 : az1;
        if ((fx * fx + fy * fy) + fz * fz < P.r2) return P.S3;
    }
    double sx[kMaxS], sy[kMaxS], sz[kMaxS];
    sub_squares(S, ci, x, sx);
    sub_squares(S, cj, y, sy);
    sub_squares(S, ck, z, sz);
    int cnt = 0;
    for (int c = 0; c < S; ++c)
        for (int b = 0; b < S; ++b) {
            for (int a = 0; a < S; ++a) cnt += ((sx[a] + sy[b]) + sz[c] < P.r2) ? 1 : 0;
        }
    return cnt;
}

// Feedback deposition function (Eq. du, with omega on every row; see pmp.h).
// G points at the particle's gathered row 0 with row stride gs.
__device__ __forceinline__ void feedback_delta(double w, const double U[NF], double q, double e, double Pv,
                                               const double vc[3], double d0, double d1, double d2, double dd,
                                               double dU[NF])
{
    const double rn = U[0] + q;
    // sqrt and the quotient by integer digit recurrence (pmp_exact.cuh): the
    // same correctly rounded values, off the FP64 pipe
    const double s = exact::positive(dd) ? exact::div_rn(w * Pv, exact::sqrt_rn(dd)) : 0.0;
    const double pr0 = s * d0, pr1 = s * d1, pr2 = s * d2;
    dU[0] = w * q;
    dU[1] = fma(w, fma(rn, vc[0], -U[1]), pr0);
    dU[2] = fma(w, fma(rn, vc[1], -U[2]), pr1);
    dU[3] = fma(w, fma(rn, vc[2], -U[3]), pr2);
    dU[4] = fma(w, e, fma(vc[2], pr2, fma(vc[1], pr1, vc[0] * pr0)));
}

// max(b, x) for b >= +0 and x not NaN, as a comparison of the 64-bit
// patterns: non-negative doubles order like their patterns, and a negative x
// (or -0) has a negative pattern.  The same value as b >= x ? b : x, off the
// FP64 pipe (an FP64 comparison occupies it like an addition).
__device__ __forceinline__ double max_nonneg(double b, double x)
{
    return __double_as_longlong(b) >= __double_as_longlong(x) ? b : x;
}

// -x by flipping the sign bit (exact, off the FP64 pipe).
__device__ __forceinline__ double neg_bits(double x)
{
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}

// Sink deposition function (Eq. accretion_function with the Truelove rate in
// the max): a = max(K w, rho - rho_Tr), Delta U = -a (1, p inv, E inv).
__device__ __forceinline__ void sink_delta(const KParams &P, const double U[NF], double K, double w, double dU[NF])
{
    const double inv = exact::div_rn(1.0, U[0]);
    const double rtr = P.ctr * sink_cs2(P, U, inv);
    const double bh = K * w;
    const double tr = U[0] - rtr;
    const double a = bh >= tr ? bh : tr;
    dU[0] = -a;
    dU[1] = -(a * (U[1] * inv));
    dU[2] = -(a * (U[2] * inv));
    dU[3] = -(a * (U[3] * inv));
    dU[4] = -(a * (U[4] * inv));
}

// Per-cell sink quantities (valid cells, x fastest), inv = 1/rho:
//   G record (gather), 4 doubles = 32 bytes (one sector):  rho, p_x, p_y, p_z
//   D record (spread, Step 4), 4 doubles = 32 bytes (one sector):  p_x inv, p_y inv, p_z inv, E inv
//   rho c_s (gather), rho - rho_Tr (deposit, limiter) and eta (Step 4) in dense arrays of their
//   own, so that a kernel reads 8 bytes per cell for each of them, not a record
constexpr int kGRec = 4;
constexpr int kDRec = 4;
// Bytes per cell the L2 windows of the sink kernels are sized with (the
// launch shapes were measured with this figure).
constexpr double kWindowBytesPerCell = 48.0;

// Gathered-row indices.
enum { FB_MSNR = 0, FB_VSNR, FB_VX, FB_VY, FB_VZ, FB_NH, FB_RM, FB_PRAD, FB_Q, FB_E, FB_PV, FB_REGIME, FB_ROWS };
enum { SK_RHO = 0, SK_VINF, SK_CINF, SK_MDOT, SK_RACC, SK_SUMW, SK_K, SK_NMEM, SK_ROWS };
enum { MS_VK = 0, MS_Q, MS_ROWS = MS_Q + NF };  // V_K, then (m, p, e) / V_K

// ---------------------------------------------------------------------------
// gathered rows from the kernel sums (shared by the single-box and batched
// gathers; the order of every operation is the oracle's)
// ---------------------------------------------------------------------------

// The per-particle formulas keep the compiler's FP64 division and sqrt: they
// run once per particle, and the integer forms of pmp_exact.cuh inlined at
// their dozen call sites made the fused plan + gather kernels' code large
// enough to stall on instruction fetch (512^3: 25.0 -> 29.0 ms).  The
// per-pair and per-cell formulas use the integer forms.

// Quotients and square roots of the per-sink formulas: the integer forms of
// pmp_exact.cuh (the same correctly rounded values, off the FP64 pipe)
// through one out-of-line copy each, so that their dozen call sites do not
// enlarge the kernels' code (512^3: sink plan + gather + deposit 23.5 -> 23.2
// ms).  The supernova rows keep the compiler's FP64 sequences: the integer
// forms made the supernova plan + gather slower (25.0 -> 26.5 ms).
static __device__ __noinline__ double row_div(double a, double b) { return exact::div_rn(a, b); }
static __device__ __noinline__ double row_sqrt(double x) { return exact::sqrt_rn(x); }

// Sec. 3.2.1 from the omega-weighted sums over the kernel: sw = sum omega,
// sr = sum omega rho, sp = sum omega p.  Writes the 12 feedback rows of one
// particle (G at its row 0, row stride gs); false if a result is not finite.
__device__ __forceinline__ bool fb_gather_rows(const KParams &P, double sw, double sr, double sp0, double sp1,
                                               double sp2, double m, double pe0, double pe1, double pe2, double Esn,
                                               double *G, long long gs)
{
    const double V = P.V;
    const double Vsnr = sw * V;
    const double Mgas = sr * V;
    const double Msnr = Mgas + m;
    const double vc0 = (sp0 * V + pe0) / Msnr;
    const double vc1 = (sp1 * V + pe1) / Msnr;
    const double vc2 = (sp2 * V + pe2) / Msnr;
    const double nH = Msnr / (P.mu_H * Vsnr);
    // both powers of n_H are exp(a log n_H): the logarithm is taken once
    const double lnH = pmp_log(nH);
    const double Msf = P.A_sf * pmp_exp(-0.26 * lnH);
    const double RM = Msnr / Msf;
    double regime, prad;
    if (RM <= P.RM_ej) {
        regime = 0.0;
        prad = 0.0;
    } else if (RM <= P.RM_st) {
        regime = 1.0;
        prad = sqrt(((2.0 * m) * P.eps_K) * Esn);
    } else {
        regime = 2.0;
        prad = P.A_p * pmp_exp(-0.17 * lnH);
    }
    const double vej2 = (pe0 * pe0 + pe1 * pe1) + pe2 * pe2;
    const double Ekin = vej2 / (2.0 * m);
    G[FB_MSNR * gs] = Msnr;
    G[FB_VSNR * gs] = Vsnr;
    G[FB_VX * gs] = vc0;
    G[FB_VY * gs] = vc1;
    G[FB_VZ * gs] = vc2;
    G[FB_NH * gs] = nH;
    G[FB_RM * gs] = RM;
    G[FB_PRAD * gs] = prad;
    G[FB_Q * gs] = m / Vsnr;
    G[FB_E * gs] = (Esn + Ekin) / Vsnr;
    G[FB_PV * gs] = prad / Vsnr;
    G[FB_REGIME * gs] = regime;
    return isfinite(Msnr) && isfinite(nH) && isfinite(prad) && isfinite(Ekin);
}

// Sec. 3.1.1, first half: from the kernel sums srho = sum rho, sp = sum p and
// src = sum rho c_s over nk cells, the ambient state, r_BH, mdot_BH and
// r_acc (cell units, clamped to [1/4, r_K / 2]).
struct SinkAmbient {
    double rho_inf, vinf2, c_inf, den, mdot, racc, ra2;
};

__device__ __forceinline__ SinkAmbient sink_ambient(const KParams &P, double srho, double sp0, double sp1, double sp2,
                                                    double src, int nk, double ms, double ps0, double ps1, double ps2)
{
    SinkAmbient a;
    a.rho_inf = row_div(srho, (double)nk);
    a.c_inf = row_div(src, srho);
    const double u0 = row_div(sp0, srho) - row_div(ps0, ms);
    const double u1 = row_div(sp1, srho) - row_div(ps1, ms);
    const double u2 = row_div(sp2, srho) - row_div(ps2, ms);
    a.vinf2 = (u0 * u0 + u1 * u1) + u2 * u2;
    const double cinf2 = a.c_inf * a.c_inf;
    a.den = a.vinf2 + cinf2;
    const double r_bh = row_div(P.G * ms, a.den);
    a.mdot = ((P.four_pi * a.rho_inf) * (r_bh * r_bh)) * row_sqrt(P.lam2 * cinf2 + a.vinf2);
    double racc = row_div(r_bh, P.dx);
    if (racc < 0.25) racc = 0.25;
    if (racc > 0.5 * P.rK) racc = 0.5 * P.rK;
    a.racc = racc;
    a.ra2 = racc * racc;
    return a;
}

// Per-axis Gaussian factor exp(-d^2 / r_acc^2) of the cell centred d away.
__device__ __forceinline__ double sink_axis_weight(double d, double ra2) { return pmp_exp(-row_div(d * d, ra2)); }

// Second half: K = mdot dt / (V sum w) and the 8 sink rows; false (and K = 0)
// if a result is not finite.
__device__ __forceinline__ bool sink_gather_rows(const KParams &P, const SinkAmbient &a, double sumw, int nk, double *G,
                                                 long long gs)
{
    double K = row_div(row_div(a.mdot * P.dt, P.V), sumw);
    const bool ok = (a.den > 0.0) && isfinite(a.mdot) && isfinite(K);
    if (!ok) K = 0.0;
    G[SK_RHO * gs] = a.rho_inf;
    G[SK_VINF * gs] = row_sqrt(a.vinf2);
    G[SK_CINF * gs] = a.c_inf;
    G[SK_MDOT * gs] = a.mdot;
    G[SK_RACC * gs] = a.racc;
    G[SK_SUMW * gs] = sumw;
    G[SK_K * gs] = K;
    G[SK_NMEM * gs] = (double)nk;
    return ok;
}

// True when every field of D is +0 or -0 (integer test; no FP64 instruction).
// A cell whose summed change is zero in every field receives nothing in
// Step 5 and is left as it is.
__device__ __forceinline__ bool all_zero(const double D[NF])
{
    unsigned long long acc = 0;
#pragma unroll
    for (int f = 0; f < NF; ++f) acc |= (unsigned long long)__double_as_longlong(D[f]) << 1;
    return acc == 0;
}

// App. A.1 rounding of one buffer value v with error bound e: r = e / |v|,
// N_bit = ceil(log2 r) + 52 + M clamped to [0, 52], and the low N_bit bits of
// the significand set to zero (truncation toward zero).  v = 0 or e = 0 is
// left as it is.
__device__ __forceinline__ double repro_round(double v, double e, int M)
{
    if (v == 0.0 || !(e > 0.0)) return v;
    const double r = exact::div_rn(e, fabs(v));
    if (!(r > 0.0)) return v;  // underflow: N_bit < 0
    int nb = 52;
    if (r < 1.0) {
        int k;
        const double m = frexp(r, &k);       // r = m 2^k, m in [1/2, 1)
        const int c = m == 0.5 ? k - 1 : k;  // ceil(log2 r)
        nb = c + 52 + M;
        nb = nb < 0 ? 0 : (nb > 52 ? 52 : nb);
    }
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    return __longlong_as_double((long long)(bits & ~((1ULL << nb) - 1ULL)));
}

// Position check: 0 <= x < n on each axis (NaN fails).
__device__ __forceinline__ int position_status(const Box &B, double x, double y, double z)
{
    if (!(x == x && y == y && z == z)) return PMP_ERR_NONFINITE;
    if (!(x >= 0.0 && x < (double)B.n0 && y >= 0.0 && y < (double)B.n1 && z >= 0.0 && z < (double)B.n2))
        return PMP_ERR_PARTICLE_OUTSIDE;
    return PMP_OK;
}

}  // namespace pmp
