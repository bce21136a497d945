// pmp_particles.cu -- particle-side kernels: gather, atomic deposit, the pair
// kernels of the sorted deposit, and Step 4 for sinks.
//
// One thread owns one particle and walks its kernel cells in the canonical
// order (z slowest, x fastest), so every per-particle sum has one fixed
// summation order.
#include "pmp_device.cuh"
#include "pmp_launch.h"

namespace pmp {

// ---------------------------------------------------------------------------
// gather
// ---------------------------------------------------------------------------

template <int R>
__global__ void __launch_bounds__(128) k_gather_fb(KParams P, Box S, const double *__restrict__ u, Parts p,
                                                   double *__restrict__ G, DevStatus *st)
{
    constexpr int W = 2 * R + 1;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.count) return;
    const long long gs = p.count;
    const double x = p.x[s], y = p.y[s], z = p.z[s];
    const double m = p.m[s], pe0 = p.px[s], pe1 = p.py[s], pe2 = p.pz[s], Esn = p.e[s];
    int bad = position_status(S, x, y, z);
    if (!bad && !(m > 0.0)) bad = PMP_ERR_NONFINITE;
    if (bad) {
        report(st, bad, s);
        for (int r = 0; r < FB_ROWS; ++r) G[r * gs + s] = 0.0;
        return;
    }
    Axis<R> ax, ay, az;
    ax.init(x, S.n0, S.per0);
    ay.init(y, S.n1, S.per1);
    az.init(z, S.n2, S.per2);
    double sw = 0.0, sr = 0.0, sp0 = 0.0, sp1 = 0.0, sp2 = 0.0;
    for (int oz = 0; oz < W; ++oz) {
        if (!az.in[oz]) continue;
        for (int oy = 0; oy < W; ++oy) {
            if (!ay.in[oy]) continue;
            for (int ox = 0; ox < W; ++ox) {
                if (!ax.in[ox]) continue;
                const double dd = (ax.sq[ox] + ay.sq[oy]) + az.sq[oz];
                if (!(dd < P.r2)) continue;
                const int cnt = covered_count(P, ax.c[ox], ay.c[oy], az.c[oz], x, y, z);
                if (cnt == 0) continue;
                const double w = (double)cnt / (double)P.S3;
                double U[NF];
                load_cell(u, S, S.at(ax.w[ox], ay.w[oy], az.w[oz]), U);
                sw = sw + w;
                sr = sr + w * U[0];
                sp0 = sp0 + w * U[1];
                sp1 = sp1 + w * U[2];
                sp2 = sp2 + w * U[3];
            }
        }
    }
    const double V = P.V;
    const double Vsnr = sw * V;
    const double Mgas = sr * V;
    const double Msnr = Mgas + m;
    const double vc0 = (sp0 * V + pe0) / Msnr;
    const double vc1 = (sp1 * V + pe1) / Msnr;
    const double vc2 = (sp2 * V + pe2) / Msnr;
    const double nH = Msnr / (P.mu_H * Vsnr);
    const double Msf = P.A_sf * pmp_pow(nH, -0.26);
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
        prad = P.A_p * pmp_pow(nH, -0.17);
    }
    const double vej2 = (pe0 * pe0 + pe1 * pe1) + pe2 * pe2;
    const double Ekin = vej2 / (2.0 * m);
    G[FB_MSNR * gs + s] = Msnr;
    G[FB_VSNR * gs + s] = Vsnr;
    G[FB_VX * gs + s] = vc0;
    G[FB_VY * gs + s] = vc1;
    G[FB_VZ * gs + s] = vc2;
    G[FB_NH * gs + s] = nH;
    G[FB_RM * gs + s] = RM;
    G[FB_PRAD * gs + s] = prad;
    G[FB_Q * gs + s] = m / Vsnr;
    G[FB_E * gs + s] = (Esn + Ekin) / Vsnr;
    G[FB_PV * gs + s] = prad / Vsnr;
    G[FB_REGIME * gs + s] = regime;
    if (!isfinite(Msnr) || !isfinite(nH) || !isfinite(prad) || !isfinite(Ekin)) report(st, PMP_ERR_NONFINITE, s);
}

template <int R>
__global__ void __launch_bounds__(128) k_gather_sink(KParams P, Box S, const double *__restrict__ u, Parts p,
                                                     double *__restrict__ G, DevStatus *st)
{
    constexpr int W = 2 * R + 1;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.count) return;
    const long long gs = p.count;
    const double x = p.x[s], y = p.y[s], z = p.z[s];
    const double ms = p.m[s], ps0 = p.px[s], ps1 = p.py[s], ps2 = p.pz[s];
    int bad = position_status(S, x, y, z);
    if (!bad && !(ms > 0.0)) bad = PMP_ERR_NONFINITE;
    if (bad) {
        report(st, bad, s);
        for (int r = 0; r < SK_ROWS; ++r) G[r * gs + s] = 0.0;
        return;
    }
    Axis<R> ax, ay, az;
    ax.init(x, S.n0, S.per0);
    ay.init(y, S.n1, S.per1);
    az.init(z, S.n2, S.per2);
    double srho = 0.0, sp0 = 0.0, sp1 = 0.0, sp2 = 0.0, src = 0.0;
    int nk = 0;
    for (int oz = 0; oz < W; ++oz) {
        if (!az.in[oz]) continue;
        for (int oy = 0; oy < W; ++oy) {
            if (!ay.in[oy]) continue;
            for (int ox = 0; ox < W; ++ox) {
                if (!ax.in[ox]) continue;
                const double dd = (ax.sq[ox] + ay.sq[oy]) + az.sq[oz];
                if (!(dd < P.r2)) continue;
                double U[NF], cs, rtr;
                load_cell(u, S, S.at(ax.w[ox], ay.w[oy], az.w[oz]), U);
                sink_cell(P, U, cs, rtr);
                srho = srho + U[0];
                sp0 = sp0 + U[1];
                sp1 = sp1 + U[2];
                sp2 = sp2 + U[3];
                src = src + U[0] * cs;
                ++nk;
            }
        }
    }
    const double rho_inf = srho / (double)nk;
    const double c_inf = src / srho;
    const double u0 = sp0 / srho - ps0 / ms;
    const double u1 = sp1 / srho - ps1 / ms;
    const double u2 = sp2 / srho - ps2 / ms;
    const double vinf2 = (u0 * u0 + u1 * u1) + u2 * u2;
    const double cinf2 = c_inf * c_inf;
    const double den = vinf2 + cinf2;
    const double r_bh = (P.G * ms) / den;
    const double mdot = ((P.four_pi * rho_inf) * (r_bh * r_bh)) * sqrt(P.lam2 * cinf2 + vinf2);
    double racc = r_bh / P.dx;
    if (racc < 0.25) racc = 0.25;
    if (racc > 0.5 * P.rK) racc = 0.5 * P.rK;
    const double ra2 = racc * racc;
    double ex[W], ey[W], ez[W];
#pragma unroll
    for (int o = 0; o < W; ++o) {
        ex[o] = pmp_exp(-(ax.sq[o] / ra2));
        ey[o] = pmp_exp(-(ay.sq[o] / ra2));
        ez[o] = pmp_exp(-(az.sq[o] / ra2));
    }
    double sumw = 0.0;
    for (int oz = 0; oz < W; ++oz) {
        if (!az.in[oz]) continue;
        for (int oy = 0; oy < W; ++oy) {
            if (!ay.in[oy]) continue;
            for (int ox = 0; ox < W; ++ox) {
                if (!ax.in[ox]) continue;
                const double dd = (ax.sq[ox] + ay.sq[oy]) + az.sq[oz];
                if (!(dd < P.r2)) continue;
                sumw = sumw + (ex[ox] * ey[oy]) * ez[oz];
            }
        }
    }
    double K = ((mdot * P.dt) / P.V) / sumw;
    const bool ok = (den > 0.0) && isfinite(mdot) && isfinite(K);
    if (!ok) {
        K = 0.0;
        report(st, PMP_ERR_NONFINITE, s);
    }
    G[SK_RHO * gs + s] = rho_inf;
    G[SK_VINF * gs + s] = sqrt(vinf2);
    G[SK_CINF * gs + s] = c_inf;
    G[SK_MDOT * gs + s] = mdot;
    G[SK_RACC * gs + s] = racc;
    G[SK_SUMW * gs + s] = sumw;
    G[SK_K * gs + s] = K;
    G[SK_NMEM * gs + s] = (double)nk;
}

// ---------------------------------------------------------------------------
// Step 1, atomic accumulation
// ---------------------------------------------------------------------------

template <int R>
__global__ void __launch_bounds__(128) k_deposit_fb_atomic(KParams P, Box S, const double *__restrict__ u, Box B,
                                                           double *__restrict__ b, Parts p,
                                                           const double *__restrict__ G, DevStatus *st)
{
    constexpr int W = 2 * R + 1;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.count) return;
    const long long gs = p.count;
    const double x = p.x[s], y = p.y[s], z = p.z[s];
    const int bad = position_status(S, x, y, z);
    if (bad) {
        report(st, bad, s);
        return;
    }
    const double q = G[FB_Q * gs + s], e = G[FB_E * gs + s], Pv = G[FB_PV * gs + s];
    const double vc[3] = {G[FB_VX * gs + s], G[FB_VY * gs + s], G[FB_VZ * gs + s]};
    Axis<R> ax, ay, az;
    ax.init(x, S.n0, S.per0);
    ay.init(y, S.n1, S.per1);
    az.init(z, S.n2, S.per2);
    for (int oz = 0; oz < W; ++oz) {
        if (!az.in[oz]) continue;
        for (int oy = 0; oy < W; ++oy) {
            if (!ay.in[oy]) continue;
            for (int ox = 0; ox < W; ++ox) {
                if (!ax.in[ox]) continue;
                const double dd = (ax.sq[ox] + ay.sq[oy]) + az.sq[oz];
                if (!(dd < P.r2)) continue;
                const int cnt = covered_count(P, ax.c[ox], ay.c[oy], az.c[oz], x, y, z);
                if (cnt == 0) continue;
                const double w = (double)cnt / (double)P.S3;
                double U[NF], dU[NF];
                load_cell(u, S, S.at(ax.w[ox], ay.w[oy], az.w[oz]), U);
                feedback_delta(w, U, q, e, Pv, vc, ax.d[ox], ay.d[oy], az.d[oz], dd, dU);
                const long long c = B.at(ax.c[ox], ay.c[oy], az.c[oz]);
#pragma unroll
                for (int f = 0; f < NF; ++f) atomicAdd(b + (long long)f * B.fs + c, dU[f]);
            }
        }
    }
}

template <int R>
__global__ void __launch_bounds__(128) k_deposit_sink_atomic(KParams P, Box S, const double *__restrict__ u, Box B,
                                                             double *__restrict__ b, Parts p,
                                                             const double *__restrict__ G, DevStatus *st)
{
    constexpr int W = 2 * R + 1;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.count) return;
    const long long gs = p.count;
    const double x = p.x[s], y = p.y[s], z = p.z[s];
    const int bad = position_status(S, x, y, z);
    if (bad) {
        report(st, bad, s);
        return;
    }
    const double K = G[SK_K * gs + s], racc = G[SK_RACC * gs + s];
    const double ra2 = racc * racc;
    Axis<R> ax, ay, az;
    ax.init(x, S.n0, S.per0);
    ay.init(y, S.n1, S.per1);
    az.init(z, S.n2, S.per2);
    double ex[W], ey[W], ez[W];
#pragma unroll
    for (int o = 0; o < W; ++o) {
        ex[o] = pmp_exp(-(ax.sq[o] / ra2));
        ey[o] = pmp_exp(-(ay.sq[o] / ra2));
        ez[o] = pmp_exp(-(az.sq[o] / ra2));
    }
    for (int oz = 0; oz < W; ++oz) {
        if (!az.in[oz]) continue;
        for (int oy = 0; oy < W; ++oy) {
            if (!ay.in[oy]) continue;
            for (int ox = 0; ox < W; ++ox) {
                if (!ax.in[ox]) continue;
                const double dd = (ax.sq[ox] + ay.sq[oy]) + az.sq[oz];
                if (!(dd < P.r2)) continue;
                double U[NF], dU[NF];
                load_cell(u, S, S.at(ax.w[ox], ay.w[oy], az.w[oz]), U);
                sink_delta(P, U, K, (ex[ox] * ey[oy]) * ez[oz], dU);
                const long long c = B.at(ax.c[ox], ay.c[oy], az.c[oz]);
#pragma unroll
                for (int f = 0; f < NF; ++f) atomicAdd(b + (long long)f * B.fs + c, dU[f]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Step 1, sorted accumulation: pair count, pair emission, per-cell sums
// ---------------------------------------------------------------------------

// Kernel cells that receive a contribution: members with omega > 0 (feedback)
// or members (sink).  emit = false counts, emit = true writes (cell, particle)
// pairs at offsets[s].
template <int R, bool EMIT>
__global__ void __launch_bounds__(128) k_pairs(KParams P, Box S, Box B, Parts p, long long *__restrict__ counts,
                                               const long long *__restrict__ offsets, unsigned *__restrict__ keys,
                                               int *__restrict__ vals, DevStatus *st)
{
    constexpr int W = 2 * R + 1;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.count) return;
    const double x = p.x[s], y = p.y[s], z = p.z[s];
    const int bad = position_status(S, x, y, z);
    if (bad) {
        if (!EMIT) {
            report(st, bad, s);
            counts[s] = 0;
        }
        return;
    }
    Axis<R> ax, ay, az;
    ax.init(x, S.n0, S.per0);
    ay.init(y, S.n1, S.per1);
    az.init(z, S.n2, S.per2);
    long long n = 0;
    long long off = EMIT ? offsets[s] : 0;
    for (int oz = 0; oz < W; ++oz) {
        if (!az.in[oz]) continue;
        for (int oy = 0; oy < W; ++oy) {
            if (!ay.in[oy]) continue;
            for (int ox = 0; ox < W; ++ox) {
                if (!ax.in[ox]) continue;
                const double dd = (ax.sq[ox] + ay.sq[oy]) + az.sq[oz];
                if (!(dd < P.r2)) continue;
                if (P.kind == PMP_KIND_FEEDBACK && covered_count(P, ax.c[ox], ay.c[oy], az.c[oz], x, y, z) == 0)
                    continue;
                if (EMIT) {
                    keys[off + n] = (unsigned)B.at(ax.c[ox], ay.c[oy], az.c[oz]);
                    vals[off + n] = (int)s;
                }
                ++n;
            }
        }
    }
    if (!EMIT) counts[s] = n;
}

// One thread per run of equal keys: the run's contributions are added to the
// buffer cell in ascending particle order (the radix sort is stable and pairs
// were emitted in particle order).
__global__ void __launch_bounds__(128) k_segment_sum(KParams P, Box S, const double *__restrict__ u, Box B,
                                                     double *__restrict__ b, Parts p, const double *__restrict__ G,
                                                     const unsigned *__restrict__ keys, const int *__restrict__ vals,
                                                     const long long *__restrict__ total_ptr)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = *total_ptr;
    if (i >= total) return;
    const unsigned key = keys[i];
    if (i > 0 && keys[i - 1] == key) return;
    const long long gs = p.count;
    const long long kk = (long long)key;
    const int ck = (int)(kk / B.pxy) - B.g;
    const int cj = (int)((kk % B.pxy) / B.px) - B.g;
    const int ci = (int)(kk % B.px) - B.g;
    const long long own = S.at(wrapi(ci, S.n0), wrapi(cj, S.n1), wrapi(ck, S.n2));
    double U[NF];
    load_cell(u, S, own, U);
    double acc[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) acc[f] = b[(long long)f * B.fs + kk];
    for (long long j = i; j < total && keys[j] == key; ++j) {
        const long long s = vals[j];
        const double x = p.x[s], y = p.y[s], z = p.z[s];
        const double d0 = ((double)ci + 0.5) - x, d1 = ((double)cj + 0.5) - y, d2 = ((double)ck + 0.5) - z;
        const double dd = (d0 * d0 + d1 * d1) + d2 * d2;
        double dU[NF];
        if (P.kind == PMP_KIND_FEEDBACK) {
            const int cnt = covered_count(P, ci, cj, ck, x, y, z);
            const double w = (double)cnt / (double)P.S3;
            const double vc[3] = {G[FB_VX * gs + s], G[FB_VY * gs + s], G[FB_VZ * gs + s]};
            feedback_delta(w, U, G[FB_Q * gs + s], G[FB_E * gs + s], G[FB_PV * gs + s], vc, d0, d1, d2, dd, dU);
        } else {
            const double racc = G[SK_RACC * gs + s];
            const double ra2 = racc * racc;
            const double w = (pmp_exp(-((d0 * d0) / ra2)) * pmp_exp(-((d1 * d1) / ra2))) * pmp_exp(-((d2 * d2) / ra2));
            sink_delta(P, U, G[SK_K * gs + s], w, dU);
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) acc[f] = acc[f] + dU[f];
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) b[(long long)f * B.fs + kk] = acc[f];
}

// ---------------------------------------------------------------------------
// Step 4: limited changes returned to sinks
// ---------------------------------------------------------------------------

template <int R>
__global__ void __launch_bounds__(128) k_return_sinks(KParams P, Box S, const double *__restrict__ u, Box B,
                                                      const double *__restrict__ b, Parts p,
                                                      const double *__restrict__ G, DevStatus *st)
{
    constexpr int W = 2 * R + 1;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.count) return;
    const long long gs = p.count;
    const double x = p.x[s], y = p.y[s], z = p.z[s];
    const int bad = position_status(S, x, y, z);
    if (bad) {
        report(st, bad, s);
        return;
    }
    const double K = G[SK_K * gs + s], racc = G[SK_RACC * gs + s];
    const double ra2 = racc * racc;
    Axis<R> ax, ay, az;
    ax.init(x, S.n0, S.per0);
    ay.init(y, S.n1, S.per1);
    az.init(z, S.n2, S.per2);
    double ex[W], ey[W], ez[W];
#pragma unroll
    for (int o = 0; o < W; ++o) {
        ex[o] = pmp_exp(-(ax.sq[o] / ra2));
        ey[o] = pmp_exp(-(ay.sq[o] / ra2));
        ez[o] = pmp_exp(-(az.sq[o] / ra2));
    }
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int oz = 0; oz < W; ++oz) {
        if (!az.in[oz]) continue;
        for (int oy = 0; oy < W; ++oy) {
            if (!ay.in[oy]) continue;
            for (int ox = 0; ox < W; ++ox) {
                if (!ax.in[ox]) continue;
                const double dd = (ax.sq[ox] + ay.sq[oy]) + az.sq[oz];
                if (!(dd < P.r2)) continue;
                double U[NF], dU[NF], D[NF];
                load_cell(u, S, S.at(ax.w[ox], ay.w[oy], az.w[oz]), U);
                sink_delta(P, U, K, (ex[ox] * ey[oy]) * ez[oz], dU);
                load_cell(b, B, B.at(ax.w[ox], ay.w[oy], az.w[oz]), D);
                const double eta = sink_eta(P, U, D);
                a0 = a0 + eta * dU[0];
                a1 = a1 + eta * dU[1];
                a2 = a2 + eta * dU[2];
                a3 = a3 + eta * dU[3];
            }
        }
    }
    p.m[s] = p.m[s] - a0 * P.V;
    p.px[s] = p.px[s] - a1 * P.V;
    p.py[s] = p.py[s] - a2 * P.V;
    p.pz[s] = p.pz[s] - a3 * P.V;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

static inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

#define PMP_DISPATCH_R(R_, CALL)                         \
    switch (R_) {                                        \
    case 1: { constexpr int RR = 1; CALL; } break;       \
    case 2: { constexpr int RR = 2; CALL; } break;       \
    case 3: { constexpr int RR = 3; CALL; } break;       \
    case 4: { constexpr int RR = 4; CALL; } break;       \
    case 5: { constexpr int RR = 5; CALL; } break;       \
    default: { constexpr int RR = 6; CALL; } break;      \
    }

void launch_gather(const KParams &P, const Box &S, const double *u, const Parts &p, double *G, DevStatus *st,
                   cudaStream_t stream)
{
    if (p.count == 0) return;
    const unsigned nb = blocks_for(p.count, 128);
    if (P.kind == PMP_KIND_FEEDBACK) {
        PMP_DISPATCH_R(P.R, (k_gather_fb<RR><<<nb, 128, 0, stream>>>(P, S, u, p, G, st)));
    } else {
        PMP_DISPATCH_R(P.R, (k_gather_sink<RR><<<nb, 128, 0, stream>>>(P, S, u, p, G, st)));
    }
}

void launch_deposit_atomic(const KParams &P, const Box &S, const double *u, const Box &B, double *b, const Parts &p,
                           const double *G, DevStatus *st, cudaStream_t stream)
{
    if (p.count == 0) return;
    const unsigned nb = blocks_for(p.count, 128);
    if (P.kind == PMP_KIND_FEEDBACK) {
        PMP_DISPATCH_R(P.R, (k_deposit_fb_atomic<RR><<<nb, 128, 0, stream>>>(P, S, u, B, b, p, G, st)));
    } else {
        PMP_DISPATCH_R(P.R, (k_deposit_sink_atomic<RR><<<nb, 128, 0, stream>>>(P, S, u, B, b, p, G, st)));
    }
}

void launch_pair_count(const KParams &P, const Box &S, const Box &B, const Parts &p, long long *counts,
                       DevStatus *st, cudaStream_t stream)
{
    if (p.count == 0) return;
    const unsigned nb = blocks_for(p.count, 128);
    PMP_DISPATCH_R(P.R, (k_pairs<RR, false><<<nb, 128, 0, stream>>>(P, S, B, p, counts, nullptr, nullptr, nullptr,
                                                                     st)));
}

void launch_pair_emit(const KParams &P, const Box &S, const Box &B, const Parts &p, const long long *offsets,
                      unsigned *keys, int *vals, DevStatus *st, cudaStream_t stream)
{
    if (p.count == 0) return;
    const unsigned nb = blocks_for(p.count, 128);
    PMP_DISPATCH_R(P.R, (k_pairs<RR, true><<<nb, 128, 0, stream>>>(P, S, B, p, nullptr, offsets, keys, vals, st)));
}

void launch_segment_sum(const KParams &P, const Box &S, const double *u, const Box &B, double *b, const Parts &p,
                        const double *G, const unsigned *keys, const int *vals, const long long *total_dev,
                        long long total, cudaStream_t stream)
{
    if (total == 0) return;
    k_segment_sum<<<blocks_for(total, 128), 128, 0, stream>>>(P, S, u, B, b, p, G, keys, vals, total_dev);
}

void launch_return_sinks(const KParams &P, const Box &S, const double *u, const Box &B, const double *b,
                         const Parts &p, const double *G, DevStatus *st, cudaStream_t stream)
{
    if (p.count == 0) return;
    const unsigned nb = blocks_for(p.count, 128);
    PMP_DISPATCH_R(P.R, (k_return_sinks<RR><<<nb, 128, 0, stream>>>(P, S, u, B, b, p, G, st)));
}

}  // namespace pmp
