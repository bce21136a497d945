// pmp_particles.cu -- particle-side kernels.
//
//   plan      one warp per particle (spatial processing order): lanes test the
//             (2R+1)^3 candidate cells; omega by a warp-wide ballot over the
//             S^3 sub-points; kernel cells with omega > 0 written in canonical
//             order (z slowest, x fastest) to the particle's fixed slot range
//   gather    one thread per particle over its cells in that order, so every
//             per-particle sum has one fixed summation order
//   deposit   one warp per 8 consecutive particles, lanes over their pairs,
//             FP64 atomics into the buffer
//   sorted    pairs stably sorted by buffer cell, one thread per cell adding
//             its pairs in particle-index order
//   return    Step 4 for sinks, one thread per sink over its cells
#include "pmp_device.cuh"
#include "pmp_launch.h"
#include "pmp_plan.cuh"

namespace pmp {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// processing order: particles keyed by host cell (spatial locality)
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned spread3(unsigned v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Key of a particle: Morton (Z-order) code of its host cell (coordinates
// shifted right by `sh` so that each fits in 10 bits); invalid positions sort
// last.  Consecutive particles of this order have overlapping kernels.
__global__ void __launch_bounds__(256) k_host_keys(Box S, Parts p, int sh, unsigned *__restrict__ keys,
                                                   unsigned *__restrict__ ids)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.count) return;
    const double x = p.x[s], y = p.y[s], z = p.z[s];
    unsigned key = 0xffffffffu;
    if (position_status(S, x, y, z) == PMP_OK) {
        const unsigned hx = (unsigned)(int)floor(x) >> sh, hy = (unsigned)(int)floor(y) >> sh,
                       hz = (unsigned)(int)floor(z) >> sh;
        key = spread3(hx) | (spread3(hy) << 1) | (spread3(hz) << 2);
    }
    keys[s] = key;
    ids[s] = (unsigned)s;
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------

// shared floats per warp: edges [3][W+1], centre squares [3][W], farthest-corner
// squares [3][W], sub-point squares [3][W*S]
__host__ __device__ constexpr int plan_warp_floats(int W, int S) { return 3 * (W + 1) + 6 * W + 3 * W * S; }

template <int R, bool FB>
__global__ void __launch_bounds__(256) k_plan(KParams P, Box S, Parts p, const unsigned *__restrict__ perm,
                                              unsigned cap, unsigned *__restrict__ counts,
                                              unsigned long long *__restrict__ slots,
                                              unsigned long long *__restrict__ hosts, DevStatus *st)
{
    constexpr int W = 2 * R + 1;
    constexpr int W3 = W * W * W;
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long t = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
    if (t >= p.count) return;  // warp-uniform
    const int Sn = P.S;
    float *edge = smem + (size_t)wib * plan_warp_floats(W, FB ? Sn : 1);  // [3][W+1]
    float *csq = edge + 3 * (W + 1);                                       // [3][W]
    float *fc2 = csq + 3 * W;                                              // [3][W]
    float *sub = fc2 + 3 * W;                                              // [3][W*S]
    const long long s = perm ? (long long)perm[t] : t;
    const double x = p.x[s], y = p.y[s], z = p.z[s];
    const int bad = position_status(S, x, y, z);
    if (bad) {
        if (lane == 0) {
            report(st, bad, s);
            counts[t] = 0;
        }
        return;
    }
    const int h0 = (int)floor(x), h1 = (int)floor(y), h2 = (int)floor(z);
    if (lane == 0 && hosts) hosts[s] = pack_host(h0, h1, h2);
    for (int i = lane; i < 3 * (W + 1); i += 32) {
        const int a = i / (W + 1), o = i - a * (W + 1);
        const int h = a == 0 ? h0 : (a == 1 ? h1 : h2);
        const double xa = a == 0 ? x : (a == 1 ? y : z);
        edge[i] = (float)((double)(h + o - R) - xa);
    }
    __syncwarp();
    for (int i = lane; i < 3 * W; i += 32) {
        const int a = i / W, o = i - a * W;
        const float e0 = edge[a * (W + 1) + o], e1 = edge[a * (W + 1) + o + 1];
        const float c = e0 + 0.5f;
        csq[i] = c * c;
        const float m = fabsf(e0) > fabsf(e1) ? fabsf(e0) : fabsf(e1);
        fc2[i] = m * m;
    }
    if (FB) {
        for (int i = lane; i < 3 * W * Sn; i += 32) {
            const int a = i / (W * Sn), r = i - a * (W * Sn), o = r / Sn, k = r - o * Sn;
            const float u = edge[a * (W + 1) + o] + (float)P.frac[k];
            sub[i] = u * u;
        }
    }
    __syncwarp();
    const R2Band band = make_band(P.r2);
    unsigned nout = 0;
    const unsigned long long base = (unsigned long long)t * cap;
    for (int k0 = 0; k0 < W3; k0 += 32) {
        const int k = k0 + lane;
        int ox = 0, oy = 0, oz = 0;
        bool mem = false, full = false;
        if (k < W3) {
            oz = k / (W * W);
            oy = k / W - oz * W;
            ox = k - (k / W) * W;
            const int c0 = h0 + ox - R, c1 = h1 + oy - R, c2 = h2 + oz - R;
            const bool dom = (S.per0 || (c0 >= 0 && c0 < S.n0)) && (S.per1 || (c1 >= 0 && c1 < S.n1)) &&
                             (S.per2 || (c2 >= 0 && c2 < S.n2));
            if (dom) {
                const float tf = (csq[ox] + csq[W + oy]) + csq[2 * W + oz];
                if (tf < band.lo) mem = true;
                else if (tf <= band.hi) mem = centre_inside_exact(P.r2, c0, c1, c2, x, y, z);
                if (FB && mem) full = (fc2[ox] + fc2[W + oy]) + fc2[2 * W + oz] < band.lo;
            }
        }
        int cnt = 0;
        if (FB) {
            cnt = full ? P.S3 : 0;
            unsigned need = __ballot_sync(kFull, mem && !full);
            while (need) {
                const int src = __ffs(need) - 1;
                need &= need - 1;
                const int cx = __shfl_sync(kFull, ox, src), cy = __shfl_sync(kFull, oy, src),
                          cz = __shfl_sync(kFull, oz, src);
                const float *sx = sub + cx * Sn, *sy = sub + (W + cy) * Sn, *sz = sub + (2 * W + cz) * Sn;
                int c = 0;
                for (int q0 = 0; q0 < P.S3; q0 += 32) {
                    const int q = q0 + lane;
                    bool in = false;
                    if (q < P.S3) {
                        int qa, qb, qc;
                        if (P.Slog >= 0) {
                            qa = q & (Sn - 1);
                            qb = (q >> P.Slog) & (Sn - 1);
                            qc = q >> (2 * P.Slog);
                        } else {
                            qa = q % Sn;
                            qb = (q / Sn) % Sn;
                            qc = q / (Sn * Sn);
                        }
                        const float tf = (sx[qa] + sy[qb]) + sz[qc];
                        if (tf < band.lo) in = true;
                        else if (tf <= band.hi)
                            in = subpoint_inside_exact(P.r2, P.frac[qa], P.frac[qb], P.frac[qc], h0 + cx - R,
                                                       h1 + cy - R, h2 + cz - R, x, y, z);
                    }
                    c += __popc(__ballot_sync(kFull, in));
                }
                if (lane == src) cnt = c;
            }
            mem = mem && cnt > 0;
        }
        const unsigned m = __ballot_sync(kFull, mem);
        if (mem) {
            const unsigned pos = nout + __popc(m & ((1u << lane) - 1u));
            if (pos < cap) slots[base + pos] = pack_pair(h0 + ox - R, h1 + oy - R, h2 + oz - R, R, cnt);
            else report(st, PMP_ERR_WORKSPACE, s);
        }
        nout += __popc(m);
    }
    if (lane == 0) counts[t] = nout < cap ? nout : cap;
}

// ---------------------------------------------------------------------------
// gather
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(128) k_gather_fb(KParams P, Box S, const double *__restrict__ u, Parts p,
                                                   PlanPtrs pl, double *__restrict__ G, DevStatus *st)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.count) return;
    const long long s = pl.perm ? (long long)pl.perm[t] : t;
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
    double sw = 0.0, sr = 0.0, sp0 = 0.0, sp1 = 0.0, sp2 = 0.0;
    const double s3 = (double)P.S3;
    const unsigned long long b0 = (unsigned long long)t * pl.cap;
    const unsigned nc = pl.counts[t];
    for (unsigned q = 0; q < nc; ++q) {
        const PairCell c = unpack_pair(pl.slots[b0 + q], P.R);
        double U[NF];
        load_cell(u, S, S.at(owner(c.i, S.n0), owner(c.j, S.n1), owner(c.k, S.n2)), U);
        if (c.cnt == P.S3) {
            sw = sw + 1.0;
            sr = sr + U[0];
            sp0 = sp0 + U[1];
            sp1 = sp1 + U[2];
            sp2 = sp2 + U[3];
        } else {
            const double w = (double)c.cnt / s3;
            sw = sw + w;
            sr = sr + w * U[0];
            sp0 = sp0 + w * U[1];
            sp1 = sp1 + w * U[2];
            sp2 = sp2 + w * U[3];
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

// Sink gather.  Writes the particle's per-axis Gaussian factors
// exp(-d^2 / r_acc^2) to wts[s][3][W] for the deposit and Step 4.
template <int R>
__global__ void __launch_bounds__(128) k_gather_sink(KParams P, Box S, const double *__restrict__ u, Parts p,
                                                     PlanPtrs pl, double *__restrict__ G, DevStatus *st)
{
    constexpr int W = 2 * R + 1;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.count) return;
    const long long s = pl.perm ? (long long)pl.perm[t] : t;
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
    const unsigned long long b0 = (unsigned long long)t * pl.cap;
    const unsigned nc = pl.counts[t];
    const long long as = pl.aux_stride;
    double srho = 0.0, sp0 = 0.0, sp1 = 0.0, sp2 = 0.0, src = 0.0;
    for (unsigned q = 0; q < nc; ++q) {
        const PairCell c = unpack_pair(pl.slots[b0 + q], P.R);
        const int wi = owner(c.i, S.n0), wj = owner(c.j, S.n1), wk = owner(c.k, S.n2);
        double U[NF];
        load_cell(u, S, S.at(wi, wj, wk), U);
        srho = srho + U[0];
        sp0 = sp0 + U[1];
        sp1 = sp1 + U[2];
        sp2 = sp2 + U[3];
        src = src + __ldg(pl.aux + AUX_RCS * as + vidx(S, wi, wj, wk));
    }
    const int nk = (int)nc;
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
    const int hx = (int)floor(x), hy = (int)floor(y), hz = (int)floor(z);
    double *ws = pl.wts + s * (3 * W);
#pragma unroll
    for (int o = 0; o < W; ++o) {
        const double ax = ((double)(hx + o - R) + 0.5) - x;
        const double ay = ((double)(hy + o - R) + 0.5) - y;
        const double az = ((double)(hz + o - R) + 0.5) - z;
        ws[o] = pmp_exp(-((ax * ax) / ra2));
        ws[W + o] = pmp_exp(-((ay * ay) / ra2));
        ws[2 * W + o] = pmp_exp(-((az * az) / ra2));
    }
    double sumw = 0.0;
    for (unsigned q = 0; q < nc; ++q) {
        const PairCell c = unpack_pair(pl.slots[b0 + q], P.R);
        sumw = sumw + (ws[c.i - hx + R] * ws[W + c.j - hy + R]) * ws[2 * W + c.k - hz + R];
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
// per-pair deposition values
// ---------------------------------------------------------------------------

__device__ __forceinline__ void fb_pair_delta(const KParams &P, const Box &S, const double *__restrict__ u,
                                              const Parts &p, const double *__restrict__ G, long long s,
                                              const PairCell &c, double dU[NF])
{
    const long long gs = p.count;
    const double x = __ldg(p.x + s), y = __ldg(p.y + s), z = __ldg(p.z + s);
    const double d0 = ((double)c.i + 0.5) - x, d1 = ((double)c.j + 0.5) - y, d2 = ((double)c.k + 0.5) - z;
    const double dd = (d0 * d0 + d1 * d1) + d2 * d2;
    const double w = c.cnt == P.S3 ? 1.0 : (double)c.cnt / (double)P.S3;
    double U[NF];
    load_cell(u, S, S.at(owner(c.i, S.n0), owner(c.j, S.n1), owner(c.k, S.n2)), U);
    const double vc[3] = {__ldg(G + FB_VX * gs + s), __ldg(G + FB_VY * gs + s), __ldg(G + FB_VZ * gs + s)};
    feedback_delta(w, U, __ldg(G + FB_Q * gs + s), __ldg(G + FB_E * gs + s), __ldg(G + FB_PV * gs + s), vc, d0, d1,
                   d2, dd, dU);
}

template <int R>
__device__ __forceinline__ void sink_pair_delta(const KParams &P, const Box &S, const Parts &p,
                                                const double *__restrict__ G, const PlanPtrs &pl, long long s,
                                                const PairCell &c, double dU[NF], long long &vcell)
{
    constexpr int W = 2 * R + 1;
    int hx, hy, hz;
    unpack_host(__ldg(pl.hosts + s), hx, hy, hz);
    const double *ws = pl.wts + s * (3 * W);
    const double w = (__ldg(ws + c.i - hx + R) * __ldg(ws + W + c.j - hy + R)) * __ldg(ws + 2 * W + c.k - hz + R);
    vcell = vidx(S, owner(c.i, S.n0), owner(c.j, S.n1), owner(c.k, S.n2));
    const long long as = pl.aux_stride;
    const double bh = __ldg(G + SK_K * p.count + s) * w;
    const double tr = __ldg(pl.aux + AUX_TR * as + vcell);
    const double a = bh >= tr ? bh : tr;
    dU[0] = -a;
    dU[1] = -(a * __ldg(pl.aux + AUX_V0 * as + vcell));
    dU[2] = -(a * __ldg(pl.aux + AUX_V1 * as + vcell));
    dU[3] = -(a * __ldg(pl.aux + AUX_V2 * as + vcell));
    dU[4] = -(a * __ldg(pl.aux + AUX_ES * as + vcell));
}

// ---------------------------------------------------------------------------
// Step 1, atomic accumulation: a warp takes 8 consecutive particles of the
// processing order and spreads their pairs over its lanes
// ---------------------------------------------------------------------------

constexpr int kPartsPerWarp = 8;

template <int R, bool FB>
__global__ void __launch_bounds__(256) k_deposit_atomic(KParams P, Box S, const double *__restrict__ u, Box B,
                                                        double *__restrict__ b, Parts p,
                                                        const double *__restrict__ G, PlanPtrs pl)
{
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long t0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kPartsPerWarp;
         t0 < p.count; t0 += nwarps * kPartsPerWarp) {
        // inclusive prefix of the 8 particles' pair counts, held by lanes 0..7
        unsigned c = 0;
        long long sid = 0;
        if (lane < kPartsPerWarp && t0 + lane < p.count) {
            c = __ldg(pl.counts + t0 + lane);
            sid = pl.perm ? (long long)__ldg(pl.perm + t0 + lane) : t0 + lane;
        }
        unsigned incl = c;
#pragma unroll
        for (int d = 1; d < kPartsPerWarp; d <<= 1) {
            const unsigned v = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += v;
        }
        const unsigned total = __shfl_sync(kFull, incl, kPartsPerWarp - 1);
        for (unsigned g0 = 0; g0 < total; g0 += 32) {
            const unsigned g = g0 + lane;
            // particle j of this pair: the first whose inclusive prefix exceeds g
            int j = 0;
            unsigned before = 0;
#pragma unroll
            for (int k = 0; k < kPartsPerWarp - 1; ++k) {
                const unsigned ik = __shfl_sync(kFull, incl, k);
                if (g >= ik) {
                    j = k + 1;
                    before = ik;
                }
            }
            const long long s = __shfl_sync(kFull, sid, j);
            if (g < total) {
                const unsigned long long slot = (unsigned long long)(t0 + j) * pl.cap + (g - before);
                const PairCell cell = unpack_pair(__ldg(pl.slots + slot), P.R);
                double dU[NF];
                if (FB) {
                    fb_pair_delta(P, S, u, p, G, s, cell, dU);
                } else {
                    long long vc;
                    sink_pair_delta<R>(P, S, p, G, pl, s, cell, dU, vc);
                }
                const long long bc = B.at(cell.i, cell.j, cell.k);
#pragma unroll
                for (int f = 0; f < NF; ++f) atomicAdd(b + (long long)f * B.fs + bc, dU[f]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Step 1, sorted accumulation
// ---------------------------------------------------------------------------

// Compact (buffer cell, slot) lists in particle-index order (the sorted mode
// plans in index order); offsets from the exclusive scan of the counts.
__global__ void __launch_bounds__(128) k_sort_keys(KParams P, Box B, long long n, PlanPtrs pl,
                                                   const unsigned long long *__restrict__ offsets,
                                                   unsigned *__restrict__ keys, unsigned *__restrict__ vals)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const unsigned long long o = offsets[t];
    const unsigned nc = pl.counts[t];
    const unsigned long long b0 = (unsigned long long)t * pl.cap;
    for (unsigned q = 0; q < nc; ++q) {
        const PairCell c = unpack_pair(pl.slots[b0 + q], P.R);
        keys[o + q] = (unsigned)B.at(c.i, c.j, c.k);
        vals[o + q] = (unsigned)(b0 + q);
    }
}

// One thread per run of equal keys (a buffer cell): the run's pairs, which the
// stable sort kept in particle-index order, are added in that order on top of
// what the buffer holds.
template <int R, bool FB>
__global__ void __launch_bounds__(128) k_segment_sum(KParams P, Box S, const double *__restrict__ u, Box B,
                                                     double *__restrict__ b, Parts p, const double *__restrict__ G,
                                                     PlanPtrs pl, const unsigned long long *__restrict__ total_ptr,
                                                     const unsigned *__restrict__ keys,
                                                     const unsigned *__restrict__ vals)
{
    const unsigned long long total = *total_ptr;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const unsigned key = keys[i];
        if (i > 0 && keys[i - 1] == key) continue;
        double acc[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) acc[f] = b[(long long)f * B.fs + key];
        for (unsigned long long j = i; j < total && keys[j] == key; ++j) {
            const unsigned long long slot = vals[j];
            const long long s = (long long)(slot / pl.cap);  // index-order plan: slot row = particle
            const PairCell c = unpack_pair(pl.slots[slot], P.R);
            double dU[NF];
            if (FB) {
                fb_pair_delta(P, S, u, p, G, s, c, dU);
            } else {
                long long vc;
                sink_pair_delta<R>(P, S, p, G, pl, s, c, dU, vc);
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) acc[f] = acc[f] + dU[f];
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) b[(long long)f * B.fs + key] = acc[f];
    }
}

// ---------------------------------------------------------------------------
// Step 4: limited changes returned to sinks
// ---------------------------------------------------------------------------

template <int R>
__global__ void __launch_bounds__(128) k_return_sinks(KParams P, Box S, Parts p, const double *__restrict__ G,
                                                      PlanPtrs pl, DevStatus *st)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.count) return;
    const long long s = pl.perm ? (long long)pl.perm[t] : t;
    const int bad = position_status(S, p.x[s], p.y[s], p.z[s]);
    if (bad) {
        report(st, bad, s);
        return;
    }
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    const unsigned long long b0 = (unsigned long long)t * pl.cap;
    const unsigned nc = pl.counts[t];
    for (unsigned q = 0; q < nc; ++q) {
        const PairCell c = unpack_pair(pl.slots[b0 + q], P.R);
        double dU[NF];
        long long vc;
        sink_pair_delta<R>(P, S, p, G, pl, s, c, dU, vc);
        const double e = __ldg(pl.eta + vc);
        if (e == 1.0) {
            a0 = a0 + dU[0];
            a1 = a1 + dU[1];
            a2 = a2 + dU[2];
            a3 = a3 + dU[3];
        } else {
            a0 = a0 + e * dU[0];
            a1 = a1 + e * dU[1];
            a2 = a2 + e * dU[2];
            a3 = a3 + e * dU[3];
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

void launch_host_keys(const Box &S, const Parts &p, unsigned *keys, unsigned *ids, cudaStream_t stream)
{
    if (p.count == 0) return;
    int nmax = S.n0 > S.n1 ? S.n0 : S.n1;
    nmax = nmax > S.n2 ? nmax : S.n2;
    int bits = 0;
    while ((1 << bits) < nmax) ++bits;
    const int sh = bits > 10 ? bits - 10 : 0;
    k_host_keys<<<blocks_for(p.count, 256), 256, 0, stream>>>(S, p, sh, keys, ids);
}

template <int R, bool FB>
static void plan_one(const KParams &P, const Box &S, const Parts &p, const PlanPtrs &pl, DevStatus *st,
                     cudaStream_t stream)
{
    constexpr int W = 2 * R + 1;
    const int warps = 8;
    const size_t sm = (size_t)warps * plan_warp_floats(W, FB ? P.S : 1) * sizeof(float);
    k_plan<R, FB><<<blocks_for(p.count, warps), warps * 32, sm, stream>>>(P, S, p, pl.perm, (unsigned)pl.cap,
                                                                         pl.counts, pl.slots, pl.hosts, st);
}

void launch_plan(const KParams &P, const Box &S, const Parts &p, const PlanPtrs &pl, DevStatus *st,
                 cudaStream_t stream)
{
    if (p.count == 0) return;
    if (P.kind == PMP_KIND_FEEDBACK) {
        PMP_DISPATCH_R(P.R, (plan_one<RR, true>(P, S, p, pl, st, stream)));
    } else {
        PMP_DISPATCH_R(P.R, (plan_one<RR, false>(P, S, p, pl, st, stream)));
    }
}

void launch_gather(const KParams &P, const Box &S, const double *u, const Parts &p, const PlanPtrs &pl, double *G,
                   DevStatus *st, cudaStream_t stream)
{
    if (p.count == 0) return;
    const unsigned nb = blocks_for(p.count, 128);
    if (P.kind == PMP_KIND_FEEDBACK) {
        k_gather_fb<<<nb, 128, 0, stream>>>(P, S, u, p, pl, G, st);
    } else {
        PMP_DISPATCH_R(P.R, (k_gather_sink<RR><<<nb, 128, 0, stream>>>(P, S, u, p, pl, G, st)));
    }
}

void launch_deposit_atomic(const KParams &P, const Box &S, const double *u, const Box &B, double *b, const Parts &p,
                           const double *G, const PlanPtrs &pl, cudaStream_t stream)
{
    if (p.count == 0) return;
    const long long warps = (p.count + kPartsPerWarp - 1) / kPartsPerWarp;
    const long long blocks_needed = (warps + 7) / 8;
    const unsigned nb = (unsigned)(blocks_needed < 152LL * 64 ? blocks_needed : 152LL * 64);
    if (P.kind == PMP_KIND_FEEDBACK) {
        k_deposit_atomic<1, true><<<nb, 256, 0, stream>>>(P, S, u, B, b, p, G, pl);
    } else {
        PMP_DISPATCH_R(P.R, (k_deposit_atomic<RR, false><<<nb, 256, 0, stream>>>(P, S, u, B, b, p, G, pl)));
    }
}

void launch_sort_keys(const KParams &P, const Box &B, const Parts &p, const PlanPtrs &pl,
                      const unsigned long long *offsets, unsigned *keys, unsigned *vals, cudaStream_t stream)
{
    if (p.count == 0) return;
    k_sort_keys<<<blocks_for(p.count, 128), 128, 0, stream>>>(P, B, p.count, pl, offsets, keys, vals);
}

void launch_segment_sum(const KParams &P, const Box &S, const double *u, const Box &B, double *b, const Parts &p,
                        const double *G, const PlanPtrs &pl, const unsigned long long *total, const unsigned *keys,
                        const unsigned *vals, cudaStream_t stream)
{
    const unsigned nb = 152u * 32u;
    if (P.kind == PMP_KIND_FEEDBACK) {
        k_segment_sum<1, true><<<nb, 128, 0, stream>>>(P, S, u, B, b, p, G, pl, total, keys, vals);
    } else {
        PMP_DISPATCH_R(P.R, (k_segment_sum<RR, false><<<nb, 128, 0, stream>>>(P, S, u, B, b, p, G, pl, total, keys,
                                                                               vals)));
    }
}

void launch_return_sinks(const KParams &P, const Box &S, const Parts &p, const double *G, const PlanPtrs &pl,
                         DevStatus *st, cudaStream_t stream)
{
    if (p.count == 0) return;
    const unsigned nb = blocks_for(p.count, 128);
    PMP_DISPATCH_R(P.R, (k_return_sinks<RR><<<nb, 128, 0, stream>>>(P, S, p, G, pl, st)));
}

}  // namespace pmp
