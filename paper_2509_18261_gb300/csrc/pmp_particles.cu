// pmp_particles.cu -- particle-side kernels.
//
//   plan      persistent; one warp per particle (spatial processing order):
//             lanes classify the candidate cells, then count the S^3
//             sub-points of the boundary cells (a lane per cell); kernel cells
//             with omega > 0 written in canonical order (z slowest, x fastest)
//             to the particle's fixed slot range
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

// Particles whose pairs a warp of the atomic deposit spreads over its lanes.
constexpr int kPartsPerWarp = 8;

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

// Per-particle prologue (one thread per particle): host cell, the fractional
// position x - floor(x) (exact in FP64) rounded to FP32 for the plan's
// filters, and the processing-order key: the Morton (Z-order) code of the host
// cell (coordinates shifted right by `sh` to fit 10 bits), so that consecutive
// particles of the order have overlapping kernels.  Invalid positions get
// host = kNoHost and sort last.
constexpr unsigned long long kNoHost = ~0ULL;

__global__ void __launch_bounds__(256) k_prologue(Box S, Parts p, int sh, unsigned *__restrict__ keys,
                                                  unsigned *__restrict__ ids, unsigned long long *__restrict__ hosts,
                                                  float4 *__restrict__ fr, DevStatus *st)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.count) return;
    const double x = p.x[s], y = p.y[s], z = p.z[s];
    const int bad = position_status(S, x, y, z);
    if (bad) {
        report(st, bad, s);
        hosts[s] = kNoHost;
        fr[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (keys) {
            keys[s] = 0xffffffffu;
            ids[s] = (unsigned)s;
        }
        return;
    }
    const double fx = floor(x), fy = floor(y), fz = floor(z);
    const int hx = (int)fx, hy = (int)fy, hz = (int)fz;
    hosts[s] = pack_host(hx, hy, hz);
    fr[s] = make_float4((float)(x - fx), (float)(y - fy), (float)(z - fz), 0.f);
    if (keys) {
        const unsigned ux = (unsigned)hx >> sh, uy = (unsigned)hy >> sh, uz = (unsigned)hz >> sh;
        keys[s] = spread3(ux) | (spread3(uy) << 1) | (spread3(uz) << 2);
        ids[s] = (unsigned)s;
    }
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------

// Candidate offsets of a kernel: (ox, oy, oz) in [0, W)^3, offset o - R per
// axis, whose cell centre can come within r_K of some point of the host cell,
// i.e. sum_a max(0, |o_a - R| - 1/2)^2 <= r_K^2 (1 + 1e-9) (the slack covers
// rounding of the FP64 distance).  Kept in canonical order (z slowest, x
// fastest); their number is the slot bound of a particle.  Built by one warp.
__device__ __forceinline__ int build_candidates(double rK, int R, unsigned *cand)
{
    const int W = 2 * R + 1, W3 = W * W * W;
    const int lane = threadIdx.x & 31;
    const double lim = rK * rK * (1.0 + 1e-9);
    int n = 0;
    for (int k0 = 0; k0 < W3; k0 += 32) {
        const int k = k0 + lane;
        bool ok = false;
        unsigned code = 0;
        if (k < W3) {
            const int oz = k / (W * W), oy = k / W - oz * W, ox = k - (k / W) * W;
            const int o[3] = {ox - R, oy - R, oz - R};
            double s = 0.0;
            for (int a = 0; a < 3; ++a) {
                const double m = fabs((double)o[a]) - 0.5;
                if (m > 0.0) s += m * m;
            }
            ok = s <= lim;
            code = (unsigned)ox | ((unsigned)oy << 8) | ((unsigned)oz << 16);
        }
        const unsigned msk = __ballot_sync(kFull, ok);
        if (ok) cand[n + __popc(msk & ((1u << lane) - 1u))] = code;
        n += __popc(msk);
    }
    return n;
}

// Per-warp shared memory of the plan: FP32 squares per axis (sub-points
// [3][W*S], centres [3][W], farthest corners [3][W]), then two u16 arrays of
// W^3 entries (count per candidate, boundary-cell list).
__host__ __device__ constexpr int plan_warp_bytes(int W, int S)
{
    return ((3 * W * S + 6 * W) * 4 + 15) / 16 * 16 + (4 * W * W * W + 15) / 16 * 16;
}

// Sub-point count of one boundary cell (centre inside, farthest corner not
// surely inside): the S^3 FP32 sums are compared with both band edges; if no
// sum falls inside the band the count below band_lo is the exact count,
// otherwise the cell is recounted with the FP64 test for the in-band points.
template <int SC>
__device__ __forceinline__ int boundary_count(const KParams &P, const float *sx, const float *sy, const float *sz,
                                              int cx, int cy, int cz, const Parts &p, long long s)
{
    constexpr int SM = SC ? SC : kMaxS;
    const int Sn = SC ? SC : P.S;
    const float blo = P.band_lo, bhi = P.band_hi;
    float vx[SM];
#pragma unroll
    for (int a = 0; a < SM; ++a) vx[a] = (SC || a < Sn) ? sx[a] : 3.0e38f;
    int lo = 0, hi = 0;
#pragma unroll
    for (int c = 0; c < SM; ++c) {
        if (!SC && c >= Sn) break;
        const float vzc = sz[c];
#pragma unroll
        for (int b = 0; b < SM; ++b) {
            if (!SC && b >= Sn) break;
            const float t = sy[b] + vzc;
#pragma unroll
            for (int a = 0; a < SM; ++a) {
                const float v = t + vx[a];
                lo += v < blo ? 1 : 0;
                hi += v <= bhi ? 1 : 0;
            }
        }
    }
    if (lo == hi) return lo;
    const double x = p.x[s], y = p.y[s], z = p.z[s];
    int cnt = 0;
    for (int c = 0; c < Sn; ++c)
        for (int b = 0; b < Sn; ++b) {
            const float t = sy[b] + sz[c];
            for (int a = 0; a < Sn; ++a) {
                const float v = t + sx[a];
                if (v < blo) ++cnt;
                else if (v <= bhi && subpoint_inside_exact(P.r2, P.frac[a], P.frac[b], P.frac[c], cx, cy, cz, x, y, z))
                    ++cnt;
            }
        }
    return cnt;
}

// Steps 1-4 of the plan for particle s (processing position t) by one warp;
// returns the particle's slot count (the same in every lane).
template <int R, bool FB, int SC>
__device__ __forceinline__ unsigned plan_particle(const KParams &P, const Box &S, const Parts &p, long long t, long long s,
                                              unsigned long long hp, float4 f4, unsigned cap, int ncand,
                                              const unsigned *cand, float *sub, float *csq, float *fc2,
                                              unsigned short *stc, unsigned short *blist, unsigned *counts,
                                              unsigned long long *slots, DevStatus *st)
{
    constexpr int W = 2 * R + 1;
    const int lane = threadIdx.x & 31;
    const int Sn = FB ? (SC ? SC : P.S) : 1;
    const float blo = P.band_lo, bhi = P.band_hi;
    int h0, h1, h2;
    unpack_host(hp, h0, h1, h2);
    // 1. per-axis squares from the FP32 edge offsets e = (o - R) - frac
    __syncwarp();
    for (int i = lane; i < 3 * W; i += 32) {
        const int a = i / W, o = i - a * W;
        const float fa = a == 0 ? f4.x : (a == 1 ? f4.y : f4.z);
        const float c = ((float)(o - R) - fa) + 0.5f;
        csq[i] = c * c;
    }
    if (FB) {
        for (int i = lane; i < 3 * W * Sn; i += 32) {
            const int a = i / (W * Sn), r = i - a * (W * Sn), o = r / Sn, k = r - o * Sn;
            const float fa = a == 0 ? f4.x : (a == 1 ? f4.y : f4.z);
            const float u = ((float)(o - R) - fa) + P.fracf[k];
            sub[i] = u * u;
        }
        __syncwarp();
        // the farthest sub-point of a cell along an axis is its first or last
        // one: if the sum of those squares is surely inside, all S^3 are
        for (int i = lane; i < 3 * W; i += 32) {
            const float s0 = sub[i * Sn], s1 = sub[i * Sn + Sn - 1];
            fc2[i] = s0 > s1 ? s0 : s1;
        }
    }
    __syncwarp();
    // 2. classification
    unsigned nout = 0, nb = 0;
    const unsigned long long base = (unsigned long long)t * cap;
    for (int k0 = 0; k0 < ncand; k0 += 32) {
        const int k = k0 + lane;
        int ox = 0, oy = 0, oz = 0;
        bool mem = false, full = false;
        if (k < ncand) {
            const unsigned code = cand[k];
            ox = code & 0xff;
            oy = (code >> 8) & 0xff;
            oz = code >> 16;
            const int c0 = h0 + ox - R, c1 = h1 + oy - R, c2 = h2 + oz - R;
            const bool dom = (S.per0 || (c0 >= 0 && c0 < S.n0)) && (S.per1 || (c1 >= 0 && c1 < S.n1)) &&
                             (S.per2 || (c2 >= 0 && c2 < S.n2));
            if (dom) {
                const float tf = (csq[ox] + csq[W + oy]) + csq[2 * W + oz];
                if (tf < blo) mem = true;
                else if (tf <= bhi) mem = centre_inside_exact(P.r2, c0, c1, c2, p.x[s], p.y[s], p.z[s]);
                if (FB && mem) full = (fc2[ox] + fc2[W + oy]) + fc2[2 * W + oz] < blo;
            }
        }
        if (FB) {
            if (k < ncand) stc[k] = mem ? (full ? (unsigned short)P.S3 : 0) : 0;
            const bool bnd = mem && !full;
            const unsigned bm = __ballot_sync(kFull, bnd);
            if (bnd) blist[nb + __popc(bm & ((1u << lane) - 1u))] = (unsigned short)k;
            nb += __popc(bm);
        } else {
            const unsigned m = __ballot_sync(kFull, mem);
            if (mem) {
                const unsigned pos = nout + __popc(m & ((1u << lane) - 1u));
                if (pos < cap) slots[base + pos] = pack_pair(h0 + ox - R, h1 + oy - R, h2 + oz - R, R, 0);
                else report(st, PMP_ERR_WORKSPACE, s);
            }
            nout += __popc(m);
        }
    }
    if (FB) {
        __syncwarp();
        // 3. sub-point counts of the boundary cells
        for (unsigned j = lane; j < nb; j += 32) {
            const int k = blist[j];
            const unsigned code = cand[k];
            const int ox = code & 0xff, oy = (code >> 8) & 0xff, oz = code >> 16;
            stc[k] = (unsigned short)boundary_count<SC>(P, sub + ox * Sn, sub + (W + oy) * Sn,
                                                        sub + (2 * W + oz) * Sn, h0 + ox - R, h1 + oy - R,
                                                        h2 + oz - R, p, s);
        }
        __syncwarp();
        // 4. cells with omega > 0, in candidate order
        for (int k0 = 0; k0 < ncand; k0 += 32) {
            const int k = k0 + lane;
            const int cnt = k < ncand ? stc[k] : 0;
            const unsigned m = __ballot_sync(kFull, cnt > 0);
            if (cnt > 0) {
                const unsigned code = cand[k];
                const int ox = code & 0xff, oy = (code >> 8) & 0xff, oz = code >> 16;
                const unsigned pos = nout + __popc(m & ((1u << lane) - 1u));
                if (pos < cap) slots[base + pos] = pack_pair(h0 + ox - R, h1 + oy - R, h2 + oz - R, R, cnt);
                else report(st, PMP_ERR_WORKSPACE, s);
            }
            nout += __popc(m);
        }
    }
    const unsigned n = nout < cap ? nout : cap;
    if (lane == 0) counts[t] = n;
    return n;
}

// The plan.  Persistent: each block builds the candidate table once, then its
// warps take particles of the processing order.  For one particle a warp
//   1. writes the per-axis FP32 squares;
//   2. classifies the candidates (lane per candidate): member if the centre
//      is inside (FP32 outside the band, else the FP64 test), full if the
//      farthest sub-point is surely inside (omega = 1), else a boundary cell;
//   3. (supernovae) counts the sub-points of the boundary cells, a lane per
//      cell;
//   4. writes the cells with omega > 0 (every member, for sinks) in
//      candidate order to the particle's slots.
template <int R, bool FB, int SC>
__global__ void __launch_bounds__(256) k_plan(KParams P, Box S, Parts p, const unsigned *__restrict__ perm,
                                              const unsigned long long *__restrict__ hosts,
                                              const float4 *__restrict__ fr, unsigned cap,
                                              unsigned *__restrict__ counts, unsigned long long *__restrict__ slots,
                                              DevStatus *st)
{
    constexpr int W = 2 * R + 1;
    constexpr int W3 = W * W * W;
    extern __shared__ __align__(16) unsigned char psm[];
    __shared__ int ncand_sh;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int Sn = FB ? (SC ? SC : P.S) : 1;
    unsigned *cand = reinterpret_cast<unsigned *>(psm);
    const int wbytes = plan_warp_bytes(W, Sn);
    unsigned char *wsm = psm + (W3 * 4 + 15) / 16 * 16 + (size_t)wib * wbytes;
    float *sub = reinterpret_cast<float *>(wsm);  // [3][W*S]
    float *csq = sub + 3 * W * Sn;                // [3][W]
    float *fc2 = csq + 3 * W;                     // [3][W]
    unsigned short *stc = reinterpret_cast<unsigned short *>(wsm + ((3 * W * Sn + 6 * W) * 4 + 15) / 16 * 16);
    unsigned short *blist = stc + W3;
    if (wib == 0) {
        const int n = build_candidates(P.rK, R, cand);
        if (lane == 0) ncand_sh = n;
    }
    __syncthreads();
    const int ncand = ncand_sh;
    const long long nwarps = (long long)gridDim.x * nw;
    // The particle data of the next iteration and the index of the one after
    // are requested one step ahead (their loads are random accesses).
    long long t = (long long)blockIdx.x * nw + wib;
    long long s = 0, s1 = 0;
    unsigned long long hp = kNoHost;
    float4 f4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t < p.count) {
        s = perm ? (long long)perm[t] : t;
        hp = hosts[s];
        f4 = fr[s];
    }
    if (t + nwarps < p.count) s1 = perm ? (long long)perm[t + nwarps] : t + nwarps;
    for (; t < p.count; t += nwarps) {
        unsigned long long hp1 = kNoHost;
        float4 f41 = make_float4(0.f, 0.f, 0.f, 0.f);
        long long s2 = 0;
        if (t + nwarps < p.count) {
            hp1 = hosts[s1];
            f41 = fr[s1];
        }
        if (t + 2 * nwarps < p.count) s2 = perm ? (long long)perm[t + 2 * nwarps] : t + 2 * nwarps;
        if (hp != kNoHost)
            plan_particle<R, FB, SC>(P, S, p, t, s, hp, f4, cap, ncand, cand, sub, csq, fc2, stc, blist, counts,
                                     slots, st);
        else if (lane == 0)
            counts[t] = 0;
        s = s1;
        hp = hp1;
        f4 = f41;
        s1 = s2;
    }
}

// ---------------------------------------------------------------------------
// gather
// ---------------------------------------------------------------------------

// Covered fractions omega = k / S^3 for k = 0..S^3, computed once per block.
constexpr int kMaxS3 = kMaxS * kMaxS * kMaxS;

// Pairs whose loads a per-particle gather loop issues together (512^3
// sweeps: supernova plan + gather 1 -> 24.0 ms, 2 -> 24.2, 3 -> 25.1, 4 ->
// 25.0, 8 -> 27.7: the fused kernel is bound by instruction issue and fetch,
// not by its loads; sink plan + gather + deposit 2 -> 24.0 ms, 4 -> 23.1-23.4,
// 8 -> 23.1).
#ifndef PMP_GATHER_UNROLL_FB
#define PMP_GATHER_UNROLL_FB 1
#endif
#ifndef PMP_GATHER_UNROLL_SINK
#define PMP_GATHER_UNROLL_SINK 4
#endif
constexpr int kUnrollFb = PMP_GATHER_UNROLL_FB;
constexpr int kUnroll = PMP_GATHER_UNROLL_SINK;

// Block size of the thread-per-sink kernels (gather, Step 4).  Step 4 keeps
// each sink's 3(2R+1) Gaussian factors in a shared-memory column (the gather
// does not: its cell-record loads need the L1 that the array would take).
constexpr int kSinkThreads = 128;

// A plan slot: through the read-only path (NC) when an earlier launch wrote
// it, else (written by this warp in the same launch) a coherent load.
template <bool NC>
__device__ __forceinline__ unsigned long long slot_load(const unsigned long long *q)
{
    if (NC) return __ldg(q);
    return *q;
}

// One kernel cell's terms of the supernova gather sums, products fused into
// the sums.  No branch on omega = 1 (wtab[S^3] = 1 and fma(1, v, s) == s + v):
// lanes of a warp mix full and partial cells, and a divergent branch would
// issue both paths on the FP64 pipe.  With IW (S a power of two) sum omega is
// kept as the integer sum of the sub-point counts: every term k / S^3 and
// every partial sum is a multiple of 2^-3log2(S) far below 2^53, so the FP64
// sum in kernel order is exact and equals (sum k) / S^3 bit for bit.
template <bool IW>
__device__ __forceinline__ void fb_gather_add(const double *wtab, int cnt, const double U[NF], double &sw,
                                              unsigned &isw, double &sr, double &sp0, double &sp1, double &sp2)
{
    const double w = wtab[cnt];
    if (IW)
        isw += (unsigned)cnt;
    else
        sw = sw + w;
    sr = fma(w, U[0], sr);
    sp0 = fma(w, U[1], sp0);
    sp1 = fma(w, U[2], sp1);
    sp2 = fma(w, U[3], sp2);
}

__device__ __forceinline__ void fill_omega_table(const KParams &P, double *wtab)
{
    for (int i = threadIdx.x; i <= P.S3; i += blockDim.x) wtab[i] = (double)i / (double)P.S3;
    __syncthreads();
}

template <bool IW, bool NC>
__device__ __forceinline__ void gather_fb_particle(const KParams &P, const Box &S, const double *__restrict__ u,
                                                   const Parts &p, const PlanPtrs &pl, double *__restrict__ G,
                                                   DevStatus *st, const double *wtab, long long t)
{
    const long long s = pl.perm ? (long long)pl.perm[t] : t;
    const long long gs = p.count;
    const double m = p.m[s], pe0 = p.px[s], pe1 = p.py[s], pe2 = p.pz[s], Esn = p.e[s];
    int bad = pl.hosts[s] == kNoHost ? PMP_ERR_PARTICLE_OUTSIDE : 0;
    if (!bad && !(m > 0.0)) bad = PMP_ERR_NONFINITE;
    if (bad) {
        if (bad == PMP_ERR_NONFINITE) report(st, bad, s);
        for (int r = 0; r < FB_ROWS; ++r) G[r * gs + s] = 0.0;
        return;
    }
    double sw = 0.0, sr = 0.0, sp0 = 0.0, sp1 = 0.0, sp2 = 0.0;
    unsigned isw = 0;
    const unsigned long long b0 = (unsigned long long)t * pl.cap;
    const unsigned nc = pl.counts[t];
    // the cells' loads are issued kUnrollFb at a time, the sums stay in kernel order
    unsigned q = 0;
    for (; q + kUnrollFb <= nc; q += kUnrollFb) {
        PairCell c[kUnrollFb];
        double U[kUnrollFb][NF];
#pragma unroll
        for (int k = 0; k < kUnrollFb; ++k) c[k] = unpack_pair(slot_load<NC>(pl.slots + b0 + q + k), P.R);
#pragma unroll
        for (int k = 0; k < kUnrollFb; ++k)
            load_cell(u, S, S.at(owner(c[k].i, S.n0), owner(c[k].j, S.n1), owner(c[k].k, S.n2)), U[k]);
#pragma unroll
        for (int k = 0; k < kUnrollFb; ++k) fb_gather_add<IW>(wtab, c[k].cnt, U[k], sw, isw, sr, sp0, sp1, sp2);
    }
    for (; q < nc; ++q) {
        const PairCell c = unpack_pair(slot_load<NC>(pl.slots + b0 + q), P.R);
        double U[NF];
        load_cell(u, S, S.at(owner(c.i, S.n0), owner(c.j, S.n1), owner(c.k, S.n2)), U);
        fb_gather_add<IW>(wtab, c.cnt, U, sw, isw, sr, sp0, sp1, sp2);
    }
    if (IW) sw = (double)isw * wtab[1];  // wtab[1] = 2^-3log2(S): exact
    if (!fb_gather_rows(P, sw, sr, sp0, sp1, sp2, m, pe0, pe1, pe2, Esn, G + s, gs)) report(st, PMP_ERR_NONFINITE, s);
}

// Grid-stride over the processing order (a window of consecutive particles
// in flight, see window_blocks).
__global__ void __launch_bounds__(128) k_gather_fb(KParams P, Box S, const double *__restrict__ u, Parts p,
                                                   PlanPtrs pl, double *__restrict__ G, DevStatus *st)
{
    __shared__ double wtab[kMaxS3 + 1];
    fill_omega_table(P, wtab);
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (P.Slog >= 0) {
        for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < p.count; t += stride)
            gather_fb_particle<true, true>(P, S, u, p, pl, G, st, wtab, t);
    } else {
        for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < p.count; t += stride)
            gather_fb_particle<false, true>(P, S, u, p, pl, G, st, wtab, t);
    }
}

// Resident blocks per SM the fused plan + gather is compiled for (its
// register budget).  512^3 sweep: 2 -> 30.6 ms, 3 -> 26.4 ms (no spills),
// 4 -> 25.0 ms (64 registers, 16 bytes spilled).
#ifndef PMP_PLAN_GATHER_MINB
#define PMP_PLAN_GATHER_MINB 4
#endif

// Plan and gather of the supernova kind in one persistent kernel.  A warp
// takes 32 consecutive particles of the processing order, plans them one
// after the other as k_plan does (warp-cooperative), then each lane gathers
// one of them as k_gather_fb does (thread per particle).  The plan is bound
// by instruction issue and the gather by the FP64 pipe, so warps in the two
// phases share an SM's issue slots and FP64 pipe instead of running one
// kernel after the other.  Slots and counts are the same as those of the two
// kernels; the gather reads the slots its warp has just written through the
// coherent path, after the warp's barrier.
template <int R, int SC>
__global__ void __launch_bounds__(256, PMP_PLAN_GATHER_MINB) k_plan_gather_fb(KParams P, Box S, const double *__restrict__ u, Parts p,
                                                        PlanPtrs pl, double *__restrict__ G, DevStatus *st)
{
    constexpr int W = 2 * R + 1;
    constexpr int W3 = W * W * W;
    extern __shared__ __align__(16) unsigned char psm[];
    __shared__ int ncand_sh;
    __shared__ double wtab[kMaxS3 + 1];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int Sn = SC ? SC : P.S;
    unsigned *cand = reinterpret_cast<unsigned *>(psm);
    const int wbytes = plan_warp_bytes(W, Sn);
    unsigned char *wsm = psm + (W3 * 4 + 15) / 16 * 16 + (size_t)wib * wbytes;
    float *sub = reinterpret_cast<float *>(wsm);  // [3][W*S]
    float *csq = sub + 3 * W * Sn;                // [3][W]
    float *fc2 = csq + 3 * W;                     // [3][W]
    unsigned short *stc = reinterpret_cast<unsigned short *>(wsm + ((3 * W * Sn + 6 * W) * 4 + 15) / 16 * 16);
    unsigned short *blist = stc + W3;
    for (int i = threadIdx.x; i <= P.S3; i += blockDim.x) wtab[i] = (double)i / (double)P.S3;
    if (wib == 0) {
        const int n = build_candidates(P.rK, R, cand);
        if (lane == 0) ncand_sh = n;
    }
    __syncthreads();
    const int ncand = ncand_sh;
    const long long nwarps = (long long)gridDim.x * nw;
    for (long long t0 = ((long long)blockIdx.x * nw + wib) * 32; t0 < p.count; t0 += nwarps * 32) {
        // lane j loads particle t0 + j's index, host cell and offsets
        const long long tl = t0 + lane;
        long long sl = 0;
        unsigned long long hl = kNoHost;
        float4 fl = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tl < p.count) {
            sl = pl.perm ? (long long)pl.perm[tl] : tl;
            hl = pl.hosts[sl];
            fl = pl.fr[sl];
        }
        const int nj = p.count - t0 < 32 ? (int)(p.count - t0) : 32;
        for (int j = 0; j < nj; ++j) {
            const long long s = __shfl_sync(kFull, sl, j);
            const unsigned long long hp = __shfl_sync(kFull, hl, j);
            float4 f4;
            f4.x = __shfl_sync(kFull, fl.x, j);
            f4.y = __shfl_sync(kFull, fl.y, j);
            f4.z = __shfl_sync(kFull, fl.z, j);
            f4.w = 0.f;
            if (hp != kNoHost)
                plan_particle<R, true, SC>(P, S, p, t0 + j, s, hp, f4, (unsigned)pl.cap, ncand, cand, sub, csq, fc2,
                                           stc, blist, pl.counts, pl.slots, st);
            else if (lane == 0)
                pl.counts[t0 + j] = 0;
        }
        __syncwarp();
        if (tl < p.count) {
            if (P.Slog >= 0)
                gather_fb_particle<true, false>(P, S, u, p, pl, G, st, wtab, tl);
            else
                gather_fb_particle<false, false>(P, S, u, p, pl, G, st, wtab, tl);
        }
    }
}

// Particle-mesh gather (MASS kind): V_K = V sum omega over the plan's cells in
// kernel order, then (m, p, e) / V_K.
__global__ void __launch_bounds__(128) k_gather_mass(KParams P, Box S, Parts p, PlanPtrs pl, double *__restrict__ G,
                                                     DevStatus *st)
{
    __shared__ double wtab[kMaxS3 + 1];
    fill_omega_table(P, wtab);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.count) return;
    const long long s = pl.perm ? (long long)pl.perm[t] : t;
    const long long gs = p.count;
    if (pl.hosts[s] == kNoHost) {
        for (int r = 0; r < MS_ROWS; ++r) G[r * gs + s] = 0.0;
        return;
    }
    double sw = 0.0;
    const unsigned long long b0 = (unsigned long long)t * pl.cap;
    const unsigned nc = pl.counts[t];
    for (unsigned q = 0; q < nc; ++q) {
        const int cnt = (int)(__ldg(pl.slots + b0 + q) >> 48);
        sw = sw + (cnt == P.S3 ? 1.0 : wtab[cnt]);
    }
    const double VK = sw * P.V;
    const double u[NF] = {p.m[s], p.px[s], p.py[s], p.pz[s], p.e ? p.e[s] : 0.0};
    G[MS_VK * gs + s] = VK;
    bool ok = isfinite(VK) && VK > 0.0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const double q = exact::div_rn(u[f], VK);
        G[(MS_Q + f) * gs + s] = q;
        ok = ok && isfinite(q);
    }
    if (!ok) report(st, PMP_ERR_NONFINITE, s);
}

// Sink gather.  Writes the particle's per-axis Gaussian factors
// exp(-d^2 / r_acc^2) to wts[s][3][W] for the deposit and Step 4.
// The rest of one sink's gather once the sums over its kernel cells (in
// kernel order) are known: Sec. 3.1.1's ambient quantities, the per-axis
// Gaussian factors, sum w and the gathered rows (row stride gs).
template <int R>
__device__ __forceinline__ void gather_sink_finish(const KParams &P, const PlanPtrs &pl, double *__restrict__ G,
                                                   long long gs, DevStatus *st, long long t, long long s, double x,
                                                   double y, double z, double ms, double ps0, double ps1,
                                                   double ps2, unsigned nc, double srho, double sp0, double sp1,
                                                   double sp2, double src)
{
    constexpr int W = 2 * R + 1;
    const unsigned long long b0 = (unsigned long long)t * pl.cap;
    const int nk = (int)nc;
    const SinkAmbient am = sink_ambient(P, srho, sp0, sp1, sp2, src, nk, ms, ps0, ps1, ps2);
    const double ra2 = am.ra2;
    const int hx = (int)floor(x), hy = (int)floor(y), hz = (int)floor(z);
    double *ws = pl.wts + s * (3 * W);
#pragma unroll
    for (int o = 0; o < W; ++o) {
        ws[o] = sink_axis_weight(((double)(hx + o - R) + 0.5) - x, ra2);
        ws[W + o] = sink_axis_weight(((double)(hy + o - R) + 0.5) - y, ra2);
        ws[2 * W + o] = sink_axis_weight(((double)(hz + o - R) + 0.5) - z, ra2);
    }
    double sumw = 0.0;
    for (unsigned q = 0; q < nc; ++q) {
        const PairCell c = unpack_pair(pl.slots[b0 + q], P.R);
        sumw = fma(ws[c.i - hx + R] * ws[W + c.j - hy + R], ws[2 * W + c.k - hz + R], sumw);
    }
    if (!sink_gather_rows(P, am, sumw, nk, G + s, gs)) report(st, PMP_ERR_NONFINITE, s);
}

// The validity test of a sink before its gather: false (rows zeroed, the
// error reported) for a position outside the box or a mass that is not
// positive.
__device__ __forceinline__ bool sink_gather_ok(const Box &S, double x, double y, double z, double ms,
                                               double *__restrict__ G, long long gs, long long s, DevStatus *st)
{
    int bad = position_status(S, x, y, z);
    if (!bad && !(ms > 0.0)) bad = PMP_ERR_NONFINITE;
    if (bad) {
        report(st, bad, s);
        for (int r = 0; r < SK_ROWS; ++r) G[r * gs + s] = 0.0;
        return false;
    }
    return true;
}

template <int R, bool NC = true>
__device__ __forceinline__ void gather_sink_particle(const KParams &P, const Box &S, const double *__restrict__ u,
                                                     const Parts &p, const PlanPtrs &pl, double *__restrict__ G,
                                                     DevStatus *st, long long t)
{
    const long long s = pl.perm ? (long long)pl.perm[t] : t;
    const long long gs = p.count;
    const double x = p.x[s], y = p.y[s], z = p.z[s];
    const double ms = p.m[s], ps0 = p.px[s], ps1 = p.py[s], ps2 = p.pz[s];
    if (!sink_gather_ok(S, x, y, z, ms, G, gs, s, st)) return;
    const unsigned long long b0 = (unsigned long long)t * pl.cap;
    const unsigned nc = pl.counts[t];
    double srho = 0.0, sp0 = 0.0, sp1 = 0.0, sp2 = 0.0, src = 0.0;
    unsigned q = 0;
    for (; q + kUnroll <= nc; q += kUnroll) {
        double2 g[kUnroll][2];
        double gc[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const PairCell c = unpack_pair(slot_load<NC>(pl.slots + b0 + q + k), P.R);
            const long long vc = vidx(S, owner(c.i, S.n0), owner(c.j, S.n1), owner(c.k, S.n2));
            const double2 *r = reinterpret_cast<const double2 *>(pl.grec + vc * kGRec);
            g[k][0] = __ldg(r);
            g[k][1] = __ldg(r + 1);
            gc[k] = __ldg(pl.gcs + vc);
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            srho = srho + g[k][0].x;
            sp0 = sp0 + g[k][0].y;
            sp1 = sp1 + g[k][1].x;
            sp2 = sp2 + g[k][1].y;
            src = src + gc[k];
        }
    }
    for (; q < nc; ++q) {
        const PairCell c = unpack_pair(slot_load<NC>(pl.slots + b0 + q), P.R);
        const long long vc = vidx(S, owner(c.i, S.n0), owner(c.j, S.n1), owner(c.k, S.n2));
        const double2 *g = reinterpret_cast<const double2 *>(pl.grec + vc * kGRec);
        const double2 g0 = __ldg(g), g1 = __ldg(g + 1);
        srho = srho + g0.x;
        sp0 = sp0 + g0.y;
        sp1 = sp1 + g1.x;
        sp2 = sp2 + g1.y;
        src = src + __ldg(pl.gcs + vc);
    }
    gather_sink_finish<R>(P, pl, G, gs, st, t, s, x, y, z, ms, ps0, ps1, ps2, nc, srho, sp0, sp1, sp2, src);
}

// Grid-stride over the processing order: the sinks in flight at a time are a
// window of consecutive sinks whose kernel cells fit in L2 (see the launcher).
template <int R>
__global__ void __launch_bounds__(kSinkThreads) k_gather_sink(KParams P, Box S, const double *__restrict__ u, Parts p,
                                                              PlanPtrs pl, double *__restrict__ G, DevStatus *st)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < p.count; t += stride)
        gather_sink_particle<R>(P, S, u, p, pl, G, st, t);
}

// Blocks per SM of the fused sink kernel (0: an L2 window of sinks in
// flight, as the sink gather; the default 6 is the measured best, see
// PMP_SINK_PASS1_MINB).
#ifndef PMP_SINK_PASS1_BPS
#define PMP_SINK_PASS1_BPS 6
#endif

// Per-warp shared memory of k_pass1_sink: the plan's FP32 centre squares
// ([3][W], padded), then for 8 sinks their Gaussian factors ([8][3W]), K and
// indices, and their host cells ([8][3]).
__host__ __device__ constexpr int pass1_sink_warp_bytes(int W)
{
    return (3 * W * 4 + 15) / 16 * 16 + (kPartsPerWarp * 3 * W + 2 * kPartsPerWarp) * 8 + kPartsPerWarp * 3 * 4;
}

// Plan, gather and ATOMIC deposit of the sink kind in one persistent kernel
// (pmp_gather_deposit; the per-cell records are written before it).  A warp
// takes 32 consecutive sinks of the processing order and
//   1. plans them one after the other (warp per sink, as k_plan);
//   2. gathers them, a lane per sink (as k_gather_sink), which also writes
//      each sink's Gaussian factors and K;
//   3. adds -a of their pairs to the one-field scratch, 8 sinks at a time,
//      lanes over the pairs (as k_deposit_atomic); k_sink_spread completes
//      Step 1.
template <int R>
// Resident blocks per SM the fused sink kernel is compiled for (78
// registers, no spills) and launched with.  512^3 sweep of (compiled for,
// launched): (any, 4) 24.6 ms, (6, 6) 23.7 ms, (6, 5) 24.8 ms, (8, 8) 31.9 ms,
// (any, 3) 30.8 ms: more sinks in flight than about one L2 of cell records
// costs more than the extra warps gain.
#ifndef PMP_SINK_PASS1_MINB
#define PMP_SINK_PASS1_MINB 6
#endif
__global__ void __launch_bounds__(128, PMP_SINK_PASS1_MINB) k_pass1_sink(KParams P, Box S, const double *__restrict__ u, Box B,
                                                    double *__restrict__ scr, Parts p, PlanPtrs pl,
                                                    double *__restrict__ G, DevStatus *st)
{
    constexpr int W = 2 * R + 1;
    constexpr int W3 = W * W * W;
    extern __shared__ __align__(16) unsigned char psm[];
    __shared__ int ncand_sh;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned *cand = reinterpret_cast<unsigned *>(psm);
    const size_t head = (size_t)(W3 * 4 + 15) / 16 * 16;
    unsigned char *wsm = psm + head + (size_t)wib * pass1_sink_warp_bytes(W);
    float *csq = reinterpret_cast<float *>(wsm);  // [3][W]
    double *wt = reinterpret_cast<double *>(wsm + (3 * W * 4 + 15) / 16 * 16);  // [8][3W]
    double *kt = wt + kPartsPerWarp * 3 * W;                                   // [8]
    long long *sidt = reinterpret_cast<long long *>(kt + kPartsPerWarp);       // [8]
    int *ht = reinterpret_cast<int *>(sidt + kPartsPerWarp);                   // [8][3]
    if (wib == 0) {
        const int n = build_candidates(P.rK, R, cand);
        if (lane == 0) ncand_sh = n;
    }
    __syncthreads();
    const int ncand = ncand_sh;
    const long long nwarps = (long long)gridDim.x * nw;
    const long long gs = p.count;
    for (long long t0 = ((long long)blockIdx.x * nw + wib) * 32; t0 < p.count; t0 += nwarps * 32) {
        const long long tl = t0 + lane;
        long long sl = 0;
        unsigned long long hl = kNoHost;
        float4 fl = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tl < p.count) {
            sl = pl.perm ? (long long)pl.perm[tl] : tl;
            hl = pl.hosts[sl];
            fl = pl.fr[sl];
        }
        const int nj = p.count - t0 < 32 ? (int)(p.count - t0) : 32;
        // 1. plan
        unsigned myc = 0;
        for (int j = 0; j < nj; ++j) {
            const long long s = __shfl_sync(kFull, sl, j);
            const unsigned long long hp = __shfl_sync(kFull, hl, j);
            float4 f4;
            f4.x = __shfl_sync(kFull, fl.x, j);
            f4.y = __shfl_sync(kFull, fl.y, j);
            f4.z = __shfl_sync(kFull, fl.z, j);
            f4.w = 0.f;
            if (hp != kNoHost) {
                const unsigned c = plan_particle<R, false, 0>(P, S, p, t0 + j, s, hp, f4, (unsigned)pl.cap, ncand,
                                                              cand, nullptr, csq, nullptr, nullptr, nullptr, pl.counts,
                                                              pl.slots, st);
                if (lane == j) myc = c;
            } else if (lane == 0) {
                pl.counts[t0 + j] = 0;
            }
        }
        __syncwarp();
        // 2. gather, lane per sink (a lane's loop keeps the loads of four
        // cells' records in flight; staging the records of six sinks at a time
        // in shared memory, with lanes over (sink, field) for the sums, left
        // fewer loads in flight and was slower: 23.1 -> 35.5 ms at 512^3)
        if (tl < p.count) gather_sink_particle<R, false>(P, S, u, p, pl, G, st, tl);
        __syncwarp();
        // 3. deposit of -a into the scratch, 8 sinks at a time
        for (int jb = 0; jb < nj; jb += kPartsPerWarp) {
            const int src = jb + (lane & (kPartsPerWarp - 1));
            const unsigned cj = __shfl_sync(kFull, myc, src);
            const long long sj = __shfl_sync(kFull, sl, src);
            const unsigned long long hj = __shfl_sync(kFull, hl, src);
            const bool mine = lane < kPartsPerWarp && jb + lane < nj;
            unsigned incl = mine ? cj : 0;
#pragma unroll
            for (int d = 1; d < kPartsPerWarp; d <<= 1) {
                const unsigned v = __shfl_up_sync(kFull, incl, d);
                if (lane >= d) incl += v;
            }
            const unsigned total = __shfl_sync(kFull, incl, kPartsPerWarp - 1);
            if (mine) {
                sidt[lane] = sj;
                kt[lane] = G[SK_K * gs + sj];
                int hx, hy, hz;
                unpack_host(hj, hx, hy, hz);
                ht[3 * lane] = hx;
                ht[3 * lane + 1] = hy;
                ht[3 * lane + 2] = hz;
            }
            __syncwarp();
            for (int i = lane; i < kPartsPerWarp * 3 * W; i += 32) {
                const int j = i / (3 * W);
                if (jb + j < nj) wt[i] = pl.wts[sidt[j] * (3 * W) + (i - j * 3 * W)];
            }
            __syncwarp();
            for (unsigned g0 = 0; g0 < total; g0 += 32) {
                const unsigned g = g0 + lane;
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
                if (g < total) {
                    const unsigned long long slot = (unsigned long long)(t0 + jb + j) * pl.cap + (g - before);
                    const PairCell cell = unpack_pair(slot_load<false>(pl.slots + slot), P.R);
                    const double *wj = wt + j * 3 * W;
                    const double w = (wj[cell.i - ht[3 * j] + R] * wj[W + cell.j - ht[3 * j + 1] + R]) *
                                     wj[2 * W + cell.k - ht[3 * j + 2] + R];
                    const double d0x =
                        __ldg(pl.dtr + vidx(S, owner(cell.i, S.n0), owner(cell.j, S.n1), owner(cell.k, S.n2)));
                    const double bh = kt[j] * w;  // >= +0: K and w are
                    const double a = max_nonneg(bh, d0x);
                    atomicAdd(scr + B.at(cell.i, cell.j, cell.k), neg_bits(a));
                    if (pl.pa) pl.pa[slot] = a;  // Step 4 reads it back (launch_return_sinks_stored)
                }
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// Step 1, atomic accumulation: a warp takes 8 consecutive particles of the
// processing order and spreads their pairs over its lanes
// ---------------------------------------------------------------------------

// Feedback deposition value of one pair from precomputed centre offsets.
__device__ __forceinline__ void fb_pair_delta_d(const double *__restrict__ u, const Box &S, const double *__restrict__ G,
                                                long long gs, long long s, const PairCell &c, double w, double d0,
                                                double d1, double d2, double dd, double dU[NF])
{
    double U[NF];
    load_cell(u, S, S.at(owner(c.i, S.n0), owner(c.j, S.n1), owner(c.k, S.n2)), U);
    const double vc[3] = {__ldg(G + FB_VX * gs + s), __ldg(G + FB_VY * gs + s), __ldg(G + FB_VZ * gs + s)};
    feedback_delta(w, U, __ldg(G + FB_Q * gs + s), __ldg(G + FB_E * gs + s), __ldg(G + FB_PV * gs + s), vc, d0, d1,
                   d2, dd, dU);
}

// With pv (sorted mode), pair q of the particle at processing position t
// (particle s) stores its value at pv[(offs[t] + q) * 5 + f], and its buffer
// cell and that place offs[t] + q at position koffs[s] + q of the sort's key
// and value lists (particle-index order), instead of adding into the buffer.
template <int R, bool FB>
#ifndef PMP_DEPOSIT_MINB
#define PMP_DEPOSIT_MINB 1
#endif
__global__ void __launch_bounds__(256, PMP_DEPOSIT_MINB) k_deposit_atomic(KParams P, Box S, const double *__restrict__ u, Box B,
                                                        double *__restrict__ b, Parts p,
                                                        const double *__restrict__ G, PlanPtrs pl,
                                                        double *__restrict__ E, double *__restrict__ scr,
                                                        double *__restrict__ pv,
                                                        const unsigned long long *__restrict__ offs,
                                                        const unsigned long long *__restrict__ koffs,
                                                        unsigned *__restrict__ skeys, unsigned *__restrict__ svals)
{
    constexpr int W = 2 * R + 1;
    constexpr int TAB = kPartsPerWarp * 3 * W;  // per warp: [8 particles][3 axes][W offsets]
    __shared__ double wtab[FB ? kMaxS3 + 1 : 1];
    __shared__ double dtab[FB ? 8 * TAB : 1], qtab[FB ? 8 * TAB : 1];
    __shared__ long long sidtab[8 * kPartsPerWarp];
    // sinks: per warp the 8 particles' Gaussian factors [8][3W], K and host cells
    __shared__ double swt[FB ? 1 : 8 * kPartsPerWarp * 3 * W];
    __shared__ double sK[FB ? 1 : 8 * kPartsPerWarp];
    __shared__ int shost[FB ? 1 : 8 * kPartsPerWarp * 3];
    if (FB) fill_omega_table(P, wtab);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double *dt = dtab + (FB ? wib * TAB : 0), *qt = qtab + (FB ? wib * TAB : 0);
    double *wt = swt + (FB ? 0 : wib * kPartsPerWarp * 3 * W);
    double *kt = sK + (FB ? 0 : wib * kPartsPerWarp);
    int *ht = shost + (FB ? 0 : wib * kPartsPerWarp * 3);
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long t0 = ((long long)blockIdx.x * (blockDim.x >> 5) + wib) * kPartsPerWarp; t0 < p.count;
         t0 += nwarps * kPartsPerWarp) {
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
        if (FB) {
            // centre offsets (c + 1/2) - x and their squares of the 8 particles
            __syncwarp();
            if (lane < kPartsPerWarp) sidtab[wib * kPartsPerWarp + lane] = sid;
            __syncwarp();
            for (int i = lane; i < TAB; i += 32) {
                const int j = i / (3 * W), r = i - j * (3 * W), a = r / W, o = r - a * W;
                const long long sj = sidtab[wib * kPartsPerWarp + j];
                if (t0 + j < p.count) {
                    const unsigned long long hp = __ldg(pl.hosts + sj);
                    if (hp != kNoHost) {
                        int hx, hy, hz;
                        unpack_host(hp, hx, hy, hz);
                        const int h = a == 0 ? hx : (a == 1 ? hy : hz);
                        const double xa = a == 0 ? __ldg(p.x + sj) : (a == 1 ? __ldg(p.y + sj) : __ldg(p.z + sj));
                        // (c + 1/2) - x, c + 1/2 built on the integer pipes (exact)
                        const double d = exact::half_odd(2 * (h + o - R) + 1) - xa;
                        dt[i] = d;
                        qt[i] = d * d;
                    }
                }
            }
            __syncwarp();
        } else {
            __syncwarp();
            if (lane < kPartsPerWarp) sidtab[wib * kPartsPerWarp + lane] = sid;
            __syncwarp();
            for (int i = lane; i < kPartsPerWarp * 3 * W; i += 32) {
                const int j = i / (3 * W);
                if (t0 + j < p.count) wt[i] = __ldg(pl.wts + sidtab[wib * kPartsPerWarp + j] * (3 * W) + (i - j * 3 * W));
            }
            if (lane < kPartsPerWarp && t0 + lane < p.count) {
                kt[lane] = __ldg(G + SK_K * p.count + sid);
                int hx, hy, hz;
                unpack_host(__ldg(pl.hosts + sid), hx, hy, hz);
                ht[3 * lane] = hx;
                ht[3 * lane + 1] = hy;
                ht[3 * lane + 2] = hz;
            }
            __syncwarp();
        }
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
                if (FB && P.kind == PMP_KIND_MASS) {
                    const double w = cell.cnt == P.S3 ? 1.0 : wtab[cell.cnt];
#pragma unroll
                    for (int f = 0; f < NF; ++f) dU[f] = w * __ldg(G + (MS_Q + f) * p.count + s);
                } else if (FB) {
                    int hx, hy, hz;
                    unpack_host(__ldg(pl.hosts + s), hx, hy, hz);
                    const int ix = j * 3 * W + (cell.i - hx + R), iy = j * 3 * W + W + (cell.j - hy + R),
                              iz = j * 3 * W + 2 * W + (cell.k - hz + R);
                    const double dd = (qt[ix] + qt[iy]) + qt[iz];
                    const double w = cell.cnt == P.S3 ? 1.0 : wtab[cell.cnt];
                    fb_pair_delta_d(u, S, G, p.count, s, cell, w, dt[ix], dt[iy], dt[iz], dd, dU);
                } else {
                    const double *wj = wt + j * 3 * W;
                    const double w = (wj[cell.i - ht[3 * j] + R] * wj[W + cell.j - ht[3 * j + 1] + R]) *
                                     wj[2 * W + cell.k - ht[3 * j + 2] + R];
                    const long long vc = vidx(S, owner(cell.i, S.n0), owner(cell.j, S.n1), owner(cell.k, S.n2));
                    const double bh = kt[j] * w;
                    const double a = max_nonneg(bh, __ldg(pl.dtr + vc));
                    if (scr) {
                        // the cell's factors (1, p/rho, E/rho) are applied by k_sink_spread
                        atomicAdd(scr + B.at(cell.i, cell.j, cell.k), neg_bits(a));
                        continue;
                    }
                    const double2 *d = reinterpret_cast<const double2 *>(pl.drec + vc * kDRec);
                    const double2 d0 = __ldg(d), d1 = __ldg(d + 1);
                    dU[0] = -a;
                    dU[1] = -(a * d0.x);
                    dU[2] = -(a * d0.y);
                    dU[3] = -(a * d1.x);
                    dU[4] = -(a * d1.y);
                }
                if (pv) {
                    const unsigned long long idx = offs[t0 + j] + (g - before);
                    double *o = pv + idx * NF;
#pragma unroll
                    for (int f = 0; f < NF; ++f) o[f] = dU[f];
                    const unsigned long long kpos = koffs[s] + (g - before);
                    skeys[kpos] = (unsigned)B.at(cell.i, cell.j, cell.k);
                    svals[kpos] = (unsigned)idx;
                    continue;
                }
                const long long bc = B.at(cell.i, cell.j, cell.k);
                if (E) {
                    // App. A.1: the error bound of the cell grows by eps |buffer| after each addition
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const long long o = (long long)f * B.fs + bc;
                        const double nv = atomicAdd(b + o, dU[f]) + dU[f];
                        atomicAdd(E + o, kEpsMachine * fabs(nv));
                    }
                } else {
#pragma unroll
                    for (int f = 0; f < NF; ++f) atomicAdd(b + (long long)f * B.fs + bc, dU[f]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Step 1, sorted accumulation
// ---------------------------------------------------------------------------



constexpr unsigned kLongRun = 32;  // runs longer than this are summed by k_segment_long
constexpr int kSegChunk = 4;       // pairs whose loads a run's thread issues together

// One thread per run of equal keys (a buffer cell) of at most kLongRun pairs:
// the run's pairs, which the stable sort kept in particle-index order, are
// added in that order on top of what the buffer holds.  Longer runs are
// queued for k_segment_long.  (Runs handed to the lanes as they finish, or
// sorted by length within blocks of 128, issue fewer FP64 additions but were
// slower: 0.67 ms here, 0.89 and 0.71 ms those, at 256^3; the kernel waits
// on its chain of dependent loads.)
__global__ void __launch_bounds__(128) k_segment_runs(Box B, double *__restrict__ b, const double *__restrict__ pv,
                                                      const unsigned long long *__restrict__ nruns_ptr,
                                                      const unsigned *__restrict__ uniq,
                                                      const unsigned *__restrict__ lens,
                                                      const unsigned *__restrict__ offs,
                                                      const unsigned *__restrict__ vals, unsigned *__restrict__ longq,
                                                      unsigned *__restrict__ nlong)
{
    const unsigned long long nruns = *nruns_ptr;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long r = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; r < nruns; r += stride) {
        const unsigned len = lens[r];
        if (len > kLongRun) {
            longq[atomicAdd(nlong, 1u)] = (unsigned)r;
            continue;
        }
        const unsigned key = uniq[r], o = offs[r];
        double acc[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) acc[f] = b[(long long)f * B.fs + key];
        // kSegChunk pairs' indices, then all their values, are loaded before
        // they are added (in run order): the loads of a chunk are in flight
        // together
        for (unsigned j0 = 0; j0 < len; j0 += kSegChunk) {
            unsigned idx[kSegChunk];
#pragma unroll
            for (int k = 0; k < kSegChunk; ++k) idx[k] = j0 + k < len ? __ldg(vals + o + j0 + k) : 0u;
            double v[kSegChunk][NF];
#pragma unroll
            for (int k = 0; k < kSegChunk; ++k) {
                const double *pk = pv + (unsigned long long)idx[k] * NF;
#pragma unroll
                for (int f = 0; f < NF; ++f) v[k][f] = j0 + k < len ? __ldg(pk + f) : 0.0;
            }
#pragma unroll
            for (int k = 0; k < kSegChunk; ++k) {
                if (j0 + k < len) {
#pragma unroll
                    for (int f = 0; f < NF; ++f) acc[f] = acc[f] + v[k][f];
                }
            }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) b[(long long)f * B.fs + key] = acc[f];
    }
}

constexpr int kLongPerWarp = 6;  // long runs a warp sums side by side (lanes 5 r + f)

// Long runs, kLongPerWarp per warp: for 32 consecutive pairs of each of its
// runs at a time, the lanes stage the pairs' stored values in shared memory,
// then lane 5 r + f adds field f of run r's pairs in run order -- for every
// run and field the same sequence of additions as a single thread would
// make.  An FP64 instruction costs the pipe the same with 5 or 30 active
// lanes, so six runs per warp take the time of one.  The loads are
// software-pipelined: the next chunk's values and the chunk after that's
// list indices are in flight while a chunk is summed, so a run of thousands
// of pairs (a Plummer core) costs about one load latency per 32 pairs.
__global__ void __launch_bounds__(128) k_segment_long(Box B, double *__restrict__ b, const double *__restrict__ pv,
                                                      const unsigned *__restrict__ uniq,
                                                      const unsigned *__restrict__ lens,
                                                      const unsigned *__restrict__ offs,
                                                      const unsigned *__restrict__ vals,
                                                      const unsigned *__restrict__ longq,
                                                      const unsigned *__restrict__ nlong_ptr)
{
    constexpr int G = kLongPerWarp;
    __shared__ double stage[4][G][32][NF];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int rme = lane / NF, fme = lane - rme * NF;  // lanes 0..29: run rme, field fme
    const unsigned nlong = *nlong_ptr;
    const unsigned ngroups = (nlong + G - 1) / G;
    const unsigned nw = gridDim.x * (blockDim.x >> 5);
    for (unsigned g = blockIdx.x * (blockDim.x >> 5) + wib; g < ngroups; g += nw) {
        unsigned key[G], o[G], len[G];
        unsigned maxlen = 0, mylen = 0, mykey = 0;
#pragma unroll
        for (int r = 0; r < G; ++r) {
            const unsigned q = g * G + r;
            len[r] = 0;
            key[r] = 0;
            o[r] = 0;
            if (q < nlong) {
                const unsigned rr = longq[q];
                key[r] = uniq[rr];
                o[r] = offs[rr];
                len[r] = lens[rr];
            }
            maxlen = len[r] > maxlen ? len[r] : maxlen;
            if (r == rme) {
                mylen = len[r];
                mykey = key[r];
            }
        }
        const bool mine = rme < G && mylen > 0;
        double acc = 0.0;
        if (mine) acc = b[(long long)fme * B.fs + mykey];
        // chunk 0's values, chunk 1's indices
        unsigned id[G];
        double v[G][NF];
#pragma unroll
        for (int r = 0; r < G; ++r) id[r] = lane < (int)len[r] ? __ldg(vals + o[r] + lane) : 0u;
#pragma unroll
        for (int r = 0; r < G; ++r) {
#pragma unroll
            for (int f = 0; f < NF; ++f)
                v[r][f] = lane < (int)len[r] ? __ldg(pv + (unsigned long long)id[r] * NF + f) : 0.0;
        }
#pragma unroll
        for (int r = 0; r < G; ++r) id[r] = 32u + lane < len[r] ? __ldg(vals + o[r] + 32u + lane) : 0u;
        for (unsigned c0 = 0; c0 < maxlen; c0 += 32) {
#pragma unroll
            for (int r = 0; r < G; ++r) {
                if (c0 + lane < len[r]) {
#pragma unroll
                    for (int f = 0; f < NF; ++f) stage[wib][r][lane][f] = v[r][f];
                }
            }
            __syncwarp();
            // in flight during the sums: chunk c0 + 32's values, chunk c0 + 64's indices
            const unsigned c1 = c0 + 32u, c2 = c0 + 64u;
#pragma unroll
            for (int r = 0; r < G; ++r) {
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    v[r][f] = c1 + lane < len[r] ? __ldg(pv + (unsigned long long)id[r] * NF + f) : 0.0;
            }
#pragma unroll
            for (int r = 0; r < G; ++r) id[r] = c2 + lane < len[r] ? __ldg(vals + o[r] + c2 + lane) : 0u;
            if (mine && mylen > c0) {
                // eight staged values at a time in registers, then added in order
                const unsigned m = mylen - c0 < 32u ? mylen - c0 : 32u;
                for (unsigned l0 = 0; l0 < m; l0 += 8) {
                    double x[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) x[k] = stage[wib][rme][l0 + k][fme];
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (l0 + k < m) acc = acc + x[k];
                }
            }
            __syncwarp();
        }
        if (mine) b[(long long)fme * B.fs + mykey] = acc;
    }
}

// ---------------------------------------------------------------------------
// Step 4: limited changes returned to sinks
// ---------------------------------------------------------------------------

// One kernel cell's terms of the Step-4 sums: the pair's removal a (as in
// the deposit, from the cell's rho - rho_Tr) limited by the cell's eta e,
// b = e a; the mass sum takes -b, the momentum sums take -b v (v = p/rho from
// the D record), fused.
__device__ __forceinline__ void sink_return_add(double K, double w, double tr, double2 v01, double v2, double e,
                                                double &a0, double &a1, double &a2, double &a3)
{
    const double bh = K * w;
    const double a = bh >= tr ? bh : tr;
    const double b = e == 1.0 ? a : e * a;
    a0 = a0 - b;
    a1 = fma(-b, v01.x, a1);
    a2 = fma(-b, v01.y, a2);
    a3 = fma(-b, v2, a3);
}

template <int R>
__device__ __forceinline__ void return_sink_particle(const KParams &P, const Box &S, const Parts &p,
                                                     const double *__restrict__ G, const PlanPtrs &pl, DevStatus *st,
                                                     double *wsm, long long t)
{
    constexpr int W = 2 * R + 1;
    const long long s = pl.perm ? (long long)pl.perm[t] : t;
    const int bad = position_status(S, p.x[s], p.y[s], p.z[s]);
    if (bad) {
        report(st, bad, s);
        return;
    }
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    const unsigned long long b0 = (unsigned long long)t * pl.cap;
    const unsigned nc = pl.counts[t];
    int hx, hy, hz;
    unpack_host(__ldg(pl.hosts + s), hx, hy, hz);
    double *wc = wsm + threadIdx.x;
    {
        const double *ws = pl.wts + s * (3 * W);
        for (int o = 0; o < 3 * W; ++o) wc[o * kSinkThreads] = __ldg(ws + o);
    }
    const double K = __ldg(G + SK_K * p.count + s);
    unsigned q = 0;
    for (; q + kUnroll <= nc; q += kUnroll) {
        double2 v01[kUnroll];
        double tr[kUnroll], v2[kUnroll], e[kUnroll], wx[kUnroll], wy[kUnroll], wz[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const PairCell c = unpack_pair(__ldg(pl.slots + b0 + q + k), P.R);
            const long long vc = vidx(S, owner(c.i, S.n0), owner(c.j, S.n1), owner(c.k, S.n2));
            const double *r = pl.drec + vc * kDRec;
            v01[k] = __ldg(reinterpret_cast<const double2 *>(r));
            v2[k] = __ldg(r + 2);
            tr[k] = __ldg(pl.dtr + vc);
            e[k] = __ldg(pl.deta + vc);
            wx[k] = wc[(c.i - hx + R) * kSinkThreads];
            wy[k] = wc[(W + c.j - hy + R) * kSinkThreads];
            wz[k] = wc[(2 * W + c.k - hz + R) * kSinkThreads];
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k)
            sink_return_add(K, (wx[k] * wy[k]) * wz[k], tr[k], v01[k], v2[k], e[k], a0, a1, a2, a3);
    }
    for (; q < nc; ++q) {
        const PairCell c = unpack_pair(__ldg(pl.slots + b0 + q), P.R);
        const long long vc = vidx(S, owner(c.i, S.n0), owner(c.j, S.n1), owner(c.k, S.n2));
        const double *r = pl.drec + vc * kDRec;
        const double w = (wc[(c.i - hx + R) * kSinkThreads] * wc[(W + c.j - hy + R) * kSinkThreads]) *
                         wc[(2 * W + c.k - hz + R) * kSinkThreads];
        sink_return_add(K, w, __ldg(pl.dtr + vc), __ldg(reinterpret_cast<const double2 *>(r)), __ldg(r + 2),
                        __ldg(pl.deta + vc), a0, a1, a2, a3);
    }
    p.m[s] = p.m[s] - a0 * P.V;
    p.px[s] = p.px[s] - a1 * P.V;
    p.py[s] = p.py[s] - a2 * P.V;
    p.pz[s] = p.pz[s] - a3 * P.V;
}

// Grid-stride over the processing order, like k_gather_sink.
template <int R>
__global__ void __launch_bounds__(kSinkThreads) k_return_sinks(KParams P, Box S, Parts p,
                                                                const double *__restrict__ G, PlanPtrs pl,
                                                                DevStatus *st)
{
    __shared__ double wsm[3 * (2 * R + 1) * kSinkThreads];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < p.count; t += stride)
        return_sink_particle<R>(P, S, p, G, pl, st, wsm, t);
}

// Step 4 from the stored removals: a warp per sink of the processing order,
// lane l over the sink's kernel cells l, l + 32, ...; each lane sums
// b = eta a and b v of its cells (v = p / rho from the D record, eta from
// deta), then the warp adds the 32 partial sums.  Per pair: one
// product and four additions of FP64 work, and loads of neighbouring cells'
// records by neighbouring lanes.
__global__ void __launch_bounds__(256) k_return_sinks_stored(KParams P, Box S, Parts p, PlanPtrs pl)
{
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < p.count; t += nwarps) {
        const long long s = pl.perm ? (long long)pl.perm[t] : t;
        if (pl.hosts[s] == kNoHost) continue;  // reported by the prologue
        const unsigned long long b0 = (unsigned long long)t * pl.cap;
        const unsigned nc = pl.counts[t];
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        for (unsigned q = lane; q < nc; q += 32) {
            const PairCell c = unpack_pair(__ldg(pl.slots + b0 + q), P.R);
            const double a = __ldg(pl.pa + b0 + q);
            const long long vc = vidx(S, owner(c.i, S.n0), owner(c.j, S.n1), owner(c.k, S.n2));
            const double *r = pl.drec + vc * kDRec;
            const double2 v01 = __ldg(reinterpret_cast<const double2 *>(r));
            const double v2 = __ldg(r + 2);
            const double b = __ldg(pl.deta + vc) * a;
            a0 = a0 - b;
            a1 = fma(-b, v01.x, a1);
            a2 = fma(-b, v01.y, a2);
            a3 = fma(-b, v2, a3);
        }
        // The warp's 32 partial sums of the four fields, reduced with the
        // fields spread over the lanes: after the first exchange each half
        // warp keeps two fields, after the second each quarter one, so a
        // lane makes 6 additions instead of 20 (each FP64 instruction costs
        // the pipe the same whatever the lanes hold).
        const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
        const double x = (hi16 ? a2 : a0) + __shfl_xor_sync(kFull, hi16 ? a0 : a2, 16);
        const double y = (hi16 ? a3 : a1) + __shfl_xor_sync(kFull, hi16 ? a1 : a3, 16);
        double z = (hi8 ? y : x) + __shfl_xor_sync(kFull, hi8 ? x : y, 8);
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) z = z + __shfl_xor_sync(kFull, z, o);
        // lane 8f holds field f: m, p_x, p_y, p_z
        if ((lane & 7) == 0) {
            double *dst = lane == 0 ? p.m : (lane == 8 ? p.px : (lane == 16 ? p.py : p.pz));
            dst[s] = dst[s] - z * P.V;
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

static inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

void launch_prologue(const Box &S, const Parts &p, unsigned *keys, unsigned *ids, const PlanPtrs &pl, DevStatus *st,
                     cudaStream_t stream)
{
    if (p.count == 0) return;
    int nmax = S.n0 > S.n1 ? S.n0 : S.n1;
    nmax = nmax > S.n2 ? nmax : S.n2;
    int bits = 0;
    while ((1 << bits) < nmax) ++bits;
    const int sh = bits > 10 ? bits - 10 : 0;
    k_prologue<<<blocks_for(p.count, 256), 256, 0, stream>>>(S, p, sh, keys, ids, pl.hosts, pl.fr, st);
}

template <int R, bool FB, int SC>
static void plan_one(const KParams &P, const Box &S, const Parts &p, const PlanPtrs &pl, DevStatus *st,
                     cudaStream_t stream)
{
    constexpr int W = 2 * R + 1;
    const int Sn = FB ? (SC ? SC : P.S) : 1;
    const size_t head = (size_t)(W * W * W * 4 + 15) / 16 * 16;
    const size_t wb = (size_t)plan_warp_bytes(W, Sn);
    int warps = 8;
    while (warps > 1 && head + warps * wb > 48 * 1024) --warps;
    const size_t sm = head + warps * wb;
    int dev = 0, nsm = 152, per_sm = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plan<R, FB, SC>, warps * 32, sm) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const long long need = (p.count + warps - 1) / warps;
    const long long grid = need < (long long)nsm * per_sm ? need : (long long)nsm * per_sm;
    k_plan<R, FB, SC><<<(unsigned)grid, warps * 32, sm, stream>>>(P, S, p, pl.perm, pl.hosts, pl.fr,
                                                                   (unsigned)pl.cap, pl.counts, pl.slots, st);
}

void launch_plan(const KParams &P, const Box &S, const Parts &p, const PlanPtrs &pl, DevStatus *st,
                 cudaStream_t stream)
{
    if (p.count == 0) return;
    if (P.kind != PMP_KIND_SINK) {  // supernova and particle-mesh kernels both carry omega
        if (P.S == 4) {
            PMP_DISPATCH_R(P.R, (plan_one<RR, true, 4>(P, S, p, pl, st, stream)));
        } else {
            PMP_DISPATCH_R(P.R, (plan_one<RR, true, 0>(P, S, p, pl, st, stream)));
        }
    } else {
        PMP_DISPATCH_R(P.R, (plan_one<RR, false, 0>(P, S, p, pl, st, stream)));
    }
}

template <int R, int SC>
static void plan_gather_one(const KParams &P, const Box &S, const double *u, const Parts &p, const PlanPtrs &pl,
                            double *G, DevStatus *st, cudaStream_t stream)
{
    constexpr int W = 2 * R + 1;
    const int Sn = SC ? SC : P.S;
    const size_t head = (size_t)(W * W * W * 4 + 15) / 16 * 16;
    const size_t wb = (size_t)plan_warp_bytes(W, Sn);
    int warps = 8;
    while (warps > 1 && head + warps * wb > 40 * 1024) --warps;
    const size_t sm = head + warps * wb;
    int dev = 0, nsm = 152, per_sm = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plan_gather_fb<R, SC>, warps * 32, sm) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const long long per_block = 32LL * warps;
    const long long need = (p.count + per_block - 1) / per_block;
    const long long grid = need < (long long)nsm * per_sm ? need : (long long)nsm * per_sm;
    k_plan_gather_fb<R, SC><<<(unsigned)grid, warps * 32, sm, stream>>>(P, S, u, p, pl, G, st);
}

void launch_plan_gather_fb(const KParams &P, const Box &S, const double *u, const Parts &p, const PlanPtrs &pl,
                           double *G, DevStatus *st, cudaStream_t stream)
{
    if (p.count == 0) return;
    if (P.S == 4) {
        PMP_DISPATCH_R(P.R, (plan_gather_one<RR, 4>(P, S, u, p, pl, G, st, stream)));
    } else {
        PMP_DISPATCH_R(P.R, (plan_gather_one<RR, 0>(P, S, u, p, pl, G, st, stream)));
    }
}

// Blocks of the thread-per-sink kernels.  They run grid-stride over the
// processing order, so the sinks in flight are a window of grid x
// kSinkThreads consecutive sinks; its kernel cells (about cells / sinks of
// them per sink, counted at kWindowBytesPerCell bytes each) are kept within
// half the L2, else every record is read from DRAM several times.
//
// The window is set in units of "L2 windows": blocks per SM such that the
// window's records take about one L2.  Measured on the 512^3 workload (sink
// gather 21.8 -> 16.0 ms, Step 4 27.2 -> 21.0 ms), the gather does best at
// about one and a half L2 windows (more resident warps hide its latency) and
// Step 4, whose shared-memory tables already limit residency, at about one.
static unsigned window_blocks(const Box &S, long long n, int threads, double bytes_per_cell, double l2_windows,
                              int forced)
{
    int dev = 0, nsm = 152, l2 = 126 << 20;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    }
    const double cells = (double)S.n0 * S.n1 * S.n2;
    const double per_particle = cells / (double)(n > 0 ? n : 1);
    long long bps = forced > 0 ? forced
                               : (long long)(l2_windows * (double)l2 /
                                                 ((double)nsm * threads * per_particle * bytes_per_cell) +
                                             0.5);
    if (bps < 1) bps = 1;
    if (bps > 16) bps = 16;
    const long long need = (n + threads - 1) / threads;
    const long long grid = (long long)nsm * bps;
    return (unsigned)(need < grid ? need : grid);
}

#ifndef PMP_SINK_GATHER_BPS
#define PMP_SINK_GATHER_BPS 0
#endif
#ifndef PMP_SINK_RETURN_BPS
#define PMP_SINK_RETURN_BPS 0
#endif
#ifndef PMP_FB_GATHER_BPS
#define PMP_FB_GATHER_BPS 0
#endif
#ifndef PMP_DEPOSIT_BPS
#define PMP_DEPOSIT_BPS 0
#endif

void launch_gather(const KParams &P, const Box &S, const double *u, const Parts &p, const PlanPtrs &pl, double *G,
                   DevStatus *st, cudaStream_t stream)
{
    if (p.count == 0) return;
    const unsigned nb = blocks_for(p.count, 128);
    if (P.kind == PMP_KIND_FEEDBACK) {
        // FP64-bound: a smaller window did not pay (512^3 sweep), full grid
        const unsigned nbf = PMP_FB_GATHER_BPS > 0 ? window_blocks(S, p.count, 128, 40.0, 1.0, PMP_FB_GATHER_BPS) : nb;
        k_gather_fb<<<nbf, 128, 0, stream>>>(P, S, u, p, pl, G, st);
    } else if (P.kind == PMP_KIND_MASS) {
        k_gather_mass<<<nb, 128, 0, stream>>>(P, S, p, pl, G, st);
    } else {
        const unsigned nbs = window_blocks(S, p.count, kSinkThreads, kWindowBytesPerCell, 1.5, PMP_SINK_GATHER_BPS);
        PMP_DISPATCH_R(P.R, (k_gather_sink<RR><<<nbs, kSinkThreads, 0, stream>>>(P, S, u, p, pl, G, st)));
    }
}

// The fused sink kernel: 4-warp blocks, each warp 32 sinks; a block has as
// many sinks in flight as a 128-thread gather block.  Its grid is
// PMP_SINK_PASS1_BPS blocks per SM (the sweep is at k_pass1_sink); with the
// macro set to 0, two L2 windows set it.  The first 512^3 sweep, before the
// kernel was compiled for its occupancy (blocks per SM): 2 -> 45.7 ms, 3 ->
// 32.8 ms, 4 -> 27.5 ms, 6 -> 37.5 ms (the separate plan, gather and deposit
// took 2.6 + 16.2 + 9.6 ms).
template <int R>
static void pass1_sink_one(const KParams &P, const Box &S, const double *u, const Box &B, double *scr,
                           const Parts &p, const PlanPtrs &pl, double *G, DevStatus *st, cudaStream_t stream)
{
    constexpr int W = 2 * R + 1;
    constexpr int warps = 4;
    const size_t sm = (size_t)(W * W * W * 4 + 15) / 16 * 16 + (size_t)warps * pass1_sink_warp_bytes(W);
    const unsigned nb = window_blocks(S, (p.count + 31) / 32 * 32, 32 * warps, kWindowBytesPerCell, 2.0, PMP_SINK_PASS1_BPS);
    const long long need = (p.count + 32LL * warps - 1) / (32LL * warps);
    const unsigned grid = (unsigned)(need < (long long)nb ? need : (long long)nb);
    k_pass1_sink<R><<<grid, 32 * warps, sm, stream>>>(P, S, u, B, scr, p, pl, G, st);
}

void launch_pass1_sink(const KParams &P, const Box &S, const double *u, const Box &B, double *scr, const Parts &p,
                       const PlanPtrs &pl, double *G, DevStatus *st, cudaStream_t stream)
{
    if (p.count == 0) return;
    PMP_DISPATCH_R(P.R, (pass1_sink_one<RR>(P, S, u, B, scr, p, pl, G, st, stream)));
}

static void launch_pair_kernel(const KParams &P, const Box &S, const double *u, const Box &B, double *b,
                               const Parts &p, const double *G, const PlanPtrs &pl, double *E, double *scr,
                               double *pv, const unsigned long long *offs, const unsigned long long *koffs,
                               unsigned *skeys, unsigned *svals, cudaStream_t stream)
{
    if (p.count == 0) return;
    // Only resident blocks: the grid-stride loop then moves all of them
    // through the processing order together, so the particles in flight are
    // one compact window (a larger grid spreads the resident blocks' chunks
    // over the whole order and every buffer line is fetched many times).
    const long long warps = (p.count + kPartsPerWarp - 1) / kPartsPerWarp;
    const long long blocks_needed = (warps + 7) / 8;
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int occ = 1;
    if (P.kind != PMP_KIND_SINK) {
        PMP_DISPATCH_R(P.R, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_deposit_atomic<RR, true>, 256, 0));
    } else {
        PMP_DISPATCH_R(P.R, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_deposit_atomic<RR, false>, 256, 0));
    }
    // resident blocks per SM (512^3 sweeps): the sink deposit does best with
    // two (18.1 -> 16.5 ms), the supernova deposit with three (23.9 -> 22.2
    // ms against two; more warps hide its loads' latency)
    const int cap = P.kind == PMP_KIND_SINK ? 2 : 3;
    occ = occ < cap ? occ : cap;
    if (PMP_DEPOSIT_BPS > 0) occ = PMP_DEPOSIT_BPS;
    if (occ < 1) occ = 1;
    const unsigned nb = (unsigned)(blocks_needed < (long long)nsm * occ ? blocks_needed : (long long)nsm * occ);
    if (P.kind != PMP_KIND_SINK) {
        PMP_DISPATCH_R(P.R, (k_deposit_atomic<RR, true><<<nb, 256, 0, stream>>>(P, S, u, B, b, p, G, pl, E, nullptr,
                                                                                 pv, offs, koffs, skeys, svals)));
    } else {
        PMP_DISPATCH_R(P.R, (k_deposit_atomic<RR, false><<<nb, 256, 0, stream>>>(P, S, u, B, b, p, G, pl, E, scr,
                                                                                  pv, offs, koffs, skeys, svals)));
    }
}

void launch_deposit_atomic(const KParams &P, const Box &S, const double *u, const Box &B, double *b, const Parts &p,
                           const double *G, const PlanPtrs &pl, double *E, double *scr, cudaStream_t stream)
{
    launch_pair_kernel(P, S, u, B, b, p, G, pl, E, scr, nullptr, nullptr, nullptr, nullptr, nullptr, stream);
}

void launch_pair_values(const KParams &P, const Box &S, const double *u, const Box &B, const Parts &p,
                        const double *G, const PlanPtrs &pl, const unsigned long long *offsets,
                        const unsigned long long *koffsets, double *pv, unsigned *keys, unsigned *vals,
                        cudaStream_t stream)
{
    launch_pair_kernel(P, S, u, B, nullptr, p, G, pl, nullptr, nullptr, pv, offsets, koffsets, keys, vals, stream);
}

__global__ void __launch_bounds__(256) k_counts_by_index(const unsigned *__restrict__ perm,
                                                         const unsigned *__restrict__ counts, long long n,
                                                         unsigned *__restrict__ counts_idx)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) counts_idx[perm ? perm[t] : t] = counts[t];
    if (t == n) counts_idx[n] = 0;
}

void launch_counts_by_index(const PlanPtrs &pl, long long n, unsigned *counts_idx, cudaStream_t stream)
{
    k_counts_by_index<<<blocks_for(n + 1, 256), 256, 0, stream>>>(pl.perm, pl.counts, n, counts_idx);
}


#ifndef PMP_SEG_LONG_BPS
#define PMP_SEG_LONG_BPS 8
#endif

void launch_segment_sum(const Box &B, double *b, const double *pv, const unsigned long long *nruns,
                        const unsigned *uniq, const unsigned *lens, const unsigned *offs, const unsigned *vals,
                        unsigned *longq, unsigned *nlong, cudaStream_t stream)
{
    const unsigned nb = 152u * 32u;
    cudaMemsetAsync(nlong, 0, sizeof(unsigned), stream);
    k_segment_runs<<<nb, 128, 0, stream>>>(B, b, pv, nruns, uniq, lens, offs, vals, longq, nlong);
    // long runs: eight four-warp blocks per SM (256^3 sweep of the blocks
    // per SM, whole segment sum: 1 -> 2.27 ms, 2 -> 1.81, 4 -> 1.66, 8 -> 1.44)
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    k_segment_long<<<(unsigned)nsm * PMP_SEG_LONG_BPS, 128, 0, stream>>>(B, b, pv, uniq, lens, offs, vals, longq,
                                                                        nlong);
}

#ifndef PMP_SINK_RETURN_STORED_BPS
#define PMP_SINK_RETURN_STORED_BPS 0
#endif

void launch_return_sinks_stored(const KParams &P, const Box &S, const Parts &p, const PlanPtrs &pl, DevStatus *st,
                                cudaStream_t stream)
{
    (void)st;
    if (p.count == 0) return;
    // resident blocks only, so the sinks in flight are one window of the
    // processing order; the window (8 sinks per block) is also kept near the
    // L2's size in cell records
    int dev = 0, nsm = 152, occ = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_return_sinks_stored, 256, 0) != cudaSuccess || occ < 1)
        occ = 1;
    const unsigned nb = window_blocks(S, p.count, 8, kWindowBytesPerCell, 1.0, PMP_SINK_RETURN_STORED_BPS);
    const long long cap = (long long)nsm * occ;
    const unsigned grid = (unsigned)((long long)nb < cap ? (long long)nb : cap);
    k_return_sinks_stored<<<grid, 256, 0, stream>>>(P, S, p, pl);
}

void launch_return_sinks(const KParams &P, const Box &S, const Parts &p, const double *G, const PlanPtrs &pl,
                         DevStatus *st, cudaStream_t stream)
{
    if (p.count == 0) return;
    const unsigned nb = window_blocks(S, p.count, kSinkThreads, kWindowBytesPerCell, 1.0, PMP_SINK_RETURN_BPS);
    PMP_DISPATCH_R(P.R, (k_return_sinks<RR><<<nb, kSinkThreads, 0, stream>>>(P, S, p, G, pl, st)));
}

}  // namespace pmp

// ---------------------------------------------------------------------------
// adjoint of a supernova pass
// ---------------------------------------------------------------------------

namespace pmp {

// L depends on particle s through Delta U^s_c (Eq. du with the readings of
// the forward pass).  With a = dL/dU_new at the owner of c (zero where the
// limiter acted) the per-pair sums are
//   Sgr = sum w a_rho, Sgp = sum w a_p, Srgp = sum w rho_c a_p, SgE = sum w a_E,
//   Sgpd = sum w a_p.dhat, SgEd = sum w a_E dhat,
//   X = sum (w/|d|) (t - dhat (dhat.t)),  t = a_p + a_E v_COM,
// and dL/dq = Sgr + v_COM.Sgp, dL/dv_COM = Srgp + q Sgp + Pv SgEd,
// dL/de = SgE, dL/dPv = Sgpd + v_COM.SgEd, dL/dx_s = -Pv X; the chain rule
// through q = m/V_snr, e = (E + |p|^2/2m)/V_snr, v_COM = (P_gas + p)/M_snr and
// Pv = |p_radial|/V_snr gives dL/d(m, E, p).  The kernel-cell set and omega
// are constant in position almost everywhere and carry no derivative.
__global__ void __launch_bounds__(128) k_backward_fb(KParams P, Box S, const double *__restrict__ u,
                                                     const double *__restrict__ gU, Parts p, PlanPtrs pl,
                                                     const unsigned char *__restrict__ pass,
                                                     const double *__restrict__ G, double *__restrict__ gout)
{
    __shared__ double wtab[kMaxS3 + 1];
    fill_omega_table(P, wtab);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.count) return;
    const long long s = pl.perm ? (long long)pl.perm[t] : t;
    const long long gs = p.count;
    if (pl.hosts[s] == kNoHost || !(p.m[s] > 0.0)) {
        for (int r = 0; r < 8; ++r) gout[r * gs + s] = 0.0;
        return;
    }
    const double x = p.x[s], y = p.y[s], z = p.z[s];
    const double m = p.m[s], pe0 = p.px[s], pe1 = p.py[s], pe2 = p.pz[s], Esn = p.e[s];
    const double Msnr = G[FB_MSNR * gs + s], Vsnr = G[FB_VSNR * gs + s];
    const double vc0 = G[FB_VX * gs + s], vc1 = G[FB_VY * gs + s], vc2 = G[FB_VZ * gs + s];
    const double prad = G[FB_PRAD * gs + s], q = G[FB_Q * gs + s], Pv = G[FB_PV * gs + s];
    const int regime = (int)G[FB_REGIME * gs + s];
    double Sgr = 0.0, Sgp0 = 0.0, Sgp1 = 0.0, Sgp2 = 0.0, Srgp0 = 0.0, Srgp1 = 0.0, Srgp2 = 0.0, SgE = 0.0;
    double Sgpd = 0.0, SgEd0 = 0.0, SgEd1 = 0.0, SgEd2 = 0.0, X0 = 0.0, X1 = 0.0, X2 = 0.0;
    const unsigned long long b0 = (unsigned long long)t * pl.cap;
    const unsigned nc = pl.counts[t];
    for (unsigned k = 0; k < nc; ++k) {
        const PairCell c = unpack_pair(pl.slots[b0 + k], P.R);
        const int oi = owner(c.i, S.n0), oj = owner(c.j, S.n1), ok = owner(c.k, S.n2);
        if (!pass[vidx(S, oi, oj, ok)]) continue;
        const long long o = S.at(oi, oj, ok);
        const double w = wtab[c.cnt];
        const double ar = __ldg(gU + o), ap0 = __ldg(gU + S.fs + o), ap1 = __ldg(gU + 2 * S.fs + o),
                     ap2 = __ldg(gU + 3 * S.fs + o), aE = __ldg(gU + 4 * S.fs + o);
        const double rho = __ldg(u + o);
        Sgr += w * ar;
        Sgp0 += w * ap0;
        Sgp1 += w * ap1;
        Sgp2 += w * ap2;
        Srgp0 += w * rho * ap0;
        Srgp1 += w * rho * ap1;
        Srgp2 += w * rho * ap2;
        SgE += w * aE;
        const double d0 = ((double)c.i + 0.5) - x, d1 = ((double)c.j + 0.5) - y, d2 = ((double)c.k + 0.5) - z;
        const double dd = d0 * d0 + d1 * d1 + d2 * d2;
        if (dd > 0.0) {
            const double dist = exact::sqrt_rn(dd);
            const double h0 = exact::div_rn(d0, dist), h1 = exact::div_rn(d1, dist), h2 = exact::div_rn(d2, dist);
            Sgpd += w * (ap0 * h0 + ap1 * h1 + ap2 * h2);
            SgEd0 += w * aE * h0;
            SgEd1 += w * aE * h1;
            SgEd2 += w * aE * h2;
            const double t0 = ap0 + aE * vc0, t1 = ap1 + aE * vc1, t2 = ap2 + aE * vc2;
            const double th = t0 * h0 + t1 * h1 + t2 * h2;
            const double f = exact::div_rn(w, dist);
            X0 += f * (t0 - h0 * th);
            X1 += f * (t1 - h1 * th);
            X2 += f * (t2 - h2 * th);
        }
    }
    const double dLdq = Sgr + (vc0 * Sgp0 + vc1 * Sgp1 + vc2 * Sgp2);
    const double dLdv0 = Srgp0 + q * Sgp0 + Pv * SgEd0, dLdv1 = Srgp1 + q * Sgp1 + Pv * SgEd1,
                 dLdv2 = Srgp2 + q * Sgp2 + Pv * SgEd2;
    const double dLde = SgE;
    const double dLdPv = Sgpd + (vc0 * SgEd0 + vc1 * SgEd1 + vc2 * SgEd2);
    double dpr_dm = 0.0, dpr_dE = 0.0;
    if (regime == 2) {
        dpr_dm = -0.17 * prad / Msnr;
    } else if (regime == 1) {
        dpr_dm = prad / (2.0 * m);
        dpr_dE = Esn != 0.0 ? prad / (2.0 * Esn) : 0.0;
    }
    const double pe2sum = pe0 * pe0 + pe1 * pe1 + pe2 * pe2;
    const double vdot = dLdv0 * vc0 + dLdv1 * vc1 + dLdv2 * vc2;
    gout[0 * gs + s] = dLdq / Vsnr - dLde * pe2sum / (2.0 * m * m * Vsnr) - vdot / Msnr + dLdPv * dpr_dm / Vsnr;
    gout[1 * gs + s] = dLde / Vsnr + dLdPv * dpr_dE / Vsnr;
    gout[2 * gs + s] = dLde * pe0 / (m * Vsnr) + dLdv0 / Msnr;
    gout[3 * gs + s] = dLde * pe1 / (m * Vsnr) + dLdv1 / Msnr;
    gout[4 * gs + s] = dLde * pe2 / (m * Vsnr) + dLdv2 / Msnr;
    gout[5 * gs + s] = -Pv * X0;
    gout[6 * gs + s] = -Pv * X1;
    gout[7 * gs + s] = -Pv * X2;
}

void launch_backward_fb(const KParams &P, const Box &S, const double *u, const double *gU, const Parts &p,
                        const PlanPtrs &pl, const unsigned char *pass, const double *G, double *gout,
                        cudaStream_t stream)
{
    if (p.count == 0) return;
    k_backward_fb<<<blocks_for(p.count, 128), 128, 0, stream>>>(P, S, u, gU, p, pl, pass, G, gout);
}

}  // namespace pmp
