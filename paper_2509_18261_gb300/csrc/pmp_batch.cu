// pmp_batch.cu -- the batched form: one PMP pass (Sec. 2.2, Steps 1-5) over
// many uneven patches of one level that tile a periodic domain.
//
// Each patch reads the ghost cells of the state through its 26 neighbours and
// sums the ghost cells of its buffer into theirs in the fixed order of App.
// A.2, so the caller never fills ghost cells.  The work is cut into items:
//
//   gather   one warp per particle: kernel membership and the omega sub-point
//            count of each of the (2R+1)^3 offsets, kept in a per-particle
//            table; the kernel sums in canonical order (lane order, one lane
//            adds)
//   deposit  OWNER: one block per tile of a patch's padded box; the particles
//            of the patch whose kernel reaches the tile are staged in shared
//            memory in index order, each thread adds their contributions to
//            its cell in that order and writes the cell once -- deterministic,
//            without atomics, and it is also the zeroing of the buffer.
//            ATOMIC: the patch's padded box is zeroed in the gather phase and
//            one warp per particle adds its pairs with FP64 atomics.
//   step 4   one warp per sink: eta at each kernel cell from the owning
//            cell's pre-update state and folded sum
//   apply    one warp per row of valid cells: the ghost sum (images from the
//            neighbours), the limiter and the update fused; a cell whose
//            summed change is zero in every field is only read
//
// PERSISTENT runs every phase in one cooperative launch, blocks taking items
// from a queue per phase, with a grid barrier between phases whose waits are
// bounded in time (a block that gives up sets PMP_ERR_TIMEOUT and every block
// returns).  PER_PATCH launches each phase once per patch (the plain form).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "pmp.h"
#include "pmp_ctx.h"
#include "pmp_device.cuh"
#include "pmp_launch.h"
#include "pmp_plan.cuh"

namespace pmp {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kCap = 512;  // candidate particles staged per chunk of a tile
constexpr unsigned kFullMask = 0xffffffffu;
constexpr unsigned long long kNoHostB = ~0ULL;
constexpr unsigned long long kWaitNs = 4000000000ULL;  // grid-barrier wait limit
constexpr int kPackThreads = 256;  // cells per pack item and block
constexpr int kRegionSlots = 6;    // region lists a batch keeps for packing

struct PatchDev {
    int n[3];
    int g;
    int px, py;      // padded extents along x and y
    int nb[26];      // neighbour patches, offsets (ox, oy, oz) with oz slowest
    long long pxy;   // padded plane
    long long off;   // arena offset of (field 0, padded cell 0)
    long long fs;    // field stride
    long long vbase; // valid cells of the patches before this one
};

enum { STRAT_OWNER_CUBE = 0, STRAT_OWNER_ROWS = 1, STRAT_ATOMIC = 2, NSTRAT = 3 };

// OWNER: the tile [lo, hi) of padded-local coordinates.  ATOMIC: particles
// [lo[0], hi[0]) (absolute indices) of the patch.
struct DepItem {
    int patch, strat;
    int lo[3], hi[3];
};
struct AppItem {
    int patch, k0, k1, pad_;
};
struct ZeroItem {
    int patch, pad_;
    long long c0, c1;  // padded flat cells [c0, c1) of the patch, all fields
};

struct Ctl {
    unsigned q[8];  // work-queue heads, one per phase
    unsigned count, gen, abort, pad_;
};

struct BArgs {
    KParams P;
    const PatchDev *T;
    int np, nzero, ndep, napp;
    const long long *first;  // [np + 1]
    double *u, *b;
    Parts p;
    double *G;
    double *eta_out;
    double *wts;                // sink: [N][3W] per-axis Gaussian factors
    unsigned short *om;         // [N][W3] omega sub-point count (0: not in the kernel)
    unsigned long long *hostp;  // [N] packed host cell, kNoHostB if invalid
    const DepItem *dep;
    const AppItem *app;
    const ZeroItem *zero;
    Ctl *ctl;
    DevStatus *st;
    unsigned hold;  // arrivals a grid barrier waits for beyond the grid (0; 1 only to test the timeout)
    int ph0, ph1;   // the phases [ph0, ph1] this launch runs (0 gather, 1 deposit, 2 Step 4, 3 apply)
};

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------

__device__ __forceinline__ int nb_slot(int ox, int oy, int oz)
{
    const int t = ((oz + 1) * 3 + (oy + 1)) * 3 + (ox + 1);
    return t > 13 ? t - 1 : t;
}

__device__ __forceinline__ long long pcell(const PatchDev *T, int i, int j, int k)
{
    const int g = T->g;
    return T->off + (long long)(k + g) * T->pxy + (long long)(j + g) * T->px + (long long)(i + g);
}

// The arena index (field 0) and field stride of the valid cell that padded
// coordinate (i, j, k) of patch p stands for.
struct Owner {
    long long c, fs;
    int q, i, j, k;
};

__device__ __forceinline__ Owner owner_of(const PatchDev *TT, int p, int i, int j, int k)
{
    const PatchDev *T = TT + p;
    const int ox = i < 0 ? -1 : (i >= T->n[0] ? 1 : 0);
    const int oy = j < 0 ? -1 : (j >= T->n[1] ? 1 : 0);
    const int oz = k < 0 ? -1 : (k >= T->n[2] ? 1 : 0);
    Owner o;
    if (!(ox | oy | oz)) {
        o.q = p;
        o.i = i;
        o.j = j;
        o.k = k;
    } else {
        o.q = T->nb[nb_slot(ox, oy, oz)];
        const PatchDev *Q = TT + o.q;
        o.i = i + (ox < 0 ? Q->n[0] : 0) - (ox > 0 ? T->n[0] : 0);
        o.j = j + (oy < 0 ? Q->n[1] : 0) - (oy > 0 ? T->n[1] : 0);
        o.k = k + (oz < 0 ? Q->n[2] : 0) - (oz > 0 ? T->n[2] : 0);
    }
    const PatchDev *Q = TT + o.q;
    o.c = pcell(Q, o.i, o.j, o.k);
    o.fs = Q->fs;
    return o;
}

// Loads that bypass L1: values written by other blocks earlier in the same
// persistent launch must come from L2.
__device__ __forceinline__ void load5(const double *a, long long c, long long fs, double V[NF])
{
#pragma unroll
    for (int f = 0; f < NF; ++f) V[f] = __ldcg(a + (long long)f * fs + c);
}

// Summed buffer of valid cell (i, j, k) of patch q: ((B_c + B_img1) + B_img2)
// + ... over its ghost images in lexicographic order of the image offset
// (oz, oy, ox) (App. A.2).  The image at offset o lies in the neighbour
// nb[-o], at c + n_neighbour (o = 1), c - n_q (o = -1) or c (o = 0) per axis;
// it exists when that coordinate is inside the neighbour's padded box, that
// is for o = 1 when c < g and for o = -1 when c >= n_q - g.  `img` reports
// whether an image held a non-zero value.
__device__ __forceinline__ void folded_at(const BArgs &a, int q, int i, int j, int k, double D[NF], bool &img)
{
    const PatchDev *T = a.T + q;
    load5(a.b, pcell(T, i, j, k), T->fs, D);
    img = false;
    const int g = T->g, n0 = T->n[0], n1 = T->n[1], n2 = T->n[2];
    const bool xl = i < g, xh = i >= n0 - g, yl = j < g, yh = j >= n1 - g, zl = k < g, zh = k >= n2 - g;
    if (!(xl | xh | yl | yh | zl | zh)) return;
    unsigned long long nz = 0;
    for (int oz = -1; oz <= 1; ++oz) {
        if ((oz == 1 && !zl) || (oz == -1 && !zh)) continue;
        for (int oy = -1; oy <= 1; ++oy) {
            if ((oy == 1 && !yl) || (oy == -1 && !yh)) continue;
            for (int ox = -1; ox <= 1; ++ox) {
                if ((ox == 1 && !xl) || (ox == -1 && !xh)) continue;
                if (!ox && !oy && !oz) continue;
                const PatchDev *Rn = a.T + T->nb[nb_slot(-ox, -oy, -oz)];
                const int gi = i + (ox > 0 ? Rn->n[0] : (ox < 0 ? -n0 : 0));
                const int gj = j + (oy > 0 ? Rn->n[1] : (oy < 0 ? -n1 : 0));
                const int gk = k + (oz > 0 ? Rn->n[2] : (oz < 0 ? -n2 : 0));
                const long long c = pcell(Rn, gi, gj, gk);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const double v = __ldcg(a.b + (long long)f * Rn->fs + c);
                    nz |= (unsigned long long)__double_as_longlong(v) << 1;
                    D[f] = D[f] + v;
                }
            }
        }
    }
    img = nz != 0;
}

// Largest p with first[p] <= s (the patch holding particle s).
__device__ __forceinline__ int patch_of(const long long *first, int np, long long s)
{
    int lo = 0, hi = np;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(first + mid) <= s) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// shared memory
// ---------------------------------------------------------------------------

template <int R>
struct SmemT {
    static constexpr int W = 2 * R + 1;
    union {
        struct {
            double red[kWarps][32][6];  // per-warp lane values for ordered sums
            double ws[kWarps][3 * W];   // sink: per-axis Gaussian factors
        } pw;
        struct {
            long long s[kCap];
            int4 h[kCap];   // host cell of the candidate
            double x[kCap], y[kCap], z[kCap];
            double d[6][kCap];  // feedback: q, e, Pv, v_COM; sink: K
        } dep;
    } u;
    double wtab[kMaxS * kMaxS * kMaxS + 1];
    int wcnt[kWarps];
    int nc;
    int item;
    int ok;
};

// ---------------------------------------------------------------------------
// gather: one warp per particle
// ---------------------------------------------------------------------------

template <int R, bool FB>
__device__ void gather_particle(const BArgs &a, long long s, SmemT<R> &sm)
{
    constexpr int W = 2 * R + 1, W3 = W * W * W;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long N = a.p.count;
    const KParams &P = a.P;
    const int p = patch_of(a.first, a.np, s);
    const PatchDev *T = a.T + p;
    const double x = a.p.x[s], y = a.p.y[s], z = a.p.z[s];
    const double m = a.p.m[s];
    int bad = 0;
    if (!(x == x && y == y && z == z)) bad = PMP_ERR_NONFINITE;
    else if (!(x >= 0.0 && x < (double)T->n[0] && y >= 0.0 && y < (double)T->n[1] && z >= 0.0 &&
               z < (double)T->n[2]))
        bad = PMP_ERR_PARTICLE_OUTSIDE;
    else if (!(m > 0.0)) bad = PMP_ERR_NONFINITE;
    unsigned short *om = a.om + s * W3;
    if (bad) {
        if (lane == 0) {
            report(a.st, bad, s);
            a.hostp[s] = kNoHostB;
            for (int r = 0; r < (FB ? FB_ROWS : SK_ROWS); ++r) a.G[r * N + s] = 0.0;
        }
        for (int k = lane; k < W3; k += 32) om[k] = 0;
        return;
    }
    const int h0 = (int)floor(x), h1 = (int)floor(y), h2 = (int)floor(z);
    if (lane == 0) a.hostp[s] = pack_host(h0, h1, h2);
    double (*red)[6] = sm.u.pw.red[wib];
    // lane f < 5 keeps sum f: one FP64 instruction per cell for all five sums
    // (an FP64 instruction with one active lane costs the pipe about what a
    // full-warp one does); the sequence of additions per sum is unchanged
    double acc = 0.0;
    int nk = 0;
    for (int k0 = 0; k0 < W3; k0 += 32) {
        const int k = k0 + lane;
        int cnt = 0;
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0, v4 = 0.0;
        if (k < W3) {
            const int oz = k / (W * W), oy = (k / W) % W, ox = k % W;
            const int ci = h0 + ox - R, cj = h1 + oy - R, ck = h2 + oz - R;
            const double d0 = ((double)ci + 0.5) - x, d1 = ((double)cj + 0.5) - y, d2 = ((double)ck + 0.5) - z;
            if ((d0 * d0 + d1 * d1) + d2 * d2 < P.r2) cnt = FB ? covered_count(P, ci, cj, ck, x, y, z) : 1;
            om[k] = (unsigned short)cnt;
            if (cnt) {
                const Owner o = owner_of(a.T, p, ci, cj, ck);
                double U[NF];
                load5(a.u, o.c, o.fs, U);
                if (FB) {
                    // omega and the cell's rho, p; lane 0 fuses the products into the sums
                    v0 = (double)cnt / (double)P.S3;
                    v1 = U[0];
                    v2 = U[1];
                    v3 = U[2];
                    v4 = U[3];
                } else {
                    double cs, rtr;
                    sink_cell(P, U, exact::div_rn(1.0, U[0]), cs, rtr);
                    v0 = U[0];
                    v1 = U[1];
                    v2 = U[2];
                    v3 = U[3];
                    v4 = U[0] * cs;
                }
            }
        }
        const unsigned mem = __ballot_sync(kFullMask, cnt != 0);
        red[lane][0] = v0;
        red[lane][1] = v1;
        red[lane][2] = v2;
        red[lane][3] = v3;
        red[lane][4] = v4;
        __syncwarp();
        if (lane < 5) {
            for (int l = 0; l < 32; ++l) {
                if (!((mem >> l) & 1u)) continue;
                if (FB) {
                    // sum 0 = sum omega (fma(1, w, s) == s + w); sums 1-4 = fma(omega, v, s)
                    const double w = red[l][0];
                    acc = fma(lane == 0 ? 1.0 : w, lane == 0 ? w : red[l][lane], acc);
                } else {
                    acc = acc + red[l][lane];
                }
            }
        }
        nk += __popc(mem);
        __syncwarp();
    }
    const double s0 = __shfl_sync(kFullMask, acc, 0), s1 = __shfl_sync(kFullMask, acc, 1),
                 s2 = __shfl_sync(kFullMask, acc, 2), s3 = __shfl_sync(kFullMask, acc, 3),
                 s4 = __shfl_sync(kFullMask, acc, 4);
    if (FB) {
        if (lane == 0 &&
            !fb_gather_rows(P, s0, s1, s2, s3, s4, m, a.p.px[s], a.p.py[s], a.p.pz[s], a.p.e[s], a.G + s, N))
            report(a.st, PMP_ERR_NONFINITE, s);
        return;
    }
    // sinks: ambient state, then the Gaussian weights and their sum
    SinkAmbient am;
    if (lane == 0) am = sink_ambient(P, s0, s1, s2, s3, s4, nk, m, a.p.px[s], a.p.py[s], a.p.pz[s]);
    const double ra2 = __shfl_sync(kFullMask, lane == 0 ? am.ra2 : 0.0, 0);
    double *ws = sm.u.pw.ws[wib];
    for (int o = lane; o < 3 * W; o += 32) {
        const int ax = o / W, oo = o - ax * W;
        const int h = ax == 0 ? h0 : (ax == 1 ? h1 : h2);
        const double c = ax == 0 ? x : (ax == 1 ? y : z);
        const double wv = sink_axis_weight(((double)(h + oo - R) + 0.5) - c, ra2);
        ws[o] = wv;
        a.wts[s * (3 * W) + o] = wv;
    }
    __syncwarp();
    double sumw = 0.0;
    for (int k0 = 0; k0 < W3; k0 += 32) {
        const int k = k0 + lane;
        double wxy = 0.0, wz = 0.0;
        bool mem = false;
        if (k < W3 && om[k]) {
            const int oz = k / (W * W), oy = (k / W) % W, ox = k % W;
            wxy = ws[ox] * ws[W + oy];
            wz = ws[2 * W + oz];
            mem = true;
        }
        const unsigned mm = __ballot_sync(kFullMask, mem);
        red[lane][0] = wxy;
        red[lane][1] = wz;
        __syncwarp();
        if (lane == 0)
            for (int l = 0; l < 32; ++l)
                if ((mm >> l) & 1u) sumw = fma(red[l][0], red[l][1], sumw);
        __syncwarp();
    }
    if (lane == 0 && !sink_gather_rows(P, am, sumw, nk, a.G + s, N)) report(a.st, PMP_ERR_NONFINITE, s);
}

// ---------------------------------------------------------------------------
// deposit, OWNER strategy: one block per tile
// ---------------------------------------------------------------------------

template <int R, bool FB>
__device__ void deposit_tile(const BArgs &a, const DepItem &it, SmemT<R> &sm)
{
    constexpr int W = 2 * R + 1, W3 = W * W * W;
    const KParams &P = a.P;
    const int p = it.patch;
    const PatchDev *T = a.T + p;
    const long long N = a.p.count;
    const long long f0 = __ldg(a.first + p), f1 = __ldg(a.first + p + 1);
    const int lo0 = it.lo[0], lo1 = it.lo[1], lo2 = it.lo[2];
    const int tx = it.hi[0] - lo0, ty = it.hi[1] - lo1, tz = it.hi[2] - lo2;
    const int ncell = tx * ty * tz;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long fs = T->fs;
    bool first_chunk = true;
    long long scan = f0;
    for (;;) {
        if (threadIdx.x == 0) sm.nc = 0;
        __syncthreads();
        while (scan < f1) {
            const long long s = scan + threadIdx.x;
            bool c = false;
            int hh0 = 0, hh1 = 0, hh2 = 0;
            if (s < f1) {
                const unsigned long long hp = __ldcg(a.hostp + s);
                if (hp != kNoHostB) {
                    unpack_host(hp, hh0, hh1, hh2);
                    c = hh0 + R >= lo0 && hh0 - R < lo0 + tx && hh1 + R >= lo1 && hh1 - R < lo1 + ty &&
                        hh2 + R >= lo2 && hh2 - R < lo2 + tz;
                }
            }
            const unsigned bal = __ballot_sync(kFullMask, c);
            if (lane == 0) sm.wcnt[wib] = __popc(bal);
            __syncthreads();
            int before = sm.nc, total = 0;
            for (int w = 0; w < kWarps; ++w) {
                if (w < wib) before += sm.wcnt[w];
                total += sm.wcnt[w];
            }
            if (c) {
                const int pos = before + __popc(bal & ((1u << lane) - 1u));
                sm.u.dep.s[pos] = s;
                sm.u.dep.h[pos] = make_int4(hh0, hh1, hh2, 0);
                sm.u.dep.x[pos] = a.p.x[s];
                sm.u.dep.y[pos] = a.p.y[s];
                sm.u.dep.z[pos] = a.p.z[s];
                if (FB) {
                    sm.u.dep.d[0][pos] = __ldcg(a.G + FB_Q * N + s);
                    sm.u.dep.d[1][pos] = __ldcg(a.G + FB_E * N + s);
                    sm.u.dep.d[2][pos] = __ldcg(a.G + FB_PV * N + s);
                    sm.u.dep.d[3][pos] = __ldcg(a.G + FB_VX * N + s);
                    sm.u.dep.d[4][pos] = __ldcg(a.G + FB_VY * N + s);
                    sm.u.dep.d[5][pos] = __ldcg(a.G + FB_VZ * N + s);
                } else {
                    sm.u.dep.d[0][pos] = __ldcg(a.G + SK_K * N + s);
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) sm.nc = before + total;
            scan += kThreads;
            __syncthreads();
            if (sm.nc + kThreads > kCap) break;
        }
        const int nc = sm.nc;
        for (int c = threadIdx.x; c < ncell; c += kThreads) {
            const int ii = c % tx, r = c / tx;
            const int i = lo0 + ii, j = lo1 + r % ty, k = lo2 + r / ty;
            const long long cb = pcell(T, i, j, k);
            double acc[NF];
            if (first_chunk) {
#pragma unroll
                for (int f = 0; f < NF; ++f) acc[f] = 0.0;
            } else {
                load5(a.b, cb, fs, acc);
            }
            bool haveU = false;
            double U[NF], tr = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0, q4 = 0.0;
            for (int t = 0; t < nc; ++t) {
                const int4 h = sm.u.dep.h[t];
                const int ox = i - h.x + R, oy = j - h.y + R, oz = k - h.z + R;
                if ((unsigned)ox > 2u * R || (unsigned)oy > 2u * R || (unsigned)oz > 2u * R) continue;
                const long long s = sm.u.dep.s[t];
                const int cnt = __ldcg(a.om + s * W3 + (oz * W + oy) * W + ox);
                if (!cnt) continue;
                if (!haveU) {
                    const Owner o = owner_of(a.T, p, i, j, k);
                    load5(a.u, o.c, o.fs, U);
                    if (!FB) {
                        const double inv = exact::div_rn(1.0, U[0]);
                        tr = U[0] - P.ctr * sink_cs2(P, U, inv);
                        q1 = U[1] * inv;
                        q2 = U[2] * inv;
                        q3 = U[3] * inv;
                        q4 = U[4] * inv;
                    }
                    haveU = true;
                }
                double dU[NF];
                if (FB) {
                    const double w = sm.wtab[cnt];
                    const double d0 = ((double)i + 0.5) - sm.u.dep.x[t];
                    const double d1 = ((double)j + 0.5) - sm.u.dep.y[t];
                    const double d2 = ((double)k + 0.5) - sm.u.dep.z[t];
                    const double dd = (d0 * d0 + d1 * d1) + d2 * d2;
                    const double vc[3] = {sm.u.dep.d[3][t], sm.u.dep.d[4][t], sm.u.dep.d[5][t]};
                    feedback_delta(w, U, sm.u.dep.d[0][t], sm.u.dep.d[1][t], sm.u.dep.d[2][t], vc, d0, d1, d2, dd,
                                   dU);
                } else {
                    const double *ws = a.wts + s * (3 * W);
                    const double w = (__ldcg(ws + ox) * __ldcg(ws + W + oy)) * __ldcg(ws + 2 * W + oz);
                    const double bh = sm.u.dep.d[0][t] * w;
                    const double am = bh >= tr ? bh : tr;
                    dU[0] = -am;
                    dU[1] = -(am * q1);
                    dU[2] = -(am * q2);
                    dU[3] = -(am * q3);
                    dU[4] = -(am * q4);
                }
#pragma unroll
                for (int f = 0; f < NF; ++f) acc[f] = acc[f] + dU[f];
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) a.b[(long long)f * fs + cb] = acc[f];
        }
        first_chunk = false;
        if (scan >= f1) break;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// deposit, ATOMIC strategy: one warp per particle, FP64 atomics
// ---------------------------------------------------------------------------

template <int R, bool FB>
__device__ void deposit_atomic_particle(const BArgs &a, int p, long long s, SmemT<R> &sm)
{
    constexpr int W = 2 * R + 1, W3 = W * W * W;
    const KParams &P = a.P;
    const int lane = threadIdx.x & 31;
    const unsigned long long hp = __ldcg(a.hostp + s);
    if (hp == kNoHostB) return;
    int h0, h1, h2;
    unpack_host(hp, h0, h1, h2);
    const PatchDev *T = a.T + p;
    const long long N = a.p.count;
    const double x = a.p.x[s], y = a.p.y[s], z = a.p.z[s];
    double g0 = 0.0, g1 = 0.0, g2 = 0.0, g3 = 0.0, g4 = 0.0, g5 = 0.0;
    if (FB) {
        g0 = __ldcg(a.G + FB_Q * N + s);
        g1 = __ldcg(a.G + FB_E * N + s);
        g2 = __ldcg(a.G + FB_PV * N + s);
        g3 = __ldcg(a.G + FB_VX * N + s);
        g4 = __ldcg(a.G + FB_VY * N + s);
        g5 = __ldcg(a.G + FB_VZ * N + s);
    } else {
        g0 = __ldcg(a.G + SK_K * N + s);
    }
    for (int k = lane; k < W3; k += 32) {
        const int cnt = __ldcg(a.om + s * W3 + k);
        if (!cnt) continue;
        const int oz = k / (W * W), oy = (k / W) % W, ox = k % W;
        const int ci = h0 + ox - R, cj = h1 + oy - R, ck = h2 + oz - R;
        const Owner o = owner_of(a.T, p, ci, cj, ck);
        double U[NF], dU[NF];
        load5(a.u, o.c, o.fs, U);
        if (FB) {
            const double d0 = ((double)ci + 0.5) - x, d1 = ((double)cj + 0.5) - y, d2 = ((double)ck + 0.5) - z;
            const double dd = (d0 * d0 + d1 * d1) + d2 * d2;
            const double vc[3] = {g3, g4, g5};
            feedback_delta(sm.wtab[cnt], U, g0, g1, g2, vc, d0, d1, d2, dd, dU);
        } else {
            const double *ws = a.wts + s * (3 * W);
            const double w = (__ldcg(ws + ox) * __ldcg(ws + W + oy)) * __ldcg(ws + 2 * W + oz);
            sink_delta(P, U, g0, w, dU);
        }
        const long long cb = pcell(T, ci, cj, ck);
#pragma unroll
        for (int f = 0; f < NF; ++f) atomicAdd(a.b + (long long)f * T->fs + cb, dU[f]);
    }
}

__device__ void zero_item(const BArgs &a, const ZeroItem &it)
{
    const PatchDev *T = a.T + it.patch;
    for (long long c = it.c0 + threadIdx.x; c < it.c1; c += kThreads) {
#pragma unroll
        for (int f = 0; f < NF; ++f) a.b[T->off + (long long)f * T->fs + c] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// Step 4 for sinks: one warp per sink
// ---------------------------------------------------------------------------

template <int R>
__device__ void return_sink(const BArgs &a, long long s, SmemT<R> &sm)
{
    constexpr int W = 2 * R + 1, W3 = W * W * W;
    const KParams &P = a.P;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned long long hp = __ldcg(a.hostp + s);
    if (hp == kNoHostB) return;
    int h0, h1, h2;
    unpack_host(hp, h0, h1, h2);
    const int p = patch_of(a.first, a.np, s);
    const long long N = a.p.count;
    const double K = __ldcg(a.G + SK_K * N + s);
    const double *ws = a.wts + s * (3 * W);
    double (*red)[6] = sm.u.pw.red[wib];
    double acc = 0.0;  // lane f < 4 keeps sum f (see gather_particle)
    for (int k0 = 0; k0 < W3; k0 += 32) {
        const int k = k0 + lane;
        bool mem = false;
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
        if (k < W3 && __ldcg(a.om + s * W3 + k)) {
            mem = true;
            const int oz = k / (W * W), oy = (k / W) % W, ox = k % W;
            const Owner o = owner_of(a.T, p, h0 + ox - R, h1 + oy - R, h2 + oz - R);
            double U[NF], dU[NF], D[NF];
            load5(a.u, o.c, o.fs, U);
            const double w = (__ldcg(ws + ox) * __ldcg(ws + W + oy)) * __ldcg(ws + 2 * W + oz);
            sink_delta(P, U, K, w, dU);
            bool img;
            folded_at(a, o.q, o.i, o.j, o.k, D, img);
            const double eta = sink_eta(P, U, D);
            // b = eta a and v = p inv; lane 0 fuses -b v into the sums
            const double inv = exact::div_rn(1.0, U[0]);
            v0 = eta * (-dU[0]);
            v1 = U[1] * inv;
            v2 = U[2] * inv;
            v3 = U[3] * inv;
        }
        const unsigned mm = __ballot_sync(kFullMask, mem);
        red[lane][0] = v0;
        red[lane][1] = v1;
        red[lane][2] = v2;
        red[lane][3] = v3;
        __syncwarp();
        if (lane < 4)
            for (int l = 0; l < 32; ++l) {
                if (!((mm >> l) & 1u)) continue;
                // mass: fma(-b, 1, c) == c - b; momentum: fma(-b, v, c)
                acc = fma(-red[l][0], lane == 0 ? 1.0 : red[l][lane], acc);
            }
        __syncwarp();
    }
    const double c0 = __shfl_sync(kFullMask, acc, 0), c1 = __shfl_sync(kFullMask, acc, 1),
                 c2 = __shfl_sync(kFullMask, acc, 2), c3 = __shfl_sync(kFullMask, acc, 3);
    if (lane == 0) {
        const double V = P.V;
        a.p.m[s] = a.p.m[s] - c0 * V;
        a.p.px[s] = a.p.px[s] - c1 * V;
        a.p.py[s] = a.p.py[s] - c2 * V;
        a.p.pz[s] = a.p.pz[s] - c3 * V;
    }
}

// ---------------------------------------------------------------------------
// Steps 2 (summation), 3 and 5 fused: one warp per row of valid cells
// ---------------------------------------------------------------------------

template <bool FB>
__device__ void apply_item(const BArgs &a, const AppItem &it, unsigned &nl, unsigned &nr)
{
    const KParams &P = a.P;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int q = it.patch;
    const PatchDev *T = a.T + q;
    const int n0 = T->n[0], n1 = T->n[1];
    const long long fs = T->fs, vb = T->vbase;
    const int rows = (it.k1 - it.k0) * n1;
    for (int r = wib; r < rows; r += kWarps) {
        const int k = it.k0 + r / n1, j = r % n1;
        for (int i = lane; i < n0; i += 32) {
            double D[NF];
            bool img;
            folded_at(a, q, i, j, k, D, img);
            const long long c = pcell(T, i, j, k);
            double eta = 1.0;
            if (!all_zero(D)) {
                double U[NF];
                load5(a.u, c, fs, U);
                if (FB) {
                    int noroot = 0;
                    const double l = sn_lambda(U, D, noroot);
                    nr += noroot;
                    eta = l;
                    a.u[c] = U[0] + D[0];
                    a.u[fs + c] = U[1] + l * D[1];
                    a.u[2 * fs + c] = U[2] + l * D[2];
                    a.u[3 * fs + c] = U[3] + l * D[3];
                    a.u[4 * fs + c] = U[4] + D[4];
                } else {
                    eta = sink_eta(P, U, D);
#pragma unroll
                    for (int f = 0; f < NF; ++f) a.u[(long long)f * fs + c] = U[f] + (eta == 1.0 ? D[f] : eta * D[f]);
                }
                nl += eta < 1.0;
            }
            if (img) {
#pragma unroll
                for (int f = 0; f < NF; ++f) a.b[(long long)f * fs + c] = D[f];
            }
            if (a.eta_out) a.eta_out[vb + ((long long)k * n1 + j) * n0 + i] = eta;
        }
    }
}

__device__ __forceinline__ void flush_counts(const BArgs &a, unsigned nl, unsigned nr)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nl += __shfl_down_sync(kFullMask, nl, o);
        nr += __shfl_down_sync(kFullMask, nr, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (nl) atomicAdd(&a.st->n_limited, (unsigned long long)nl);
        if (nr) atomicAdd(&a.st->n_noroot, (unsigned long long)nr);
    }
}

template <int R>
__device__ void fill_wtab(const KParams &P, SmemT<R> &sm)
{
    for (int i = threadIdx.x; i <= P.S3; i += kThreads) sm.wtab[i] = (double)i / (double)P.S3;
}

// ---------------------------------------------------------------------------
// the persistent pass
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch.  The wait is bounded: a block
// that has waited kWaitNs sets PMP_ERR_TIMEOUT and the abort word, and every
// waiting block returns false once it sees the abort word.
template <int R>
__device__ bool grid_sync(const BArgs &a, SmemT<R> &sm)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        volatile unsigned *gen = &a.ctl->gen;
        volatile unsigned *ab = &a.ctl->abort;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&a.ctl->count, 1u) + 1u;
        if (arrived == gridDim.x + a.hold) {
            atomicExch(&a.ctl->count, 0u);
            __threadfence();
            atomicAdd(&a.ctl->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g0) {
                if (*ab) {
                    good = 0;
                    break;
                }
                if (global_ns() - t0 > kWaitNs) {
                    report(a.st, PMP_ERR_TIMEOUT, -1);
                    atomicExch(&a.ctl->abort, 1u);
                    good = 0;
                    break;
                }
                __nanosleep(200);
            }
        }
        __threadfence();
        sm.ok = good;
    }
    __syncthreads();
    return sm.ok != 0;
}

template <int R>
__device__ __forceinline__ int next_item(unsigned *q, SmemT<R> &sm)
{
    __syncthreads();
    if (threadIdx.x == 0) sm.item = (int)atomicAdd(q, 1u);
    __syncthreads();
    return sm.item;
}

template <int R, bool FB>
__global__ void __launch_bounds__(kThreads, 2) k_batch_persistent(BArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemT<R> &sm = *reinterpret_cast<SmemT<R> *>(smem_raw);
    const int wib = threadIdx.x >> 5;
    if (FB) fill_wtab(a.P, sm);
    const long long N = a.p.count;
    const long long ngrp = (N + kWarps - 1) / kWarps;
    // a grid barrier only between two phases this launch runs
    const int last = FB && a.ph1 == 2 ? 1 : a.ph1;
    // phase 0: zeroing for the atomic strategy, then the gather (8 particles per item)
    if (a.ph0 <= 0) {
        for (;;) {
            const int it = next_item(&a.ctl->q[0], sm);
            if (it >= a.nzero + ngrp) break;
            if (it < a.nzero) {
                zero_item(a, a.zero[it]);
            } else {
                const long long s = (long long)(it - a.nzero) * kWarps + wib;
                if (s < N) gather_particle<R, FB>(a, s, sm);
            }
        }
        if (last == 0 || !grid_sync(a, sm)) return;
    }
    // phase 1: deposit
    if (a.ph0 <= 1) {
        for (;;) {
            const int it = next_item(&a.ctl->q[1], sm);
            if (it >= a.ndep) break;
            const DepItem d = a.dep[it];
            if (d.strat == STRAT_ATOMIC) {
                for (long long s = d.lo[0] + wib; s < d.hi[0]; s += kWarps)
                    deposit_atomic_particle<R, FB>(a, d.patch, s, sm);
            } else {
                deposit_tile<R, FB>(a, d, sm);
            }
        }
        if (last == 1 || !grid_sync(a, sm)) return;
    }
    // phase 2: Step 4 (sinks)
    if (!FB && a.ph0 <= 2) {
        for (;;) {
            const int it = next_item(&a.ctl->q[2], sm);
            if (it >= ngrp) break;
            const long long s = (long long)it * kWarps + wib;
            if (s < N) return_sink<R>(a, s, sm);
        }
        if (last == 2 || !grid_sync(a, sm)) return;
    }
    // phase 3: summation, limiter, update
    unsigned nl = 0, nr = 0;
    for (;;) {
        const int it = next_item(&a.ctl->q[3], sm);
        if (it >= a.napp) break;
        apply_item<FB>(a, a.app[it], nl, nr);
    }
    flush_counts(a, nl, nr);
}

// ---------------------------------------------------------------------------
// the plain form: one launch per phase and patch
// ---------------------------------------------------------------------------

template <int R, bool FB>
__global__ void __launch_bounds__(kThreads) k_batch_gather(BArgs a, long long s0, long long s1)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemT<R> &sm = *reinterpret_cast<SmemT<R> *>(smem_raw);
    const long long s = s0 + (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    if (s < s1) gather_particle<R, FB>(a, s, sm);
}

template <int R, bool FB>
__global__ void __launch_bounds__(kThreads) k_batch_deposit(BArgs a, int i0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemT<R> &sm = *reinterpret_cast<SmemT<R> *>(smem_raw);
    if (FB) fill_wtab(a.P, sm);
    __syncthreads();
    const DepItem d = a.dep[i0 + blockIdx.x];
    if (d.strat == STRAT_ATOMIC) {
        for (long long s = d.lo[0] + (threadIdx.x >> 5); s < d.hi[0]; s += kWarps)
            deposit_atomic_particle<R, FB>(a, d.patch, s, sm);
    } else {
        deposit_tile<R, FB>(a, d, sm);
    }
}

__global__ void __launch_bounds__(kThreads) k_batch_zero(BArgs a, int i0)
{
    zero_item(a, a.zero[i0 + blockIdx.x]);
}

template <int R>
__global__ void __launch_bounds__(kThreads) k_batch_return(BArgs a, long long s0, long long s1)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemT<R> &sm = *reinterpret_cast<SmemT<R> *>(smem_raw);
    const long long s = s0 + (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    if (s < s1) return_sink<R>(a, s, sm);
}

template <bool FB>
__global__ void __launch_bounds__(kThreads) k_batch_apply(BArgs a, int i0)
{
    unsigned nl = 0, nr = 0;
    apply_item<FB>(a, a.app[i0 + blockIdx.x], nl, nr);
    flush_counts(a, nl, nr);
}

// ---------------------------------------------------------------------------
// packing and unpacking of exchange regions (the batched form on several ranks)
// ---------------------------------------------------------------------------

// A region of one local patch: cells lo <= c < hi (padded coordinates), its
// five fields at msg[off + f * vol + cell] (x fastest).
struct PackRegion {
    int patch;
    int lo[3], hi[3];
    int pad_;
    long long off, vol;
};
// kPackCells consecutive cells of one region.
struct PackItem {
    int region, pad_;
    long long c0;
};

__device__ __forceinline__ void region_cell(const PackRegion &r, long long c, int &i, int &j, int &k)
{
    const int nx = r.hi[0] - r.lo[0], ny = r.hi[1] - r.lo[1];
    i = r.lo[0] + (int)(c % nx);
    const long long t = c / nx;
    j = r.lo[1] + (int)(t % ny);
    k = r.lo[2] + (int)(t / ny);
}

// pack (to_msg) or unpack one item per block; folded: the folded sums of the
// buffer (App. A.2 order) instead of the stored values (valid cells only)
__global__ void __launch_bounds__(kPackThreads) k_batch_pack(BArgs a, const PackRegion *__restrict__ regs,
                                                             const PackItem *__restrict__ items, const double *src,
                                                             double *dst, int to_msg, int folded)
{
    const PackItem it = items[blockIdx.x];
    const PackRegion r = regs[it.region];
    const long long c = it.c0 + threadIdx.x;
    if (c >= r.vol) return;
    int i, j, k;
    region_cell(r, c, i, j, k);
    const PatchDev *T = a.T + r.patch;
    const long long pc = pcell(T, i, j, k);
    if (folded) {
        double D[NF];
        bool img;
        folded_at(a, r.patch, i, j, k, D, img);
#pragma unroll
        for (int f = 0; f < NF; ++f) dst[r.off + (long long)f * r.vol + c] = D[f];
        return;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const long long m = r.off + (long long)f * r.vol + c, e = pc + (long long)f * T->fs;
        if (to_msg)
            dst[m] = src[e];
        else
            dst[e] = src[m];
    }
}

}  // namespace
}  // namespace pmp

// ===========================================================================
// host side
// ===========================================================================

using pmp::AppItem;
using pmp::BArgs;
using pmp::Ctl;
using pmp::DepItem;
using pmp::PatchDev;
using pmp::ZeroItem;

struct pmp_batch {
    pmp_ctx *ctx;
    int np, ng, R, W3;
    double dx;
    long long arena_len;
    std::vector<pmp_patch> patches;
    std::vector<long long> first;  // [np + 1]
    std::vector<int> strat;        // per patch
    // device
    PatchDev *T;
    long long *first_d;
    Ctl *ctl;
    DepItem *dep;
    AppItem *app;
    ZeroItem *zero;
    size_t dep_cap, app_cap, zero_cap;
    unsigned short *om;
    unsigned long long *hostp;
    double *wts;
    long long part_cap;
    // host item lists, grouped by patch (heavy patches first); ranges per patch
    std::vector<DepItem> dep_h;
    std::vector<AppItem> app_h;
    std::vector<ZeroItem> zero_h;
    std::vector<int> dep_lo, dep_hi, app_lo, app_hi, zero_lo, zero_hi;
    int grid;
    size_t smem;
    // CUDA graph of the persistent launch, for one set of argument pointers,
    // captured on a private stream (the context's may be the legacy stream,
    // which cannot capture) and launched on the context's stream
    cudaGraphExec_t graph;
    cudaStream_t cap_stream;
    const void *gkey[8];
    unsigned hold;  // see pmp_batch_hold_barriers
    int n_owned;    // patches [0, n_owned) are worked on; the rest are only read
    // region lists for pack / unpack (pmp_batch_set_regions), per slot: the
    // regions and work items of up to kPackCells cells each
    pmp::PackRegion *reg[pmp::kRegionSlots];
    pmp::PackItem *pitem[pmp::kRegionSlots];
    int nreg[pmp::kRegionSlots], npitem[pmp::kRegionSlots];
    std::vector<pmp::PackRegion> reg_h[pmp::kRegionSlots];
};

namespace {

using pmp::KParams;

template <class T>
cudaError_t grow(T **ptr, size_t *cap, size_t need)
{
    if (need <= *cap && *ptr) return cudaSuccess;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    const size_t n = need > 0 ? need : 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(ptr), n * sizeof(T));
    if (e == cudaSuccess) *cap = n;
    return e;
}

long long padded_cells(const pmp_patch &p, int g)
{
    return ((long long)p.n[0] + 2 * g) * ((long long)p.n[1] + 2 * g) * ((long long)p.n[2] + 2 * g);
}

// Tiles of a patch's padded box for an OWNER strategy.
void tiles(const pmp_patch &pp, int g, int p, int strat, std::vector<DepItem> &out)
{
    const int P0 = pp.n[0] + 2 * g, P1 = pp.n[1] + 2 * g, P2 = pp.n[2] + 2 * g;
    int tx, ty, tz;
    if (strat == pmp::STRAT_OWNER_ROWS) {
        tx = P0;
        ty = 8;
        tz = 4;
    } else {
        tx = 8;
        ty = 8;
        tz = 8;
    }
    for (int k = 0; k < P2; k += tz)
        for (int j = 0; j < P1; j += ty)
            for (int i = 0; i < P0; i += tx) {
                DepItem d;
                d.patch = p;
                d.strat = strat;
                d.lo[0] = i - g;
                d.lo[1] = j - g;
                d.lo[2] = k - g;
                d.hi[0] = std::min(i + tx, P0) - g;
                d.hi[1] = std::min(j + ty, P1) - g;
                d.hi[2] = std::min(k + tz, P2) - g;
                out.push_back(d);
            }
}

// Builds the item lists for the current particle ranges and strategies, and
// uploads them.
pmp_status build_items(pmp_batch *b)
{
    const int np = b->np, g = b->ng;
    std::vector<int> order(b->n_owned);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (b->first[x + 1] - b->first[x]) > (b->first[y + 1] - b->first[y]);
    });
    b->dep_h.clear();
    b->app_h.clear();
    b->zero_h.clear();
    b->dep_lo.assign(np, 0);
    b->dep_hi.assign(np, 0);
    b->app_lo.assign(np, 0);
    b->app_hi.assign(np, 0);
    b->zero_lo.assign(np, 0);
    b->zero_hi.assign(np, 0);
    for (int p : order) {
        const pmp_patch &pp = b->patches[p];
        const int st = b->strat[p];
        b->dep_lo[p] = (int)b->dep_h.size();
        b->zero_lo[p] = (int)b->zero_h.size();
        if (st == pmp::STRAT_ATOMIC) {
            const long long pc = padded_cells(pp, g);
            for (long long c = 0; c < pc; c += 16384) {
                ZeroItem z;
                z.patch = p;
                z.pad_ = 0;
                z.c0 = c;
                z.c1 = std::min(c + 16384, pc);
                b->zero_h.push_back(z);
            }
            for (long long s = b->first[p]; s < b->first[p + 1]; s += 64) {
                DepItem d;
                std::memset(&d, 0, sizeof(d));
                d.patch = p;
                d.strat = st;
                d.lo[0] = (int)s;
                d.hi[0] = (int)std::min(s + 64, b->first[p + 1]);
                b->dep_h.push_back(d);
            }
        } else {
            tiles(pp, g, p, st, b->dep_h);
        }
        b->dep_hi[p] = (int)b->dep_h.size();
        b->zero_hi[p] = (int)b->zero_h.size();
        b->app_lo[p] = (int)b->app_h.size();
        const long long plane = (long long)pp.n[0] * pp.n[1];
        const int kz = (int)std::max(1LL, std::min((long long)pp.n[2], 4096LL / std::max(1LL, plane) + 1));
        for (int k = 0; k < pp.n[2]; k += kz) {
            AppItem a;
            a.patch = p;
            a.k0 = k;
            a.k1 = std::min(k + kz, pp.n[2]);
            a.pad_ = 0;
            b->app_h.push_back(a);
        }
        b->app_hi[p] = (int)b->app_h.size();
    }
    if (grow(&b->dep, &b->dep_cap, b->dep_h.size()) != cudaSuccess ||
        grow(&b->app, &b->app_cap, b->app_h.size()) != cudaSuccess ||
        grow(&b->zero, &b->zero_cap, b->zero_h.size()) != cudaSuccess)
        return PMP_ERR_CUDA;
    if ((!b->dep_h.empty() && cudaMemcpy(b->dep, b->dep_h.data(), b->dep_h.size() * sizeof(DepItem),
                                         cudaMemcpyHostToDevice) != cudaSuccess) ||
        (!b->app_h.empty() && cudaMemcpy(b->app, b->app_h.data(), b->app_h.size() * sizeof(AppItem),
                                         cudaMemcpyHostToDevice) != cudaSuccess) ||
        (!b->zero_h.empty() && cudaMemcpy(b->zero, b->zero_h.data(), b->zero_h.size() * sizeof(ZeroItem),
                                          cudaMemcpyHostToDevice) != cudaSuccess))
        return PMP_ERR_CUDA;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return PMP_OK;
}

BArgs make_args(pmp_batch *b, double *state, double *buffer, const pmp_particles *p, double *gathered,
                double *eta_out)
{
    BArgs a;
    std::memset(&a, 0, sizeof(a));
    a.P = pmp::make_kparams(b->ctx->p, b->dx);
    a.T = b->T;
    a.np = b->np;
    a.nzero = (int)b->zero_h.size();
    a.ndep = (int)b->dep_h.size();
    a.napp = (int)b->app_h.size();
    a.first = b->first_d;
    a.u = state;
    a.b = buffer;
    a.p.count = p->count;
    a.p.x = p->x;
    a.p.y = p->y;
    a.p.z = p->z;
    a.p.m = p->m;
    a.p.px = p->px;
    a.p.py = p->py;
    a.p.pz = p->pz;
    a.p.e = p->e;
    a.G = gathered;
    a.eta_out = eta_out;
    a.wts = b->wts;
    a.om = b->om;
    a.hostp = b->hostp;
    a.dep = b->dep;
    a.app = b->app;
    a.zero = b->zero;
    a.ctl = b->ctl;
    a.st = b->ctx->st;
    a.hold = b->hold;
    a.ph0 = 0;
    a.ph1 = 3;
    return a;
}

template <int R, bool FB>
cudaError_t launch_persistent(pmp_batch *b, const BArgs &a, cudaStream_t st)
{
    auto kern = pmp::k_batch_persistent<R, FB>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)b->grid);
    cfg.blockDim = dim3(pmp::kThreads);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int R, bool FB>
cudaError_t configure(pmp_batch *b)
{
    const size_t sm = sizeof(pmp::SmemT<R>);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(pmp::k_batch_persistent<R, FB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(pmp::k_batch_gather<R, FB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(pmp::k_batch_deposit<R, FB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm)) != cudaSuccess)
        return e;
    if (!FB && (e = cudaFuncSetAttribute(pmp::k_batch_return<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm)) != cudaSuccess)
        return e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pmp::k_batch_persistent<R, FB>, pmp::kThreads,
                                                           sm)) != cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    b->grid = per_sm * sms;
    b->smem = sm;
    return cudaSuccess;
}

cudaError_t do_configure(pmp_batch *b)
{
    cudaError_t e = cudaSuccess;
    const bool fb = b->ctx->p.kind == PMP_KIND_FEEDBACK;
    if (fb) {
        PMP_DISPATCH_R(b->R, (e = configure<RR, true>(b)));
    } else {
        PMP_DISPATCH_R(b->R, (e = configure<RR, false>(b)));
    }
    return e;
}

// The persistent pass: reset the queue and barrier words, one cooperative launch.
cudaError_t enqueue_persistent(pmp_batch *b, const BArgs &a, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(b->ctl, 0, sizeof(Ctl), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&b->ctx->st->n_limited, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const bool fb = b->ctx->p.kind == PMP_KIND_FEEDBACK;
    if (fb) {
        PMP_DISPATCH_R(b->R, (e = launch_persistent<RR, true>(b, a, st)));
    } else {
        PMP_DISPATCH_R(b->R, (e = launch_persistent<RR, false>(b, a, st)));
    }
    return e;
}

template <int R, bool FB>
cudaError_t per_patch(pmp_batch *b, const BArgs &a, cudaStream_t st)
{
    using namespace pmp;
    const size_t sm = b->smem;
    if (a.ph0 <= 1) {
        for (int p = 0; p < b->np; ++p)
            if (b->zero_hi[p] > b->zero_lo[p])
                k_batch_zero<<<(unsigned)(b->zero_hi[p] - b->zero_lo[p]), kThreads, 0, st>>>(a, b->zero_lo[p]);
        for (int p = 0; p < b->np; ++p) {
            const long long s0 = b->first[p], s1 = b->first[p + 1];
            if (s1 > s0)
                k_batch_gather<R, FB><<<(unsigned)((s1 - s0 + kWarps - 1) / kWarps), kThreads, sm, st>>>(a, s0, s1);
        }
        for (int p = 0; p < b->np; ++p)
            if (b->dep_hi[p] > b->dep_lo[p])
                k_batch_deposit<R, FB><<<(unsigned)(b->dep_hi[p] - b->dep_lo[p]), kThreads, sm, st>>>(a, b->dep_lo[p]);
    }
    if (a.ph1 < 2) return cudaGetLastError();
    if (!FB) {
        for (int p = 0; p < b->np; ++p) {
            const long long s0 = b->first[p], s1 = b->first[p + 1];
            if (s1 > s0)
                k_batch_return<R><<<(unsigned)((s1 - s0 + kWarps - 1) / kWarps), kThreads, sm, st>>>(a, s0, s1);
        }
    }
    for (int p = 0; p < b->np; ++p)
        if (b->app_hi[p] > b->app_lo[p])
            k_batch_apply<FB><<<(unsigned)(b->app_hi[p] - b->app_lo[p]), kThreads, 0, st>>>(a, b->app_lo[p]);
    return cudaGetLastError();
}

cudaError_t enqueue_per_patch(pmp_batch *b, const BArgs &a, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(&b->ctx->st->n_limited, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const bool fb = b->ctx->p.kind == PMP_KIND_FEEDBACK;
    if (fb) {
        PMP_DISPATCH_R(b->R, (e = per_patch<RR, true>(b, a, st)));
    } else {
        PMP_DISPATCH_R(b->R, (e = per_patch<RR, false>(b, a, st)));
    }
    return e;
}

// Only the gather, then only the deposit items [i0, i1) (the autotuner's
// timed trials).
template <int R, bool FB>
cudaError_t trial_gather(pmp_batch *b, const BArgs &a, cudaStream_t st)
{
    using namespace pmp;
    const long long n = b->first[b->np];
    if (n > 0) k_batch_gather<R, FB><<<(unsigned)((n + kWarps - 1) / kWarps), kThreads, b->smem, st>>>(a, 0, n);
    return cudaGetLastError();
}

template <int R, bool FB>
cudaError_t trial_deposit(pmp_batch *b, const BArgs &a, const std::vector<int> &patches, cudaStream_t st)
{
    using namespace pmp;
    for (int p : patches)
        if (b->zero_hi[p] > b->zero_lo[p])
            k_batch_zero<<<(unsigned)(b->zero_hi[p] - b->zero_lo[p]), kThreads, 0, st>>>(a, b->zero_lo[p]);
    for (int p : patches)
        if (b->dep_hi[p] > b->dep_lo[p])
            k_batch_deposit<R, FB><<<(unsigned)(b->dep_hi[p] - b->dep_lo[p]), kThreads, b->smem, st>>>(a, b->dep_lo[p]);
    return cudaGetLastError();
}

pmp_status check_particles(const pmp_batch *b, const pmp_particles *p, double *gathered)
{
    if (!p || p->count != b->first[b->np]) return PMP_ERR_ARG;
    if (p->count > 0) {
        if (!p->x || !p->y || !p->z || !p->m || !p->px || !p->py || !p->pz || !gathered) return PMP_ERR_ARG;
        if (b->ctx->p.kind == PMP_KIND_FEEDBACK && !p->e) return PMP_ERR_ARG;
    }
    return PMP_OK;
}

// Patch-size bin (padded cells) x occupancy bin (particles per 1000 valid
// cells) of a patch, for the autotuner.
constexpr int kSizeBins = 4, kOccBins = 5;
int bin_of(const pmp_batch *b, int p)
{
    const pmp_patch &pp = b->patches[p];
    const long long pc = padded_cells(pp, b->ng);
    const int sb = pc < 16384 ? 0 : (pc < 65536 ? 1 : (pc < 262144 ? 2 : 3));
    const long long nv = (long long)pp.n[0] * pp.n[1] * pp.n[2];
    const long long cnt = b->first[p + 1] - b->first[p];
    const double occ = 1000.0 * (double)cnt / (double)nv;
    const int ob = cnt == 0 ? 0 : (occ < 1.0 ? 1 : (occ < 10.0 ? 2 : (occ < 100.0 ? 3 : 4)));
    return sb * kOccBins + ob;
}

}  // namespace

extern "C" {

static pmp_status batch_create(pmp_ctx *ctx, const pmp_patch *patches, int32_t n_patches, int32_t n_owned, int32_t ng,
                               double dx, int64_t arena_len, pmp_batch **out)
{
    if (!out) return PMP_ERR_ARG;
    *out = nullptr;
    if (!ctx || !patches || n_patches < 1 || ng < 0 || !std::isfinite(dx) || !(dx > 0.0) || arena_len < 1)
        return PMP_ERR_ARG;
    if (n_owned < 0 || n_owned > n_patches) return PMP_ERR_ARG;
    if (ctx->p.kind == PMP_KIND_MASS) return PMP_ERR_ARG;  // the batched form covers supernovae and sinks
    const int R = (int)std::ceil(ctx->p.r_K);
    if (ng < R) return PMP_ERR_GHOST_TOO_THIN;
    // geometry checks: extents, arena bounds, disjoint patches, a consistent
    // rectilinear neighbour table
    std::vector<std::pair<long long, long long>> spans;
    for (int p = 0; p < n_patches; ++p) {
        const pmp_patch &pp = patches[p];
        for (int a = 0; a < 3; ++a) {
            if (pp.n[a] < 1 || pp.n[a] < ng) return PMP_ERR_ARG;
            if (pp.n[a] + 2LL * ng > 0x1fffff) return PMP_ERR_ARG;
        }
        const long long pc = padded_cells(pp, ng);
        if (pp.field_stride < pc || pp.offset < 0) return PMP_ERR_ARG;
        const long long end = pp.offset + (long long)(pmp::NF - 1) * pp.field_stride + pc;
        if (end > arena_len) return PMP_ERR_ARG;
        spans.push_back({pp.offset, pp.offset + (long long)pmp::NF * pp.field_stride});
    }
    {
        std::vector<std::pair<long long, long long>> s = spans;
        std::sort(s.begin(), s.end());
        for (size_t i = 1; i < s.size(); ++i)
            if (s[i].first < s[i - 1].second) return PMP_ERR_ARG;
    }
    for (int p = 0; p < n_patches; ++p) {
        const pmp_patch &pp = patches[p];
        int t = 0;
        for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    if (!ox && !oy && !oz) continue;
                    const int q = pp.neighbour[t++];
                    if (q < 0 || q >= n_patches) return PMP_ERR_ARG;
                    if (p >= n_owned) continue;  // proxies and the zero patch: only read
                    const int o[3] = {ox, oy, oz};
                    for (int a = 0; a < 3; ++a)
                        if (o[a] == 0 && patches[q].n[a] != pp.n[a]) return PMP_ERR_ARG;
                    // the reverse offset leads back (between owned patches)
                    const int rt = ((1 - oz) * 3 + (1 - oy)) * 3 + (1 - ox);
                    if (q < n_owned && patches[q].neighbour[rt > 13 ? rt - 1 : rt] != p) return PMP_ERR_ARG;
                }
    }
    pmp_batch *b = new (std::nothrow) pmp_batch();
    if (!b) return PMP_ERR_ARG;
    b->ctx = ctx;
    b->np = n_patches;
    b->n_owned = n_owned;
    b->ng = ng;
    b->R = R;
    b->W3 = (2 * R + 1) * (2 * R + 1) * (2 * R + 1);
    b->dx = dx;
    b->arena_len = arena_len;
    b->patches.assign(patches, patches + n_patches);
    b->first.assign(n_patches + 1, 0);
    b->strat.assign(n_patches, pmp::STRAT_OWNER_CUBE);
    std::vector<PatchDev> T(n_patches);
    long long vb = 0;
    for (int p = 0; p < n_patches; ++p) {
        const pmp_patch &pp = patches[p];
        PatchDev &d = T[p];
        std::memset(&d, 0, sizeof(d));
        for (int a = 0; a < 3; ++a) d.n[a] = pp.n[a];
        d.g = ng;
        d.px = pp.n[0] + 2 * ng;
        d.py = pp.n[1] + 2 * ng;
        for (int t = 0; t < 26; ++t) d.nb[t] = pp.neighbour[t];
        d.pxy = (long long)d.px * d.py;
        d.off = pp.offset;
        d.fs = pp.field_stride;
        d.vbase = vb;
        vb += (long long)pp.n[0] * pp.n[1] * pp.n[2];
    }
    pmp_status s = PMP_OK;
    if (cudaMalloc(&b->T, sizeof(PatchDev) * n_patches) != cudaSuccess ||
        cudaMalloc(&b->first_d, sizeof(long long) * (n_patches + 1)) != cudaSuccess ||
        cudaMalloc(&b->ctl, sizeof(Ctl)) != cudaSuccess ||
        cudaMemcpy(b->T, T.data(), sizeof(PatchDev) * n_patches, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->first_d, b->first.data(), sizeof(long long) * (n_patches + 1), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        s = PMP_ERR_CUDA;
    if (!s && do_configure(b) != cudaSuccess) s = PMP_ERR_CUDA;
    if (!s) s = build_items(b);
    if (s) {
        pmp_batch_destroy(b);
        return s;
    }
    *out = b;
    return PMP_OK;
}

pmp_status pmp_batch_create(pmp_ctx *ctx, const pmp_patch *patches, int32_t n_patches, int32_t ng, double dx,
                            int64_t arena_len, pmp_batch **out)
{
    return batch_create(ctx, patches, n_patches, n_patches, ng, dx, arena_len, out);
}

pmp_status pmp_batch_create_partial(pmp_ctx *ctx, const pmp_patch *patches, int32_t n_patches, int32_t n_owned,
                                    int32_t ng, double dx, int64_t arena_len, pmp_batch **out)
{
    return batch_create(ctx, patches, n_patches, n_owned, ng, dx, arena_len, out);
}

void pmp_batch_destroy(pmp_batch *b)
{
    if (!b) return;
    for (int k = 0; k < pmp::kRegionSlots; ++k) {
        cudaFree(b->reg[k]);
        cudaFree(b->pitem[k]);
    }
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFree(b->T);
    cudaFree(b->first_d);
    cudaFree(b->ctl);
    cudaFree(b->dep);
    cudaFree(b->app);
    cudaFree(b->zero);
    cudaFree(b->om);
    cudaFree(b->hostp);
    cudaFree(b->wts);
    delete b;
}

pmp_status pmp_batch_set_particles(pmp_batch *b, const int64_t *first)
{
    if (!b || !first || first[0] != 0) return PMP_ERR_ARG;
    for (int p = 0; p < b->np; ++p)
        if (first[p + 1] < first[p]) return PMP_ERR_ARG;
    const long long n = first[b->np];
    if (n > 0x7fffffffLL) return PMP_ERR_ARG;
    if (cudaStreamSynchronize(b->ctx->stream) != cudaSuccess) return PMP_ERR_CUDA;
    b->first.assign(first, first + b->np + 1);
    if (cudaMemcpy(b->first_d, b->first.data(), sizeof(long long) * (b->np + 1), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return PMP_ERR_CUDA;
    if (n > b->part_cap || !b->om) {
        cudaFree(b->om);
        cudaFree(b->hostp);
        cudaFree(b->wts);
        b->om = nullptr;
        b->hostp = nullptr;
        b->wts = nullptr;
        b->part_cap = 0;
        const size_t n1 = (size_t)(n > 0 ? n : 1);
        const int W = 2 * b->R + 1;
        if (cudaMalloc(&b->om, n1 * (size_t)b->W3 * sizeof(unsigned short)) != cudaSuccess ||
            cudaMalloc(&b->hostp, n1 * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMalloc(&b->wts, n1 * 3 * (size_t)W * sizeof(double)) != cudaSuccess)
            return PMP_ERR_CUDA;
        b->part_cap = (long long)n1;
    }
    return build_items(b);
}

pmp_status pmp_batch_set_strategy(pmp_batch *b, int32_t strategy)
{
    if (!b || strategy < 0 || strategy >= pmp::NSTRAT) return PMP_ERR_ARG;
    if (cudaStreamSynchronize(b->ctx->stream) != cudaSuccess) return PMP_ERR_CUDA;
    b->strat.assign(b->np, strategy);
    return build_items(b);
}

pmp_status pmp_batch_strategies(const pmp_batch *b, int32_t *per_patch)
{
    if (!b || !per_patch) return PMP_ERR_ARG;
    for (int p = 0; p < b->np; ++p) per_patch[p] = b->strat[p];
    return PMP_OK;
}

pmp_status pmp_batch_autotune(pmp_batch *b, const double *state, double *buffer, pmp_particles *particles,
                              double *gathered, int32_t deterministic, int32_t reps, int32_t *bin_choice)
{
    if (!b || !state || !buffer || reps < 1) return PMP_ERR_ARG;
    pmp_status s = check_particles(b, particles, gathered);
    if (s) return s;
    if (b->first[b->np] > 0 && !b->om) return PMP_ERR_ARG;
    cudaStream_t st = b->ctx->stream;
    const bool fb = b->ctx->p.kind == PMP_KIND_FEEDBACK;
    std::vector<std::vector<int>> bins(kSizeBins * kOccBins);
    for (int p = 0; p < b->np; ++p) bins[bin_of(b, p)].push_back(p);
    const int nstrat = deterministic ? 2 : pmp::NSTRAT;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return PMP_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PMP_ERR_CUDA;
    }
    std::vector<int> saved = b->strat;
    std::vector<int> choice(bins.size(), -1);
    cudaError_t ce = cudaSuccess;
    for (size_t bi = 0; bi < bins.size() && ce == cudaSuccess; ++bi) {
        if (bins[bi].empty()) continue;
        float best = 3.0e38f;
        for (int stg = 0; stg < nstrat && ce == cudaSuccess; ++stg) {
            for (int p : bins[bi]) b->strat[p] = stg;
            if ((s = build_items(b)) != PMP_OK) break;
            BArgs a = make_args(b, const_cast<double *>(state), buffer, particles, gathered, nullptr);
            if (fb) {
                PMP_DISPATCH_R(b->R, (ce = trial_gather<RR, true>(b, a, st)));
            } else {
                PMP_DISPATCH_R(b->R, (ce = trial_gather<RR, false>(b, a, st)));
            }
            float tbest = 3.0e38f;
            for (int r = 0; r < reps && ce == cudaSuccess; ++r) {
                cudaEventRecord(e0, st);
                if (fb) {
                    PMP_DISPATCH_R(b->R, (ce = trial_deposit<RR, true>(b, a, bins[bi], st)));
                } else {
                    PMP_DISPATCH_R(b->R, (ce = trial_deposit<RR, false>(b, a, bins[bi], st)));
                }
                cudaEventRecord(e1, st);
                if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
                float ms = 0.0f;
                if (ce == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
                tbest = std::min(tbest, ms);
            }
            if (tbest < best) {
                best = tbest;
                choice[bi] = stg;
            }
        }
        if (s) break;
        for (int p : bins[bi]) b->strat[p] = choice[bi];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ce != cudaSuccess || s) {
        b->strat = saved;
        build_items(b);
        return s ? s : PMP_ERR_CUDA;
    }
    if (bin_choice)
        for (size_t bi = 0; bi < bins.size(); ++bi) bin_choice[bi] = choice[bi];
    return build_items(b);
}

pmp_status pmp_cycle_batched(pmp_batch *b, double *state, double *buffer, pmp_particles *particles,
                             double *gathered, double *eta_out, int32_t launch)
{
    if (!b || !state || !buffer) return PMP_ERR_ARG;
    if (launch != PMP_BATCH_PERSISTENT && launch != PMP_BATCH_PER_PATCH && launch != PMP_BATCH_GRAPH)
        return PMP_ERR_ARG;
    if (((reinterpret_cast<uintptr_t>(state) | reinterpret_cast<uintptr_t>(buffer)) & 7) != 0) return PMP_ERR_ARG;
    if (state == buffer) return PMP_ERR_ARG;
    {
        const double *s0 = state, *s1 = state + b->arena_len, *b0 = buffer, *b1 = buffer + b->arena_len;
        if (s0 < b1 && b0 < s1) return PMP_ERR_ARG;
    }
    pmp_status s = check_particles(b, particles, gathered);
    if (s) return s;
    if (b->first[b->np] > 0 && !b->om) return PMP_ERR_ARG;
    cudaStream_t st = b->ctx->stream;
    const BArgs a = make_args(b, state, buffer, particles, gathered, eta_out);
    cudaError_t e = cudaSuccess;
    if (launch == PMP_BATCH_PER_PATCH) {
        e = enqueue_per_patch(b, a, st);
    } else if (launch == PMP_BATCH_PERSISTENT) {
        e = enqueue_persistent(b, a, st);
    } else {
        const void *key[8] = {state, buffer, particles->x, particles->m, particles->px, gathered, eta_out,
                              particles->e};
        if (b->graph && std::memcmp(key, b->gkey, sizeof(key)) != 0) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        if (!b->graph) {
            cudaGraph_t g = nullptr;
            if (!b->cap_stream) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t e1 = enqueue_persistent(b, a, b->cap_stream);
                e = cudaStreamEndCapture(b->cap_stream, &g);
                if (e1 != cudaSuccess) e = e1;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e == cudaSuccess) std::memcpy(b->gkey, key, sizeof(key));
            else b->graph = nullptr;
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, st);
    }
    return e == cudaSuccess ? PMP_OK : PMP_ERR_CUDA;
}

pmp_status pmp_cycle_batched_part(pmp_batch *b, double *state, double *buffer, pmp_particles *particles,
                                  double *gathered, double *eta_out, int32_t launch, int32_t part)
{
    if (part == PMP_BATCH_PART_ALL) return pmp_cycle_batched(b, state, buffer, particles, gathered, eta_out, launch);
    if (!b || !state || !buffer) return PMP_ERR_ARG;
    if (part != PMP_BATCH_PART_DEPOSIT && part != PMP_BATCH_PART_FINISH) return PMP_ERR_ARG;
    if (launch != PMP_BATCH_PERSISTENT && launch != PMP_BATCH_PER_PATCH) return PMP_ERR_ARG;
    if (((reinterpret_cast<uintptr_t>(state) | reinterpret_cast<uintptr_t>(buffer)) & 7) != 0) return PMP_ERR_ARG;
    {
        const double *s0 = state, *s1 = state + b->arena_len, *b0 = buffer, *b1 = buffer + b->arena_len;
        if (s0 < b1 && b0 < s1) return PMP_ERR_ARG;
    }
    pmp_status s = check_particles(b, particles, gathered);
    if (s) return s;
    if (b->first[b->np] > 0 && !b->om) return PMP_ERR_ARG;
    BArgs a = make_args(b, state, buffer, particles, gathered, eta_out);
    a.ph0 = part == PMP_BATCH_PART_DEPOSIT ? 0 : 2;
    a.ph1 = part == PMP_BATCH_PART_DEPOSIT ? 1 : 3;
    const cudaError_t e = launch == PMP_BATCH_PER_PATCH ? enqueue_per_patch(b, a, b->ctx->stream)
                                                        : enqueue_persistent(b, a, b->ctx->stream);
    return e == cudaSuccess ? PMP_OK : PMP_ERR_CUDA;
}

pmp_status pmp_batch_set_regions(pmp_batch *b, int32_t slot, const pmp_region *regions, int32_t n)
{
    if (!b || slot < 0 || slot >= pmp::kRegionSlots || n < 0 || (n > 0 && !regions)) return PMP_ERR_ARG;
    std::vector<pmp::PackRegion> R(n);
    std::vector<pmp::PackItem> I;
    for (int r = 0; r < n; ++r) {
        const pmp_region &g = regions[r];
        if (g.patch < 0 || g.patch >= b->np || g.offset < 0) return PMP_ERR_ARG;
        const pmp_patch &pp = b->patches[g.patch];
        pmp::PackRegion &d = R[r];
        std::memset(&d, 0, sizeof(d));
        d.patch = g.patch;
        for (int a = 0; a < 3; ++a) {
            if (g.lo[a] < -b->ng || g.hi[a] > pp.n[a] + b->ng || g.lo[a] >= g.hi[a]) return PMP_ERR_ARG;
            d.lo[a] = g.lo[a];
            d.hi[a] = g.hi[a];
        }
        d.off = g.offset;
        d.vol = (long long)(g.hi[0] - g.lo[0]) * (g.hi[1] - g.lo[1]) * (g.hi[2] - g.lo[2]);
        for (long long c = 0; c < d.vol; c += pmp::kPackThreads) {
            pmp::PackItem it;
            it.region = r;
            it.pad_ = 0;
            it.c0 = c;
            I.push_back(it);
        }
    }
    if (cudaStreamSynchronize(b->ctx->stream) != cudaSuccess) return PMP_ERR_CUDA;
    cudaFree(b->reg[slot]);
    cudaFree(b->pitem[slot]);
    b->reg[slot] = nullptr;
    b->pitem[slot] = nullptr;
    b->nreg[slot] = b->npitem[slot] = 0;
    b->reg_h[slot].clear();
    if (n == 0) return PMP_OK;
    if (cudaMalloc(&b->reg[slot], sizeof(pmp::PackRegion) * R.size()) != cudaSuccess ||
        cudaMalloc(&b->pitem[slot], sizeof(pmp::PackItem) * I.size()) != cudaSuccess ||
        cudaMemcpy(b->reg[slot], R.data(), sizeof(pmp::PackRegion) * R.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->pitem[slot], I.data(), sizeof(pmp::PackItem) * I.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return PMP_ERR_CUDA;
    b->nreg[slot] = n;
    b->npitem[slot] = (int)I.size();
    b->reg_h[slot] = R;
    return PMP_OK;
}

static pmp_status pack_impl(pmp_batch *b, int32_t slot, const double *src, double *dst, int to_msg, int folded)
{
    if (!b || slot < 0 || slot >= pmp::kRegionSlots || !src || !dst) return PMP_ERR_ARG;
    if (b->npitem[slot] == 0) return PMP_OK;
    pmp_particles none;
    std::memset(&none, 0, sizeof(none));
    const double *arena = to_msg ? src : dst;
    BArgs a = make_args(b, const_cast<double *>(arena), const_cast<double *>(arena), &none, nullptr, nullptr);
    pmp::k_batch_pack<<<(unsigned)b->npitem[slot], pmp::kPackThreads, 0, b->ctx->stream>>>(
        a, b->reg[slot], b->pitem[slot], src, dst, to_msg, folded);
    return cudaGetLastError() == cudaSuccess ? PMP_OK : PMP_ERR_CUDA;
}

pmp_status pmp_batch_pack(pmp_batch *b, int32_t slot, const double *arena, double *msg, int32_t folded)
{
    if (folded != 0 && folded != 1) return PMP_ERR_ARG;
    if (b && folded && slot >= 0 && slot < pmp::kRegionSlots) {
        // folded sums are formed at valid cells of owned patches only
        for (const auto &r : b->reg_h[slot]) {
            if (r.patch >= b->n_owned) return PMP_ERR_ARG;
            for (int a = 0; a < 3; ++a)
                if (r.lo[a] < 0 || r.hi[a] > b->patches[r.patch].n[a]) return PMP_ERR_ARG;
        }
    }
    return pack_impl(b, slot, arena, msg, 1, folded);
}

pmp_status pmp_batch_unpack(pmp_batch *b, int32_t slot, const double *msg, double *arena)
{
    return pack_impl(b, slot, msg, arena, 0, 0);
}

pmp_status pmp_batch_hold_barriers(pmp_batch *b, int32_t arrivals)
{
    if (!b || arrivals < 0 || arrivals > 1) return PMP_ERR_ARG;
    if (cudaStreamSynchronize(b->ctx->stream) != cudaSuccess) return PMP_ERR_CUDA;
    b->hold = (unsigned)arrivals;
    if (b->graph) {  // the captured launch holds the old arguments
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return PMP_OK;
}

pmp_status pmp_batch_info(const pmp_batch *b, int32_t *grid, int64_t *items)
{
    if (!b) return PMP_ERR_ARG;
    if (grid) *grid = b->grid;
    if (items) {
        items[0] = (int64_t)b->zero_h.size();
        items[1] = (int64_t)b->dep_h.size();
        items[2] = (int64_t)b->app_h.size();
    }
    return PMP_OK;
}

}  // extern "C"
