// pmp_mesh.cu -- cell-side kernels: buffer zeroing, the ghost fold (Step 2 on
// one GPU) and the limited apply (Steps 3 + 5).
#include "pmp_device.cuh"
#include "pmp_launch.h"
#include "pmp_plan.cuh"

namespace pmp {

// Zero fields [0, 5) over cells [0, ncells), 16-byte stores where aligned.
__global__ void __launch_bounds__(256) k_zero(double *__restrict__ b, long long fs, long long ncells)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int f = 0; f < NF; ++f) {
        double *base = b + (long long)f * fs;
        const long long head = (reinterpret_cast<uintptr_t>(base) & 15) ? 1 : 0;
        const long long nvec = (ncells - head) / 2;
        double2 *v = reinterpret_cast<double2 *>(base + head);
        for (long long i = tid; i < nvec; i += stride) v[i] = make_double2(0.0, 0.0);
        if (tid == 0) {
            if (head) base[0] = 0.0;
            if (head + 2 * nvec < ncells) base[ncells - 1] = 0.0;
        }
    }
}

// Step 2: one warp per valid row (j, k).  Rows inside the y and z ghost
// shells are folded whole; other rows only at the x ends.  Images are added
// in lexicographic order of (oz, oy, ox).
__global__ void __launch_bounds__(256) k_fold(Box B, double *__restrict__ b)
{
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long nrows = (long long)B.n1 * B.n2;
    if (warp >= nrows) return;
    const int j = (int)(warp % B.n1), k = (int)(warp / B.n1);
    const int g = B.g;
    const bool yz_shell = (B.per1 && (j < g || j >= B.n1 - g)) || (B.per2 && (k < g || k >= B.n2 - g));
    int ends = 0;  // cells per end of the row to visit
    if (yz_shell) ends = B.n0;
    else if (B.per0) ends = g < B.n0 ? g : B.n0;
    else return;
    const int nvisit = yz_shell ? B.n0 : (2 * ends < B.n0 ? 2 * ends : B.n0);
    for (int t = lane; t < nvisit; t += 32) {
        int i;
        if (yz_shell || 2 * ends >= B.n0) i = t;
        else i = t < ends ? t : B.n0 - 2 * ends + t;
        const long long c = B.at(i, j, k);
        double v[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) v[f] = b[(long long)f * B.fs + c];
        for (int oz = -1; oz <= 1; ++oz) {
            if (oz && !B.per2) continue;
            const int gk = k + oz * B.n2;
            if (gk < -g || gk >= B.n2 + g) continue;
            for (int oy = -1; oy <= 1; ++oy) {
                if (oy && !B.per1) continue;
                const int gj = j + oy * B.n1;
                if (gj < -g || gj >= B.n1 + g) continue;
                for (int ox = -1; ox <= 1; ++ox) {
                    if (ox && !B.per0) continue;
                    if (!ox && !oy && !oz) continue;
                    const int gi = i + ox * B.n0;
                    if (gi < -g || gi >= B.n0 + g) continue;
                    const long long im = B.at(gi, gj, gk);
#pragma unroll
                    for (int f = 0; f < NF; ++f) v[f] = v[f] + b[(long long)f * B.fs + im];
                }
            }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) b[(long long)f * B.fs + c] = v[f];
    }
}

// FP32 pre-check of the Eq. lambda constraint at lambda = 1, on values
// converted from the FP64 operands: f = e_int0 rho'/rho + |p + dp|^2/(2 rho')
// - E' with e_int0 = E - |p|^2/(2 rho).  With rho' >= rho (a deposit that adds
// mass), every FP32 rounding, the cancellations in E - |p|^2/(2 rho) and in
// p + dp included, perturbs f by at most a few 2^-23 M, where M = (E +
// |p|^2/(2 rho)) rho'/rho + |p + dp|^2/(2 rho') + |E'|; in all well under
// 2^-18 M, while the FP64 expression is within 2^-48 M of exact.  f < -2^-14 M
// therefore means the FP64 test passes (lambda = 1) as well.  Returns false
// when undecided (including rho' < rho, over- or underflow), so the caller
// runs the FP64 limiter, whose first step is the exact test.
__device__ __forceinline__ bool sn_lambda_holds_f32(const double U[NF], const double D[NF])
{
    const float r = f32_trunc(U[0]), p0 = f32_trunc(U[1]), p1 = f32_trunc(U[2]), p2 = f32_trunc(U[3]),
                E = f32_trunc(U[4]);
    const float dr = f32_trunc(D[0]), d0 = f32_trunc(D[1]), d1 = f32_trunc(D[2]), d2 = f32_trunc(D[3]),
                dE = f32_trunc(D[4]);
    const float r1 = r + dr, E1 = E + dE;
    const float pp = (p0 * p0 + p1 * p1) + p2 * p2;
    const float k0 = pp / (2.0f * r);
    const float q = r1 / r;
    const float n0 = p0 + d0, n1 = p1 + d1, n2 = p2 + d2;
    const float kn = ((n0 * n0 + n1 * n1) + n2 * n2) / (2.0f * r1);
    const float f = ((E - k0) * q + kn) - E1;
    const float M = (fabsf(E) + k0) * q + kn + fabsf(E1);
    return dr >= 0.0f && M > 1e-30f && M < 1e30f && f < -6.103515625e-05f * M;
}

// Valid cell v (x fastest) -> (i, j, k), in 32-bit arithmetic when the box
// has fewer than 2^32 valid cells (a 64-bit division costs several times the
// instructions of a 32-bit one).
__device__ __forceinline__ void cell_of(const Box &S, long long v, long long nvalid, int &i, int &j, int &k)
{
    if (nvalid <= 0xffffffffLL) {
        const unsigned w = (unsigned)v, n0 = (unsigned)S.n0, n1 = (unsigned)S.n1;
        const unsigned r = w / n0;
        i = (int)(w - r * n0);
        const unsigned kk = r / n1;
        j = (int)(r - kk * n1);
        k = (int)kk;
    } else {
        i = (int)(v % S.n0);
        const long long r = v / S.n0;
        j = (int)(r % S.n1);
        k = (int)(r / S.n1);
    }
}

// Adds the block's total of `mine` to *ctr with one atomic.  Every thread of
// the block calls it (it holds a barrier); `sh` has a slot per warp.  One
// atomic per warp on a single counter serialises at its L2 slice: millions
// of them at 512^3.
__device__ __forceinline__ void block_add(unsigned long long *ctr, unsigned mine, unsigned *sh)
{
    const unsigned w = __reduce_add_sync(0xffffffffu, mine);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
        if (t) atomicAdd(ctr, t);
    }
}

// True when the three momentum changes are zero (+0 or -0), tested on the
// bits so that the FP64 pipe is left to the arithmetic.
__device__ __forceinline__ bool no_dp(const double D[NF])
{
    const unsigned long long m = (unsigned long long)__double_as_longlong(D[1]) |
                                 (unsigned long long)__double_as_longlong(D[2]) |
                                 (unsigned long long)__double_as_longlong(D[3]);
    return (m << 1) == 0;
}

constexpr int kApplyThreads = 256;
constexpr int kFbPend = 64;  // cells a warp holds back for its FP64 limiter batch

// Steps 3 + 5 for feedback in one streaming pass.  Cells that receive
// nothing, receive no momentum, or whose Eq. lambda constraint holds at
// lambda = 1 by the FP32 pre-check are updated at once; a warp keeps the
// others, with the state and summed change it has just loaded, in a
// shared-memory list and runs the FP64 limiter on 32 of them whenever that
// many are pending (a full-warp FP64 branch, overlapped with the other warps'
// streaming; no cell is read twice).
#ifndef PMP_FB_APPLY_MINB
#define PMP_FB_APPLY_MINB 3
#endif
__global__ void __launch_bounds__(kApplyThreads, PMP_FB_APPLY_MINB) k_apply_fb_stream(Box S, double *__restrict__ u, Box B,
                                                                      const double *__restrict__ b,
                                                                      double *__restrict__ eta_out, DevStatus *st)
{
    constexpr int kW = kApplyThreads / 32;
    __shared__ double pend[kW][kFbPend][2 * NF];
    __shared__ long long pcell[kW][kFbPend];
    __shared__ unsigned sh[kW];
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned nl = 0, nr = 0;
    int npend = 0;  // the same in every lane
    // the limiter on pending entry q (one lane)
    auto limit = [&](int q) {
        const long long v = pcell[wid][q];
        const double *e_ = pend[wid][q];
        double U[NF], D[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            U[f] = e_[f];
            D[f] = e_[NF + f];
        }
        int i, j, k;
        cell_of(S, v, nvalid, i, j, k);
        const long long cs = S.at(i, j, k);
        // pending cells receive momentum (no_dp was false)
        int noroot;
        double rho1, E1;
        const double l = sn_lambda_dp(U, D, noroot, rho1, E1);
        nl += l < 1.0;
        nr += noroot;
        if (eta_out) eta_out[v] = l;
        u[cs] = rho1;
        u[S.fs + cs] = U[1] + l * D[1];
        u[2 * S.fs + cs] = U[2] + l * D[2];
        u[3 * S.fs + cs] = U[3] + l * D[3];
        u[4 * S.fs + cs] = E1;
    };
    const long long step = (long long)gridDim.x * kApplyThreads;
    for (long long v0 = ((long long)blockIdx.x * kW + wid) * 32; v0 < nvalid; v0 += step) {
        const long long v = v0 + lane;
        bool need = false;
        double U[NF], D[NF];
        if (v < nvalid) {
            int i, j, k;
            cell_of(S, v, nvalid, i, j, k);
            const long long cs = S.at(i, j, k), cb = B.at(i, j, k);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                D[f] = __ldg(b + (long long)f * B.fs + cb);
                U[f] = u[(long long)f * S.fs + cs];
            }
            if (all_zero(D)) {
                if (eta_out) eta_out[v] = 1.0;
            } else if (no_dp(D) || sn_lambda_holds_f32(U, D)) {
                if (eta_out) eta_out[v] = 1.0;
#pragma unroll
                for (int f = 0; f < NF; ++f) u[(long long)f * S.fs + cs] = U[f] + D[f];
            } else {
                need = true;
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, need);
        if (need) {
            const int q = npend + __popc(m & lt);
            pcell[wid][q] = v;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                pend[wid][q][f] = U[f];
                pend[wid][q][NF + f] = D[f];
            }
        }
        npend += __popc(m);
        __syncwarp();
        if (npend >= 32) {
            limit(npend - 32 + lane);
            npend -= 32;
            __syncwarp();
        }
    }
    if (lane < npend) limit(lane);
    block_add(&st->n_limited, nl, sh);
    __syncthreads();
    block_add(&st->n_noroot, nr, sh);
}

// Per-cell sink records, each value in the order the sink formulas state it:
// G = (rho, p) and rho c_s for the gather; D = (p inv, E inv) with inv =
// 1/rho for the spread and Step 4; rho - rho_Tr (Eq. truelove) for the
// deposit and the limiter; eta = 1 until Step 3 limits the cell.
__global__ void __launch_bounds__(256) k_sink_aux(KParams P, Box S, const double *__restrict__ u,
                                                  double *__restrict__ grec, double *__restrict__ gcs,
                                                  double *__restrict__ drec, double *__restrict__ dtr,
                                                  double *__restrict__ deta)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvalid) return;
    const int i = (int)(v % S.n0);
    const long long r = v / S.n0;
    const int j = (int)(r % S.n1), k = (int)(r / S.n1);
    double U[NF], cs, rtr;
    load_cell(u, S, S.at(i, j, k), U);
    const double inv = exact::div_rn(1.0, U[0]);
    sink_cell(P, U, inv, cs, rtr);
    double2 *g = reinterpret_cast<double2 *>(grec + v * kGRec);
    g[0] = make_double2(U[0], U[1]);
    g[1] = make_double2(U[2], U[3]);
    gcs[v] = U[0] * cs;
    double2 *d = reinterpret_cast<double2 *>(drec + v * kDRec);
    d[0] = make_double2(U[1] * inv, U[2] * inv);
    d[1] = make_double2(U[3] * inv, U[4] * inv);
    dtr[v] = U[0] - rtr;
    deta[v] = 1.0;
}

// Step 1 for sinks in the ATOMIC mode, second half.  Every pair's change is
// Delta U = -a (1, p inv, E inv) with the factors of its cell (the owner, for
// a ghost image), so the deposit sums only s = sum(-a) per buffer cell into a
// one-field scratch, and here the cell's buffer gains s (1, p inv, E inv)
// from its owner's D record (fused multiply-adds: this pass is bound by the
// FP64 pipe, not by HBM, at five separate operations per cell).  In real
// arithmetic this is the sum of the pairs' five-field changes; in FP64 it
// differs from that sum by the order of the additions and the rounding of
// the products, as any atomic order does.
// A block takes padded rows (j, k), its threads the cells i of the row.
__global__ void __launch_bounds__(256) k_sink_spread(Box S, Box B, double *__restrict__ b,
                                                     const double *__restrict__ scr, const double *__restrict__ drec)
{
    const long long py = B.pxy / B.px;
    const long long rows = B.ncells / B.px;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int k = (int)(row / py) - B.g, j = (int)(row % py) - B.g;
        const long long c0 = row * B.px;
        for (int ii = threadIdx.x; ii < B.px; ii += blockDim.x) {
            const long long c = c0 + ii;
            const double sc = scr[c];
            if ((__double_as_longlong(sc) << 1) == 0) continue;  // +-0: no pair reached the cell
            const int i = ii - B.g;
            const double2 *d = reinterpret_cast<const double2 *>(
                drec + vidx(S, owner(i, S.n0), owner(j, S.n1), owner(k, S.n2)) * kDRec);
            const double2 d0 = __ldg(d), d1 = __ldg(d + 1);
            b[c] += sc;
            b[B.fs + c] = fma(sc, d0.x, b[B.fs + c]);
            b[2 * B.fs + c] = fma(sc, d0.y, b[2 * B.fs + c]);
            b[3 * B.fs + c] = fma(sc, d1.x, b[3 * B.fs + c]);
            b[4 * B.fs + c] = fma(sc, d1.y, b[4 * B.fs + c]);
        }
    }
}

// FP32 pre-test of the sink limiter's fast case: true only when the FP64
// tests a <= RN(cap rho) and a <= RN(rho - rho_min) both hold, for a > 0.
// af and rf are a and rho truncated to FP32 (within 2^-23 below), cap is
// rounded down and rho_min up, and the comparison carries a 2^-16 relative
// margin on each side: up = af (1 + 2^-16) exceeds a, and t1 = (cap rho) (1 -
// 2^-16), t2 = (rho - rho_min) (1 - 2^-16), each with at most three FP32
// roundings, stay below the FP64 values.  An operand outside the FP32 normal
// range gives NaN or a subnormal bound, and so false; t1 is kept below 1e30
// so that no product overflows.  False means "undecided": the caller runs
// the FP64 tests.
__device__ __forceinline__ bool sink_eta_one_f32(const KParams &P, double rho, double d0)
{
    const float af = -f32_trunc(d0), rf = f32_trunc(rho);
    const float up = af * 1.0000152587890625f;
    const float t1 = (P.cap_lo * rf) * 0.9999847412109375f;
    const float t2 = (rf - P.rho_min_hi) * 0.9999847412109375f;
    return up < t1 && up < t2 && t1 < 1e30f;
}

// Sink limiter (Sec. 3.1.1 with the density floor) in FP64 for a cell with
// removal a = -D[0] > 0 that the FP32 pre-test left undecided; t is rho -
// rho_Tr from the cell's D record.  Same operations as sink_eta.
__device__ __forceinline__ double sink_eta_fp64(const KParams &P, double rho, double d0, double t)
{
    const double a = -d0;
    const double capr = P.cap * rho;
    const double fl = rho - P.rho_min;
    if (a <= capr && a <= fl) return 1.0;
    double al = a < capr ? a : capr;
    al = al > t ? al : t;
    al = al < fl ? al : fl;
    if (al < 0.0) al = 0.0;
    return al < a ? al / a : 1.0;
}

// a = -D[0] > 0 exactly when D[0] is negative: sign set, not -0, not NaN
// (decided on the bits, no FP64 instruction).
__device__ __forceinline__ bool removal_positive(double d0)
{
    const unsigned long long b0 = (unsigned long long)__double_as_longlong(d0);
    const unsigned long long mag2 = b0 << 1;
    return (b0 >> 63) != 0 && mag2 != 0 && mag2 <= (0x7ff0000000000000ULL << 1);
}

// One cell's Steps 3 + 5 for sinks once eta is known: eta to eta_out and,
// for a cell that went through the FP64 limiter (LIM), to deta, where Step 4
// reads it (the cell records pass writes eta = 1 for every cell, so the other
// cells need no write here); U += eta Delta U^sum (one eta for every field; a
// cell whose change is zero in every field is left as it is).
template <bool LIM>
__device__ __forceinline__ void sink_update(const Box &S, double *__restrict__ u, long long v, long long cs,
                                            const double U[NF], const double D[NF], double e,
                                            double *__restrict__ deta, double *__restrict__ eta_out)
{
    if (LIM) deta[v] = e;
    if (eta_out) eta_out[v] = e;
    if (all_zero(D)) return;
    if (e == 1.0) {
#pragma unroll
        for (int f = 0; f < NF; ++f) u[(long long)f * S.fs + cs] = U[f] + D[f];
    } else {
#pragma unroll
        for (int f = 0; f < NF; ++f) u[(long long)f * S.fs + cs] = U[f] + e * D[f];
    }
}

constexpr int kSinkPend = 64;  // cells a warp holds back for its FP64 limiter batch

// Steps 3 + 5 for sinks in one pass over the valid cells, a warp taking 32
// consecutive cells at a time.  eta = 1 wherever it is decided without FP64
// work -- no removal (from the bits of Delta rho^sum) or the FP32 pre-test
// above -- and those cells are updated at once.  The cells left undecided
// (about one in twenty) are held back, with their loaded state and summed
// change, in the warp's shared-memory list; whenever it holds 32 of them the
// warp runs the FP64 limiter on all 32 lanes.  Issued cell by cell in place,
// that branch would take the FP64 pipe for every warp in which one lane
// takes it.  Every decision is the FP64 one.  Step 4 reads only the records,
// the particles and the plan, never the state, so it can follow this pass.
// Limited cells are counted per block.
#ifndef PMP_SINK_APPLY_MINB
#define PMP_SINK_APPLY_MINB 3
#endif
__global__ void __launch_bounds__(kApplyThreads, PMP_SINK_APPLY_MINB) k_sink_eta_apply(KParams P, Box S, double *__restrict__ u, Box B,
                                                                     const double *__restrict__ b,
                                                                     const double *__restrict__ dtr,
                                                                     double *__restrict__ deta,
                                                                     double *__restrict__ eta_out, DevStatus *st)
{
    constexpr int kW = kApplyThreads / 32;
    __shared__ double pend[kW][kSinkPend][2 * NF];
    __shared__ long long pcell[kW][kSinkPend];
    __shared__ unsigned sh[kW];
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned nl = 0;
    int npend = 0;  // the same in every lane
    // the limiter on pending entry q (one lane)
    auto limit = [&](int q) {
        const long long v = pcell[wid][q];
        const double *e_ = pend[wid][q];
        double U[NF], D[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            U[f] = e_[f];
            D[f] = e_[NF + f];
        }
        int i, j, k;
        cell_of(S, v, nvalid, i, j, k);
        const double e = sink_eta_fp64(P, U[0], D[0], __ldg(dtr + v));
        nl += e < 1.0;
        sink_update<true>(S, u, v, S.at(i, j, k), U, D, e, deta, eta_out);
    };
    const long long step = (long long)gridDim.x * kApplyThreads;
    for (long long v0 = ((long long)blockIdx.x * kW + wid) * 32; v0 < nvalid; v0 += step) {
        const long long v = v0 + lane;
        bool need = false;
        long long cs = 0;
        double U[NF], D[NF];
        if (v < nvalid) {
            int i, j, k;
            cell_of(S, v, nvalid, i, j, k);
            cs = S.at(i, j, k);
            const long long cb = B.at(i, j, k);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                D[f] = __ldg(b + (long long)f * B.fs + cb);
                U[f] = u[(long long)f * S.fs + cs];
            }
            need = removal_positive(D[0]) && !sink_eta_one_f32(P, U[0], D[0]);
        }
        const unsigned m = __ballot_sync(0xffffffffu, need);
        if (need) {
            const int q = npend + __popc(m & lt);
            pcell[wid][q] = v;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                pend[wid][q][f] = U[f];
                pend[wid][q][NF + f] = D[f];
            }
        } else if (v < nvalid) {
            sink_update<false>(S, u, v, cs, U, D, 1.0, deta, eta_out);
        }
        npend += __popc(m);
        __syncwarp();
        if (npend >= 32) {
            limit(npend - 32 + lane);
            npend -= 32;
            __syncwarp();
        }
    }
    if (lane < npend) limit(lane);
    block_add(&st->n_limited, nl, sh);
}

// Adjoint of the limited apply: pass[c] = 1 where the supernova limiter left
// the cell's change unscaled (lambda = 1), 0 where it acted; gradients flow
// only through the former.
__global__ void __launch_bounds__(256) k_pass_mask(Box S, const double *__restrict__ u, Box B,
                                                   const double *__restrict__ b, unsigned char *__restrict__ pass)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvalid) return;
    const int i = (int)(v % S.n0);
    const long long r = v / S.n0;
    const int j = (int)(r % S.n1), k = (int)(r / S.n1);
    const long long cs = S.at(i, j, k), cb = B.at(i, j, k);
    double U[NF], D[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        U[f] = __ldg(u + (long long)f * S.fs + cs);
        D[f] = __ldg(b + (long long)f * B.fs + cb);
    }
    bool ok = (D[1] == 0.0 && D[2] == 0.0 && D[3] == 0.0) || sn_lambda_holds_f32(U, D);
    if (!ok) {
        int nr;
        ok = sn_lambda(U, D, nr) == 1.0;
    }
    pass[v] = ok ? 1 : 0;
}

void launch_pass_mask(const Box &S, const double *u, const Box &B, const double *b, unsigned char *pass,
                      cudaStream_t stream)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    k_pass_mask<<<(unsigned)((nvalid + 255) / 256), 256, 0, stream>>>(S, u, B, b, pass);
}

void launch_zero(const Box &B, double *b, cudaStream_t stream)
{
    k_zero<<<152 * 8, 256, 0, stream>>>(b, B.fs, B.ncells);
}

// Auxiliary conserved fields under accretion (the extensions of Sec. 3.1.1
// beyond minimal hydrodynamics: the dual-energy internal energy and species
// densities), at fixed specific value: every pair's change of field X is
// -a X/rho with the cell's X/rho, so the summed change is (X/rho) Delta rho^sum
// and the limited update X := X + eta ((X / rho) Delta rho^sum), eta the
// cell's accretion limiter.  Runs before Step 5 (rho is the pre-update one).
__global__ void __launch_bounds__(256) k_apply_extra(KParams P, Box S, const double *__restrict__ u, Box B,
                                                     const double *__restrict__ b, double *__restrict__ X, int nx,
                                                     long long xs)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvalid) return;
    const int i = (int)(v % S.n0);
    const long long r = v / S.n0;
    const int j = (int)(r % S.n1), k = (int)(r / S.n1);
    double D[NF];
    load_cell(b, B, B.at(i, j, k), D);
    if (all_zero(D)) return;
    double U[NF];
    load_cell(u, S, S.at(i, j, k), U);
    const double eta = sink_eta(P, U, D);
    const long long c = S.at(i, j, k);
    for (int f = 0; f < nx; ++f) {
        const double x = X[(long long)f * xs + c];
        X[(long long)f * xs + c] = x + eta * ((x / U[0]) * D[0]);
    }
}

void launch_apply_extra(const KParams &P, const Box &S, const double *u, const Box &B, const double *b, double *X,
                        int nx, long long xs, cudaStream_t stream)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    k_apply_extra<<<(unsigned)((nvalid + 255) / 256), 256, 0, stream>>>(P, S, u, B, b, X, nx, xs);
}

// Sink creation (Sec. 3.1.2), pass 1: a valid cell qualifies when the
// retained accretion buffer is zero in every field there (no sink within
// r_K), rho > rho_Tr (Eq. truelove with the cell's c_s), and rho is strictly
// larger than at every other cell whose centre lies within r_K (periodic
// images on periodic axes).  Reads only.
__global__ void __launch_bounds__(256) k_create_flags(KParams P, Box S, const double *__restrict__ u, Box B,
                                                      const double *__restrict__ b, unsigned *__restrict__ flags)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvalid) return;
    const int i = (int)(v % S.n0);
    const long long r = v / S.n0;
    const int j = (int)(r % S.n1), k = (int)(r / S.n1);
    unsigned ok = 0;
    double D[NF];
    load_cell(b, B, B.at(i, j, k), D);
    if (all_zero(D)) {
        double U[NF];
        load_cell(u, S, S.at(i, j, k), U);
        if (U[0] > sink_rho_tr(P, U)) {
            ok = 1;
            const int R = P.R;
            for (int oz = -R; oz <= R && ok; ++oz)
                for (int oy = -R; oy <= R && ok; ++oy)
                    for (int ox = -R; ox <= R && ok; ++ox) {
                        if (!ox && !oy && !oz) continue;
                        const double d2 = (double)(ox * ox + oy * oy) + (double)(oz * oz);
                        if (!(d2 < P.r2)) continue;
                        int a = i + ox, bb = j + oy, c = k + oz;
                        if (a < 0 || a >= S.n0) {
                            if (!S.per0) continue;
                            a = wrapi(a, S.n0);
                        }
                        if (bb < 0 || bb >= S.n1) {
                            if (!S.per1) continue;
                            bb = wrapi(bb, S.n1);
                        }
                        if (c < 0 || c >= S.n2) {
                            if (!S.per2) continue;
                            c = wrapi(c, S.n2);
                        }
                        if (a == i && bb == j && c == k) continue;
                        if (!(U[0] > __ldg(u + S.at(a, bb, c)))) ok = 0;
                    }
        }
    }
    flags[v] = ok;
}

// Pass 2: each qualifying cell with position p < cap (the exclusive scan of
// the flags, so sinks come in cell order) becomes sink p at the cell centre
// with m = (rho - rho_Tr) V and p = m v; the cell keeps v and E/rho with
// rho := rho_Tr.  The last cell writes the total.
__global__ void __launch_bounds__(256) k_create_apply(KParams P, Box S, double *__restrict__ u,
                                                      const unsigned *__restrict__ flags,
                                                      const unsigned long long *__restrict__ pos, long long cap,
                                                      double *x, double *y, double *z, double *m, double *px,
                                                      double *py, double *pz, long long *count)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvalid) return;
    const unsigned f = flags[v];
    const unsigned long long q = pos[v];
    if (v == nvalid - 1) *count = (long long)(q + f);
    if (!f || (long long)q >= cap) return;
    const int i = (int)(v % S.n0);
    const long long r = v / S.n0;
    const int j = (int)(r % S.n1), k = (int)(r / S.n1);
    const long long c = S.at(i, j, k);
    double U[NF];
    load_cell(u, S, c, U);
    const double rtr = sink_rho_tr(P, U);
    const double v0 = exact::div_rn(U[1], U[0]), v1 = exact::div_rn(U[2], U[0]), v2 = exact::div_rn(U[3], U[0]);
    const double es = exact::div_rn(U[4], U[0]);
    const double ms = (U[0] - rtr) * P.V;
    x[q] = (double)i + 0.5;
    y[q] = (double)j + 0.5;
    z[q] = (double)k + 0.5;
    m[q] = ms;
    px[q] = ms * v0;
    py[q] = ms * v1;
    pz[q] = ms * v2;
    u[c] = rtr;
    u[S.fs + c] = rtr * v0;
    u[2 * S.fs + c] = rtr * v1;
    u[3 * S.fs + c] = rtr * v2;
    u[4 * S.fs + c] = rtr * es;
}

void launch_create_flags(const KParams &P, const Box &S, const double *u, const Box &B, const double *b,
                         unsigned *flags, cudaStream_t stream)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    k_create_flags<<<(unsigned)((nvalid + 255) / 256), 256, 0, stream>>>(P, S, u, B, b, flags);
}

void launch_create_apply(const KParams &P, const Box &S, double *u, const unsigned *flags,
                         const unsigned long long *pos, long long cap, double *x, double *y, double *z, double *m,
                         double *px, double *py, double *pz, long long *count, cudaStream_t stream)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    k_create_apply<<<(unsigned)((nvalid + 255) / 256), 256, 0, stream>>>(P, S, u, flags, pos, cap, x, y, z, m, px,
                                                                         py, pz, count);
}

// App. A.1 rounding, every padded buffer cell and field (grid-stride).
__global__ void __launch_bounds__(256) k_round(Box B, double *__restrict__ b, const double *__restrict__ E, int M)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < B.ncells; c += stride) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const long long o = (long long)f * B.fs + c;
            const double e = E[o];
            if (e > 0.0) b[o] = repro_round(b[o], e, M);
        }
    }
}

void launch_round(const Box &B, double *b, const double *E, int M, cudaStream_t stream)
{
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long need = (B.ncells + 255) / 256;
    const long long grid = need < (long long)nsm * 8 ? need : (long long)nsm * 8;
    k_round<<<(unsigned)(grid > 0 ? grid : 1), 256, 0, stream>>>(B, b, E, M);
}

void launch_fold(const Box &B, double *b, cudaStream_t stream)
{
    const long long nrows = (long long)B.n1 * B.n2;
    const long long threads = nrows * 32;
    k_fold<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(B, b);
}

void launch_sink_aux(const KParams &P, const Box &S, const double *u, double *grec, double *gcs, double *drec,
                     double *dtr, double *deta, cudaStream_t stream)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    k_sink_aux<<<(unsigned)((nvalid + 255) / 256), 256, 0, stream>>>(P, S, u, grec, gcs, drec, dtr, deta);
}

void launch_sink_spread(const Box &S, const Box &B, double *b, const double *scr, const double *drec,
                        cudaStream_t stream)
{
    const long long rows = B.ncells / B.px;
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long grid = rows < 8LL * nsm ? rows : 8LL * nsm;
    if (grid > 0) k_sink_spread<<<(unsigned)grid, 256, 0, stream>>>(S, B, b, scr, drec);
}

// Resident grid of a grid-stride cell kernel: SMs x resident blocks, capped
// by the blocks the work needs.
template <typename K>
static unsigned resident_grid(K kernel, int threads, long long need)
{
    int dev = 0, nsm = 152, per_sm = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long cap = (long long)nsm * per_sm;
    const long long g = need < cap ? need : cap;
    return (unsigned)(g > 0 ? g : 1);
}

void launch_sink_eta_apply(const KParams &P, const Box &S, double *u, const Box &B, const double *b, const double *dtr,
                           double *deta, double *eta_out, DevStatus *st, cudaStream_t stream)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    if (nvalid == 0) return;
    const unsigned grid = resident_grid(k_sink_eta_apply, kApplyThreads, (nvalid + kApplyThreads - 1) / kApplyThreads);
    k_sink_eta_apply<<<grid, kApplyThreads, 0, stream>>>(P, S, u, B, b, dtr, deta, eta_out, st);
}

void launch_apply_fb_stream(const Box &S, double *u, const Box &B, const double *b, double *eta_out, DevStatus *st,
                            cudaStream_t stream)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    if (nvalid == 0) return;
    const unsigned grid = resident_grid(k_apply_fb_stream, kApplyThreads, (nvalid + kApplyThreads - 1) / kApplyThreads);
    k_apply_fb_stream<<<grid, kApplyThreads, 0, stream>>>(S, u, B, b, eta_out, st);
}

// Step 5 of the particle-mesh deposit (no Step 3 in Sec. 2.2's PM/PIC subset):
// U += Delta U^sum, eta = 1.
__global__ void __launch_bounds__(256) k_apply_add(Box S, double *__restrict__ u, Box B, const double *__restrict__ b,
                                                   double *__restrict__ eta_out)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvalid) return;
    const int i = (int)(v % S.n0);
    const long long r = v / S.n0;
    const int j = (int)(r % S.n1), k = (int)(r / S.n1);
    const long long cs = S.at(i, j, k), cb = B.at(i, j, k);
    double D[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) D[f] = __ldg(b + (long long)f * B.fs + cb);
    if (eta_out) eta_out[v] = 1.0;
    if (all_zero(D)) return;
#pragma unroll
    for (int f = 0; f < NF; ++f) u[(long long)f * S.fs + cs] = u[(long long)f * S.fs + cs] + D[f];
}

void launch_apply(const KParams &P, const Box &S, double *u, const Box &B, const double *b, double *eta_out,
                  DevStatus *st, cudaStream_t stream)
{
    const long long nvalid = (long long)S.n0 * S.n1 * S.n2;
    if (nvalid == 0) return;
    if (P.kind == PMP_KIND_MASS) {
        k_apply_add<<<(unsigned)((nvalid + 255) / 256), 256, 0, stream>>>(S, u, B, b, eta_out);
    } else {
        launch_apply_fb_stream(S, u, B, b, eta_out, st, stream);
    }
}

}  // namespace pmp
