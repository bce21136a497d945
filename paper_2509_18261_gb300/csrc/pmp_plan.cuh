// pmp_plan.cuh -- the per-pass plan: each particle's kernel cells, found once
// and reused by gather, deposit, Step 4 and the adjoint.
//
// Decisions that compare an FP64 sum of three squares with r_K^2 (kernel
// membership; the sub-point count of the covered fraction omega) are taken
// first in FP32.  The FP32 offsets are built from the FP64 cell-edge offsets
// fl(c - x) converted to FP32 plus an exact FP32 fraction; each differs from
// the exact offset by at most 2^-24 (|c - x| + |offset|), so the FP32 sum of
// squares is within about 1.3 * 2^-20 (R+1)^2 of the exact sum, below
// 2^-14 r_K^2 for every allowed r_K.  A result outside the band
// r_K^2 (1 -/+ 2^-14) therefore decides the FP64 comparison exactly; inside
// it the FP64 sum is formed in the canonical order and compared.  Every
// decision equals the one the plain FP64 definition takes.
#pragma once

#include "pmp_device.cuh"

namespace pmp {

struct R2Band {
    double r2;
    float lo, hi;  // r2 (1 -/+ 2^-14), rounded outward
};

__device__ __forceinline__ R2Band make_band(double r2)
{
    R2Band b;
    b.r2 = r2;
    b.lo = __double2float_rd(r2 * (1.0 - 6.103515625e-05));
    b.hi = __double2float_ru(r2 * (1.0 + 6.103515625e-05));
    return b;
}

// Packed pair: unwrapped cell coordinates + R in bits 0-47 (16 each), the
// omega sub-point count in bits 48-63.
__device__ __forceinline__ unsigned long long pack_pair(int i, int j, int k, int R, int cnt)
{
    return (unsigned long long)(unsigned)(i + R) | ((unsigned long long)(unsigned)(j + R) << 16) |
           ((unsigned long long)(unsigned)(k + R) << 32) | ((unsigned long long)(unsigned)cnt << 48);
}

struct PairCell {
    int i, j, k, cnt;
};

__device__ __forceinline__ PairCell unpack_pair(unsigned long long v, int R)
{
    PairCell c;
    c.i = (int)(v & 0xffffULL) - R;
    c.j = (int)((v >> 16) & 0xffffULL) - R;
    c.k = (int)((v >> 32) & 0xffffULL) - R;
    c.cnt = (int)(v >> 48);
    return c;
}

__device__ __forceinline__ unsigned long long pack_host(int hx, int hy, int hz)
{
    return (unsigned long long)(unsigned)hx | ((unsigned long long)(unsigned)hy << 21) |
           ((unsigned long long)(unsigned)hz << 42);
}

__device__ __forceinline__ void unpack_host(unsigned long long v, int &hx, int &hy, int &hz)
{
    hx = (int)(v & 0x1fffffULL);
    hy = (int)((v >> 21) & 0x1fffffULL);
    hz = (int)((v >> 42) & 0x1fffffULL);
}

// Owning valid coordinate of an unwrapped one (|c| stays within one period).
__device__ __forceinline__ int owner(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// Index of a valid cell in a compact (no ghost) per-cell array.
__device__ __forceinline__ long long vidx(const Box &B, int i, int j, int k)
{
    return ((long long)k * B.n1 + j) * B.n0 + i;
}

// Exact FP64 membership test of a cell centre, in the canonical order.
static __device__ __noinline__ bool centre_inside_exact(double r2, int ci, int cj, int ck, double x, double y, double z)
{
    const double d0 = ((double)ci + 0.5) - x, d1 = ((double)cj + 0.5) - y, d2 = ((double)ck + 0.5) - z;
    return (d0 * d0 + d1 * d1) + d2 * d2 < r2;
}

// Exact FP64 sub-point test, in the canonical order.
static __device__ __noinline__ bool subpoint_inside_exact(double r2, double fa, double fb, double fc, int ci, int cj, int ck,
                                                   double x, double y, double z)
{
    const double sx = ((double)ci + fa) - x;
    const double sy = ((double)cj + fb) - y;
    const double sz = ((double)ck + fc) - z;
    return (sx * sx + sy * sy) + sz * sz < r2;
}

}  // namespace pmp
