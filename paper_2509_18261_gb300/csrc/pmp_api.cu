// pmp_api.cu -- the C ABI declared in include/pmp.h: argument checks, context
// and status words, and the order in which each call enqueues its kernels.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pmp.h"
#include "pmp_device.cuh"
#include "pmp_launch.h"
#include "pmp_ctx.h"

// The supernova plan and gather as one kernel (1) or as two (0).
#ifndef PMP_FB_PLAN_GATHER_FUSED
#define PMP_FB_PLAN_GATHER_FUSED 1
#endif

namespace {

using pmp::Box;
using pmp::make_box;
using pmp::overlaps;
using pmp::KParams;
using pmp::Parts;

// State/buffer compatibility and the ghost-width rule (Sec. 2.2, Step 1: the
// buffer's ghost zones must contain the kernel).
pmp_status check_pair(const pmp_ctx *ctx, const pmp_mesh *state, const pmp_mesh *buffer, Box *S, Box *B)
{
    pmp_status s = make_box(state, S);
    if (s) return s;
    s = make_box(buffer, B);
    if (s) return s;
    for (int a = 0; a < 3; ++a)
        if (state->n[a] != buffer->n[a] || state->periodic[a] != buffer->periodic[a]) return PMP_ERR_ARG;
    if (state->dx != buffer->dx) return PMP_ERR_ARG;
    if (overlaps(state, buffer)) return PMP_ERR_ARG;
    if (buffer->ng < (int)std::ceil(ctx->p.r_K)) return PMP_ERR_GHOST_TOO_THIN;
    for (int a = 0; a < 3; ++a)
        if (buffer->periodic[a] && buffer->ng > buffer->n[a]) return PMP_ERR_GHOST_TOO_THIN;
    return PMP_OK;
}

pmp_status make_parts(const pmp_ctx *ctx, const pmp_particles *p, Parts *q)
{
    if (!p || p->count < 0 || p->count > 0x7fffffffLL) return PMP_ERR_ARG;
    if (p->count > 0) {
        if (!p->x || !p->y || !p->z || !p->m || !p->px || !p->py || !p->pz) return PMP_ERR_ARG;
        if (ctx->p.kind == PMP_KIND_FEEDBACK && !p->e) return PMP_ERR_ARG;  // MASS: e optional
    }
    q->count = p->count;
    q->x = p->x;
    q->y = p->y;
    q->z = p->z;
    q->m = p->m;
    q->px = p->px;
    q->py = p->py;
    q->pz = p->pz;
    q->e = p->e;
    return PMP_OK;
}

pmp_status last_launch()
{
    return cudaGetLastError() == cudaSuccess ? PMP_OK : PMP_ERR_CUDA;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Upper bound on the kernel cells of one particle: offsets o in [-R, R]^3 whose
// cell centre can come within r_K of some point of the host cell, i.e.
// sum_a max(0, |o_a| - 1/2)^2 <= r_K^2 (with a little slack for rounding).
long long max_pairs_per_particle(double rK)
{
    const int R = (int)std::ceil(rK);
    const double lim = rK * rK * (1.0 + 1e-9);
    long long n = 0;
    for (int a = -R; a <= R; ++a)
        for (int b = -R; b <= R; ++b)
            for (int c = -R; c <= R; ++c) {
                double s = 0.0;
                for (int o : {a, b, c}) {
                    const double m = std::fabs((double)o) - 0.5;
                    if (m > 0.0) s += m * m;
                }
                if (s <= lim) ++n;
            }
    return n;
}

struct Layout {
    size_t keys, ids, keys2, ids2, counts, slots, hosts, fr, wts, aux, pa, mask, offsets, koffsets, kcounts, skeys, skeys2,
        svals, svals2, soffs, slong, scnt, spv;
    size_t temp, temp_bytes, total;
    long long cap, aux_stride;
};

Layout layout(const pmp_params &p, long long n, long long nvalid, int mode)
{
    Layout L;
    std::memset(&L, 0, sizeof(L));
    const int R = (int)std::ceil(p.r_K);
    const int W = 2 * R + 1;
    const bool sink = p.kind == PMP_KIND_SINK;
    const bool sorted = mode == PMP_MODE_SORTED;
    L.cap = max_pairs_per_particle(p.r_K);
    L.aux_stride = nvalid;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align256(off + bytes);
        return at;
    };
    const size_t n1 = (size_t)(n > 0 ? n : 1);
    const size_t pairs = n1 * (size_t)L.cap;
    L.keys = take(4 * n1);
    L.ids = take(4 * n1);
    L.keys2 = take(4 * n1);
    L.ids2 = take(4 * n1);
    L.counts = take(4 * (n1 + 1));
    L.slots = take(8 * pairs);
    L.hosts = take(8 * n1);
    L.fr = take(16 * n1);
    if (sink) {
        L.wts = take(8 * n1 * 3 * (size_t)W);
        // D records, G records, rho c_s, rho - rho_Tr, eta
        L.aux = take(8 * (size_t)(pmp::kDRec + pmp::kGRec + 3) * (size_t)(nvalid > 0 ? nvalid : 1));
        // ATOMIC: each pair's removal a, stored by the fused deposit for Step 4
        if (mode == PMP_MODE_ATOMIC) L.pa = take(8 * pairs);
    } else {
        L.mask = take((size_t)(nvalid > 0 ? nvalid : 1));  // the adjoint's per-cell pass mask
    }
    if (sorted) {
        L.offsets = take(8 * (n1 + 1));
        L.koffsets = take(8 * (n1 + 1));
        L.kcounts = take(4 * (n1 + 1));
        L.skeys = take(4 * pairs);
        L.skeys2 = take(4 * pairs);
        L.svals = take(4 * pairs);
        L.svals2 = take(4 * pairs);
        L.soffs = take(4 * pairs);  // first pair of each run of equal cells
        L.slong = take(4 * pairs);  // runs longer than a warp
        L.scnt = take(16);          // number of runs, number of long runs
        L.spv = take(8 * 5 * pairs);  // every pair's deposition value, index order
    }
    L.temp_bytes = pmp::cub_temp_bytes(n, (long long)pairs, sorted);
    L.temp = take(L.temp_bytes);
    L.total = off;
    return L;
}

long long nvalid_rows(const Layout &L) { return L.aux_stride; }

// A tail with the buffer mesh's layout follows the rest of the workspace:
// ROUNDED mode, the error-bound buffer E of App. A.1 ([5][field_stride]
// doubles); ATOMIC mode for sinks, the one-field scratch of the deposit
// ([field_stride] doubles).
size_t ebuf_offset(const Layout &L) { return align256(L.total); }
size_t ebuf_bytes(const pmp_mesh *buffer) { return sizeof(double) * 5 * (size_t)buffer->field_stride; }
size_t tail_bytes(const pmp_params &p, int mode, const pmp_mesh *buffer)
{
    if (mode == PMP_MODE_ROUNDED) return ebuf_bytes(buffer);
    if (mode == PMP_MODE_ATOMIC && p.kind == PMP_KIND_SINK) return sizeof(double) * (size_t)buffer->field_stride;
    return 0;
}

bool valid_mode(int32_t mode) { return mode == PMP_MODE_ATOMIC || mode == PMP_MODE_SORTED || mode == PMP_MODE_ROUNDED; }

pmp::PlanPtrs plan_ptrs(const Layout &L, void *ws, const pmp_params &p, int mode)
{
    char *w = static_cast<char *>(ws);
    pmp::PlanPtrs pl;
    std::memset(&pl, 0, sizeof(pl));
    (void)mode;
    pl.perm = reinterpret_cast<const unsigned *>(w + L.ids2);
    pl.counts = reinterpret_cast<unsigned *>(w + L.counts);
    pl.slots = reinterpret_cast<unsigned long long *>(w + L.slots);
    pl.hosts = reinterpret_cast<unsigned long long *>(w + L.hosts);
    pl.fr = reinterpret_cast<float4 *>(w + L.fr);
    if (p.kind == PMP_KIND_SINK) {
        pl.wts = reinterpret_cast<double *>(w + L.wts);
        // the two 32-byte records first: at the region's 256-byte-aligned
        // start, every record is one sector
        const size_t nv = (size_t)(nvalid_rows(L) > 0 ? nvalid_rows(L) : 1);
        pl.drec = reinterpret_cast<double *>(w + L.aux);
        pl.grec = pl.drec + (size_t)pmp::kDRec * nv;
        pl.gcs = pl.grec + (size_t)pmp::kGRec * nv;
        pl.dtr = pl.gcs + nv;
        pl.deta = pl.dtr + nv;
        pl.pa = mode == PMP_MODE_ATOMIC ? reinterpret_cast<double *>(w + L.pa) : nullptr;
    }
    pl.cap = (unsigned long long)L.cap;
    return pl;
}

pmp_status check_workspace(const Layout &L, const void *ws, size_t bytes)
{
    if (!ws || bytes < L.total || (reinterpret_cast<uintptr_t>(ws) & 255)) return PMP_ERR_WORKSPACE;
    return PMP_OK;
}

long long nvalid_of(const pmp_mesh *m) { return (long long)m->n[0] * m->n[1] * m->n[2]; }

}  // namespace

namespace pmp {

pmp_status make_box(const pmp_mesh *m, Box *b)
{
    if (!m || !m->data) return PMP_ERR_ARG;
    for (int a = 0; a < 3; ++a) {
        if (m->n[a] < 1) return PMP_ERR_ARG;
        if (m->periodic[a] != 0 && m->periodic[a] != 1) return PMP_ERR_ARG;
    }
    if (m->ng < 0 || !std::isfinite(m->dx) || !(m->dx > 0.0)) return PMP_ERR_ARG;
    const long long px = (long long)m->n[0] + 2LL * m->ng, py = (long long)m->n[1] + 2LL * m->ng,
                    pz = (long long)m->n[2] + 2LL * m->ng;
    const long long nc = px * py * pz;
    if (m->field_stride < nc) return PMP_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(m->data) & 7) != 0) return PMP_ERR_ARG;
    b->n0 = m->n[0];
    b->n1 = m->n[1];
    b->n2 = m->n[2];
    b->g = m->ng;
    b->per0 = m->periodic[0];
    b->per1 = m->periodic[1];
    b->per2 = m->periodic[2];
    b->pad_ = 0;
    b->px = px;
    b->pxy = px * py;
    b->fs = m->field_stride;
    b->ncells = nc;
    return PMP_OK;
}

// True when the byte ranges of two meshes' data intersect: five fields
// field_stride apart, the last one ending after its padded cells.  Both
// meshes have passed make_box.
bool overlaps(const pmp_mesh *a, const pmp_mesh *b)
{
    auto extent = [](const pmp_mesh *m) {
        const size_t cells = (size_t)(m->n[0] + 2 * m->ng) * (size_t)(m->n[1] + 2 * m->ng) * (size_t)(m->n[2] + 2 * m->ng);
        return sizeof(double) * (4 * (size_t)m->field_stride + cells);
    };
    const char *a0 = reinterpret_cast<const char *>(a->data), *b0 = reinterpret_cast<const char *>(b->data);
    return a0 < b0 + extent(b) && b0 < a0 + extent(a);
}

pmp_status check_params(const pmp_params *p)
{
    if (!p) return PMP_ERR_ARG;
    if (p->kind != PMP_KIND_FEEDBACK && p->kind != PMP_KIND_SINK && p->kind != PMP_KIND_MASS) return PMP_ERR_ARG;
    if (!std::isfinite(p->r_K) || p->r_K < 1.0 || p->r_K > (double)pmp::kMaxR) return PMP_ERR_ARG;
    if (p->kind == PMP_KIND_MASS) return p->subsample < 1 || p->subsample > pmp::kMaxS ? PMP_ERR_ARG : PMP_OK;
    if (!std::isfinite(p->gamma) || !(p->gamma > 1.0)) return PMP_ERR_ARG;
    if (p->kind == PMP_KIND_FEEDBACK) {
        if (p->subsample < 1 || p->subsample > pmp::kMaxS) return PMP_ERR_ARG;
        if (!std::isfinite(p->A_sf) || !(p->A_sf > 0.0) || !std::isfinite(p->A_p) || p->A_p < 0.0) return PMP_ERR_ARG;
        if (!std::isfinite(p->mu_H) || !(p->mu_H > 0.0) || !std::isfinite(p->eps_K) || p->eps_K < 0.0) return PMP_ERR_ARG;
        if (!std::isfinite(p->RM_ej) || !std::isfinite(p->RM_st) || p->RM_ej > p->RM_st) return PMP_ERR_ARG;
    } else {
        if (!std::isfinite(p->G) || !(p->G > 0.0) || !std::isfinite(p->dt) || p->dt < 0.0) return PMP_ERR_ARG;
        if (!std::isfinite(p->lambda_bh) || p->lambda_bh < 0.0 || !std::isfinite(p->J) || !(p->J > 0.0)) return PMP_ERR_ARG;
        if (!std::isfinite(p->cap) || !(p->cap > 0.0) || p->cap > 1.0 || !std::isfinite(p->rho_min) || p->rho_min < 0.0)
            return PMP_ERR_ARG;
    }
    return PMP_OK;
}

// Derived constants, each in the order the formulas state it.
KParams make_kparams(const pmp_params &p, double dx)
{
    KParams k;
    std::memset(&k, 0, sizeof(k));
    k.rK = p.r_K;
    k.r2 = p.r_K * p.r_K;
    k.dt = p.dt;
    k.G = p.G;
    k.gg = p.gamma * (p.gamma - 1.0);
    k.lam2 = p.lambda_bh * p.lambda_bh;
    k.ctr = p.kind == PMP_KIND_SINK ? ((p.J * p.J) * pmp::kPi) / (p.G * (dx * dx)) : 0.0;
    k.cap = p.cap;
    k.rho_min = p.rho_min;
    // cap rounded down and rho_min rounded up to FP32 (the sink limiter's FP32 pre-test)
    k.cap_lo = (float)p.cap;
    if ((double)k.cap_lo > p.cap) k.cap_lo = std::nextafter(k.cap_lo, 0.0f);
    k.rho_min_hi = (float)p.rho_min;
    if ((double)k.rho_min_hi < p.rho_min) k.rho_min_hi = std::nextafter(k.rho_min_hi, 3.0e38f);
    k.A_sf = p.A_sf;
    k.A_p = p.A_p;
    k.mu_H = p.mu_H;
    k.RM_ej = p.RM_ej;
    k.RM_st = p.RM_st;
    k.eps_K = p.eps_K;
    k.V = (dx * dx) * dx;
    k.dx = dx;
    k.four_pi = 4.0 * pmp::kPi;
    k.S = p.kind == PMP_KIND_SINK ? 1 : p.subsample;
    k.S3 = k.S * k.S * k.S;
    for (int a = 0; a < 8; ++a) k.frac[a] = a < k.S ? ((double)a + 0.5) / (double)k.S : 0.0;
    k.Slog = -1;
    for (int b = 0; b < 4; ++b)
        if (k.S == (1 << b)) k.Slog = b;
    for (int a = 0; a < 8; ++a) k.fracf[a] = (float)k.frac[a];
    // FP32 band r2 (1 -/+ 2^-14), rounded outward
    const double lo = k.r2 * (1.0 - 6.103515625e-05), hi = k.r2 * (1.0 + 6.103515625e-05);
    k.band_lo = (float)lo;
    if ((double)k.band_lo > lo) k.band_lo = std::nextafter(k.band_lo, 0.0f);
    k.band_hi = (float)hi;
    if ((double)k.band_hi < hi) k.band_hi = std::nextafter(k.band_hi, 3.0e38f);
    k.R = (int)std::ceil(p.r_K);
    k.kind = p.kind;
    return k;
}

}  // namespace pmp

using pmp::check_params;
using pmp::make_kparams;
using pmp_detail::Timed;
using pmp_detail::take_event;

extern "C" {

pmp_status pmp_create(pmp_ctx **out, const pmp_params *params, pmp_stream stream)
{
    if (!out) return PMP_ERR_ARG;
    *out = nullptr;
    pmp_status s = check_params(params);
    if (s) return s;
    pmp_ctx *c = new (std::nothrow) pmp_ctx;
    if (!c) return PMP_ERR_ARG;
    c->p = *params;
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    c->st = nullptr;
    c->plan_ws = nullptr;
    c->plan_n = -1;
    c->plan_nvalid = -1;
    c->plan_mode = PMP_MODE_ATOMIC;
    c->plan_has_a = false;
    c->repro_M = 28;
    c->timing = false;
    if (cudaGetDevice(&c->device) != cudaSuccess || cudaMalloc(&c->st, sizeof(pmp::DevStatus)) != cudaSuccess ||
        cudaMemset(c->st, 0, sizeof(pmp::DevStatus)) != cudaSuccess) {
        if (c->st) cudaFree(c->st);
        delete c;
        return PMP_ERR_CUDA;
    }
    *out = c;
    return PMP_OK;
}

void pmp_destroy(pmp_ctx *ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &m : ctx->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    cudaFree(ctx->st);
    delete ctx;
}

// Sink creation workspace: flags (4 B) and scan positions (8 B) per valid
// cell, then the scan's temporary storage.
struct CreateLayout {
    size_t flags, pos, temp, temp_bytes, total;
};

static CreateLayout create_layout(long long nv)
{
    CreateLayout L;
    const size_t n1 = (size_t)(nv > 0 ? nv : 1);
    size_t off = 0;
    L.flags = off;
    off = align256(off + 4 * n1);
    L.pos = off;
    off = align256(off + 8 * n1);
    L.temp = off;
    L.temp_bytes = pmp::scan_temp_bytes(nv);
    L.total = align256(off + L.temp_bytes);
    return L;
}

pmp_status pmp_create_sinks_workspace_size(const pmp_ctx *ctx, const pmp_mesh *state, size_t *bytes)
{
    if (!ctx || !state || !bytes || ctx->p.kind != PMP_KIND_SINK) return PMP_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (state->n[a] < 1) return PMP_ERR_ARG;
    *bytes = create_layout(nvalid_of(state)).total;
    return PMP_OK;
}

pmp_status pmp_create_sinks(pmp_ctx *ctx, pmp_mesh *state, const pmp_mesh *buffer, int64_t capacity, double *x,
                            double *y, double *z, double *m, double *px, double *py, double *pz, int64_t *count,
                            void *workspace, size_t workspace_bytes)
{
    if (!ctx || ctx->p.kind != PMP_KIND_SINK || !count || capacity < 0) return PMP_ERR_ARG;
    if (capacity > 0 && (!x || !y || !z || !m || !px || !py || !pz)) return PMP_ERR_ARG;
    Box S, B;
    pmp_status s = make_box(state, &S);
    if (s) return s;
    s = make_box(buffer, &B);
    if (s) return s;
    for (int a = 0; a < 3; ++a)
        if (state->n[a] != buffer->n[a] || state->periodic[a] != buffer->periodic[a]) return PMP_ERR_ARG;
    if (state->dx != buffer->dx || overlaps(state, buffer)) return PMP_ERR_ARG;
    const long long nv = nvalid_of(state);
    if (nv > 0xfffffffeLL) return PMP_ERR_ARG;
    const CreateLayout L = create_layout(nv);
    if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return PMP_ERR_WORKSPACE;
    const KParams P = make_kparams(ctx->p, state->dx);
    char *w = static_cast<char *>(workspace);
    unsigned *flags = reinterpret_cast<unsigned *>(w + L.flags);
    unsigned long long *pos = reinterpret_cast<unsigned long long *>(w + L.pos);
    cudaStream_t st = ctx->stream;
    if (cudaMemsetAsync(count, 0, sizeof(int64_t), st) != cudaSuccess) return PMP_ERR_CUDA;
    {
        Timed tm(ctx, "create_flags");
        pmp::launch_create_flags(P, S, state->data, B, buffer->data, flags, st);
    }
    if (pmp::scan_counts(w + L.temp, L.temp_bytes, flags, pos, nv, st) != cudaSuccess) return PMP_ERR_CUDA;
    {
        Timed tm(ctx, "create_apply");
        pmp::launch_create_apply(P, S, state->data, flags, pos, capacity, x, y, z, m, px, py, pz,
                                 reinterpret_cast<long long *>(count), st);
    }
    return last_launch();
}

pmp_status pmp_apply_extra(pmp_ctx *ctx, const pmp_mesh *state, const pmp_mesh *buffer, double *extra, int32_t n_extra,
                           int64_t extra_stride)
{
    if (!ctx || ctx->p.kind != PMP_KIND_SINK || n_extra < 0) return PMP_ERR_ARG;
    Box S, B;
    pmp_status s = make_box(state, &S);
    if (s) return s;
    s = make_box(buffer, &B);
    if (s) return s;
    for (int a = 0; a < 3; ++a)
        if (state->n[a] != buffer->n[a] || state->periodic[a] != buffer->periodic[a]) return PMP_ERR_ARG;
    if (overlaps(state, buffer)) return PMP_ERR_ARG;
    if (n_extra == 0) return PMP_OK;
    if (!extra || extra_stride < S.ncells || (reinterpret_cast<uintptr_t>(extra) & 7)) return PMP_ERR_ARG;
    const KParams P = make_kparams(ctx->p, state->dx);
    {
        Timed tm(ctx, "apply_extra");
        pmp::launch_apply_extra(P, S, state->data, B, buffer->data, extra, n_extra, extra_stride, ctx->stream);
    }
    return last_launch();
}

pmp_status pmp_set_rounding_margin(pmp_ctx *ctx, int32_t M)
{
    if (!ctx || M < 0 || M > 104) return PMP_ERR_ARG;
    ctx->repro_M = M;
    return PMP_OK;
}

pmp_status pmp_timing_enable(pmp_ctx *ctx, int32_t on)
{
    if (!ctx) return PMP_ERR_ARG;
    ctx->timing = on != 0;
    return PMP_OK;
}

pmp_status pmp_timing_read(pmp_ctx *ctx, pmp_kernel_time *out, int32_t max, int32_t *n)
{
    if (!ctx || !n || (max > 0 && !out)) return PMP_ERR_ARG;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return PMP_ERR_CUDA;
    std::vector<pmp_kernel_time> acc;
    for (auto &m : ctx->marks) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, m.a, m.b);
        size_t k = 0;
        while (k < acc.size() && std::string(acc[k].name) != m.name) ++k;
        if (k == acc.size()) {
            pmp_kernel_time z;
            std::memset(&z, 0, sizeof(z));
            std::strncpy(z.name, m.name, sizeof(z.name) - 1);
            acc.push_back(z);
        }
        acc[k].launches += 1;
        acc[k].ms += ms;
        ctx->pool.push_back(m.a);
        ctx->pool.push_back(m.b);
    }
    ctx->marks.clear();
    *n = (int32_t)acc.size();
    for (int32_t k = 0; k < *n && k < max; ++k) out[k] = acc[k];
    return PMP_OK;
}

pmp_status pmp_set_stream(pmp_ctx *ctx, pmp_stream stream)
{
    if (!ctx) return PMP_ERR_ARG;
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    return PMP_OK;
}

int32_t pmp_gathered_rows(int32_t kind)
{
    return kind == PMP_KIND_FEEDBACK ? (int32_t)pmp::FB_ROWS
           : kind == PMP_KIND_SINK   ? (int32_t)pmp::SK_ROWS
           : kind == PMP_KIND_MASS   ? (int32_t)pmp::MS_ROWS
                                     : 0;
}

pmp_status pmp_workspace_size(const pmp_ctx *ctx, const pmp_mesh *buffer, int64_t n_particles, int32_t mode,
                              size_t *bytes)
{
    if (!ctx || !buffer || !bytes || n_particles < 0 || n_particles > 0x7fffffffLL) return PMP_ERR_ARG;
    if (!valid_mode(mode)) return PMP_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (buffer->n[a] < 1) return PMP_ERR_ARG;
    if (buffer->field_stride < 0) return PMP_ERR_ARG;
    const Layout L = layout(ctx->p, n_particles, nvalid_of(buffer), mode);
    const size_t tail = tail_bytes(ctx->p, mode, buffer);
    *bytes = tail ? ebuf_offset(L) + tail : L.total;
    return PMP_OK;
}

pmp_status pmp_zero_buffer(pmp_ctx *ctx, pmp_mesh *buffer)
{
    if (!ctx) return PMP_ERR_ARG;
    Box B;
    pmp_status s = make_box(buffer, &B);
    if (s) return s;
    {
        Timed tm(ctx, "zero");
        pmp::launch_zero(B, buffer->data, ctx->stream);
    }
    return last_launch();
}

// pmp_gather; with `fused` (sinks, ATOMIC, buffer checked by the caller)
// also Step 1 into that buffer, in the same launch as plan and gather.
static pmp_status gather_impl(pmp_ctx *ctx, const pmp_mesh *state, const pmp_particles *particles, double *gathered,
                              int32_t mode, void *workspace, size_t workspace_bytes, pmp_mesh *fused)
{
    if (!ctx || (!gathered && particles && particles->count > 0)) return PMP_ERR_ARG;
    if (!valid_mode(mode)) return PMP_ERR_ARG;
    Box S;
    Parts q;
    pmp_status s = make_box(state, &S);
    if (s) return s;
    s = make_parts(ctx, particles, &q);
    if (s) return s;
    const int R = (int)std::ceil(ctx->p.r_K);
    for (int a = 0; a < 3; ++a) {
        if (state->n[a] + 2 * R > 0xffff) return PMP_ERR_ARG;
        // a kernel cell wraps by at most one period
        if (state->periodic[a] && R > state->n[a]) return PMP_ERR_GHOST_TOO_THIN;
    }
    const long long nv = nvalid_of(state);
    if (nv > 0xfffffffeLL) return PMP_ERR_ARG;
    const Layout L = layout(ctx->p, q.count, nv, mode);
    if (mode == PMP_MODE_SORTED && (unsigned long long)q.count * (unsigned long long)L.cap > 0xffffffffULL)
        return PMP_ERR_ARG;  // slot indices of the sorted lists are 32-bit
    s = check_workspace(L, workspace, workspace_bytes);
    if (s) return s;
    ctx->plan_ws = nullptr;
    ctx->plan_has_a = false;
    const KParams P = make_kparams(ctx->p, state->dx);
    const pmp::PlanPtrs pl = plan_ptrs(L, workspace, ctx->p, mode);
    char *w = static_cast<char *>(workspace);
    void *temp = w + L.temp;
    cudaStream_t st = ctx->stream;
    if (q.count > 0) {
        // processing order: particles sorted by the Morton code of their host
        // cell (every mode; results do not depend on it)
        unsigned *keys = reinterpret_cast<unsigned *>(w + L.keys), *ids = reinterpret_cast<unsigned *>(w + L.ids);
        unsigned *keys2 = reinterpret_cast<unsigned *>(w + L.keys2), *ids2 = reinterpret_cast<unsigned *>(w + L.ids2);
        {
            Timed tm(ctx, "prologue");
            pmp::launch_prologue(S, q, keys, ids, pl, ctx->st, st);
        }
        Timed tm(ctx, "order_sort");
        int nmax = state->n[0] > state->n[1] ? state->n[0] : state->n[1];
        nmax = nmax > state->n[2] ? nmax : state->n[2];
        int bits = 0;
        while ((1 << bits) < nmax) ++bits;
        const int end_bit = 3 * (bits < 10 ? (bits > 0 ? bits : 1) : 10);
        if (pmp::sort_host_keys(temp, L.temp_bytes, keys, keys2, ids, ids2, q.count, end_bit, st) != cudaSuccess)
            return PMP_ERR_CUDA;
    }
    if (ctx->p.kind == PMP_KIND_SINK) {
        Timed tm(ctx, "cell_records");
        pmp::launch_sink_aux(P, S, state->data, pl.grec, pl.gcs, pl.drec, pl.dtr, pl.deta, st);
    }
    if (q.count > 0) {
        if (fused) {
            Box B;
            s = make_box(fused, &B);
            if (s) return s;
            // sinks: -a per pair into the scratch tail, then the cells' factors
            double *scr = reinterpret_cast<double *>(w + ebuf_offset(L));
            if (cudaMemsetAsync(scr, 0, tail_bytes(ctx->p, mode, fused), st) != cudaSuccess) return PMP_ERR_CUDA;
            {
                Timed tm(ctx, "gather_deposit");
                pmp::launch_pass1_sink(P, S, state->data, B, scr, q, pl, gathered, ctx->st, st);
            }
            Timed tm(ctx, "spread");
            pmp::launch_sink_spread(S, B, fused->data, scr, pl.drec, st);
        } else if (ctx->p.kind == PMP_KIND_FEEDBACK && PMP_FB_PLAN_GATHER_FUSED) {
            Timed tm(ctx, "plan_gather");
            pmp::launch_plan_gather_fb(P, S, state->data, q, pl, gathered, ctx->st, st);
        } else {
            {
                Timed tm(ctx, "plan");
                pmp::launch_plan(P, S, q, pl, ctx->st, st);
            }
            Timed tm(ctx, "gather");
            pmp::launch_gather(P, S, state->data, q, pl, gathered, ctx->st, st);
        }
    }
    s = last_launch();
    if (s) return s;
    ctx->plan_ws = workspace;
    ctx->plan_n = q.count;
    ctx->plan_nvalid = nv;
    ctx->plan_mode = mode;
    // the fused sink deposit stored each pair's removal for Step 4
    ctx->plan_has_a = fused && ctx->p.kind == PMP_KIND_SINK && mode == PMP_MODE_ATOMIC && q.count > 0;
    return PMP_OK;
}

pmp_status pmp_gather(pmp_ctx *ctx, const pmp_mesh *state, const pmp_particles *particles, double *gathered,
                      int32_t mode, void *workspace, size_t workspace_bytes)
{
    return gather_impl(ctx, state, particles, gathered, mode, workspace, workspace_bytes, nullptr);
}

pmp_status pmp_gather_deposit(pmp_ctx *ctx, const pmp_mesh *state, const pmp_particles *particles, double *gathered,
                              pmp_mesh *buffer, int32_t mode, void *workspace, size_t workspace_bytes)
{
    if (!ctx || !valid_mode(mode) || (particles && particles->count < 0)) return PMP_ERR_ARG;
    // Sinks in the ATOMIC mode: plan, gather and deposit in one kernel.  The
    // supernova kind runs plan + gather, then the deposit: since the square
    // root and the division of Eq. du moved off the FP64 pipe, a kernel of all
    // three phases is bound by instruction fetch and is slower than the two.
    if (ctx->p.kind == PMP_KIND_SINK && mode == PMP_MODE_ATOMIC) {
        Box S, B;
        pmp_status s = check_pair(ctx, state, buffer, &S, &B);
        if (s) return s;
        if (!particles || particles->count == 0)
            return gather_impl(ctx, state, particles, gathered, mode, workspace, workspace_bytes, nullptr);
        const size_t tail = tail_bytes(ctx->p, mode, buffer);
        if (tail && (!workspace || workspace_bytes < ebuf_offset(layout(ctx->p, particles->count,
                                                                         nvalid_of(state), mode)) + tail))
            return PMP_ERR_WORKSPACE;
        return gather_impl(ctx, state, particles, gathered, mode, workspace, workspace_bytes, buffer);
    }
    pmp_status s = gather_impl(ctx, state, particles, gathered, mode, workspace, workspace_bytes, nullptr);
    if (s || !particles || particles->count == 0) return s;
    return pmp_deposit(ctx, state, particles, gathered, buffer, mode, workspace, workspace_bytes);
}

static pmp_status check_plan(const pmp_ctx *ctx, long long n, long long nvalid, const void *ws)
{
    if (!ws || ctx->plan_ws != ws || ctx->plan_n != n || ctx->plan_nvalid != nvalid) return PMP_ERR_WORKSPACE;
    return PMP_OK;
}

pmp_status pmp_deposit(pmp_ctx *ctx, const pmp_mesh *state, const pmp_particles *particles, const double *gathered,
                       pmp_mesh *buffer, int32_t mode, void *workspace, size_t workspace_bytes)
{
    if (!ctx || (!gathered && particles && particles->count > 0)) return PMP_ERR_ARG;
    if (!valid_mode(mode)) return PMP_ERR_ARG;
    Box S, B;
    Parts q;
    pmp_status s = check_pair(ctx, state, buffer, &S, &B);
    if (s) return s;
    s = make_parts(ctx, particles, &q);
    if (s) return s;
    if (q.count == 0) return PMP_OK;
    const long long nv = nvalid_of(state);
    const Layout L = layout(ctx->p, q.count, nv, mode);
    s = check_workspace(L, workspace, workspace_bytes);
    if (s) return s;
    const size_t tail = tail_bytes(ctx->p, mode, buffer);
    if (tail && workspace_bytes < ebuf_offset(L) + tail) return PMP_ERR_WORKSPACE;
    s = check_plan(ctx, q.count, nv, workspace);
    if (s) return s;
    if (ctx->plan_mode != mode) return PMP_ERR_WORKSPACE;
    const KParams P = make_kparams(ctx->p, state->dx);
    const pmp::PlanPtrs pl = plan_ptrs(L, workspace, ctx->p, mode);
    cudaStream_t st = ctx->stream;
    if (mode == PMP_MODE_ATOMIC && ctx->p.kind == PMP_KIND_SINK) {
        // one atomic per pair into the scratch, then the cells' factors
        double *scr = reinterpret_cast<double *>(static_cast<char *>(workspace) + ebuf_offset(L));
        if (cudaMemsetAsync(scr, 0, tail, st) != cudaSuccess) return PMP_ERR_CUDA;
        {
            Timed tm(ctx, "deposit");
            pmp::launch_deposit_atomic(P, S, state->data, B, buffer->data, q, gathered, pl, nullptr, scr, st);
        }
        {
            Timed tm(ctx, "spread");
            pmp::launch_sink_spread(S, B, buffer->data, scr, pl.drec, st);
        }
        return last_launch();
    }
    if (mode == PMP_MODE_ATOMIC) {
        {
            Timed tm(ctx, "deposit");
            pmp::launch_deposit_atomic(P, S, state->data, B, buffer->data, q, gathered, pl, nullptr, nullptr, st);
        }
        return last_launch();
    }
    if (mode == PMP_MODE_ROUNDED) {
        double *E = reinterpret_cast<double *>(static_cast<char *>(workspace) + ebuf_offset(L));
        if (cudaMemsetAsync(E, 0, ebuf_bytes(buffer), st) != cudaSuccess) return PMP_ERR_CUDA;
        {
            Timed tm(ctx, "deposit");
            pmp::launch_deposit_atomic(P, S, state->data, B, buffer->data, q, gathered, pl, E, nullptr, st);
        }
        {
            Timed tm(ctx, "round");
            pmp::launch_round(B, buffer->data, E, ctx->repro_M, st);
        }
        return last_launch();
    }
    if (B.ncells > 0xffffffffLL) return PMP_ERR_ARG;
    char *w = static_cast<char *>(workspace);
    unsigned long long *offsets = reinterpret_cast<unsigned long long *>(w + L.offsets);
    if (cudaMemsetAsync(pl.counts + q.count, 0, sizeof(unsigned), st) != cudaSuccess) return PMP_ERR_CUDA;
    if (pmp::scan_counts(w + L.temp, L.temp_bytes, pl.counts, offsets, q.count + 1, st) != cudaSuccess)
        return PMP_ERR_CUDA;
    // the same counts in particle-index order, for the pair sort's input lists
    unsigned *kcounts = reinterpret_cast<unsigned *>(w + L.kcounts);
    unsigned long long *koffsets = reinterpret_cast<unsigned long long *>(w + L.koffsets);
    pmp::launch_counts_by_index(pl, q.count, kcounts, st);
    if (pmp::scan_counts(w + L.temp, L.temp_bytes, kcounts, koffsets, q.count + 1, st) != cudaSuccess)
        return PMP_ERR_CUDA;
    unsigned long long total = 0;
    if (cudaMemcpyAsync(&total, offsets + q.count, sizeof(total), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PMP_ERR_CUDA;
    if (total > (unsigned long long)q.count * (unsigned long long)L.cap) return PMP_ERR_WORKSPACE;
    if (total == 0) return PMP_OK;
    unsigned *k1 = reinterpret_cast<unsigned *>(w + L.skeys), *k2 = reinterpret_cast<unsigned *>(w + L.skeys2);
    unsigned *v1 = reinterpret_cast<unsigned *>(w + L.svals), *v2 = reinterpret_cast<unsigned *>(w + L.svals2);
    double *pv = reinterpret_cast<double *>(w + L.spv);
    {
        Timed tm(ctx, "pair_values");
        pmp::launch_pair_values(P, S, state->data, B, q, gathered, pl, offsets, koffsets, pv, k1, v1, st);
    }
    int end_bit = 1;
    while (end_bit < 32 && (1LL << end_bit) < B.ncells) ++end_bit;
    {
        Timed tm(ctx, "sort_pairs");
        if (pmp::sort_pairs(w + L.temp, L.temp_bytes, k1, k2, v1, v2, (long long)total, end_bit, st) != cudaSuccess)
            return PMP_ERR_CUDA;
    }
    // runs of equal cells: unique cells into k1, lengths into v1 (both free
    // after the sort), first pairs into soffs
    unsigned *offs = reinterpret_cast<unsigned *>(w + L.soffs), *longq = reinterpret_cast<unsigned *>(w + L.slong);
    unsigned long long *nruns = reinterpret_cast<unsigned long long *>(w + L.scnt);
    unsigned *nlong = reinterpret_cast<unsigned *>(w + L.scnt + 8);
    {
        Timed tm(ctx, "runs");
        if (pmp::encode_runs(w + L.temp, L.temp_bytes, k2, k1, v1, nruns, (long long)total, st) != cudaSuccess ||
            pmp::scan_lengths(w + L.temp, L.temp_bytes, v1, offs, (long long)total, st) != cudaSuccess)
            return PMP_ERR_CUDA;
    }
    {
        Timed tm(ctx, "segment_sum");
        pmp::launch_segment_sum(B, buffer->data, pv, nruns, k1, v1, offs, v2, longq, nlong, st);
    }
    return last_launch();
}

pmp_status pmp_fold_ghosts(pmp_ctx *ctx, pmp_mesh *buffer)
{
    if (!ctx) return PMP_ERR_ARG;
    Box B;
    pmp_status s = make_box(buffer, &B);
    if (s) return s;
    for (int a = 0; a < 3; ++a)
        if (buffer->periodic[a] && buffer->ng > buffer->n[a]) return PMP_ERR_GHOST_TOO_THIN;
    {
        Timed tm(ctx, "fold");
        pmp::launch_fold(B, buffer->data, ctx->stream);
    }
    return last_launch();
}

pmp_status pmp_apply_limited(pmp_ctx *ctx, pmp_mesh *state, const pmp_mesh *buffer, pmp_particles *particles,
                             const double *gathered, double *eta_out, void *workspace, size_t workspace_bytes)
{
    if (!ctx) return PMP_ERR_ARG;
    Box S, B;
    pmp_status s = make_box(state, &S);
    if (s) return s;
    s = make_box(buffer, &B);
    if (s) return s;
    for (int a = 0; a < 3; ++a)
        if (state->n[a] != buffer->n[a] || state->periodic[a] != buffer->periodic[a]) return PMP_ERR_ARG;
    if (overlaps(state, buffer)) return PMP_ERR_ARG;
    const KParams P = make_kparams(ctx->p, state->dx);
    cudaStream_t st = ctx->stream;
    if (ctx->p.kind == PMP_KIND_SINK) {
        const long long n = particles ? particles->count : 0;
        const long long nv = nvalid_of(state);
        const Layout L = layout(ctx->p, n, nv, ctx->plan_mode);
        s = check_workspace(L, workspace, workspace_bytes);
        if (s) return s;
        s = check_plan(ctx, n, nv, workspace);
        if (s) return s;
        const pmp::PlanPtrs pl = plan_ptrs(L, workspace, ctx->p, ctx->plan_mode);
        Parts q{};
        if (n > 0) {
            if (!gathered) return PMP_ERR_ARG;
            s = make_parts(ctx, particles, &q);
            if (s) return s;
        }
        if (cudaMemsetAsync(&ctx->st->n_limited, 0, 2 * sizeof(unsigned long long), st) != cudaSuccess)
            return PMP_ERR_CUDA;
        {
            // Steps 3 + 5; Step 4 reads only the records and the particles
            Timed tm(ctx, "apply");
            pmp::launch_sink_eta_apply(P, S, state->data, B, buffer->data, pl.dtr, pl.deta, eta_out, ctx->st, st);
        }
        if (n > 0 && ctx->plan_has_a) {
            Timed tm(ctx, "return");
            pmp::launch_return_sinks_stored(P, S, q, pl, ctx->st, st);
        } else if (n > 0) {
            Timed tm(ctx, "return");
            pmp::launch_return_sinks(P, S, q, gathered, pl, ctx->st, st);
        }
        return last_launch();
    }
    if (cudaMemsetAsync(&ctx->st->n_limited, 0, 2 * sizeof(unsigned long long), st) != cudaSuccess)
        return PMP_ERR_CUDA;
    {
        Timed tm(ctx, "apply");
        pmp::launch_apply(P, S, state->data, B, buffer->data, eta_out, ctx->st, st);
    }
    return last_launch();
}

pmp_status pmp_backward(pmp_ctx *ctx, const pmp_mesh *state_in, const pmp_mesh *buffer, const pmp_particles *particles,
                        const double *gathered, const double *gU, double *g_out, void *workspace,
                        size_t workspace_bytes)
{
    if (!ctx || ctx->p.kind != PMP_KIND_FEEDBACK) return PMP_ERR_ARG;
    Box S, B;
    Parts q;
    pmp_status s = make_box(state_in, &S);
    if (s) return s;
    s = make_box(buffer, &B);
    if (s) return s;
    for (int a = 0; a < 3; ++a)
        if (state_in->n[a] != buffer->n[a] || state_in->periodic[a] != buffer->periodic[a]) return PMP_ERR_ARG;
    s = make_parts(ctx, particles, &q);
    if (s) return s;
    if (q.count > 0 && (!gathered || !gU || !g_out)) return PMP_ERR_ARG;
    const long long nv = nvalid_of(state_in);
    const Layout L = layout(ctx->p, q.count, nv, ctx->plan_mode);
    s = check_workspace(L, workspace, workspace_bytes);
    if (s) return s;
    s = check_plan(ctx, q.count, nv, workspace);
    if (s) return s;
    if (q.count == 0) return PMP_OK;
    const KParams P = make_kparams(ctx->p, state_in->dx);
    const pmp::PlanPtrs pl = plan_ptrs(L, workspace, ctx->p, ctx->plan_mode);
    unsigned char *pass = reinterpret_cast<unsigned char *>(static_cast<char *>(workspace) + L.mask);
    {
        Timed tm(ctx, "backward_mask");
        pmp::launch_pass_mask(S, state_in->data, B, buffer->data, pass, ctx->stream);
    }
    {
        Timed tm(ctx, "backward");
        pmp::launch_backward_fb(P, S, state_in->data, gU, q, pl, pass, gathered, g_out, ctx->stream);
    }
    return last_launch();
}

pmp_status pmp_get_error(pmp_ctx *ctx, int32_t *code, int64_t *index)
{
    if (!ctx || !code || !index) return PMP_ERR_ARG;
    pmp::DevStatus h;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess ||
        cudaMemcpy(&h, ctx->st, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
        return PMP_ERR_CUDA;
    *code = h.code;
    *index = h.code ? h.index : -1;
    if (cudaMemset(ctx->st, 0, 2 * sizeof(int) + sizeof(long long)) != cudaSuccess) return PMP_ERR_CUDA;
    return PMP_OK;
}

pmp_status pmp_limiter_counts(pmp_ctx *ctx, int64_t *counts)
{
    if (!ctx || !counts) return PMP_ERR_ARG;
    pmp::DevStatus h;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess ||
        cudaMemcpy(&h, ctx->st, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
        return PMP_ERR_CUDA;
    counts[0] = (int64_t)h.n_limited;
    counts[1] = (int64_t)h.n_noroot;
    return PMP_OK;
}

}  // extern "C"
