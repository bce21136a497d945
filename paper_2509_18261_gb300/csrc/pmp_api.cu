// pmp_api.cu -- the C ABI declared in include/pmp.h: argument checks, context
// and status words, and the order in which each call enqueues its kernels.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>

#include "pmp.h"
#include "pmp_device.cuh"
#include "pmp_launch.h"

struct pmp_ctx {
    pmp_params p;
    cudaStream_t stream;
    pmp::DevStatus *st;  // device
    int device;
};

namespace {

using pmp::Box;
using pmp::KParams;
using pmp::Parts;

bool finite(double v) { return std::isfinite(v); }

pmp_status check_params(const pmp_params *p)
{
    if (!p) return PMP_ERR_ARG;
    if (p->kind != PMP_KIND_FEEDBACK && p->kind != PMP_KIND_SINK) return PMP_ERR_ARG;
    if (!finite(p->r_K) || p->r_K < 1.0 || p->r_K > (double)pmp::kMaxR) return PMP_ERR_ARG;
    if (!finite(p->gamma) || !(p->gamma > 1.0)) return PMP_ERR_ARG;
    if (p->kind == PMP_KIND_FEEDBACK) {
        if (p->subsample < 1 || p->subsample > pmp::kMaxS) return PMP_ERR_ARG;
        if (!finite(p->A_sf) || !(p->A_sf > 0.0) || !finite(p->A_p) || p->A_p < 0.0) return PMP_ERR_ARG;
        if (!finite(p->mu_H) || !(p->mu_H > 0.0) || !finite(p->eps_K) || p->eps_K < 0.0) return PMP_ERR_ARG;
        if (!finite(p->RM_ej) || !finite(p->RM_st) || p->RM_ej > p->RM_st) return PMP_ERR_ARG;
    } else {
        if (!finite(p->G) || !(p->G > 0.0) || !finite(p->dt) || p->dt < 0.0) return PMP_ERR_ARG;
        if (!finite(p->lambda_bh) || p->lambda_bh < 0.0 || !finite(p->J) || !(p->J > 0.0)) return PMP_ERR_ARG;
        if (!finite(p->cap) || !(p->cap > 0.0) || p->cap > 1.0 || !finite(p->rho_min) || p->rho_min < 0.0)
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
    k.A_sf = p.A_sf;
    k.A_p = p.A_p;
    k.mu_H = p.mu_H;
    k.RM_ej = p.RM_ej;
    k.RM_st = p.RM_st;
    k.eps_K = p.eps_K;
    k.V = (dx * dx) * dx;
    k.dx = dx;
    k.four_pi = 4.0 * pmp::kPi;
    k.S = p.kind == PMP_KIND_FEEDBACK ? p.subsample : 1;
    k.S3 = k.S * k.S * k.S;
    k.R = (int)std::ceil(p.r_K);
    k.kind = p.kind;
    return k;
}

pmp_status make_box(const pmp_mesh *m, Box *b)
{
    if (!m || !m->data) return PMP_ERR_ARG;
    for (int a = 0; a < 3; ++a) {
        if (m->n[a] < 1) return PMP_ERR_ARG;
        if (m->periodic[a] != 0 && m->periodic[a] != 1) return PMP_ERR_ARG;
    }
    if (m->ng < 0 || !finite(m->dx) || !(m->dx > 0.0)) return PMP_ERR_ARG;
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

bool overlaps(const pmp_mesh *a, const pmp_mesh *b)
{
    const char *a0 = reinterpret_cast<const char *>(a->data), *b0 = reinterpret_cast<const char *>(b->data);
    const char *a1 = a0 + sizeof(double) * (size_t)(4 * a->field_stride + 1);
    const char *b1 = b0 + sizeof(double) * (size_t)(4 * b->field_stride + 1);
    return a0 < b1 && b0 < a1;
}

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
        if (ctx->p.kind == PMP_KIND_FEEDBACK && !p->e) return PMP_ERR_ARG;
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

struct SortedLayout {
    size_t counts, offsets, kin, kout, vin, vout, temp, temp_bytes, total;
    long long cap;
};

SortedLayout sorted_layout(int R, long long n)
{
    SortedLayout L;
    const long long W = 2LL * R + 1;
    L.cap = n * W * W * W;
    size_t off = 0;
    L.counts = off;
    off = align256(off + sizeof(long long) * (size_t)(n + 1));
    L.offsets = off;
    off = align256(off + sizeof(long long) * (size_t)(n + 1));
    L.kin = off;
    off = align256(off + sizeof(unsigned) * (size_t)L.cap);
    L.kout = off;
    off = align256(off + sizeof(unsigned) * (size_t)L.cap);
    L.vin = off;
    off = align256(off + sizeof(int) * (size_t)L.cap);
    L.vout = off;
    off = align256(off + sizeof(int) * (size_t)L.cap);
    L.temp = off;
    L.temp_bytes = pmp::sort_temp_bytes(L.cap > 0 ? L.cap : 1, n);
    off = align256(off + L.temp_bytes);
    L.total = off;
    return L;
}

}  // namespace

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
    cudaFree(ctx->st);
    delete ctx;
}

pmp_status pmp_set_stream(pmp_ctx *ctx, pmp_stream stream)
{
    if (!ctx) return PMP_ERR_ARG;
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    return PMP_OK;
}

int32_t pmp_gathered_rows(int32_t kind)
{
    return kind == PMP_KIND_FEEDBACK ? (int32_t)pmp::FB_ROWS : kind == PMP_KIND_SINK ? (int32_t)pmp::SK_ROWS : 0;
}

pmp_status pmp_workspace_size(const pmp_ctx *ctx, const pmp_mesh *buffer, int64_t n_particles, int32_t mode,
                              size_t *bytes)
{
    if (!ctx || !buffer || !bytes || n_particles < 0) return PMP_ERR_ARG;
    if (mode == PMP_MODE_ATOMIC) {
        *bytes = 0;
        return PMP_OK;
    }
    if (mode != PMP_MODE_SORTED) return PMP_ERR_ARG;
    *bytes = sorted_layout((int)std::ceil(ctx->p.r_K), n_particles).total;
    return PMP_OK;
}

pmp_status pmp_zero_buffer(pmp_ctx *ctx, pmp_mesh *buffer)
{
    if (!ctx) return PMP_ERR_ARG;
    Box B;
    pmp_status s = make_box(buffer, &B);
    if (s) return s;
    pmp::launch_zero(B, buffer->data, ctx->stream);
    return last_launch();
}

pmp_status pmp_gather(pmp_ctx *ctx, const pmp_mesh *state, const pmp_particles *particles, double *gathered)
{
    if (!ctx || (!gathered && particles && particles->count > 0)) return PMP_ERR_ARG;
    Box S;
    Parts q;
    pmp_status s = make_box(state, &S);
    if (s) return s;
    s = make_parts(ctx, particles, &q);
    if (s) return s;
    const KParams P = make_kparams(ctx->p, state->dx);
    pmp::launch_gather(P, S, state->data, q, gathered, ctx->st, ctx->stream);
    return last_launch();
}

pmp_status pmp_deposit(pmp_ctx *ctx, const pmp_mesh *state, const pmp_particles *particles, const double *gathered,
                       pmp_mesh *buffer, int32_t mode, void *workspace, size_t workspace_bytes)
{
    if (!ctx || (!gathered && particles && particles->count > 0)) return PMP_ERR_ARG;
    Box S, B;
    Parts q;
    pmp_status s = check_pair(ctx, state, buffer, &S, &B);
    if (s) return s;
    s = make_parts(ctx, particles, &q);
    if (s) return s;
    const KParams P = make_kparams(ctx->p, state->dx);
    if (mode == PMP_MODE_ATOMIC) {
        pmp::launch_deposit_atomic(P, S, state->data, B, buffer->data, q, gathered, ctx->st, ctx->stream);
        return last_launch();
    }
    if (mode != PMP_MODE_SORTED) return PMP_ERR_ARG;
    if (B.ncells > 0xffffffffLL) return PMP_ERR_ARG;
    const SortedLayout L = sorted_layout(P.R, q.count);
    if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return PMP_ERR_WORKSPACE;
    if (q.count == 0) return PMP_OK;
    char *w = static_cast<char *>(workspace);
    long long *counts = reinterpret_cast<long long *>(w + L.counts);
    long long *offsets = reinterpret_cast<long long *>(w + L.offsets);
    unsigned *kin = reinterpret_cast<unsigned *>(w + L.kin), *kout = reinterpret_cast<unsigned *>(w + L.kout);
    int *vin = reinterpret_cast<int *>(w + L.vin), *vout = reinterpret_cast<int *>(w + L.vout);
    void *temp = w + L.temp;
    if (cudaMemsetAsync(counts + q.count, 0, sizeof(long long), ctx->stream) != cudaSuccess) return PMP_ERR_CUDA;
    pmp::launch_pair_count(P, S, B, q, counts, ctx->st, ctx->stream);
    if (last_launch()) return PMP_ERR_CUDA;
    if (pmp::scan_counts(temp, L.temp_bytes, counts, offsets, q.count + 1, ctx->stream) != cudaSuccess)
        return PMP_ERR_CUDA;
    long long total = 0;
    if (cudaMemcpyAsync(&total, offsets + q.count, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return PMP_ERR_CUDA;
    if (total < 0 || total > L.cap) return PMP_ERR_WORKSPACE;
    if (total == 0) return PMP_OK;
    pmp::launch_pair_emit(P, S, B, q, offsets, kin, vin, ctx->st, ctx->stream);
    if (last_launch()) return PMP_ERR_CUDA;
    int end_bit = 1;
    while (end_bit < 32 && (1LL << end_bit) < B.ncells) ++end_bit;
    if (pmp::sort_pairs(temp, L.temp_bytes, kin, kout, vin, vout, total, end_bit, ctx->stream) != cudaSuccess)
        return PMP_ERR_CUDA;
    pmp::launch_segment_sum(P, S, state->data, B, buffer->data, q, gathered, kout, vout, offsets + q.count, total,
                            ctx->stream);
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
    pmp::launch_fold(B, buffer->data, ctx->stream);
    return last_launch();
}

pmp_status pmp_apply_limited(pmp_ctx *ctx, pmp_mesh *state, const pmp_mesh *buffer, pmp_particles *particles,
                             const double *gathered, double *eta_out)
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
    if (ctx->p.kind == PMP_KIND_SINK && particles && particles->count > 0) {
        if (!gathered) return PMP_ERR_ARG;
        Parts q;
        s = make_parts(ctx, particles, &q);
        if (s) return s;
        pmp::launch_return_sinks(P, S, state->data, B, buffer->data, q, gathered, ctx->st, ctx->stream);
        if (last_launch()) return PMP_ERR_CUDA;
    }
    if (cudaMemsetAsync(&ctx->st->n_limited, 0, 2 * sizeof(unsigned long long), ctx->stream) != cudaSuccess)
        return PMP_ERR_CUDA;
    pmp::launch_apply(P, S, state->data, B, buffer->data, eta_out, ctx->st, ctx->stream);
    return last_launch();
}

pmp_status pmp_backward(pmp_ctx *ctx, const pmp_mesh *state_in, const pmp_mesh *buffer, const pmp_particles *particles,
                        const double *gathered, const double *gU, double *g_out)
{
    (void)state_in;
    (void)buffer;
    (void)particles;
    (void)gathered;
    (void)gU;
    (void)g_out;
    if (!ctx) return PMP_ERR_ARG;
    return PMP_ERR_ARG;
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
