// pmp_noalloc.cu -- Step 1 for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator-free runtime, plugins that are handed
// only pre-allocated buffers, or hosts whose process must not grow its device
// footprint after start-up.  pmp_deposit_noalloc serves them: it performs the
// supernova gather and the atomic deposit like pmp_gather + pmp_deposit, but
// takes its plan scratch from a fixed array compiled into the library instead
// of a caller-provided workspace, and it creates no context.
#include <cmath>
#include <cstring>
#include <mutex>

#include "pmp.h"
#include "pmp_device.cuh"
#include "pmp_launch.h"

namespace {

// The scratch: every GPU that loads the library holds this array until the
// process exits.
constexpr size_t kScratchBytes = (size_t)PMP_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

long long cells_bound(double rK)
{
    const int R = (int)std::ceil(rK);
    const double lim = rK * rK * (1.0 + 1e-9);
    long long n = 0;
    for (int a = -R; a <= R; ++a)
        for (int b = -R; b <= R; ++b)
            for (int c = -R; c <= R; ++c) {
                double s = 0.0;
                const int o[3] = {a, b, c};
                for (int k = 0; k < 3; ++k) {
                    const double m = std::fabs((double)o[k]) - 0.5;
                    if (m > 0.0) s += m * m;
                }
                if (s <= lim) ++n;
            }
    return n;
}

}  // namespace

extern "C" pmp_status pmp_deposit_noalloc(const pmp_params *params, const pmp_mesh *state,
                                          const pmp_particles *particles, double *gathered, pmp_mesh *buffer,
                                          pmp_stream stream)
{
    // ---- host-side checks (nothing is enqueued on failure)
    if (!params || !state || !particles || !buffer) return PMP_ERR_ARG;
    const pmp_params &p = *params;
    if (p.kind != PMP_KIND_FEEDBACK) return PMP_ERR_ARG;
    if (!std::isfinite(p.r_K) || p.r_K < 1.0 || p.r_K > (double)pmp::kMaxR) return PMP_ERR_ARG;
    if (p.subsample < 1 || p.subsample > pmp::kMaxS || !(p.gamma > 1.0) || !(p.A_sf > 0.0) || !(p.mu_H > 0.0) ||
        p.A_p < 0.0 || p.eps_K < 0.0 || p.RM_ej > p.RM_st)
        return PMP_ERR_ARG;
    const long long n = particles->count;
    if (n < 0 || n > 0x7fffffffLL) return PMP_ERR_ARG;
    if (n > 0 && (!particles->x || !particles->y || !particles->z || !particles->m || !particles->px ||
                  !particles->py || !particles->pz || !particles->e || !gathered))
        return PMP_ERR_ARG;
    if (!state->data || !buffer->data || state->dx != buffer->dx || !(state->dx > 0.0)) return PMP_ERR_ARG;
    const int R = (int)std::ceil(p.r_K);
    for (int a = 0; a < 3; ++a) {
        if (state->n[a] < 1 || state->n[a] != buffer->n[a] || state->periodic[a] != buffer->periodic[a])
            return PMP_ERR_ARG;
        if (state->n[a] + 2 * R > 0xffff) return PMP_ERR_ARG;
        if (buffer->periodic[a] && buffer->ng > buffer->n[a]) return PMP_ERR_GHOST_TOO_THIN;
    }
    if (state->ng < 0 || buffer->ng < R) return buffer->ng < R ? PMP_ERR_GHOST_TOO_THIN : PMP_ERR_ARG;
    auto ncells = [](const pmp_mesh *m) {
        return ((long long)m->n[0] + 2LL * m->ng) * ((long long)m->n[1] + 2LL * m->ng) *
               ((long long)m->n[2] + 2LL * m->ng);
    };
    if (state->field_stride < ncells(state) || buffer->field_stride < ncells(buffer)) return PMP_ERR_ARG;
    // scratch layout: status | counts | slots | hosts | fractional positions
    const long long cap = cells_bound(p.r_K);
    const size_t n1 = (size_t)(n > 0 ? n : 1);
    const size_t o_counts = 256;
    const size_t o_slots = a256(o_counts + 4 * (n1 + 1));
    const size_t o_hosts = a256(o_slots + 8 * n1 * (size_t)cap);
    const size_t o_fr = a256(o_hosts + 8 * n1);
    const size_t need = a256(o_fr + 16 * n1);
    if (need > kScratchBytes) return PMP_ERR_WORKSPACE;  // too many particles for the fixed scratch

    // ---- set-up, once per device: the device address of the scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PMP_ERR_CUDA;
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return PMP_ERR_CUDA;
            g_scratch_addr[dev] = ptr;
        }
        base = g_scratch_addr[dev];
    }
    if (n == 0) return PMP_OK;

    // ---- the same kernels as pmp_gather + pmp_deposit (index order)
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(base);
    pmp::DevStatus *status = reinterpret_cast<pmp::DevStatus *>(w);
    if (cudaMemsetAsync(status, 0, sizeof(pmp::DevStatus), st) != cudaSuccess) return PMP_ERR_CUDA;
    pmp::Box S, B;
    auto box = [](const pmp_mesh *m, pmp::Box *b) {
        b->n0 = m->n[0];
        b->n1 = m->n[1];
        b->n2 = m->n[2];
        b->g = m->ng;
        b->per0 = m->periodic[0];
        b->per1 = m->periodic[1];
        b->per2 = m->periodic[2];
        b->pad_ = 0;
        b->px = (long long)m->n[0] + 2LL * m->ng;
        b->pxy = b->px * ((long long)m->n[1] + 2LL * m->ng);
        b->fs = m->field_stride;
        b->ncells = b->pxy * ((long long)m->n[2] + 2LL * m->ng);
    };
    box(state, &S);
    box(buffer, &B);
    pmp::KParams k;
    std::memset(&k, 0, sizeof(k));
    const double dx = state->dx;
    k.rK = p.r_K;
    k.r2 = p.r_K * p.r_K;
    k.gg = p.gamma * (p.gamma - 1.0);
    k.A_sf = p.A_sf;
    k.A_p = p.A_p;
    k.mu_H = p.mu_H;
    k.RM_ej = p.RM_ej;
    k.RM_st = p.RM_st;
    k.eps_K = p.eps_K;
    k.V = (dx * dx) * dx;
    k.dx = dx;
    k.four_pi = 4.0 * pmp::kPi;
    k.S = p.subsample;
    k.S3 = k.S * k.S * k.S;
    k.R = R;
    k.kind = PMP_KIND_FEEDBACK;
    k.Slog = -1;
    for (int b = 0; b < 4; ++b)
        if (k.S == (1 << b)) k.Slog = b;
    for (int a = 0; a < 8; ++a) {
        k.frac[a] = a < k.S ? ((double)a + 0.5) / (double)k.S : 0.0;
        k.fracf[a] = (float)k.frac[a];
    }
    const double lo = k.r2 * (1.0 - 6.103515625e-05), hi = k.r2 * (1.0 + 6.103515625e-05);
    k.band_lo = (float)lo;
    if ((double)k.band_lo > lo) k.band_lo = std::nextafter(k.band_lo, 0.0f);
    k.band_hi = (float)hi;
    if ((double)k.band_hi < hi) k.band_hi = std::nextafter(k.band_hi, 3.0e38f);
    pmp::Parts q;
    q.count = n;
    q.x = particles->x;
    q.y = particles->y;
    q.z = particles->z;
    q.m = particles->m;
    q.px = particles->px;
    q.py = particles->py;
    q.pz = particles->pz;
    q.e = particles->e;
    pmp::PlanPtrs pl;
    std::memset(&pl, 0, sizeof(pl));
    pl.perm = nullptr;
    pl.counts = reinterpret_cast<unsigned *>(w + o_counts);
    pl.slots = reinterpret_cast<unsigned long long *>(w + o_slots);
    pl.hosts = reinterpret_cast<unsigned long long *>(w + o_hosts);
    pl.fr = reinterpret_cast<float4 *>(w + o_fr);
    pl.cap = (unsigned long long)cap;
    pmp::launch_prologue(S, q, nullptr, nullptr, pl, status, st);
    pmp::launch_plan_gather_fb(k, S, state->data, q, pl, gathered, status, st);
    pmp::launch_deposit_atomic(k, S, state->data, B, buffer->data, q, gathered, pl, nullptr, nullptr, st);
    return cudaGetLastError() == cudaSuccess ? PMP_OK : PMP_ERR_CUDA;
}
