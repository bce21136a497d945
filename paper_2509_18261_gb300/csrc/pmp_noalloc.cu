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

#include "pmp.h"
#include "pmp_device.cuh"
#include "pmp_launch.h"
#include "pmp_ctx.h"

namespace {

// The scratch: every GPU that loads the library holds this array until the
// process exits.
constexpr size_t kScratchBytes = (size_t)PMP_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

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
    // ---- host-side checks (nothing is enqueued on failure); the same rules
    // as the context entry points: parameters, both meshes, their pairing
    if (!params || !state || !particles || !buffer) return PMP_ERR_ARG;
    if (pmp::check_params(params) != PMP_OK || params->kind != PMP_KIND_FEEDBACK) return PMP_ERR_ARG;
    const pmp_params &p = *params;
    const long long n = particles->count;
    if (n < 0 || n > 0x7fffffffLL) return PMP_ERR_ARG;
    if (n > 0 && (!particles->x || !particles->y || !particles->z || !particles->m || !particles->px ||
                  !particles->py || !particles->pz || !particles->e || !gathered))
        return PMP_ERR_ARG;
    pmp::Box S, B;
    pmp_status s = pmp::make_box(state, &S);
    if (s) return s;
    s = pmp::make_box(buffer, &B);
    if (s) return s;
    if (state->dx != buffer->dx) return PMP_ERR_ARG;
    // the deposit reads the state while it adds into the buffer: no aliasing
    if (pmp::overlaps(state, buffer)) return PMP_ERR_ARG;
    const int R = (int)std::ceil(p.r_K);
    for (int a = 0; a < 3; ++a) {
        if (state->n[a] != buffer->n[a] || state->periodic[a] != buffer->periodic[a]) return PMP_ERR_ARG;
        if (state->n[a] + 2 * R > 0xffff) return PMP_ERR_ARG;
    }
    if (buffer->ng < R) return PMP_ERR_GHOST_TOO_THIN;
    for (int a = 0; a < 3; ++a) {
        if (buffer->periodic[a] && buffer->ng > buffer->n[a]) return PMP_ERR_GHOST_TOO_THIN;
        if (state->periodic[a] && R > state->n[a]) return PMP_ERR_GHOST_TOO_THIN;
    }
    // scratch layout: status | counts | slots | hosts | fractional positions
    const long long cap = cells_bound(p.r_K);
    const size_t n1 = (size_t)(n > 0 ? n : 1);
    const size_t o_counts = 256;
    const size_t o_slots = a256(o_counts + 4 * (n1 + 1));
    const size_t o_hosts = a256(o_slots + 8 * n1 * (size_t)cap);
    const size_t o_fr = a256(o_hosts + 8 * n1);
    const size_t need = a256(o_fr + 16 * n1);
    if (need > kScratchBytes) return PMP_ERR_WORKSPACE;  // too many particles for the fixed scratch

    // ---- the scratch's device address on the current device.  Looked up on
    // every call (it allocates nothing and costs little), so a call made
    // after a device reset or on another device never uses a stale address.
    void *base = nullptr;
    if (cudaGetSymbolAddress(&base, g_noalloc_scratch) != cudaSuccess || !base) return PMP_ERR_CUDA;
    if (n == 0) return PMP_OK;

    // ---- the same kernels as pmp_gather + pmp_deposit (index order)
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(base);
    pmp::DevStatus *status = reinterpret_cast<pmp::DevStatus *>(w);
    if (cudaMemsetAsync(status, 0, sizeof(pmp::DevStatus), st) != cudaSuccess) return PMP_ERR_CUDA;
    const pmp::KParams k = pmp::make_kparams(p, state->dx);
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
