// pmp_ctx.h -- the context object behind pmp_ctx* and helpers shared by the
// translation units that implement the C ABI (internal).
#pragma once

#include <vector>

#include <cuda_runtime.h>

#include "pmp.h"
#include "pmp_device.cuh"

struct pmp_ctx {
    pmp_params p;
    cudaStream_t stream;
    pmp::DevStatus *st;  // device
    int device;
    // the plan recorded by the last pmp_gather
    const void *plan_ws;
    long long plan_n;
    long long plan_nvalid;
    int plan_mode;
    bool plan_has_a;  // the plan's workspace holds each sink pair's removal (fused ATOMIC deposit)
    int repro_M;  // App. A.1 safety margin M of the ROUNDED mode
    // per-kernel CUDA-event timing (pmp_timing_enable)
    bool timing;
    struct Mark {
        const char *name;
        cudaEvent_t a, b;
    };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
};

namespace pmp_detail {

inline cudaEvent_t take_event(pmp_ctx *c)
{
    cudaEvent_t e;
    if (!c->pool.empty()) {
        e = c->pool.back();
        c->pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
    }
    return e;
}

// Brackets the kernel launched in its scope with two events on the context's
// stream when timing is on.
struct Timed {
    pmp_ctx *c;
    size_t idx;
    Timed(pmp_ctx *ctx, const char *name) : c(ctx), idx((size_t)-1)
    {
        if (!c->timing) return;
        pmp_ctx::Mark m{name, take_event(c), take_event(c)};
        if (!m.a || !m.b) return;
        cudaEventRecord(m.a, c->stream);
        c->marks.push_back(m);
        idx = c->marks.size() - 1;
    }
    ~Timed()
    {
        if (idx != (size_t)-1) cudaEventRecord(c->marks[idx].b, c->stream);
    }
};

}  // namespace pmp_detail


namespace pmp {

// Geometry of a mesh for the kernels, after checking it: n >= 1, periodic
// flags 0 or 1, ng >= 0, dx finite and positive, field_stride at least the
// padded cell count, data non-NULL and 8-byte aligned (else PMP_ERR_ARG).
pmp_status make_box(const pmp_mesh *m, Box *b);
// True when the five-field extents of two meshes share a byte.
bool overlaps(const pmp_mesh *a, const pmp_mesh *b);
// Validates a parameter set (PMP_OK or PMP_ERR_ARG).
pmp_status check_params(const pmp_params *p);
// Derived constants of a parameter set for cell size dx.
KParams make_kparams(const pmp_params &p, double dx);

}  // namespace pmp
