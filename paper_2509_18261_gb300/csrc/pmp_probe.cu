// pmp_probe.cu -- measurement kernels for the roofline of the particle
// kernels (no paper counterpart): the FP64 fused multiply-add rate and the
// FP64 atomicAdd rate of the GPU the library runs on, so that achieved rates
// are set against peaks measured on the same part rather than nominal ones.
#include <cstdint>

#include "pmp.h"
#include "pmp_exact.cuh"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;  // independent FMA chains per thread (latency hidden)

// Every thread runs kChains independent chains of `iters` DFMA each; the
// chains' values stay bounded (a contraction towards a fixed point), and one
// sum per thread is stored so that no chain is dead code.
__global__ void __launch_bounds__(kProbeThreads) k_probe_fp64(double *__restrict__ out, int iters, double a, double b)
{
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = 1.0 + 1e-3 * (double)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Grid-stride: addition t goes to target (t * 2654435761) mod n_targets (a
// scattered, mostly uncontended pattern for large n_targets; every thread
// adds 1.0).
__global__ void __launch_bounds__(kProbeThreads) k_probe_atomic(double *__restrict__ target, long long n_targets,
                                                               long long n_adds)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n_adds; t += stride) {
        const unsigned long long h = (unsigned long long)t * 2654435761ULL;
        atomicAdd(target + (long long)(h % (unsigned long long)n_targets), 1.0);
    }
}

// Element-wise quotient and square root by the library's integer / FP32
// forms (pmp_exact.cuh), the ones the particle and cell kernels use.
__global__ void __launch_bounds__(kProbeThreads) k_exact_math(const double *__restrict__ a,
                                                             const double *__restrict__ b, long long n,
                                                             double *__restrict__ quot, double *__restrict__ root)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double x = a[i];
        quot[i] = pmp::exact::div_rn(x, b[i]);
        root[i] = pmp::exact::sqrt_rn(x);
    }
}

}  // namespace

extern "C" {

int32_t pmp_probe_threads(void) { return kProbeThreads; }

int32_t pmp_probe_chains(void) { return kChains; }

pmp_status pmp_probe_fp64(double *out, int32_t blocks, int32_t iters, pmp_stream stream)
{
    if (!out || blocks < 1 || iters < 1) return PMP_ERR_ARG;
    k_probe_fp64<<<blocks, kProbeThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(out, iters, 0.999999,
                                                                                     1e-6);
    return cudaGetLastError() == cudaSuccess ? PMP_OK : PMP_ERR_CUDA;
}

pmp_status pmp_probe_atomic(double *target, int64_t n_targets, int64_t n_adds, int32_t blocks, pmp_stream stream)
{
    if (!target || n_targets < 1 || n_adds < 0 || blocks < 1) return PMP_ERR_ARG;
    k_probe_atomic<<<blocks, kProbeThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(target, n_targets,
                                                                                       n_adds);
    return cudaGetLastError() == cudaSuccess ? PMP_OK : PMP_ERR_CUDA;
}

pmp_status pmp_exact_math(const double *a, const double *b, int64_t n, double *quot, double *root,
                          pmp_stream stream)
{
    if (n < 0 || (n > 0 && (!a || !b || !quot || !root))) return PMP_ERR_ARG;
    if (n == 0) return PMP_OK;
    const long long blocks = (n + kProbeThreads - 1) / kProbeThreads;
    k_exact_math<<<(unsigned)(blocks < 152LL * 16 ? blocks : 152LL * 16), kProbeThreads, 0,
                   reinterpret_cast<cudaStream_t>(stream)>>>(a, b, n, quot, root);
    return cudaGetLastError() == cudaSuccess ? PMP_OK : PMP_ERR_CUDA;
}

}  // extern "C"
