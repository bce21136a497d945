// pmp_launch.h -- host-side launchers of the PMP kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "pmp_device.cuh"

namespace pmp {

void launch_gather(const KParams &P, const Box &S, const double *u, const Parts &p, double *G, DevStatus *st,
                   cudaStream_t stream);
void launch_deposit_atomic(const KParams &P, const Box &S, const double *u, const Box &B, double *b, const Parts &p,
                           const double *G, DevStatus *st, cudaStream_t stream);
void launch_pair_count(const KParams &P, const Box &S, const Box &B, const Parts &p, long long *counts,
                       DevStatus *st, cudaStream_t stream);
void launch_pair_emit(const KParams &P, const Box &S, const Box &B, const Parts &p, const long long *offsets,
                      unsigned *keys, int *vals, DevStatus *st, cudaStream_t stream);
void launch_segment_sum(const KParams &P, const Box &S, const double *u, const Box &B, double *b, const Parts &p,
                        const double *G, const unsigned *keys, const int *vals, const long long *total_dev,
                        long long total, cudaStream_t stream);
void launch_return_sinks(const KParams &P, const Box &S, const double *u, const Box &B, const double *b,
                         const Parts &p, const double *G, DevStatus *st, cudaStream_t stream);
void launch_zero(const Box &B, double *b, cudaStream_t stream);
void launch_fold(const Box &B, double *b, cudaStream_t stream);
void launch_apply(const KParams &P, const Box &S, double *u, const Box &B, const double *b, double *eta_out,
                  DevStatus *st, cudaStream_t stream);

// sorted-mode scan and sort (CUB), in pmp_sort.cu
size_t sort_temp_bytes(long long max_pairs, long long count);
cudaError_t scan_counts(void *temp, size_t temp_bytes, const long long *counts, long long *offsets, long long n,
                        cudaStream_t stream);
cudaError_t sort_pairs(void *temp, size_t temp_bytes, const unsigned *kin, unsigned *kout, const int *vin, int *vout,
                       long long n, int end_bit, cudaStream_t stream);

}  // namespace pmp
