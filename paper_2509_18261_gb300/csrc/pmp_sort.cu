// pmp_sort.cu -- prefix sum of pair counts and the stable radix sort of
// (cell, particle) pairs for the sorted deposit (CUB primitives).
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "pmp_launch.h"

namespace pmp {

size_t sort_temp_bytes(long long max_pairs, long long count)
{
    size_t a = 0, b = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, a, (const long long *)nullptr, (long long *)nullptr, count + 1);
    cub::DeviceRadixSort::SortPairs(nullptr, b, (const unsigned *)nullptr, (unsigned *)nullptr, (const int *)nullptr,
                                    (int *)nullptr, max_pairs, 0, 32);
    return a > b ? a : b;
}

cudaError_t scan_counts(void *temp, size_t temp_bytes, const long long *counts, long long *offsets, long long n,
                        cudaStream_t stream)
{
    return cub::DeviceScan::ExclusiveSum(temp, temp_bytes, counts, offsets, n, stream);
}

cudaError_t sort_pairs(void *temp, size_t temp_bytes, const unsigned *kin, unsigned *kout, const int *vin, int *vout,
                       long long n, int end_bit, cudaStream_t stream)
{
    return cub::DeviceRadixSort::SortPairs(temp, temp_bytes, kin, kout, vin, vout, n, 0, end_bit, stream);
}

}  // namespace pmp
