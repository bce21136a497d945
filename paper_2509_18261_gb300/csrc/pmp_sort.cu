// pmp_sort.cu -- CUB primitives of the plan and the sorted deposit: the radix
// sort of particles by host cell, the prefix sum of pair counts, and the
// stable radix sort of (buffer cell, pair) keys.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_run_length_encode.cuh>
#include <cub/device/device_scan.cuh>

#include "pmp_launch.h"

namespace pmp {

size_t cub_temp_bytes(long long n, long long max_pairs, bool sorted)
{
    size_t a = 0, b = 0, c = 0;
    const long long nn = n > 0 ? n : 1;
    cub::DeviceRadixSort::SortPairs(nullptr, a, (const unsigned *)nullptr, (unsigned *)nullptr,
                                    (const unsigned *)nullptr, (unsigned *)nullptr, nn, 0, 32);
    if (sorted)
        cub::DeviceScan::ExclusiveScan(nullptr, b, (const unsigned *)nullptr, (unsigned long long *)nullptr,
                                       cuda::std::plus<unsigned long long>(), 0ULL, nn + 1);
    size_t d = 0, e = 0;
    if (sorted) {
        const long long mp = max_pairs > 0 ? max_pairs : 1;
        cub::DeviceRadixSort::SortPairs(nullptr, c, (const unsigned *)nullptr, (unsigned *)nullptr,
                                        (const unsigned *)nullptr, (unsigned *)nullptr, mp, 0, 32);
        cub::DeviceRunLengthEncode::Encode(nullptr, d, (const unsigned *)nullptr, (unsigned *)nullptr,
                                           (unsigned *)nullptr, (unsigned long long *)nullptr, mp);
        cub::DeviceScan::ExclusiveSum(nullptr, e, (const unsigned *)nullptr, (unsigned *)nullptr, mp);
    }
    size_t m = a > b ? a : b;
    m = m > c ? m : c;
    m = m > d ? m : d;
    return m > e ? m : e;
}

cudaError_t sort_host_keys(void *temp, size_t temp_bytes, const unsigned *kin, unsigned *kout, const unsigned *vin,
                           unsigned *vout, long long n, int end_bit, cudaStream_t stream)
{
    return cub::DeviceRadixSort::SortPairs(temp, temp_bytes, kin, kout, vin, vout, n, 0, end_bit, stream);
}

// Exclusive prefix sum of 32-bit counts accumulated in 64 bits.
size_t scan_temp_bytes(long long n)
{
    size_t b = 0;
    cub::DeviceScan::ExclusiveScan(nullptr, b, (const unsigned *)nullptr, (unsigned long long *)nullptr,
                                   cuda::std::plus<unsigned long long>(), 0ULL, n > 0 ? n : 1);
    return b;
}

cudaError_t scan_counts(void *temp, size_t temp_bytes, const unsigned *counts, unsigned long long *offsets,
                        long long n, cudaStream_t stream)
{
    return cub::DeviceScan::ExclusiveScan(temp, temp_bytes, counts, offsets, cuda::std::plus<unsigned long long>(),
                                          0ULL, n, stream);
}

cudaError_t encode_runs(void *temp, size_t temp_bytes, const unsigned *keys, unsigned *uniq, unsigned *lens,
                        unsigned long long *nruns, long long n, cudaStream_t stream)
{
    return cub::DeviceRunLengthEncode::Encode(temp, temp_bytes, keys, uniq, lens, nruns, n, stream);
}

cudaError_t scan_lengths(void *temp, size_t temp_bytes, const unsigned *lens, unsigned *offs, long long n,
                         cudaStream_t stream)
{
    return cub::DeviceScan::ExclusiveSum(temp, temp_bytes, lens, offs, n, stream);
}

cudaError_t sort_pairs(void *temp, size_t temp_bytes, const unsigned *kin, unsigned *kout, const unsigned *vin,
                       unsigned *vout, long long n, int end_bit, cudaStream_t stream)
{
    return cub::DeviceRadixSort::SortPairs(temp, temp_bytes, kin, kout, vin, vout, n, 0, end_bit, stream);
}

}  // namespace pmp
