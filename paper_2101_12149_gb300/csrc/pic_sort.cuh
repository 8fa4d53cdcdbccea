// Constants and kernels of the counting sort (pic_sort.cu) that other
// translation units launch on their own arrays (pic_noalloc.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace pic {

constexpr int kSortBlock = 256;                      // threads per sort CTA
constexpr int kScanItems = 16;                       // counts per thread in k_scan
constexpr int kScanChunk = kSortBlock * kScanItems;  // counts per k_scan CTA (one look-back word each)
static_assert(kScanItems % 4 == 0, "k_scan moves counts four at a time");

// count[key] += 1 for every key in [0, C); a key outside sets ERRBIT_RANGE in err.
__global__ void k_hist(const int* key, int64_t np, int* count, int64_t C, unsigned* err);
// offsets = exclusive prefix sum of count[0..C), offsets[C] = the total; status
// holds nchunks look-back words and a ticket, zeroed before the launch.
__global__ void k_scan(const int* count, int* offsets, int64_t C, unsigned long long* status, int nchunks,
                       unsigned* err);

}  // namespace pic
