#pragma once
#include "common.cuh"

namespace flood {
// out[i] = sum_{j<i} in[j] for i in [0, n], so out has n+1 entries (out[n] = total).
// in and out may not alias. Totals must fit in int32.
int exclusive_scan(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s, Scratch& scr);
int exclusive_scan(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s, Bump& scr);
// Scratch bytes exclusive_scan carves from its allocator for n entries (256-byte pieces).
size_t exclusive_scan_scratch_bytes(int64_t n);
}  // namespace flood
