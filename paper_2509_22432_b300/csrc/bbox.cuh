// Axis-aligned bounding box of an (n, 3) float32 cloud and its finiteness
// check, in one pass (used by the cell grid and by the FPS point ordering).
//
// Coordinates are reduced as order-preserving unsigned words so that min and
// max are plain integer atomics: a non-negative float maps to its bits with
// the sign bit set, a negative one to its complemented bits.
#pragma once

#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace flood {
namespace {

constexpr int kBoxThreads = 256;

__device__ __forceinline__ uint32_t ordered_bits(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__host__ __device__ inline float from_ordered(uint32_t u) {
    const uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &b, 4);
    return f;
}

// box[0..2] = ordered min, box[3..5] = ordered max; non-finite coordinates are
// left out of the box and raise FLAG_NONFINITE. Each block reduces its points
// through shuffles and shared memory and adds one atomic per word, so the
// six words see a few hundred atomics, not one per warp.
__global__ void __launch_bounds__(kBoxThreads) k_bbox(const float* X, int64_t n, uint32_t* box, uint32_t* flags) {
    __shared__ uint32_t s_red[6][kBoxThreads / 32];
    uint32_t mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
    bool bad = false;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = X[3 * i + c];
            if (!isfinite(v)) {
                bad = true;
                continue;
            }
            const uint32_t o = ordered_bits(v);
            mn[c] = min(mn[c], o);
            mx[c] = max(mx[c], o);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        mn[c] = __reduce_min_sync(0xffffffffu, mn[c]);
        mx[c] = __reduce_max_sync(0xffffffffu, mx[c]);
        if (lane == 0) {
            s_red[c][warp] = mn[c];
            s_red[3 + c][warp] = mx[c];
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, FLAG_NONFINITE);
    __syncthreads();
    if (warp == 0) {
        const int w = lane % (kBoxThreads / 32);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const uint32_t a = __reduce_min_sync(0xffffffffu, s_red[c][w]);
            const uint32_t b = __reduce_max_sync(0xffffffffu, s_red[3 + c][w]);
            if (lane == 0) {
                atomicMin(&box[c], a);
                atomicMax(&box[3 + c], b);
            }
        }
    }
}

// Blocks for k_bbox: about eight points per thread, at most two blocks per SM.
inline unsigned bbox_blocks(int64_t n, int sms) {
    const int64_t per = int64_t(kBoxThreads) * 8;
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, int64_t(sms) * 2)));
}

__global__ void k_box_init(uint32_t* box, uint32_t* flags) {
    box[0] = box[1] = box[2] = 0xffffffffu;
    box[3] = box[4] = box[5] = 0u;
    *flags = 0;
}

}  // namespace
}  // namespace flood
