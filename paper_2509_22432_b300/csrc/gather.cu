// flood_gather_rows: the landmark rows L = X[idx] of FPS's picks, on the
// device (the triangulation and the filtration take L, §3: L = X[FPS picks]).
#include "common.cuh"

namespace flood {
namespace {

constexpr int kGatherThreads = 256;

// One thread per (row, coordinate): coalesced writes of L, reads of X by row.
__global__ void __launch_bounds__(kGatherThreads) k_gather_rows(const float* X, int64_t n, int dim,
                                                                const int64_t* idx, int64_t n_idx, float* L,
                                                                uint32_t* flags) {
    const int64_t t = blockIdx.x * int64_t(kGatherThreads) + threadIdx.x;
    if (t >= n_idx * dim) return;
    const int64_t r = t / dim, c = t - r * dim;
    const int64_t i = idx[r];
    if (i < 0 || i >= n) {
        if (c == 0) atomicOr(flags, FLAG_RANGE);
        return;
    }
    L[t] = X[i * dim + c];
}

}  // namespace
}  // namespace flood

using namespace flood;

extern "C" int flood_gather_rows(const float* X, int64_t n_points, int32_t dim, const int64_t* idx, int64_t n_idx,
                                 float* L, void* stream_) {
    if (!X || (n_idx > 0 && (!idx || !L)) || n_points < 1 || dim < 1 || dim > 8 || n_idx < 0 ||
        n_idx >= (int64_t(1) << 40)) {
        set_error("flood_gather_rows: need X != NULL (and idx, L when n_idx > 0), n_points >= 1, 1 <= dim <= 8, "
                  "0 <= n_idx < 2^40");
        return FLOOD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    if (int rc = pending_error(s)) return rc;
    if (n_idx == 0) return FLOOD_OK;
    Scratch scr(s);
    uint32_t* flags = nullptr;
    if (int rc = scr.alloc(&flags, 1)) return rc;
    FLOOD_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t), s));
    const unsigned nb = static_cast<unsigned>(ceil_div(n_idx * dim, kGatherThreads));
    k_gather_rows<<<nb, kGatherThreads, 0, s>>>(X, n_points, dim, idx, n_idx, L, flags);
    note_launch(1);
    FLOOD_CUDA(cudaGetLastError());
    return defer_status(s, flags, "flood_gather_rows");
}
