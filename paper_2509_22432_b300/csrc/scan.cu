// Exclusive prefix sum of int32 counts (device), used for the cell table and
// for work-item offsets. Three-phase: per-block scans, a recursive scan of
// the block totals, then a uniform add.
#include "scan.cuh"

namespace flood {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* s_warp, int32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < (kScanThreads / 32) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[31];
    const int32_t before = warp > 0 ? s_warp[warp - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int32_t* in, int32_t* out, int64_t n,
                                                             int32_t* tile_sums) {
    __shared__ int32_t s_warp[32];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        sum += v[i];
    }
    int32_t total;
    int32_t run = block_exclusive_scan(sum, s_warp, total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_add(int32_t* out, int64_t n, const int32_t* tile_offsets) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x;
    const int32_t add = tile_offsets[blockIdx.x];
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t t = i + static_cast<int64_t>(j) * kScanThreads;
        if (t < n) out[t] += add;
    }
}

__global__ void k_set_total(const int32_t* in, int32_t* out, int64_t n) {
    // out[n] = out[n-1] + in[n-1]
    out[n] = (n > 0) ? out[n - 1] + in[n - 1] : 0;
}

template <class Alloc>
int scan_rec(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s, Alloc& scr) {
    if (n <= 0) return FLOOD_OK;
    const int64_t tiles = ceil_div(n, kScanTile);
    if (tiles == 1) {
        k_scan_tiles<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr); note_launch();
        FLOOD_CUDA(cudaGetLastError());
        return FLOOD_OK;
    }
    int32_t *sums = nullptr, *offs = nullptr;
    int rc = scr.alloc(&sums, tiles);
    if (rc) return rc;
    rc = scr.alloc(&offs, tiles);
    if (rc) return rc;
    k_scan_tiles<<<static_cast<unsigned>(tiles), kScanThreads, 0, s>>>(in, out, n, sums); note_launch();
    FLOOD_CUDA(cudaGetLastError());
    rc = scan_rec(sums, offs, tiles, s, scr);
    if (rc) return rc;
    k_scan_add<<<static_cast<unsigned>(tiles), kScanThreads, 0, s>>>(out, n, offs); note_launch();
    FLOOD_CUDA(cudaGetLastError());
    return FLOOD_OK;
}

// Second half of the two-launch scan (up to kFlatTiles tiles): each block
// adds the sum of the tile sums before its tile (a block reduction), and the
// last block writes the total to out[n].
constexpr int64_t kFlatTiles = 1024;

__global__ void __launch_bounds__(kScanThreads) k_scan_add_prefix(int32_t* out, int64_t n, const int32_t* tile_sums,
                                                                  int64_t n_tiles) {
    __shared__ int32_t s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool last = blockIdx.x == n_tiles - 1;
    const int64_t upto = last ? n_tiles : blockIdx.x;  // the last block also sums its own tile: the total
    int32_t before = 0, own = 0;
    for (int64_t t = threadIdx.x; t < upto; t += kScanThreads) {
        const int32_t v = tile_sums[t];
        if (t < blockIdx.x) before += v;
        else own += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        before += __shfl_xor_sync(0xffffffffu, before, o);
        own += __shfl_xor_sync(0xffffffffu, own, o);
    }
    if (lane == 0) s_warp[warp] = before;
    __syncthreads();
    int32_t add = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) add += s_warp[w];
    __syncthreads();
    if (lane == 0) s_warp[warp] = own;
    __syncthreads();
    if (last && threadIdx.x == 0) {
        int32_t o = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) o += s_warp[w];
        out[n] = add + o;
    }
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x;
    if (add != 0)
        for (int j = 0; j < kScanItems; ++j) {
            const int64_t t = i + static_cast<int64_t>(j) * kScanThreads;
            if (t < n) out[t] += add;
        }
}

template <class Alloc>
int scan_total(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s, Alloc& scr) {
    const int64_t tiles = ceil_div(n, kScanTile);
    if (n > 0 && tiles > 1 && tiles <= kFlatTiles) {  // two launches: tile scans, then prefixes and the total
        int32_t* sums = nullptr;
        int rc = scr.alloc(&sums, tiles);
        if (rc) return rc;
        k_scan_tiles<<<static_cast<unsigned>(tiles), kScanThreads, 0, s>>>(in, out, n, sums);
        k_scan_add_prefix<<<static_cast<unsigned>(tiles), kScanThreads, 0, s>>>(out, n, sums, tiles);
        note_launch(2);
        FLOOD_CUDA(cudaGetLastError());
        return FLOOD_OK;
    }
    int rc = scan_rec(in, out, n, s, scr);
    if (rc) return rc;
    k_set_total<<<1, 1, 0, s>>>(in, out, n); note_launch();
    FLOOD_CUDA(cudaGetLastError());
    return FLOOD_OK;
}

}  // namespace

size_t exclusive_scan_scratch_bytes(int64_t n) {
    const int64_t tiles = ceil_div(n, kScanTile);
    if (n > 0 && tiles > 1 && tiles <= kFlatTiles) return (size_t(4) * tiles + 255) & ~size_t(255);
    size_t b = 0;
    for (int64_t tiles = ceil_div(n, kScanTile); n > 0 && tiles > 1; n = tiles, tiles = ceil_div(n, kScanTile))
        b += 2 * ((size_t(4) * tiles + 255) & ~size_t(255));  // block sums and their offsets
    return b;
}

int exclusive_scan(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s, Scratch& scr) {
    return scan_total(in, out, n, s, scr);
}

int exclusive_scan(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s, Bump& scr) {
    return scan_total(in, out, n, s, scr);
}

}  // namespace flood
