// flood_build_grid: uniform cell grid over X (replaces the paper's axis
// presort + masking matrix of §4.2 / App. A.1 as the spatial index).
//
// Steps: (1) bounding box and finiteness in one pass, (2) host picks the cell
// size and dense table dimensions, (3) cell id per point + histogram,
// (4) exclusive scan -> cell_start, (5) scatter into cell order as float4
// (x, y, z, original row). Cells are ordered x fastest, so a row of cells
// along x is one contiguous range of the sorted array.
#include <math.h>
#include <stdlib.h>

#include "bbox.cuh"
#include "geometry.cuh"
#include "scan.cuh"

namespace flood {

namespace {

constexpr int kThreads = 256;
constexpr int64_t kMaxCells = int64_t(1) << 27;

__global__ void __launch_bounds__(kThreads) k_cell_ids(const float* X, int64_t n, GridView g, int32_t* cell,
                                                      int32_t* count) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int cx = cell_coord(X[3 * i + 0], g.ox, g.inv_cell, g.dx);
    const int cy = cell_coord(X[3 * i + 1], g.oy, g.inv_cell, g.dy);
    const int cz = cell_coord(X[3 * i + 2], g.oz, g.inv_cell, g.dz);
    const int32_t c = static_cast<int32_t>((static_cast<int64_t>(cz) * g.dy + cy) * g.dx + cx);
    cell[i] = c;
    atomicAdd(&count[c], 1);
}

__global__ void __launch_bounds__(kThreads) k_scatter(const float* X, int64_t n, const int32_t* cell,
                                                     const int32_t* cell_start, int32_t* fill, float4* pts) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int32_t c = cell[i];
    const int32_t pos = cell_start[c] + atomicAdd(&fill[c], 1);
    pts[pos] = make_float4(X[3 * i + 0], X[3 * i + 1], X[3 * i + 2], __int_as_float(static_cast<int>(i)));
}

// One bit per block of 4 x 4 x 4 cells: set when any of its cells is non-empty.
__global__ void k_block_bits(GridView g, uint32_t* bits) {
    const int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t nb = int64_t(g.bx) * g.by * g.bz;
    if (b >= nb) return;
    const int bx = static_cast<int>(b % g.bx), by = static_cast<int>((b / g.bx) % g.by),
              bz = static_cast<int>(b / (int64_t(g.bx) * g.by));
    bool any = false;
    for (int z = 4 * bz; z < min(4 * bz + 4, g.dz) && !any; ++z)
        for (int y = 4 * by; y < min(4 * by + 4, g.dy) && !any; ++y) {
            const int64_t row = (static_cast<int64_t>(z) * g.dy + y) * g.dx;
            const int x0 = 4 * bx, x1 = min(4 * bx + 4, g.dx);
            any = g.cell_start[row + x1] > g.cell_start[row + x0];
        }
    if (any) atomicOr(&bits[b >> 5], 1u << (b & 31));
}

// Chebyshev distance transform of the block occupancy, in three separable
// passes (distance along x to an occupied block, then the max-min combination
// along y and along z), each over a window of +-kBdistCap blocks. Distances
// are capped at kBdistCap, so every stored value is a lower bound.
constexpr int kBdistCap = 15;

__global__ void k_bdist_x(GridView g, uint8_t* out) {
    const int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t nb = int64_t(g.bx) * g.by * g.bz;
    if (b >= nb) return;
    const int bx = static_cast<int>(b % g.bx);
    const int64_t row = b - bx;
    int d = kBdistCap;
    for (int dx = -kBdistCap; dx <= kBdistCap; ++dx) {
        const int x = bx + dx;
        if (x < 0 || x >= g.bx) continue;
        const int64_t bit = row + x;
        if (g.occupied[bit >> 5] & (1u << (bit & 31))) d = min(d, abs(dx));
    }
    out[b] = static_cast<uint8_t>(d);
}

// stride: blocks between neighbours along the axis; extent: blocks along it.
__global__ void k_bdist_pass(const uint8_t* in, uint8_t* out, int64_t nb, int64_t stride, int extent) {
    const int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (b >= nb) return;
    const int c = static_cast<int>((b / stride) % extent);
    int d = kBdistCap;
    for (int dc = -kBdistCap; dc <= kBdistCap; ++dc) {
        const int cc = c + dc;
        if (cc < 0 || cc >= extent) continue;
        d = min(d, max(abs(dc), static_cast<int>(in[b + dc * stride])));
    }
    out[b] = static_cast<uint8_t>(d);
}

}  // namespace

// Default edge length: the cube root of the volume per point times 2, with
// flat or collinear boxes falling back to area or length per point.
static float default_cell_size(const float e[3], int64_t n) {
    float s[3] = {e[0], e[1], e[2]};
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (s[b] > s[a]) {
                float t = s[a];
                s[a] = s[b];
                s[b] = t;
            }
    const double np = static_cast<double>(n);
    double h;
    if (s[2] > 1e-6 * s[0])
        h = 2.0 * cbrt(static_cast<double>(s[0]) * s[1] * s[2] / np);
    else if (s[1] > 1e-6 * s[0])
        h = 2.0 * sqrt(static_cast<double>(s[0]) * s[1] / np);
    else
        h = 2.0 * s[0] / np;
    if (!(h > 0)) h = 1.0;
    return static_cast<float>(h);
}

}  // namespace flood

using namespace flood;

extern "C" int flood_build_grid(const float* X, int64_t n_points, float cell_size, flood_grid** out,
                                void* stream_) {
    if (!out) {
        set_error("flood_build_grid: out is NULL");
        return FLOOD_EINVAL;
    }
    *out = nullptr;
    if (!X || n_points < 1 || n_points >= (int64_t(1) << 31)) {
        set_error("flood_build_grid: need X != NULL and 1 <= n_points < 2^31");
        return FLOOD_EINVAL;
    }
    if (!(cell_size <= 0.0f) && !isfinite(cell_size)) {
        set_error("flood_build_grid: cell_size must be finite");
        return FLOOD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    Scratch scr(s);
    uint32_t* d_box = nullptr;  // 6 ordered words + flags
    int rc = scr.alloc(&d_box, 8);
    if (rc) return rc;
    k_box_init<<<1, 1, 0, s>>>(d_box, d_box + 6); note_launch();
    const int sms = device_sm_count();
    k_bbox<<<bbox_blocks(n_points, sms), kBoxThreads, 0, s>>>(X, n_points, d_box, d_box + 6); note_launch();
    FLOOD_CUDA(cudaGetLastError());
    uint32_t h_box[8];
    FLOOD_CUDA(cudaMemcpyAsync(h_box, d_box, sizeof(uint32_t) * 7, cudaMemcpyDeviceToHost, s));
    FLOOD_CUDA(cudaStreamSynchronize(s));
    if (h_box[6]) return status_from_flags(h_box[6], "flood_build_grid");

    flood_grid* g = static_cast<flood_grid*>(calloc(1, sizeof(flood_grid)));
    if (!g) {
        set_error("flood_build_grid: host allocation failed");
        return FLOOD_ENOMEM;
    }
    g->n_points = n_points;
    float ext[3];
    for (int c = 0; c < 3; ++c) {
        g->bbox_lo[c] = from_ordered(h_box[c]);
        g->bbox_hi[c] = from_ordered(h_box[3 + c]);
        ext[c] = g->bbox_hi[c] - g->bbox_lo[c];
        g->origin[c] = g->bbox_lo[c];
    }
    float h = cell_size > 0.0f ? cell_size : default_cell_size(ext, n_points);
    const float emax = std::max(ext[0], std::max(ext[1], ext[2]));
    if (h < emax * 1e-6f) h = emax * 1e-6f;
    if (!(h > 0.0f)) h = 1.0f;
    for (;;) {
        int64_t cells = 1;
        for (int c = 0; c < 3; ++c) {
            g->dims[c] = static_cast<int32_t>(std::min<double>(floor(ext[c] / h) + 1.0, 1 << 30));
            cells *= g->dims[c];
        }
        if (cells <= kMaxCells) {
            g->n_cells = cells;
            break;
        }
        h *= 1.25f;
    }
    g->cell_size = h;
    g->inv_cell = 1.0f / h;

    for (int c = 0; c < 3; ++c) g->bdims[c] = (g->dims[c] + 3) / 4;
    const int64_t n_blocks = int64_t(g->bdims[0]) * g->bdims[1] * g->bdims[2];
    const int64_t n_words = (n_blocks + 31) / 32;
    // from the stream-ordered pool (cheap once warm); flood_grid_destroy's
    // cudaFree waits for all work before releasing them
    cudaError_t e1 = cudaMallocAsync(&g->pts, sizeof(float4) * n_points, s);
    cudaError_t e2 = cudaMallocAsync(&g->cell_start, sizeof(int32_t) * (g->n_cells + 1), s);
    cudaError_t e3 = cudaMallocAsync(&g->occupied, sizeof(uint32_t) * n_words, s);
    cudaError_t e4 = cudaMallocAsync(&g->bdist, static_cast<size_t>(n_blocks), s);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess) {
        cudaGetLastError();
        flood_grid_destroy(g);
        set_error("flood_build_grid: device allocation failed");
        return FLOOD_ENOMEM;
    }
    g->device_bytes = int64_t(sizeof(float4)) * n_points + int64_t(sizeof(int32_t)) * (g->n_cells + 1) +
                      int64_t(sizeof(uint32_t)) * n_words + n_blocks;

    int32_t *d_cell = nullptr, *d_count = nullptr;
    uint8_t* d_bd = nullptr;
    if ((rc = scr.alloc(&d_cell, n_points)) || (rc = scr.alloc(&d_count, g->n_cells)) ||
        (rc = scr.alloc(&d_bd, n_blocks))) {
        flood_grid_destroy(g);
        return rc;
    }
    GridView v = view_of(g);
    const unsigned nb = static_cast<unsigned>(ceil_div(n_points, kThreads));
    cudaMemsetAsync(d_count, 0, sizeof(int32_t) * g->n_cells, s);
    k_cell_ids<<<nb, kThreads, 0, s>>>(X, n_points, v, d_cell, d_count); note_launch();
    rc = exclusive_scan(d_count, g->cell_start, g->n_cells, s, scr);
    if (rc == FLOOD_OK) {
        cudaMemsetAsync(d_count, 0, sizeof(int32_t) * g->n_cells, s);
        k_scatter<<<nb, kThreads, 0, s>>>(X, n_points, d_cell, g->cell_start, d_count, g->pts); note_launch();
        cudaMemsetAsync(g->occupied, 0, sizeof(uint32_t) * n_words, s);
        const unsigned nbb = static_cast<unsigned>(ceil_div(n_blocks, kThreads));
        k_block_bits<<<nbb, kThreads, 0, s>>>(view_of(g), g->occupied);
        k_bdist_x<<<nbb, kThreads, 0, s>>>(view_of(g), g->bdist);
        k_bdist_pass<<<nbb, kThreads, 0, s>>>(g->bdist, d_bd, n_blocks, g->bdims[0], g->bdims[1]);
        k_bdist_pass<<<nbb, kThreads, 0, s>>>(d_bd, g->bdist, n_blocks, int64_t(g->bdims[0]) * g->bdims[1],
                                              g->bdims[2]);
        note_launch(4);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "flood_build_grid kernels");
    }
    if (rc == FLOOD_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "flood_build_grid");
    }
    if (rc != FLOOD_OK) {
        flood_grid_destroy(g);
        return rc;
    }
    *out = g;
    return FLOOD_OK;
}

extern "C" int flood_grid_get_info(const flood_grid* g, flood_grid_info* out) {
    if (!g || !out) {
        set_error("flood_grid_get_info: NULL argument");
        return FLOOD_EINVAL;
    }
    out->n_points = g->n_points;
    out->n_cells = g->n_cells;
    out->cell_size = g->cell_size;
    out->device_bytes = g->device_bytes;
    for (int c = 0; c < 3; ++c) {
        out->dims[c] = g->dims[c];
        out->origin[c] = g->origin[c];
        out->bbox_lo[c] = g->bbox_lo[c];
        out->bbox_hi[c] = g->bbox_hi[c];
    }
    return FLOOD_OK;
}

extern "C" void flood_grid_destroy(flood_grid* g) {
    if (!g) return;
    if (g->pts) cudaFree(g->pts);
    if (g->cell_start) cudaFree(g->cell_start);
    if (g->occupied) cudaFree(g->occupied);
    if (g->bdist) cudaFree(g->bdist);
    free(g);
}
