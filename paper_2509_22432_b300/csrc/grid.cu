// flood_build_grid: uniform cell grid over X (replaces the paper's axis
// presort + masking matrix of §4.2 / App. A.1 as the spatial index).
//
// Steps, all on the device and without a host readback: (1) bounding box and
// finiteness in one pass, (2) one thread picks the cell size and the table
// dimensions from the box (enlarging the cell until the table fits the
// capacity the host allocated from n), (3) cell id per point + histogram,
// (4) exclusive scan -> cell_start, (5) scatter into cell order as float4
// (x, y, z, original row), (6) block occupancy and its distance transform.
// Cells are ordered x fastest, so a row of cells along x is one contiguous
// range of the sorted array.
#include <math.h>
#include <stdlib.h>

#include "bbox.cuh"
#include "geometry.cuh"
#include "scan.cuh"

namespace flood {

namespace {

constexpr int kThreads = 256;
constexpr int64_t kMaxCells = int64_t(1) << 27;

// Default edge length: the cube root of the volume per point times 2, with
// flat or collinear boxes falling back to area or length per point.
__device__ double default_cell_size(const float e[3], int64_t n) {
    float s[3] = {e[0], e[1], e[2]};
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (s[b] > s[a]) {
                const float t = s[a];
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
    return h;
}

// One thread: the grid geometry from the bounding box. The requested edge
// (or the default) is enlarged by 1.25x steps until the table has at most
// `cap` cells; a cloud with a non-finite coordinate gets a one-cell grid (the
// call reports the error) so that later kernels stay in bounds.
__global__ void k_grid_geometry(const uint32_t* box, const uint32_t* flags, int64_t n, float cell_size, int64_t cap,
                                GridView ptrs, GridGeom* geom) {
    GridGeom& G = *geom;
    G.v.pts = ptrs.pts;
    G.v.cell_start = ptrs.cell_start;
    G.v.occupied = ptrs.occupied;
    G.v.bdist = ptrs.bdist;
    float ext[3];
    for (int c = 0; c < 3; ++c) {
        G.bbox_lo[c] = from_ordered(box[c]);
        G.bbox_hi[c] = from_ordered(box[3 + c]);
        ext[c] = G.bbox_hi[c] - G.bbox_lo[c];
    }
    const bool bad = *flags != 0u || !(ext[0] >= 0.0f && ext[1] >= 0.0f && ext[2] >= 0.0f);
    float h = cell_size > 0.0f ? cell_size : static_cast<float>(default_cell_size(ext, n));
    const float emax = fmaxf(ext[0], fmaxf(ext[1], ext[2]));
    if (h < emax * 1e-6f) h = emax * 1e-6f;
    if (!(h > 0.0f)) h = 1.0f;
    int dims[3] = {1, 1, 1};
    if (!bad) {
        for (;;) {
            int64_t cells = 1;
            for (int c = 0; c < 3; ++c) {
                dims[c] = static_cast<int>(fmin(floor(static_cast<double>(__fdiv_rn(ext[c], h))) + 1.0, 1 << 30));
                cells *= dims[c];
            }
            if (cells <= cap) break;
            h *= 1.25f;
        }
    } else {
        for (int c = 0; c < 3; ++c) G.bbox_lo[c] = G.bbox_hi[c] = 0.0f;
        h = 1.0f;
    }
    G.v.dx = dims[0];
    G.v.dy = dims[1];
    G.v.dz = dims[2];
    G.v.bx = (dims[0] + 3) / 4;
    G.v.by = (dims[1] + 3) / 4;
    G.v.bz = (dims[2] + 3) / 4;
    G.v.ox = G.bbox_lo[0];
    G.v.oy = G.bbox_lo[1];
    G.v.oz = G.bbox_lo[2];
    G.v.cell = h;
    G.v.inv_cell = 1.0f / h;
    G.n_cells = int64_t(dims[0]) * dims[1] * dims[2];
    G.n_blocks = int64_t(G.v.bx) * G.v.by * G.v.bz;
    G.v.n_cells = G.n_cells;
    G.v.n_pts = static_cast<int32_t>(n);
}

__global__ void __launch_bounds__(kThreads) k_cell_ids(const float* X, int64_t n, const GridView* gp, int32_t* cell,
                                                      int32_t* count, uint32_t* flags) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const GridView g = *gp;
    const int cx = cell_coord(X[3 * i + 0], g.ox, g.inv_cell, g.dx);
    const int cy = cell_coord(X[3 * i + 1], g.oy, g.inv_cell, g.dy);
    const int cz = cell_coord(X[3 * i + 2], g.oz, g.inv_cell, g.dz);
    const int32_t c = static_cast<int32_t>((static_cast<int64_t>(cz) * g.dy + cy) * g.dx + cx);
    cell[i] = c;
    if (FLOOD_OOB(c, g.n_cells, flags)) return;
    atomicAdd(&count[c], 1);
}

// Counting-sort scatter; `fill` holds the histogram and is counted down (the
// order of points within a cell is arbitrary and changes no result: minima
// do not depend on it and nearest-point ties go to the lowest original row).
__global__ void __launch_bounds__(kThreads) k_scatter(const float* X, int64_t n, const int32_t* cell,
                                                     const int32_t* cell_start, int32_t* fill, float4* pts,
                                                     int64_t cap_cells, uint32_t* flags) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int32_t c = cell[i];
    if (FLOOD_OOB(c, cap_cells, flags)) return;
    const int32_t pos = cell_start[c] + atomicSub(&fill[c], 1) - 1;
    if (FLOOD_OOB(pos, n, flags)) return;
    pts[pos] = make_float4(X[3 * i + 0], X[3 * i + 1], X[3 * i + 2], __int_as_float(static_cast<int>(i)));
}

// One bit per block of 4 x 4 x 4 cells: set when any of its cells is non-empty.
__global__ void k_block_bits(const GridGeom* geom, uint32_t* bits) {
    const int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (b >= geom->n_blocks) return;
    const GridView g = geom->v;
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

__global__ void k_bdist_x(const GridGeom* geom, uint8_t* out) {
    const int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (b >= geom->n_blocks) return;
    const GridView g = geom->v;
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

// axis 1: along y, axis 2: along z.
__global__ void k_bdist_pass(const GridGeom* geom, const uint8_t* in, uint8_t* out, int axis) {
    const int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t nb = geom->n_blocks;
    if (b >= nb) return;
    const GridView g = geom->v;
    const int64_t stride = axis == 1 ? int64_t(g.bx) : int64_t(g.bx) * g.by;
    const int extent = axis == 1 ? g.by : g.bz;
    const int c = static_cast<int>((b / stride) % extent);
    int d = kBdistCap;
    for (int dc = -kBdistCap; dc <= kBdistCap; ++dc) {
        const int cc = c + dc;
        if (cc < 0 || cc >= extent) continue;
        d = min(d, max(abs(dc), static_cast<int>(in[b + dc * stride])));
    }
    out[b] = static_cast<uint8_t>(d);
}

// Capacity of the cell table for n points: the default edge gives about n/8
// cells and a covering-radius-based edge about n/8 to 2n, so 4n (at least
// 2^16, at most 2^27) leaves room; a finer requested edge is coarsened on
// the device, which changes no result.
int64_t cell_capacity(int64_t n) { return std::min<int64_t>(kMaxCells, std::max<int64_t>(int64_t(1) << 16, 4 * n)); }

}  // namespace

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
    if (int rc = pending_error(s)) return rc;
    flood_grid* g = static_cast<flood_grid*>(calloc(1, sizeof(flood_grid)));
    if (!g) {
        set_error("flood_build_grid: host allocation failed");
        return FLOOD_ENOMEM;
    }
    g->n_points = n_points;
    g->cap_cells = cell_capacity(n_points);
    g->cap_blocks = (g->cap_cells + 3) / 4 + 1;  // blocks of any dims with at most cap_cells cells
    const int64_t n_words = (g->cap_blocks + 31) / 32;
    // from the stream-ordered pool (cheap once warm); flood_grid_destroy's
    // cudaFree waits for all work before releasing them
    cudaError_t e1 = cudaMallocAsync(&g->pts, sizeof(float4) * n_points, s);
    cudaError_t e2 = cudaMallocAsync(&g->cell_start, sizeof(int32_t) * (g->cap_cells + 1), s);
    cudaError_t e3 = cudaMallocAsync(&g->occupied, sizeof(uint32_t) * n_words, s);
    cudaError_t e4 = cudaMallocAsync(&g->bdist, static_cast<size_t>(g->cap_blocks), s);
    cudaError_t e5 = cudaMallocAsync(&g->geom, sizeof(GridGeom), s);
    cudaError_t e6 = cudaEventCreateWithFlags(&g->ready, cudaEventDisableTiming);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess || e5 != cudaSuccess ||
        e6 != cudaSuccess) {
        cudaGetLastError();
        flood_grid_destroy(g);
        set_error("flood_build_grid: device allocation failed");
        return FLOOD_ENOMEM;
    }
    g->device_bytes = int64_t(sizeof(float4)) * n_points + int64_t(sizeof(int32_t)) * (g->cap_cells + 1) +
                      int64_t(sizeof(uint32_t)) * n_words + g->cap_blocks + int64_t(sizeof(GridGeom));
    GridView ptrs{};
    ptrs.pts = g->pts;
    ptrs.cell_start = g->cell_start;
    ptrs.occupied = g->occupied;
    ptrs.bdist = g->bdist;
    int rc = FLOOD_OK;
    {
        Scratch scr(s);
        uint32_t* d_box = nullptr;  // 6 ordered words + flags
        int32_t *d_cell = nullptr, *d_count = nullptr;
        uint8_t* d_bd = nullptr;
        if ((rc = scr.alloc(&d_box, 8)) || (rc = scr.alloc(&d_cell, n_points)) ||
            (rc = scr.alloc(&d_count, g->cap_cells)) || (rc = scr.alloc(&d_bd, g->cap_blocks))) {
            flood_grid_destroy(g);
            return rc;
        }
        const unsigned nb = static_cast<unsigned>(ceil_div(n_points, kThreads));
        const unsigned nbb = static_cast<unsigned>(ceil_div(g->cap_blocks, kThreads));
        cudaMemsetAsync(d_count, 0, sizeof(int32_t) * g->cap_cells, s);
        cudaMemsetAsync(g->occupied, 0, sizeof(uint32_t) * n_words, s);
        k_box_init<<<1, 1, 0, s>>>(d_box, d_box + 6);
        k_bbox<<<bbox_blocks(n_points, device_sm_count()), kBoxThreads, 0, s>>>(X, n_points, d_box, d_box + 6);
        k_grid_geometry<<<1, 1, 0, s>>>(d_box, d_box + 6, n_points, cell_size, g->cap_cells, ptrs, g->geom);
        k_cell_ids<<<nb, kThreads, 0, s>>>(X, n_points, view_of(g), d_cell, d_count, d_box + 6);
        note_launch(4);
        // cells past the used ones count 0, so their offsets all equal n_points
        rc = exclusive_scan(d_count, g->cell_start, g->cap_cells, s, scr);
        if (rc == FLOOD_OK) {
            k_scatter<<<nb, kThreads, 0, s>>>(X, n_points, d_cell, g->cell_start, d_count, g->pts, g->cap_cells,
                                              d_box + 6);
            k_block_bits<<<nbb, kThreads, 0, s>>>(g->geom, g->occupied);
            k_bdist_x<<<nbb, kThreads, 0, s>>>(g->geom, g->bdist);
            k_bdist_pass<<<nbb, kThreads, 0, s>>>(g->geom, g->bdist, d_bd, 1);
            k_bdist_pass<<<nbb, kThreads, 0, s>>>(g->geom, d_bd, g->bdist, 2);
            note_launch(5);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) rc = cuda_fail(e, "flood_build_grid kernels");
        }
        if (rc == FLOOD_OK) rc = defer_status(s, d_box + 6, "flood_build_grid");
        if (rc == FLOOD_OK) {
            cudaError_t e = cudaEventRecord(g->ready, s);
            if (e != cudaSuccess) rc = cuda_fail(e, "flood_build_grid");
        }
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
    GridGeom h;
    FLOOD_CUDA(cudaEventSynchronize(g->ready));
    FLOOD_CUDA(cudaMemcpy(&h, g->geom, sizeof(h), cudaMemcpyDeviceToHost));
    out->n_points = g->n_points;
    out->n_cells = h.n_cells;
    out->cell_size = h.v.cell;
    out->device_bytes = g->device_bytes;
    out->dims[0] = h.v.dx;
    out->dims[1] = h.v.dy;
    out->dims[2] = h.v.dz;
    out->origin[0] = h.v.ox;
    out->origin[1] = h.v.oy;
    out->origin[2] = h.v.oz;
    for (int c = 0; c < 3; ++c) {
        out->bbox_lo[c] = h.bbox_lo[c];
        out->bbox_hi[c] = h.bbox_hi[c];
    }
    return FLOOD_OK;
}

namespace flood {
// Release a grid in stream order (cudaFreeAsync on s): for callers that know
// every use of the grid is ordered before s (the serving loop, whose streams
// have completed the grid's work when a request finishes). Unlike
// flood_grid_destroy it does not wait for the whole device.
void grid_release_async(flood_grid* g, cudaStream_t s) {
    if (!g) return;
    if (g->pts) cudaFreeAsync(g->pts, s);
    if (g->cell_start) cudaFreeAsync(g->cell_start, s);
    if (g->occupied) cudaFreeAsync(g->occupied, s);
    if (g->bdist) cudaFreeAsync(g->bdist, s);
    if (g->geom) cudaFreeAsync(g->geom, s);
    if (g->ready) cudaEventDestroy(g->ready);
    free(g);
}
}  // namespace flood

extern "C" void flood_grid_destroy(flood_grid* g) {
    if (!g) return;
    if (g->pts) cudaFree(g->pts);
    if (g->cell_start) cudaFree(g->cell_start);
    if (g->occupied) cudaFree(g->occupied);
    if (g->bdist) cudaFree(g->bdist);
    if (g->geom) cudaFree(g->geom);
    if (g->ready) cudaEventDestroy(g->ready);
    free(g);
}
