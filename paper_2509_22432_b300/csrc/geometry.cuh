// Device-side geometry shared by the filtration and backward kernels: the
// cell grid view, the barycentric sample of a simplex (Lemma 1) and its cull
// box. Every quantity here depends only on (simplex, sample) so that results
// are identical however the work is tiled.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace flood {

struct GridView {
    const float4* pts;
    const int32_t* cell_start;
    const uint32_t* occupied;
    const uint8_t* bdist;
    int dx, dy, dz;
    int bx, by, bz;
    float ox, oy, oz;
    float inv_cell;
    float cell;
    int64_t n_cells;  // cells in use (cell_start has n_cells + 1 entries that matter)
    int32_t n_pts;    // points of the grid
};

// Device-resident geometry of a grid. The host fills the pointers of v at
// allocation; k_grid_geometry fills everything else from X's bounding box,
// so no host readback is needed to build or use a grid.
struct GridGeom {
    GridView v;
    float bbox_lo[3], bbox_hi[3];
    int64_t n_cells;
    int64_t n_blocks;
};

}  // namespace flood

struct flood_grid {
    int64_t n_points;
    int64_t cap_cells;    // capacity of the cell table; the grid uses at most this many cells
    int64_t cap_blocks;   // capacity of the 4 x 4 x 4 block arrays
    float4* pts;          // points sorted by cell: (x, y, z, original row as int bits)
    int32_t* cell_start;  // cap_cells + 1 offsets into pts (entries past the used cells equal n_points)
    uint32_t* occupied;   // one bit per block of 4 x 4 x 4 cells that holds any point
    uint8_t* bdist;       // per block: Chebyshev distance in blocks to the nearest occupied one (capped, a lower bound)
    flood::GridGeom* geom;  // device
    cudaEvent_t ready;    // recorded after the build's last kernel (flood_grid_get_info waits for it)
    int64_t device_bytes;
};

namespace flood {

// Interior compositions of m into k+1 parts >= 1 (barycentric c_i with
// lambda_i = c_i / m, Lemma 1), lexicographic in (c_0, ..., c_k), as bytes.
std::vector<uint8_t> interior_table(int m, int k);
// Device copy of interior_table(m, k) (host: that table), cached per device.
int device_interior_table(int m, int k, const std::vector<uint8_t>& host, const uint8_t** out);
// Frees a grid in stream order on s (every use of it must be ordered before s).
void grid_release_async(flood_grid* g, cudaStream_t s);

// d(v, X) and its rounded-up bound (0 for a point of X) for every landmark;
// src gets (v, 0). Defined with the filtration kernels.
int launch_vertices(const float* L, int32_t n_L, const flood_grid* grid, float* val, int32_t* src, float* vbound,
                    uint32_t* flags, cudaStream_t s);

// The device copy of a grid's view (kernels load it into registers).
inline const GridView* view_of(const flood_grid* g) { return &g->geom->v; }

// Cell coordinate of v along one axis; monotone in v and clamped to the grid,
// so a point inside [lo, hi] always lands between the cells of lo and hi.
__device__ __forceinline__ int cell_coord(float v, float o, float inv_cell, int dim) {
    float t = __fmul_rn(__fsub_rn(v, o), inv_cell);
    t = fminf(fmaxf(t, 0.0f), static_cast<float>(dim - 1));
    return static_cast<int>(t);
}

// First shell (Chebyshev distance in cells from the box [lo, hi]) that can
// hold a point: if every 4 x 4 x 4 block touching the box is D >= 1 blocks
// from the nearest occupied block, no point lies within 4 (D - 1) cells of
// the box, so shells 0 .. 4 (D - 1) are empty. Boxes over more than 64
// blocks start at shell 0. Warp-collective: the lanes read the (at most 64)
// blocks' distances together.
__device__ __forceinline__ int first_shell(const GridView& g, const int lo[3], const int hi[3], int lane) {
    const int x0 = lo[0] >> 2, y0 = lo[1] >> 2, z0 = lo[2] >> 2;
    const int nx = (hi[0] >> 2) - x0 + 1, ny = (hi[1] >> 2) - y0 + 1, nz = (hi[2] >> 2) - z0 + 1;
    if (nx * ny * nz > 64) return 0;
    int d = 255;
    for (int i = lane; i < nx * ny * nz; i += 32) {
        const int x = x0 + i % nx, y = y0 + (i / nx) % ny, z = z0 + i / (nx * ny);
        d = min(d, static_cast<int>(g.bdist[(static_cast<int64_t>(z) * g.by + y) * g.bx + x]));
    }
    d = static_cast<int>(__reduce_min_sync(0xffffffffu, static_cast<uint32_t>(d)));
    return d >= 1 ? 4 * (d - 1) + 1 : 0;
}

// Vertex coordinates of a k-simplex: origin v0 and edge vectors e_j = v_j - v0.
struct Simplex {
    float v0[3];
    float e[3][3];  // e[j-1] = v_j - v0, j = 1..k
};

__device__ __forceinline__ void load_simplex(const float* L, const int32_t* ids, int k, Simplex& s) {
    const int32_t i0 = ids[0];
    s.v0[0] = L[3 * i0 + 0];
    s.v0[1] = L[3 * i0 + 1];
    s.v0[2] = L[3 * i0 + 2];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j < k) {
            const int32_t ij = ids[j + 1];
#pragma unroll
            for (int c = 0; c < 3; ++c) s.e[j][c] = __fsub_rn(L[3 * ij + c], s.v0[c]);
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) s.e[j][c] = 0.0f;
        }
    }
}

// Offset p' = p - v0 = sum_{j>=1} (c_j/m) e_j of the sample with barycentric
// parts c (Lemma 1: lambda_j = c_j / m). `comp` holds c_0..c_k as bytes.
__device__ __forceinline__ void sample_offset(const Simplex& s, const uint8_t* comp, int k, float m,
                                              float& px, float& py, float& pz) {
    px = 0.0f;
    py = 0.0f;
    pz = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j < k) {
            const float w = __fdiv_rn(static_cast<float>(comp[j + 1]), m);
            px = __fmaf_rn(w, s.e[j][0], px);
            py = __fmaf_rn(w, s.e[j][1], py);
            pz = __fmaf_rn(w, s.e[j][2], pz);
        }
    }
}

// Offset p' = sum_{j>=1} lambda_j e_j of a sample given by its barycentric
// coordinates (lambda_0 is implied: p = v0 + p'). With lambda_j = fl(c_j/m)
// this is bit for bit the grid sample of sample_offset.
__device__ __forceinline__ void sample_offset_lambda(const Simplex& s, const float* lam, int k, float& px,
                                                     float& py, float& pz) {
    px = 0.0f;
    py = 0.0f;
    pz = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j < k) {
            const float w = lam[j + 1];
            px = __fmaf_rn(w, s.e[j][0], px);
            py = __fmaf_rn(w, s.e[j][1], py);
            pz = __fmaf_rn(w, s.e[j][2], pz);
        }
    }
}

// Squared distance from a sample offset to the nearest vertex of the simplex:
// u_p^2 = min_j |p - v_j|^2, an upper bound of d(p, X)^2 because v_j ∈ X.
__device__ __forceinline__ float vertex_bound_sq(const Simplex& s, int k, float px, float py, float pz) {
    float u = __fmaf_rn(px, px, __fmaf_rn(py, py, __fmul_rn(pz, pz)));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j < k) {
            const float dx = __fsub_rn(px, s.e[j][0]);
            const float dy = __fsub_rn(py, s.e[j][1]);
            const float dz = __fsub_rn(pz, s.e[j][2]);
            u = fminf(u, __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz))));
        }
    }
    return u;
}

// Cull box of a simplex, in cells: the bounding box of its samples enlarged by
// R = max_p u_p (inflated to cover FP32 rounding). Every sample's nearest
// point of X lies inside it.
struct CellBox {
    int32_t c0[3];
    int32_t n[3];
};

__device__ __forceinline__ CellBox cull_box(const GridView& g, const float v0[3], const float lo[3],
                                            const float hi[3], float R) {
    const float ax = fmaxf(fabsf(v0[0]), fmaxf(fabsf(v0[1]), fabsf(v0[2])));
    const float ext = fmaxf(fmaxf(fabsf(lo[0]), fabsf(hi[0])),
                            fmaxf(fmaxf(fabsf(lo[1]), fabsf(hi[1])), fmaxf(fabsf(lo[2]), fabsf(hi[2]))));
    const float pad = R * (1.0f + 1.0f / 65536.0f) + (ax + ext + R) * (1.0f / 262144.0f);
    CellBox b;
    const float o[3] = {g.ox, g.oy, g.oz};
    const int d[3] = {g.dx, g.dy, g.dz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float a = __fsub_rn(__fadd_rn(v0[c], lo[c]), pad);
        const float z = __fadd_rn(__fadd_rn(v0[c], hi[c]), pad);
        const int i0 = cell_coord(a, o[c], g.inv_cell, d[c]);
        const int i1 = cell_coord(z, o[c], g.inv_cell, d[c]);
        b.c0[c] = i0;
        b.n[c] = i1 - i0 + 1;
    }
    return b;
}

// Point range [begin, end) of row r of a cell box (rows run along x).
__device__ __forceinline__ void box_row(const GridView& g, const CellBox& b, int r, int32_t& begin,
                                        int32_t& end) {
    const int cy = b.c0[1] + r % b.n[1];
    const int cz = b.c0[2] + r / b.n[1];
    const int64_t base = (static_cast<int64_t>(cz) * g.dy + cy) * g.dx + b.c0[0];
    begin = g.cell_start[base];
    end = g.cell_start[base + b.n[0]];
}

// Exact nearest point of X to q, warp-collective: cull boxes of radius R,
// 2R, 4R, ... around q until the best squared distance found is within the
// box's radius (every point outside the box is farther) or the box covers the
// whole grid. Returns min over X of (d^2 bits << 32 | original row) with
// d = x - q per coordinate as in the flood kernels (ties to the lowest row),
// or ~0 if X were empty. At most 64 rounds (R doubles each round).
__device__ __forceinline__ unsigned long long warp_nearest(const GridView& g, float qx, float qy, float qz, float R,
                                                           int lane) {
    const float q[3] = {qx, qy, qz}, zero[3] = {0.0f, 0.0f, 0.0f};
    unsigned long long best = ~0ull;
    for (int it = 0; it < 64; ++it) {
        const CellBox b = cull_box(g, q, zero, zero, R);
        const int rows = b.n[1] * b.n[2];
        for (int r = 0; r < rows; ++r) {
            int32_t rb, re;
            box_row(g, b, r, rb, re);
            for (int32_t i = rb + lane; i < re; i += 32) {
                const float4 x = g.pts[i];
                const float dx = __fsub_rn(x.x, qx), dy = __fsub_rn(x.y, qy), dz = __fsub_rn(x.z, qz);
                const float d2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
                const unsigned long long key = (static_cast<unsigned long long>(__float_as_uint(d2)) << 32) |
                                               static_cast<uint32_t>(__float_as_int(x.w));
                best = key < best ? key : best;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
            best = y < best ? y : best;
        }
        const bool whole = b.c0[0] == 0 && b.c0[1] == 0 && b.c0[2] == 0 && b.n[0] == g.dx && b.n[1] == g.dy &&
                           b.n[2] == g.dz;
        if (best != ~0ull && (whole || __uint_as_float(static_cast<uint32_t>(best >> 32)) <= __fmul_rn(R, R)))
            break;
        R = __fmul_rn(R, 2.0f);
    }
    return best;
}

// Upper bound of d(p, X) from the simplex's vertices when they need not be
// points of X: min_j (|p - v_j| + d(v_j, X)) (triangle inequality), rounded
// up; vb[j] is d(v_j, X) rounded up (0 for a vertex that is a point of X).
__device__ __forceinline__ float vertex_bound_general(const Simplex& s, int k, float px, float py, float pz,
                                                      const float vb[4]) {
    float u = __fadd_ru(__fsqrt_ru(__fmaf_rn(px, px, __fmaf_rn(py, py, __fmul_rn(pz, pz)))), vb[0]);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j < k) {
            const float dx = __fsub_rn(px, s.e[j][0]);
            const float dy = __fsub_rn(py, s.e[j][1]);
            const float dz = __fsub_rn(pz, s.e[j][2]);
            u = fminf(u, __fadd_ru(__fsqrt_ru(__fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)))), vb[j + 1]));
        }
    }
    return __fmul_ru(u, 1.0f + 1.0f / 65536.0f);  // margin over the rounding of the distances
}

}  // namespace flood
