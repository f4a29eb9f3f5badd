// General ambient dimension d = 2..5: farthest point sampling, a d-dimensional
// cell grid and flood values of every simplex of Del(L) for clouds in R^d.
//
// §3 defines the Flood complex for any d; §5.3 studies how the runtime grows
// with d (Fig. 4c: swisscheese-like clouds, |X| = 1M, |L| = 1k, d = 2..5).
// The three-dimensional path (fps.cu, grid.cu, filtration.cu) is specialised
// for float4 (x, y, z, id) records and a 3-D block distance field; this path
// keeps d as a template parameter and trades those structures for ones that
// hold up when the number of simplices and samples grows steeply with d.
//
// FPS: one persistent cooperative kernel; each pick is one exchange of block
// maxima through tagged slots (two slot banks, alternating by pick parity).
// Keys are the binary32 squared distances summed left to right with every
// operation rounded (no contraction), ties to the lowest index.
//
// Flood values, per dimension k = 0..d (a dimension needs the final values of
// the one below, its facets):
//   resolve   one thread per (simplex, interior sample): the sample point, the
//             facet maximum LB, and an exact upper bound u from the nearest
//             points of the vertices. The sample cannot change the value once
//             its running nearest distance is <= LB (Lemma 2's argument with a
//             live bound instead of a ball), which is the usual outcome within
//             the sample's own cell and its 3^d - 1 neighbours, visited nearest
//             first (a lane that finishes takes the next item, so long and
//             short searches share warps); the rest either finish exactly
//             there or go to
//   fallback  one warp per remaining sample: Chebyshev shells of cells around
//             the sample, clipped to the grid, until the distance is exact or
//             falls to max(LB, the simplex's running maximum);
//   finalize  f = max(LB, sqrt(max exact sample distance)).
// Every skip and stop is decided with bounds rounded toward the safe side, so
// the value equals the maximum over the interior samples of the minimum over
// all of X of the rounded squared distance, whatever the cell size.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bbox.cuh"
#include "common.cuh"
#include "scan.cuh"

struct flood_grid_nd {
    int32_t d;
    int64_t n_points;
    int32_t cap_cells;
    float4* a4;           // coordinates 0..3 of the points in cell order (unused ones 0)
    float* a1;            // coordinate 4 (d = 5 only)
    int32_t* cell_start;  // cap_cells + 1 offsets into a4 / a1
    void* geom;           // NdGeom (device)
    cudaEvent_t ready;
    int64_t device_bytes;
};

namespace flood {
namespace {

constexpr int kNdMaxD = 5;
constexpr int kNdThreads = 256;
constexpr int kNdFpsThreads = 1024;  // one block per SM: the pick exchange reads one slot per SM
constexpr int64_t kNdChunk = int64_t(1) << 22;   // items per resolve launch (and fallback capacity)
constexpr float kOneMinus = 0.99999904632568359375f;  // 1 - 2^-20
constexpr double kNdPointsPerCell = 6.0;

// ---------------------------------------------------------------- constant tables
// Binomial coefficients C(n, r), n <= FLOOD_MAX_M + kNdMaxD, r <= kNdMaxD.
constexpr int kBinomN = FLOOD_MAX_M + kNdMaxD + 1;
struct Binom {
    uint32_t c[kBinomN][kNdMaxD + 1];
};
constexpr Binom make_binom() {
    Binom b{};
    for (int n = 0; n < kBinomN; ++n)
        for (int r = 0; r <= kNdMaxD; ++r)
            b.c[n][r] = r == 0 ? 1u : (n == 0 ? 0u : b.c[n - 1][r - 1] + b.c[n - 1][r]);
    return b;
}
__constant__ Binom c_binom = make_binom();

// Offsets of the cells of Chebyshev distance <= 1 from a cell in d dimensions,
// ordered by the number of non-zero components (own cell, face neighbours,
// edge neighbours, ...): roughly nearest first. Packed two bits per axis
// (offset + 1).
struct Ring1 {
    uint16_t o[243];
    int32_t n;
};
constexpr Ring1 make_ring1(int D) {
    Ring1 t{};
    int total = 1;
    for (int a = 0; a < D; ++a) total *= 3;
    int n = 0;
    for (int w = 0; w <= D; ++w)
        for (int code = 0; code < total; ++code) {
            int x = code, nz = 0;
            uint32_t packed = 0;
            for (int a = 0; a < D; ++a) {
                const int o = x % 3 - 1;
                x /= 3;
                nz += o != 0;
                packed |= static_cast<uint32_t>(o + 1) << (2 * a);
            }
            if (nz != w) continue;
            t.o[n++] = static_cast<uint16_t>(packed);
        }
    t.n = n;
    return t;
}
__constant__ Ring1 c_ring1[4] = {make_ring1(2), make_ring1(3), make_ring1(4), make_ring1(5)};

// ---------------------------------------------------------------- geometry
// Dense row-major cell table over the bounding box: cell (c_0..c_{d-1}) of
// edge h has lower corner lo + c h. A point goes to the cell of
// floor((x - lo) / h) evaluated in binary32 and clamped to the table; every
// point of cell c then lies within `slack` of the nominal box
// [lo + c h, lo + (c + 1) h] (slack covers the rounding of both the cell index
// and the box corners), and the first and last cell of an axis are open
// towards the outside.
struct NdGeom {
    float lo[kNdMaxD], hi[kNdMaxD];
    float h, inv_h, slack;
    int32_t dims[kNdMaxD];
    int32_t stride[kNdMaxD];
    int32_t n_cells;
    int32_t n_points;
};

__device__ __forceinline__ float corner(const NdGeom& g, int a, int c) {
    return __fmaf_rn(static_cast<float>(c), g.h, g.lo[a]);
}

template <int D>
__device__ __forceinline__ void cell_of(const NdGeom& g, const float (&p)[D], int (&c)[D]) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
        float t = __fmul_rn(__fsub_rn(p[a], g.lo[a]), g.inv_h);
        t = fminf(fmaxf(t, 0.0f), static_cast<float>(g.dims[a] - 1));
        c[a] = static_cast<int>(t);
    }
}

// Lower bound on the rounded squared distance from p to any point of cell c.
template <int D>
__device__ __forceinline__ float cell_bound(const NdGeom& g, const float (&p)[D], const int (&c)[D]) {
    float s = 0.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        float gap = 0.0f;
        if (c[a] > 0) gap = fmaxf(gap, __fsub_rd(__fsub_rd(corner(g, a, c[a]), g.slack), p[a]));
        if (c[a] < g.dims[a] - 1) gap = fmaxf(gap, __fsub_rd(p[a], __fadd_ru(corner(g, a, c[a] + 1), g.slack)));
        s = __fadd_rd(s, __fmul_rd(gap, gap));
    }
    return __fmul_rd(s, kOneMinus);
}

// Lower bound on the rounded squared distance from p to any point outside the
// cells within Chebyshev distance r of cell c (+inf if there are none).
template <int D>
__device__ __forceinline__ float ring_bound(const NdGeom& g, const float (&p)[D], const int (&c)[D], int r) {
    float gmin = INFINITY;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (c[a] - r > 0) gmin = fminf(gmin, fmaxf(0.0f, __fsub_rd(p[a], __fadd_ru(corner(g, a, c[a] - r), g.slack))));
        if (c[a] + r < g.dims[a] - 1)
            gmin = fminf(gmin, fmaxf(0.0f, __fsub_rd(__fsub_rd(corner(g, a, c[a] + r + 1), g.slack), p[a])));
    }
    if (gmin == INFINITY) return INFINITY;
    return __fmul_rd(__fmul_rd(gmin, gmin), kOneMinus);
}

// Rounded squared distance used for flood values (contracted, fixed order).
template <int D>
__device__ __forceinline__ float dist2(const float (&p)[D], float4 a, float b) {
    float dx = __fsub_rn(p[0], a.x);
    float acc = __fmul_rn(dx, dx);
    if (D > 1) {
        dx = __fsub_rn(p[1], a.y);
        acc = __fmaf_rn(dx, dx, acc);
    }
    if (D > 2) {
        dx = __fsub_rn(p[2], a.z);
        acc = __fmaf_rn(dx, dx, acc);
    }
    if (D > 3) {
        dx = __fsub_rn(p[3], a.w);
        acc = __fmaf_rn(dx, dx, acc);
    }
    if (D > 4) {
        dx = __fsub_rn(p[4], b);
        acc = __fmaf_rn(dx, dx, acc);
    }
    return acc;
}

// FPS key: binary32 squared distance, squares summed left to right, every
// operation rounded on its own (the same key as the three-dimensional FPS).
template <int D>
__device__ __forceinline__ float fps_key_nd(const float (&x)[D], const float (&l)[D]) {
    float d0 = __fsub_rn(x[0], l[0]);
    float acc = __fmul_rn(d0, d0);
#pragma unroll
    for (int a = 1; a < D; ++a) {
        const float da = __fsub_rn(x[a], l[a]);
        acc = __fadd_rn(acc, __fmul_rn(da, da));
    }
    return acc;
}

// Largest q >= 0 with sqrt(q) <= lb (sqrt correctly rounded, hence monotone):
// a sample whose squared distance is <= this cannot raise a value >= lb.
__device__ __forceinline__ float sq_threshold(float lb) {
    if (!(lb > 0.0f)) return 0.0f;
    float q = __fmul_rn(lb, lb);
    for (int i = 0; i < 8 && __fsqrt_rn(q) > lb; ++i) q = __uint_as_float(__float_as_uint(q) - 1u);
    for (int i = 0; i < 8; ++i) {
        const float nq = __uint_as_float(__float_as_uint(q) + 1u);
        if (!(__fsqrt_rn(nq) <= lb)) break;
        q = nq;
    }
    return q;
}

// Composition of rank j among the compositions of m into k+1 positive parts,
// in lexicographic order of (c_0, ..., c_k) (Lemma 1's interior grid).
__device__ __forceinline__ void unrank_interior(int64_t j, int m, int k, int (&c)[kNdMaxD + 1]) {
    int s = m - (k + 1);  // total above one per part
    for (int i = 0; i < k; ++i) {
        const int rest = k - i;  // parts after part i
        int v = 0;
        for (; v < s; ++v) {
            // completions with c_i = v + 1: the s - v extra units over `rest` parts
            const int64_t cnt = c_binom.c[s - v + rest - 1][rest - 1];
            if (j < cnt) break;
            j -= cnt;
        }
        c[i] = v + 1;
        s -= v;
    }
    c[k] = s + 1;
}

// lam[j][i] = c_i / m (binary32: c_i times the rounded reciprocal of m) for
// every interior composition j of m into k+1 parts.
__global__ void k_nd_lambda(float* lam, int64_t n, int m, int k) {
    const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (j >= n) return;
    int c[kNdMaxD + 1];
    unrank_interior(j, m, k, c);
    const float inv = __frcp_rn(static_cast<float>(m));
    for (int i = 0; i <= k; ++i) lam[j * (k + 1) + i] = __fmul_rn(static_cast<float>(c[i]), inv);
}

// ---------------------------------------------------------------- grid build
template <int D>
__global__ void __launch_bounds__(kBoxThreads) k_bbox_nd(const float* X, int64_t n, uint32_t* box, uint32_t* flags) {
    __shared__ uint32_t s_red[2 * kNdMaxD][kBoxThreads / 32];
    uint32_t mn[D], mx[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        mn[a] = 0xffffffffu;
        mx[a] = 0u;
    }
    bool bad = false;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const float v = X[D * i + a];
            if (!isfinite(v)) {
                bad = true;
                continue;
            }
            const uint32_t o = ordered_bits(v);
            mn[a] = min(mn[a], o);
            mx[a] = max(mx[a], o);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        mn[a] = __reduce_min_sync(0xffffffffu, mn[a]);
        mx[a] = __reduce_max_sync(0xffffffffu, mx[a]);
        if (lane == 0) {
            s_red[a][warp] = mn[a];
            s_red[kNdMaxD + a][warp] = mx[a];
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, FLAG_NONFINITE);
    __syncthreads();
    if (warp == 0) {
        const int w = lane % (kBoxThreads / 32);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const uint32_t lo = __reduce_min_sync(0xffffffffu, s_red[a][w]);
            const uint32_t hi = __reduce_max_sync(0xffffffffu, s_red[kNdMaxD + a][w]);
            if (lane == 0) {
                atomicMin(&box[a], lo);
                atomicMax(&box[kNdMaxD + a], hi);
            }
        }
    }
}

__global__ void k_box_init_nd(uint32_t* box, uint32_t* flags) {
    for (int a = 0; a < kNdMaxD; ++a) {
        box[a] = 0xffffffffu;
        box[kNdMaxD + a] = 0u;
    }
    *flags = 0;
}

// Cell edge and table dimensions, on the device (no readback). Without a
// requested edge, h targets about kNdPointsPerCell points per cell over the
// axes the cloud spans (a cloud flat along some axes gets one cell there); h
// grows until the table fits its capacity. (Measured on the swisscheese-like
// clouds of d = 2..5: about six points per cell is the fastest setting at
// every d; one per cell costs 1.3x-3x.)
template <int D>
__global__ void k_nd_geometry(const uint32_t* box, const uint32_t* flags, int64_t n, float cell_size, int32_t cap,
                              NdGeom* out) {
    NdGeom g{};
    float emax = 0.0f, amax = 0.0f;
    for (int a = 0; a < D; ++a) {
        g.lo[a] = *flags ? 0.0f : from_ordered(box[a]);
        g.hi[a] = *flags ? 0.0f : from_ordered(box[kNdMaxD + a]);
        emax = fmaxf(emax, g.hi[a] - g.lo[a]);
        amax = fmaxf(amax, fmaxf(fabsf(g.lo[a]), fabsf(g.hi[a])));
    }
    double h = cell_size;
    if (!(h > 0.0)) {
        double vol = 1.0;
        int deff = 0;
        for (int a = 0; a < D; ++a)
            if (double(g.hi[a]) - g.lo[a] > 1e-6 * emax) {
                vol *= double(g.hi[a]) - g.lo[a];
                ++deff;
            }
        h = deff ? pow(kNdPointsPerCell * vol / double(n), 1.0 / deff) : 1.0;
    }
    if (!(h > 0.0) || !isfinite(h)) h = emax > 0.0f ? emax : 1.0;
    float hf = static_cast<float>(h);
    for (int it = 0; it < 4096; ++it) {  // the table is sized with the binary32 edge it will use
        hf = static_cast<float>(h);
        double cells = 1.0;
        for (int a = 0; a < D; ++a) cells *= floor((double(g.hi[a]) - g.lo[a]) / double(hf)) + 1.0;
        if (cells <= double(cap)) break;
        h *= 1.1;
    }
    g.h = hf;
    g.inv_h = 1.0f / g.h;
    g.n_cells = 1;
    for (int a = 0; a < D; ++a) {
        const double e = double(g.hi[a]) - g.lo[a];
        g.dims[a] = static_cast<int32_t>(floor(e / double(g.h))) + 1;
        g.n_cells *= g.dims[a];
    }
    for (int a = D; a < kNdMaxD; ++a) g.dims[a] = 1;
    g.stride[D - 1] = 1;
    for (int a = D - 2; a >= 0; --a) g.stride[a] = g.stride[a + 1] * g.dims[a + 1];
    for (int a = D; a < kNdMaxD; ++a) g.stride[a] = 0;
    g.slack = ldexpf(amax + emax + g.h, -19);
    g.n_points = static_cast<int32_t>(n);
    *out = g;
}

template <int D>
__global__ void __launch_bounds__(kNdThreads) k_nd_cell_ids(const float* X, int64_t n, const NdGeom* geom,
                                                            int32_t* cell, int32_t* count, int32_t cap,
                                                            uint32_t* flags) {
    const int64_t i = blockIdx.x * int64_t(kNdThreads) + threadIdx.x;
    if (i >= n) return;
    const NdGeom& g = *geom;
    float p[D];
    int c[D];
#pragma unroll
    for (int a = 0; a < D; ++a) p[a] = X[D * i + a];
    cell_of<D>(g, p, c);
    int32_t id = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) id += c[a] * g.stride[a];
    if (id < 0 || id >= g.n_cells || id >= cap) {  // cannot happen for finite input
        atomicOr(flags, FLAG_INTERNAL);
        id = 0;
    }
    cell[i] = id;
    atomicAdd(&count[id], 1);
}

template <int D>
__global__ void __launch_bounds__(kNdThreads) k_nd_scatter(const float* X, int64_t n, const int32_t* cell,
                                                           const int32_t* start, int32_t* count, float4* a4,
                                                           float* a1, uint32_t* flags) {
    const int64_t i = blockIdx.x * int64_t(kNdThreads) + threadIdx.x;
    if (i >= n) return;
    const int32_t c = cell[i];
    const int64_t pos = start[c] + atomicSub(&count[c], 1) - 1;
    if (FLOOD_OOB(pos, n, flags)) return;
    const float* x = X + D * i;
    a4[pos] = make_float4(x[0], D > 1 ? x[1] : 0.0f, D > 2 ? x[2] : 0.0f, D > 3 ? x[3] : 0.0f);
    if (D > 4) a1[pos] = x[4];
}

// ---------------------------------------------------------------- FPS in d dimensions
// One block of 1024 threads per SM. Thread g of the G threads owns points
// g, g + G, g + 2G, ...: the first R of them live in registers (coordinates
// and current distance), the next E in the block's shared memory (one
// coordinate plane and a distance plane per row), and any further ones are
// read from X at every round with their distance in `dist`.
//
// Rounds: every thread folds the previous round's picks into its points'
// distances and keeps its best point (candidate word: key bits << 31 |
// (2^31 - 1 - index): the larger key, then the lower index) and its second
// key; each warp reduces to its best candidate and a bound on its other
// points. Warp 0 publishes the block's two best candidates with their
// coordinates and a bound U_b on every other point of the block (the larger
// of its third-best warp candidate and all warps' bounds) in tagged words.
// Warps 0..7 poll an eighth of the blocks each until every word carries the
// round's tag and keep its eight best candidates (the ninth joins that
// eighth's bound). Warp 0 then picks greedily: the best kept candidate
// (always the next FPS pick: no other point beats it), then, after lowering
// the other kept candidates' keys by it, the next best while its key stays
// positive and strictly above the largest bound (every point not kept has a
// key at most that bound, now and after any pick). Every block makes the
// same picks, bit for bit those of plain FPS. Points owned by threads spread
// over the whole cloud make the bounds low: at 1M points in R^5 a round
// makes about 18 picks.
// A slot word carries the round's tag r & 3 in its top bits; a block cannot
// publish round r + 2 (same parity bank) before every block has finished
// reading round r + 1.
struct NdFpsArgs {
    const float* X;
    int64_t n;
    int32_t n_landmarks;
    int64_t start;
    int64_t* out_idx;
    float* out_key;
    float* dist;      // distances of the points beyond the register and shared tiers
    uint64_t* slots;  // [2][kNdFpsMaxBlocks][kNdSlotWords]
    uint32_t* flags;
    uint32_t poll_limit;
    int32_t shared_rows;  // E
};

constexpr int kNdFpsMaxBlocks = 160;
constexpr int kNdPollers = 8;                                // warps 0..7 poll
constexpr int kNdQuarter = kNdFpsMaxBlocks / kNdPollers;     // blocks per poller warp
constexpr int kNdTop = 2;                                    // candidates a block publishes
constexpr int kNdKeep = 8;                                   // candidates a poller keeps
constexpr int kNdEntryWords = 8;                             // cand, up to 5 coordinates, padding
constexpr int kNdSlotWords = kNdTop * kNdEntryWords;         // 128 bytes per block and bank
constexpr int kNdMaxPicks = 32;
constexpr int kNdPairs = (kNdQuarter * kNdTop + 31) / 32;    // (block, entry) pairs per poller lane
static_assert(kNdPollers * kNdKeep == 64, "warp 0 merges two kept candidates per lane");
constexpr uint64_t kNdCandMask = (uint64_t(1) << 62) - 1;

__device__ __forceinline__ uint64_t nd_cand(float key, int64_t i) {
    return (static_cast<uint64_t>(__float_as_uint(key) & 0x7fffffffu) << 31) |
           static_cast<uint64_t>(0x7fffffffu - static_cast<uint32_t>(i));
}
__device__ __forceinline__ float nd_cand_key(uint64_t c) {
    return __uint_as_float(static_cast<uint32_t>(c >> 31) & 0x7fffffffu);
}
__device__ __forceinline__ int64_t nd_cand_row(uint64_t c) {
    return static_cast<int64_t>(0x7fffffffu - static_cast<uint32_t>(c & 0x7fffffffu));
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
    const uint32_t hi = static_cast<uint32_t>(v >> 32);
    const uint32_t mh = __reduce_max_sync(0xffffffffu, hi);
    const uint32_t ml = __reduce_max_sync(0xffffffffu, hi == mh ? static_cast<uint32_t>(v) : 0u);
    return (static_cast<uint64_t>(mh) << 32) | ml;
}

__device__ __forceinline__ float warp_max_key(float v) {  // values >= -1: through the order-preserving bits
    return from_ordered(__reduce_max_sync(0xffffffffu, ordered_bits(v)));
}

// 30-bit code of a bound, rounded up (decodes to a bound again).
__device__ __forceinline__ uint32_t nd_up30(float v) {
    const uint32_t u = ordered_bits(v);
    return (u > 0xfffffffcu ? 0xffffffffu : (u + 3u) & ~3u) >> 2;
}
__device__ __forceinline__ float nd_from30(uint32_t c) { return from_ordered(c << 2); }

__device__ __forceinline__ void bar_sync_n(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Poller warp h: blocks [h kNdQuarter, (h + 1) kNdQuarter) of round r's bank,
// until every word carries the round's tag. Its kNdKeep best candidates and
// their coordinates go to qc / qx, its bound on every other point of those
// blocks to *qb. Returns false if the wait gave up.
template <int D>
__device__ __forceinline__ bool nd_poll(const NdFpsArgs& a, int r, int h, int lane, int B, uint64_t* qc,
                                        float (*qx)[D], float* qb) {
    const uint64_t tag = static_cast<uint64_t>(r & 3) << 62;
    const uint64_t* bank = a.slots + static_cast<size_t>(r & 1) * kNdFpsMaxBlocks * kNdSlotWords;
    uint64_t c[kNdPairs];
    uint32_t u[kNdPairs];
    float x[kNdPairs][D];
    bool ok = false;
    for (uint32_t polls = 0; polls < a.poll_limit; ++polls) {
        bool fresh = true;
#pragma unroll
        for (int q = 0; q < kNdPairs; ++q) {
            const int pr = lane + 32 * q, b = h * kNdQuarter + pr / kNdTop, e = pr % kNdTop;
            c[q] = 0ull;
            u[q] = nd_up30(-1.0f);
#pragma unroll
            for (int k = 0; k < D; ++k) x[q][k] = 0.0f;
            if (pr >= kNdQuarter * kNdTop || b >= B) continue;
            const uint64_t* ew = bank + static_cast<size_t>(b) * kNdSlotWords + e * kNdEntryWords;
            uint64_t w[kNdEntryWords];
            ld_relaxed_v4_u64(ew, w[0], w[1], w[2], w[3]);
            ld_relaxed_v4_u64(ew + 4, w[4], w[5], w[6], w[7]);
            uint64_t stale = 0ull;
#pragma unroll
            for (int k = 0; k < kNdEntryWords; ++k) stale |= w[k] ^ tag;
            fresh = fresh && (stale >> 62) == 0ull;
            c[q] = w[0] & kNdCandMask;
            if (e == 0) u[q] = static_cast<uint32_t>(w[1] >> 32) & 0x3fffffffu;
#pragma unroll
            for (int k = 0; k < D; ++k) x[q][k] = __uint_as_float(static_cast<uint32_t>(w[1 + k]));
        }
        if (__all_sync(0xffffffffu, fresh)) {
            ok = true;
            break;
        }
    }
    uint32_t ub = 0u;
#pragma unroll
    for (int q = 0; q < kNdPairs; ++q) ub = max(ub, u[q]);
    ub = __reduce_max_sync(0xffffffffu, ub);
#pragma unroll 1
    for (int k = 0; k <= kNdKeep; ++k) {
        uint64_t v = 0ull;
        int vq = 0;
#pragma unroll
        for (int q = 0; q < kNdPairs; ++q)
            if (c[q] > v) {
                v = c[q];
                vq = q;
            }
        const uint64_t m = warp_max_u64(v);
        if (k == kNdKeep) {  // the best candidate left out joins the bound
            if (lane == 0) *qb = fmaxf(nd_from30(ub), m ? nd_cand_key(m) : -1.0f);
            break;
        }
        const int owner = __ffs(__ballot_sync(0xffffffffu, v == m)) - 1;
        if (lane == owner) {
            qc[k] = m;
#pragma unroll
            for (int q = 0; q < kNdPairs; ++q)
                if (q == vq) {
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) qx[k][kk] = x[q][kk];
                    c[q] = 0ull;
                }
        }
    }
    return ok;
}

template <int D, int R>
__global__ void __launch_bounds__(kNdFpsThreads, 1) k_fps_nd(NdFpsArgs a) {
    extern __shared__ float s_rows[];  // [E][D + 1][kNdFpsThreads]: coordinates, then distance
    __shared__ uint64_t s_wc[kNdFpsThreads / 32];     // each warp's best candidate ...
    __shared__ float s_wx[kNdFpsThreads / 32][D];     // ... its coordinates
    __shared__ float s_ws[kNdFpsThreads / 32];        // ... and the bound on the warp's other points
    __shared__ uint64_t s_qc[kNdPollers][kNdKeep];    // kept candidates of each poller
    __shared__ float s_qx[kNdPollers][kNdKeep][D];
    __shared__ float s_qb[kNdPollers];
    __shared__ int s_qok[kNdPollers];
    __shared__ uint64_t s_pc[kNdMaxPicks];            // the round's picks: candidate words ...
    __shared__ float s_pick[kNdMaxPicks][D];          // ... and coordinates
    __shared__ int s_np;                              // picks of the round; <= 0: stop
    if (*a.flags) return;  // input rejected (non-finite coordinates): every block leaves at once
    const int64_t G = int64_t(gridDim.x) * kNdFpsThreads;
    const int64_t g = blockIdx.x * int64_t(kNdFpsThreads) + threadIdx.x;
    const int B = gridDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int E = a.shared_rows;
    float px[R][D], pd[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = g + r * G;
        pd[r] = INFINITY;
#pragma unroll
        for (int c = 0; c < D; ++c) px[r][c] = i < a.n ? a.X[D * i + c] : 0.0f;
    }
    for (int e = 0; e < E; ++e) {
        const int64_t i = g + (R + e) * G;
        float* row = s_rows + size_t(e) * (D + 1) * kNdFpsThreads + threadIdx.x;
#pragma unroll
        for (int c = 0; c < D; ++c) row[c * kNdFpsThreads] = i < a.n ? a.X[D * i + c] : 0.0f;
        row[D * kNdFpsThreads] = INFINITY;
    }
    if (g == 0) {
        a.out_idx[0] = a.start;
        if (a.out_key) a.out_key[0] = INFINITY;
    }
    if (a.n_landmarks <= 1) return;  // the start point is the only pick
    if (threadIdx.x == 0) {
        s_np = 1;  // the start point is the pick the first round folds
#pragma unroll
        for (int c = 0; c < D; ++c) s_pick[0][c] = a.X[D * a.start + c];
    }
    __syncthreads();
    int j = 1;  // picks recorded
    for (int r = 1;; ++r) {
        const int np = s_np;
        // ---- fold the picks; this thread's best candidate (with coordinates) and second key
        uint64_t best = 0ull;
        float second = -1.0f, bx[D];
#pragma unroll
        for (int c = 0; c < D; ++c) bx[c] = 0.0f;
        auto consider = [&](float v, int64_t i, const float(&x)[D]) {
            const uint64_t pk = nd_cand(v, i);
            if (pk > best) {
                second = fmaxf(second, best ? nd_cand_key(best) : -1.0f);
                best = pk;
#pragma unroll
                for (int c = 0; c < D; ++c) bx[c] = x[c];
            } else {
                second = fmaxf(second, v);
            }
        };
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int64_t i = g + q * G;
            if (i < a.n) {
                for (int t = 0; t < np; ++t) pd[q] = fminf(pd[q], fps_key_nd<D>(px[q], s_pick[t]));
                consider(pd[q], i, px[q]);
            }
        }
        for (int e = 0; e < E; ++e) {
            const int64_t i = g + (R + e) * G;
            if (i >= a.n) break;
            float* row = s_rows + size_t(e) * (D + 1) * kNdFpsThreads + threadIdx.x;
            float x[D];
#pragma unroll
            for (int c = 0; c < D; ++c) x[c] = row[c * kNdFpsThreads];
            float d = row[D * kNdFpsThreads];
            for (int t = 0; t < np; ++t) d = fminf(d, fps_key_nd<D>(x, s_pick[t]));
            row[D * kNdFpsThreads] = d;
            consider(d, i, x);
        }
        for (int64_t i = g + (R + E) * G; i < a.n; i += G) {
            float x[D];
#pragma unroll
            for (int c = 0; c < D; ++c) x[c] = a.X[D * i + c];
            float d = r == 1 ? INFINITY : a.dist[i];
            for (int t = 0; t < np; ++t) d = fminf(d, fps_key_nd<D>(x, s_pick[t]));
            a.dist[i] = d;
            consider(d, i, x);
        }
        const uint64_t wb = warp_max_u64(best);
        const int wo = __ffs(__ballot_sync(0xffffffffu, best == wb)) - 1;
        const float ws = warp_max_key(lane == wo ? second : (best ? nd_cand_key(best) : -1.0f));
        if (lane == wo) {
            s_wc[warp] = wb;
#pragma unroll
            for (int c = 0; c < D; ++c) s_wx[warp][c] = bx[c];
        }
        if (lane == 0) s_ws[warp] = ws;
        __syncthreads();
        // ---- warp 0: the block's two best candidates and the bound on its other points, published
        if (warp == 0) {
            const uint64_t c = s_wc[lane];
            const uint64_t m1 = warp_max_u64(c);
            const int o1 = __ffs(__ballot_sync(0xffffffffu, c == m1)) - 1;
            const uint64_t c2 = lane == o1 ? 0ull : c;
            const uint64_t m2 = warp_max_u64(c2);
            const int o2 = __ffs(__ballot_sync(0xffffffffu, c2 == m2)) - 1;
            const uint64_t m3 = warp_max_u64(lane == o1 || lane == o2 ? 0ull : c);
            const float ub = fmaxf(m3 ? nd_cand_key(m3) : -1.0f, warp_max_key(s_ws[lane]));
            if (lane < kNdTop) {
                const uint64_t tag = static_cast<uint64_t>(r & 3) << 62;
                uint64_t* ew = a.slots + static_cast<size_t>(r & 1) * kNdFpsMaxBlocks * kNdSlotWords +
                               static_cast<size_t>(blockIdx.x) * kNdSlotWords + lane * kNdEntryWords;
                const int o = lane == 0 ? o1 : o2;
                uint64_t w[kNdEntryWords];
                w[0] = tag | (lane == 0 ? m1 : m2);
#pragma unroll
                for (int k = 1; k < kNdEntryWords; ++k) w[k] = tag;
#pragma unroll
                for (int k = 0; k < D; ++k) w[1 + k] |= __float_as_uint(s_wx[o][k]);
                if (lane == 0) w[1] |= static_cast<uint64_t>(nd_up30(ub)) << 32;
                st_relaxed_v4_u64(ew, w[0], w[1], w[2], w[3]);
                st_relaxed_v4_u64(ew + 4, w[4], w[5], w[6], w[7]);
            }
        }
        // ---- warps 0..7: poll; warp 0 merges and picks
        if (warp < kNdPollers) {
            bar_sync_n(1, kNdPollers * 32);  // warp 0 has published
            const bool ok = nd_poll<D>(a, r, warp, lane, B, s_qc[warp], s_qx[warp], &s_qb[warp]);
            if (lane == 0) s_qok[warp] = ok;
            bar_sync_n(2, kNdPollers * 32);
        }
        if (warp == 0) {
            // lane l holds kept candidates l and l + 32 (candidate e is entry e % kNdKeep of poller e / kNdKeep)
            const int h0 = lane / kNdKeep, h1 = (lane + 32) / kNdKeep, kk = lane % kNdKeep;
            const uint64_t me0 = s_qc[h0][kk], me1 = s_qc[h1][kk];
            float x0[D], x1[D];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                x0[c] = s_qx[h0][kk][c];
                x1[c] = s_qx[h1][kk][c];
            }
            float U = -1.0f;
            bool ok = true;
#pragma unroll
            for (int h = 0; h < kNdPollers; ++h) {
                U = fmaxf(U, s_qb[h]);
                ok = ok && s_qok[h];
            }
            const int cap = min(a.n_landmarks - j, kNdMaxPicks);
            const int64_t row0 = nd_cand_row(me0), row1 = nd_cand_row(me1);
            float cur0 = nd_cand_key(me0), cur1 = nd_cand_key(me1);
            bool live0 = me0 != 0ull, live1 = me1 != 0ull;
            int n = 0;
            while (n < cap) {
                const uint64_t wa = live0 ? nd_cand(cur0, row0) : 0ull;  // non-zero for every live candidate
                const uint64_t wq = live1 ? nd_cand(cur1, row1) : 0ull;
                const uint64_t w = wa > wq ? wa : wq;
                const uint64_t mw = warp_max_u64(w);
                if (mw == 0ull) {  // nothing left: with no pick at all, the points have run out
                    if (n == 0) {
                        if (lane == 0) s_pc[0] = 0ull;
                        n = 1;
                    }
                    break;
                }
                const float mk = nd_cand_key(mw);
                if (n > 0 && !(mk > 0.0f && mk > U)) break;
                const int o = __ffs(__ballot_sync(0xffffffffu, w == mw)) - 1;
                const bool sec = wq == mw;  // (on lane o)
                float qv[D];
#pragma unroll
                for (int c = 0; c < D; ++c) qv[c] = __shfl_sync(0xffffffffu, sec ? x1[c] : x0[c], o);
                if (lane == o) {
                    s_pc[n] = mw;
#pragma unroll
                    for (int c = 0; c < D; ++c) s_pick[n][c] = qv[c];
                    if (sec)
                        live1 = false;
                    else
                        live0 = false;
                }
                ++n;
                cur0 = fminf(cur0, fps_key_nd<D>(x0, qv));
                cur1 = fminf(cur1, fps_key_nd<D>(x1, qv));
            }
            __syncwarp();
            const uint64_t first = s_pc[0];
            const bool degenerate = first == 0ull || !(nd_cand_key(first) > 0.0f);
            if (lane == 0) {
                if (!ok) atomicOr(a.flags, FLAG_TIMEOUT);
                if (ok && degenerate && blockIdx.x == 0) atomicOr(a.flags, FLAG_DEGENERATE);
                s_np = ok && !degenerate ? n : -1;
            }
            if (ok && !degenerate && blockIdx.x == 0 && lane < n) {
                const uint64_t pc = s_pc[lane];
                a.out_idx[j + lane] = nd_cand_row(pc);
                if (a.out_key) a.out_key[j + lane] = nd_cand_key(pc);
            }
        }
        __syncthreads();
        const int nn = s_np;
        if (nn <= 0) return;  // a wait gave up, or the points ran out: the status reports it
        j += nn;
        if (j >= a.n_landmarks) return;
    }
}

// ---------------------------------------------------------------- flood values in d dimensions
struct NdFilt {
    const NdGeom* geom;
    const float4* a4;
    const float* a1;
    const int32_t* cs;      // cell_start
    const float* L;
    int32_t n_L;
    const int32_t* simp;    // (n, k+1) vertex ids (NULL for k = 0)
    const int32_t* fac;     // (n, k+1) facet rows, k >= 2
    int64_t n;              // simplices of this dimension
    int64_t n_lower;        // simplices of dimension k-1 (range of facet rows)
    int32_t k, m;
    int64_t I;              // interior samples per simplex (1 for k = 0)
    const float* lower;     // values of dimension k-1 (vertex values for k = 1)
    const int32_t* vnn;     // per vertex: cell-order position of a nearest point of X
    int32_t* vnn_out;       // k = 0: written
    uint32_t* qmax;         // per simplex: bits of the largest exact sample distance^2 that mattered
    float* values;          // per simplex: output
    int64_t item0, n_items; // this launch's items [item0, item0 + n_items)
    uint4* fb;              // fallback items: (item lo, item hi, best bits, position)
    uint32_t* fb_count;
    uint32_t fb_cap;        // capacity of fb
    unsigned long long* next;  // items of this launch handed out so far (first pass)
    const float* lam;       // (I, k+1) barycentric weights c_i / m of the interior samples
    unsigned long long* stats;  // kNdStats counters of this dimension
    uint32_t* flags;
};

// Work counters of one dimension (flood_nd_stats).
enum : int {
    ST_ITEMS = 0,       // (simplex, interior sample) items
    ST_PRUNED,          // settled by the vertices' nearest points alone (u <= LB)
    ST_RESOLVED,        // settled (<= LB) within the 3^d cells around the sample
    ST_EXACT,           // exact within those cells
    ST_FALLBACK,        // handed to the shell search
    ST_PAIRS,           // (sample, point) distances evaluated, first pass
    ST_PAIRS_FB,        // (sample, point) distances evaluated, shell search
    ST_CELLS,           // cells whose points were read
    kNdStats
};

// Point, facet bound and vertex bound of one item. Returns false (and raises
// a flag) if an id is out of range or a coordinate is not finite.
template <int D>
__device__ __forceinline__ bool nd_item(const NdFilt& f, int64_t item, int64_t& s, float (&p)[D], float& lb,
                                        float& u) {
    s = item / f.I;
    const int64_t j = item - s * f.I;
    lb = 0.0f;
    u = INFINITY;
    if (f.k == 0) {
        if (s >= f.n_L) return false;
#pragma unroll
        for (int a = 0; a < D; ++a) p[a] = f.L[D * s + a];
    } else {
        const float* lw = f.lam + j * (f.k + 1);
        int32_t v[kNdMaxD + 1];
        for (int i = 0; i <= f.k; ++i) {
            v[i] = f.simp[s * (f.k + 1) + i];
            if (v[i] < 0 || v[i] >= f.n_L) {
                atomicOr(f.flags, FLAG_RANGE);
                return false;
            }
        }
#pragma unroll
        for (int a = 0; a < D; ++a) p[a] = 0.0f;
        for (int i = 0; i <= f.k; ++i) {
            const float lam = __ldg(lw + i);
#pragma unroll
            for (int a = 0; a < D; ++a) p[a] = __fmaf_rn(lam, f.L[D * v[i] + a], p[a]);
        }
        // facet maximum: the vertices' values for an edge, else the facets' values
        if (f.k == 1) {
            lb = fmaxf(f.lower[v[0]], f.lower[v[1]]);
        } else {
            for (int i = 0; i <= f.k; ++i) {
                const int32_t t = f.fac[s * (f.k + 1) + i];
                if (t < 0 || t >= f.n_lower) {
                    atomicOr(f.flags, FLAG_RANGE);
                    return false;
                }
                lb = fmaxf(lb, f.lower[t]);
            }
        }
        // exact upper bound: the distance to a nearest point of each vertex is one of the candidates
        for (int i = 0; i <= f.k; ++i) {
            const int32_t q = f.vnn[v[i]];
            if (FLOOD_OOB(q, f.geom->n_points, f.flags)) return false;
            u = fminf(u, dist2<D>(p, f.a4[q], D > 4 ? f.a1[q] : 0.0f));
        }
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
        if (!isfinite(p[a])) {
            atomicOr(f.flags, FLAG_NONFINITE);
            return false;
        }
    return true;
}

// Scan the points of one cell: running minimum (and its position). Stops
// early once best <= T (the item is settled; the rest of the cell cannot
// matter); T = -1 scans the whole cell.
template <int D, bool kVertex>
__device__ __forceinline__ void scan_cell(const NdFilt& f, const float (&p)[D], int32_t cell, float& best,
                                          int32_t& pos, uint32_t& pairs, float T = -1.0f) {
    if (FLOOD_OOB(cell, f.geom->n_cells, f.flags)) return;
    const int32_t s0 = __ldg(f.cs + cell), s1 = __ldg(f.cs + cell + 1);
    int32_t i = s0;
    for (; i + 1 < s1; i += 2) {  // two independent loads in flight
        const float4 r0 = __ldg(f.a4 + i), r1 = __ldg(f.a4 + i + 1);
        const float e0 = D > 4 ? __ldg(f.a1 + i) : 0.0f, e1 = D > 4 ? __ldg(f.a1 + i + 1) : 0.0f;
        const float d0 = dist2<D>(p, r0, e0), d1 = dist2<D>(p, r1, e1);
        if (d0 < best) {
            best = d0;
            if (kVertex) pos = i;
        }
        if (d1 < best) {
            best = d1;
            if (kVertex) pos = i + 1;
        }
        if (best <= T) {
            pairs += static_cast<uint32_t>(i + 2 - s0);
            return;
        }
    }
    if (i < s1) {
        const float d = dist2<D>(p, __ldg(f.a4 + i), D > 4 ? __ldg(f.a1 + i) : 0.0f);
        if (d < best) {
            best = d;
            if (kVertex) pos = i;
        }
    }
    pairs += static_cast<uint32_t>(s1 - s0);
}

__device__ __forceinline__ void add_stats(const NdFilt& f, const uint32_t (&st)[kNdStats]) {
    __shared__ unsigned long long s_st[kNdStats];
    if (threadIdx.x < kNdStats) s_st[threadIdx.x] = 0ull;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kNdStats; ++i) {
        unsigned long long v = st[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);  // per-warp sums fit easily
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_st[i], v);
    }
    __syncthreads();
    if (threadIdx.x < kNdStats && s_st[threadIdx.x]) atomicAdd(&f.stats[threadIdx.x], s_st[threadIdx.x]);
}

// Exact squared distance of an item: vertices record it with the nearest
// point's position; higher simplices keep the largest per simplex.
template <bool kVertex>
__device__ __forceinline__ void settle(const NdFilt& f, int64_t s, float best, int32_t pos) {
    if (kVertex) {
        f.qmax[s] = __float_as_uint(best);
        f.vnn_out[s] = pos;
    } else {
        atomicMax(f.qmax + s, __float_as_uint(best));
    }
}

// First pass. Items differ a lot in how many cells they need, so a lane does
// not keep one item to the end while the others wait: every lane holds one
// item at a time and the warp advances all of them by one Ring1 entry per
// iteration. When at least half of the lanes are idle (or all are), the idle
// ones take the next items of the warp's share (kPool consecutive items at a
// time from the launch's counter: consecutive samples of a simplex, whose
// data then comes from L1), so most iterations run with most lanes busy.
// An item settles when its distance falls to T (it cannot raise the value),
// or is exact when the 3^d cells around its cell hold a point nearer than
// anything outside them; the rest go to the shell search (fallback).
constexpr int kPool = 64;

template <int D, bool kVertex>
__global__ void __launch_bounds__(kNdThreads) k_nd_resolve(NdFilt f) {
    __shared__ uint16_t s_off[243];
    const Ring1& R = c_ring1[D - 2];
    for (int t = threadIdx.x; t < R.n; t += blockDim.x) s_off[t] = R.o[t];
    __syncthreads();
    const int n_off = R.n;
    const NdGeom& g = *f.geom;
    const int lane = threadIdx.x & 31;
    uint32_t st[kNdStats] = {};
    uint32_t pairs = 0;
    // this lane's item
    bool have = false;
    int64_t item = 0, s = 0;
    float p[D], gm2[D], gp2[D];
    int c[D];
    int32_t cell0 = 0, pos = 0;
    float T = 0.0f, best = INFINITY;
    int t = 0;
    // the warp's share of the launch's items
    int64_t pool = 0, pool_end = 0;
    bool exhausted = false;
    for (;;) {
        unsigned need = __ballot_sync(0xffffffffu, !have);
        if (!exhausted && (__popc(need) >= 16 || need == 0xffffffffu)) {
            while (need && !exhausted) {
                if (pool >= pool_end) {
                    unsigned long long b0 = 0;
                    if (lane == 0) b0 = atomicAdd(f.next, static_cast<unsigned long long>(kPool));
                    b0 = __shfl_sync(0xffffffffu, b0, 0);
                    if (b0 >= static_cast<unsigned long long>(f.n_items)) {
                        exhausted = true;
                        break;
                    }
                    pool = static_cast<int64_t>(b0);
                    pool_end = std::min<int64_t>(pool + kPool, f.n_items);
                }
                const int take = min(__popc(need), static_cast<int>(pool_end - pool));
                const int rank = __popc(need & ((1u << lane) - 1u));
                if (!have && rank < take) {
                    float lb, u;
                    item = f.item0 + pool + rank;
                    if (nd_item<D>(f, item, s, p, lb, u)) {
                        ++st[ST_ITEMS];
                        T = sq_threshold(lb);
                        best = u;
                        if (!kVertex && best <= T) {
                            ++st[ST_PRUNED];
                        } else {
                            cell_of<D>(g, p, c);
                            cell0 = 0;
#pragma unroll
                            for (int a = 0; a < D; ++a) {
                                cell0 += c[a] * g.stride[a];
                                // gaps to the lower and upper face of the own cell (the neighbours' near faces)
                                const float lo = fmaxf(0.0f, __fsub_rd(p[a], __fadd_ru(corner(g, a, c[a]), g.slack)));
                                const float hi =
                                    fmaxf(0.0f, __fsub_rd(__fsub_rd(corner(g, a, c[a] + 1), g.slack), p[a]));
                                gm2[a] = __fmul_rd(lo, lo);
                                gp2[a] = __fmul_rd(hi, hi);
                            }
                            pos = 0;
                            t = 0;
                            have = true;
                        }
                    }
                }
                pool += take;
                need = __ballot_sync(0xffffffffu, !have);
            }
        }
        if (!__any_sync(0xffffffffu, have)) {
            if (exhausted) break;
            continue;
        }
        if (!have) continue;
        if (t < n_off) {
            const uint32_t w = s_off[t++];
            bool inside = true;
            int32_t cell = cell0;
            float b = 0.0f;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const int o = static_cast<int>((w >> (2 * a)) & 3u) - 1;
                const int cc = c[a] + o;
                inside = inside && cc >= 0 && cc < g.dims[a];
                cell += o * g.stride[a];
                b = o < 0 ? __fadd_rd(b, gm2[a]) : (o > 0 ? __fadd_rd(b, gp2[a]) : b);
            }
            if (inside && __fmul_rd(b, kOneMinus) < best) {
                scan_cell<D, kVertex>(f, p, cell, best, pos, pairs, T);
                ++st[ST_CELLS];
                if (best <= T) {
                    ++st[ST_RESOLVED];
                    if (kVertex) settle<true>(f, s, best, pos);
                    have = false;
                }
            }
        } else {
            if (best <= ring_bound<D>(g, p, c, 1)) {
                ++st[ST_EXACT];
                settle<kVertex>(f, s, best, pos);
            } else {
                ++st[ST_FALLBACK];
                const uint32_t slot = atomicAdd(f.fb_count, 1u);
                if (slot < f.fb_cap)
                    f.fb[slot] = make_uint4(static_cast<uint32_t>(item), static_cast<uint32_t>(item >> 32),
                                            __float_as_uint(best), static_cast<uint32_t>(pos));
                else
                    atomicOr(f.flags, FLAG_INTERNAL);
            }
            have = false;
        }
    }
    st[ST_PAIRS] = pairs;
    add_stats(f, st);
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t w = shfl_xor_u64(v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Cells at Chebyshev distance exactly r from c, clipped to the table:
// enumerated as the cells of the clipped outer box [c - r, c + r] outside the
// clipped inner box [c - r + 1, c + r - 1], split by the first axis on which a
// cell leaves the inner box.
template <int D>
struct Shell {
    int lo[D], len[D];     // clipped outer box per axis
    int ilo[D], ilen[D];   // clipped inner box per axis
    int side[D][2];        // outer values that are not inner (c - r, c + r when inside the table)
    int nside[D];
    int64_t part[D];       // cells whose first non-inner axis is a
    int64_t total;
    __device__ void init(const NdGeom& g, const int (&c)[D], int r) {
        total = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int o0 = max(0, c[a] - r), o1 = min(g.dims[a] - 1, c[a] + r);
            const int i0 = max(0, c[a] - r + 1), i1 = min(g.dims[a] - 1, c[a] + r - 1);
            lo[a] = o0;
            len[a] = o1 - o0 + 1;
            ilo[a] = i0;
            ilen[a] = i1 - i0 + 1;
            nside[a] = 0;
            if (c[a] - r >= 0) side[a][nside[a]++] = c[a] - r;
            if (c[a] + r <= g.dims[a] - 1) side[a][nside[a]++] = c[a] + r;
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            int64_t n = nside[a];
            for (int b = 0; b < a; ++b) n *= ilen[b];
            for (int b = a + 1; b < D; ++b) n *= len[b];
            part[a] = n;
            total += n;
        }
    }
    __device__ void cell(int64_t t, int (&cc)[D]) const {
        int a = 0;
        while (a < D - 1 && t >= part[a]) {
            t -= part[a];
            ++a;
        }
        // mixed radix, last axis fastest: axes > a over the outer box, axis a over its sides, axes < a inner
        for (int b = D - 1; b > a; --b) {
            cc[b] = lo[b] + static_cast<int>(t % len[b]);
            t /= len[b];
        }
        cc[a] = side[a][static_cast<int>(t % nside[a])];
        t /= nside[a];
        for (int b = a - 1; b >= 0; --b) {
            cc[b] = ilo[b] + static_cast<int>(t % ilen[b]);
            t /= ilen[b];
        }
    }
};

// Second pass: one warp per item left by the first, shells r = 2, 3, ... of
// cells around the sample's cell, 32 cells at a time, the lanes' minima merged
// after every batch. Stops when the distance is exact (the next shell cannot
// hold anything closer) or cannot raise the value (<= max(LB, the simplex's
// running maximum), re-read after each shell).
template <int D, bool kVertex>
__global__ void __launch_bounds__(kNdThreads) k_nd_fallback(NdFilt f) {
    uint32_t st[kNdStats] = {};
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (kNdThreads / 32);
    const uint32_t n = min(*f.fb_count, f.fb_cap);
    const NdGeom& g = *f.geom;
    uint32_t pairs = 0, cells = 0;
    for (int64_t e = blockIdx.x * int64_t(kNdThreads / 32) + (threadIdx.x >> 5); e < n; e += warps) {
        const uint4 it = f.fb[e];
        const int64_t item = static_cast<int64_t>(it.x) | (static_cast<int64_t>(it.y) << 32);
        int64_t s;
        float p[D], lb, u;
        if (!nd_item<D>(f, item, s, p, lb, u)) continue;  // same outcome on every lane
        const float T = sq_threshold(lb);
        // (distance bits << 32 | position): the minimum is the smallest distance, then the lowest position
        uint64_t best = (static_cast<uint64_t>(it.z) << 32) | it.w;
        int c[D];
        cell_of<D>(g, p, c);
        float stop = T;
        if (!kVertex) stop = fmaxf(T, __uint_as_float(*reinterpret_cast<volatile uint32_t*>(f.qmax + s)));
        for (int r = 2;; ++r) {
            const float rb = ring_bound<D>(g, p, c, r - 1);
            if (__uint_as_float(static_cast<uint32_t>(best >> 32)) <= rb) {  // exact already
                if (lane == 0) settle<kVertex>(f, s, __uint_as_float(static_cast<uint32_t>(best >> 32)),
                                               static_cast<int32_t>(best & 0xffffffffu));
                break;
            }
            Shell<D> sh;
            sh.init(g, c, r);
            for (int64_t base = 0; base < sh.total; base += 32) {
                const int64_t t = base + lane;
                float bl = __uint_as_float(static_cast<uint32_t>(best >> 32));
                int32_t pl = static_cast<int32_t>(best & 0xffffffffu);
                if (t < sh.total) {
                    int cc[D];
                    sh.cell(t, cc);
                    int32_t cell = 0;
#pragma unroll
                    for (int a = 0; a < D; ++a) cell += cc[a] * g.stride[a];
                    if (cell_bound<D>(g, p, cc) < bl) {
                        scan_cell<D, true>(f, p, cell, bl, pl, pairs);
                        ++cells;
                    }
                }
                best = warp_min_u64((static_cast<uint64_t>(__float_as_uint(bl)) << 32) | static_cast<uint32_t>(pl));
            }
            const float b = __uint_as_float(static_cast<uint32_t>(best >> 32));
            if (b <= stop) {  // cannot raise the value
                if (kVertex && lane == 0) settle<true>(f, s, b, static_cast<int32_t>(best & 0xffffffffu));
                break;
            }
            if (!kVertex) stop = fmaxf(T, __uint_as_float(*reinterpret_cast<volatile uint32_t*>(f.qmax + s)));
        }
    }
    st[ST_PAIRS_FB] = pairs;
    st[ST_CELLS] = cells;
    add_stats(f, st);
}

// f = max(LB, sqrt(largest exact sample distance^2)); vertices: sqrt(d(v, X)^2).
template <bool kVertex>
__global__ void __launch_bounds__(kNdThreads) k_nd_finalize(NdFilt f) {
    const int64_t i = blockIdx.x * int64_t(kNdThreads) + threadIdx.x;
    if (i >= f.n) return;
    const float q = __fsqrt_rn(__uint_as_float(f.qmax[i]));
    float lb = 0.0f;
    if (!kVertex) {
        if (f.k == 1) {
            const int32_t v0 = f.simp[2 * i], v1 = f.simp[2 * i + 1];
            if (v0 < 0 || v0 >= f.n_L || v1 < 0 || v1 >= f.n_L) {
                atomicOr(f.flags, FLAG_RANGE);
                return;
            }
            lb = fmaxf(f.lower[v0], f.lower[v1]);
        } else {
            for (int j = 0; j <= f.k; ++j) {
                const int32_t t = f.fac[i * (f.k + 1) + j];
                if (t < 0 || t >= f.n_lower) {
                    atomicOr(f.flags, FLAG_RANGE);
                    return;
                }
                lb = fmaxf(lb, f.lower[t]);
            }
        }
    }
    f.values[i] = fmaxf(lb, q);
}

// ---------------------------------------------------------------- host side
inline int64_t binom64(int n, int r) {
    if (r < 0 || n < r) return 0;
    int64_t v = 1;
    for (int i = 1; i <= r; ++i) v = v * (n - r + i) / i;
    return v;
}

struct LastNd {
    HostStats buf;
    int32_t d = 0;
    bool valid = false;
};
thread_local LastNd g_last_nd;

template <int D>
int launch_fps_nd(const float* X, int64_t n, int32_t n_l, int64_t start, int64_t* out_idx, float* out_key,
                  cudaStream_t s, Scratch& scr, uint32_t** flags_out) {
    constexpr int R = D <= 2 ? 6 : (D == 3 ? 5 : (D == 4 ? 4 : 3));  // points per thread in registers
    auto fn = k_fps_nd<D, R>;
    const int sms = device_sm_count();
    const int64_t want = ceil_div(n, int64_t(kNdFpsThreads) * R);
    const int blocks_max =
        static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, std::min(sms, kNdFpsMaxBlocks))));
    // shared rows for the points past the registers, as many as one block per SM can hold
    int dev = 0, smem_optin = 0;
    FLOOD_CUDA(cudaGetDevice(&dev));
    FLOOD_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t row_bytes = size_t(D + 1) * kNdFpsThreads * sizeof(float);
    const size_t static_bytes = 4096;  // the kernel's own shared variables, with room to spare
    const int64_t e_max = smem_optin > int(static_bytes) ? (smem_optin - static_bytes) / row_bytes : 0;
    const int64_t e_want = std::max<int64_t>(0, ceil_div(n, int64_t(blocks_max) * kNdFpsThreads) - R);
    const int E = static_cast<int>(std::min(e_max, e_want));
    const size_t smem = size_t(E) * row_bytes;
    FLOOD_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem)));
    int per_sm = 0;
    FLOOD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kNdFpsThreads, smem));
    if (per_sm < 1) {
        set_error("flood_fps_nd: the kernel does not fit on an SM");
        return FLOOD_EINTERNAL;
    }
    const int blocks = blocks_max;  // one per SM at most: all resident (cooperative launch)
    uint32_t* box = nullptr;
    uint64_t* slots = nullptr;
    float* dist = nullptr;
    int rc;
    const bool overflow = n > int64_t(blocks) * kNdFpsThreads * (R + E);
    if ((rc = scr.alloc(&box, 2 * kNdMaxD + 1)) || (rc = scr.alloc(&slots, 2 * kNdFpsMaxBlocks * kNdSlotWords)) ||
        (rc = scr.alloc(&dist, overflow ? n : 1)))
        return rc;
    uint32_t* flags = box + 2 * kNdMaxD;
    *flags_out = flags;
    FLOOD_CUDA(cudaMemsetAsync(slots, 0, sizeof(uint64_t) * 2 * kNdFpsMaxBlocks * kNdSlotWords, s));
    k_box_init_nd<<<1, 1, 0, s>>>(box, flags);
    k_bbox_nd<D><<<bbox_blocks(n, sms), kBoxThreads, 0, s>>>(X, n, box, flags);
    NdFpsArgs a{X, n, n_l, start, out_idx, out_key, dist, slots, flags, kWaitPolls, E};
    void* args[] = {&a};
    FLOOD_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(fn), dim3(blocks), dim3(kNdFpsThreads), args, smem,
                                           s));
    note_launch(3);
    return FLOOD_OK;
}

template <int D>
int build_grid_nd(flood_grid_nd* g, const float* X, float cell_size, cudaStream_t s) {
    const int64_t n = g->n_points;
    Scratch scr(s);
    uint32_t* box = nullptr;
    int32_t *cell = nullptr, *count = nullptr;
    int rc;
    if ((rc = scr.alloc(&box, 2 * kNdMaxD + 1)) || (rc = scr.alloc(&cell, n)) || (rc = scr.alloc(&count, g->cap_cells)))
        return rc;
    uint32_t* flags = box + 2 * kNdMaxD;
    NdGeom* geom = static_cast<NdGeom*>(g->geom);
    const unsigned nb = static_cast<unsigned>(ceil_div(n, kNdThreads));
    FLOOD_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t) * g->cap_cells, s));
    k_box_init_nd<<<1, 1, 0, s>>>(box, flags);
    k_bbox_nd<D><<<bbox_blocks(n, device_sm_count()), kBoxThreads, 0, s>>>(X, n, box, flags);
    k_nd_geometry<D><<<1, 1, 0, s>>>(box, flags, n, cell_size, g->cap_cells, geom);
    k_nd_cell_ids<D><<<nb, kNdThreads, 0, s>>>(X, n, geom, cell, count, g->cap_cells, flags);
    note_launch(4);
    // cells past the used ones count 0: their offsets all equal n
    if ((rc = exclusive_scan(count, g->cell_start, g->cap_cells, s, scr))) return rc;
    k_nd_scatter<D><<<nb, kNdThreads, 0, s>>>(X, n, cell, g->cell_start, count, g->a4, g->a1, flags);
    note_launch(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "flood_build_grid_nd kernels");
    if ((rc = defer_status(s, flags, "flood_build_grid_nd"))) return rc;
    FLOOD_CUDA(cudaEventRecord(g->ready, s));
    return FLOOD_OK;
}

template <int D>
int run_filtration_nd(const flood_grid_nd* grid, const float* L, int32_t n_L, const int32_t* const* simplices,
                      const int32_t* const* facets, const int64_t* n_simplices, int32_t m, float* const* values,
                      cudaStream_t s) {
    Scratch scr(s);
    int rc;
    uint32_t* flags = nullptr;
    unsigned long long* stats = nullptr;
    int32_t* vnn = nullptr;
    uint4* fb = nullptr;
    int64_t n_max = n_L, launches = 0;
    int64_t I[kNdMaxD + 1];
    for (int k = 0; k <= D; ++k) {
        I[k] = k == 0 ? 1 : binom64(m - 1, k);
        const int64_t nk = k == 0 ? n_L : n_simplices[k];
        n_max = std::max(n_max, nk);
        launches += ceil_div(nk * I[k], kNdChunk);
    }
    uint32_t *qmax = nullptr, *fb_count = nullptr;
    unsigned long long* next = nullptr;
    const int64_t n_counts = std::max<int64_t>(1, launches);
    if ((rc = scr.alloc(&flags, 1)) || (rc = scr.alloc(&stats, (kNdMaxD + 1) * kNdStats)) ||
        (rc = scr.alloc(&vnn, n_L)) || (rc = scr.alloc(&fb, kNdChunk)) || (rc = scr.alloc(&qmax, n_max)) ||
        (rc = scr.alloc(&fb_count, n_counts)) || (rc = scr.alloc(&next, n_counts)))
        return rc;
    float* lam[kNdMaxD + 1] = {};
    for (int k = 1; k <= D; ++k)
        if (n_simplices[k] > 0 && I[k] > 0) {
            if ((rc = scr.alloc(&lam[k], I[k] * (k + 1)))) return rc;
            k_nd_lambda<<<static_cast<unsigned>(ceil_div(I[k], kNdThreads)), kNdThreads, 0, s>>>(lam[k], I[k], m, k);
            note_launch(1);
        }
    // the passes run as many blocks as fit at once, striding over their items
    int per_sm_v = 0, per_sm = 0;
    FLOOD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_v, k_nd_resolve<D, true>, kNdThreads, 0));
    FLOOD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nd_resolve<D, false>, kNdThreads, 0));
    const int64_t resident_v = int64_t(device_sm_count()) * std::max(1, per_sm_v);
    const int64_t resident = int64_t(device_sm_count()) * std::max(1, per_sm);
    float* vals[kNdMaxD + 1];
    for (int k = 0; k <= D; ++k) {
        const int64_t nk = k == 0 ? n_L : n_simplices[k];
        vals[k] = values[k];
        if (!vals[k] && (rc = scr.alloc(&vals[k], nk))) return rc;
    }
    FLOOD_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t), s));
    FLOOD_CUDA(cudaMemsetAsync(vnn, 0, sizeof(int32_t) * n_L, s));  // every vertex settles; 0 if its row was rejected
    FLOOD_CUDA(cudaMemsetAsync(stats, 0, sizeof(unsigned long long) * (kNdMaxD + 1) * kNdStats, s));
    FLOOD_CUDA(cudaMemsetAsync(fb_count, 0, sizeof(uint32_t) * n_counts, s));
    FLOOD_CUDA(cudaMemsetAsync(next, 0, sizeof(unsigned long long) * n_counts, s));
    const int fb_blocks = device_sm_count() * 8;
    int64_t chunk_no = 0;
    for (int k = 0; k <= D; ++k) {
        const int64_t nk = k == 0 ? n_L : n_simplices[k];
        if (nk == 0) continue;
        NdFilt f{};
        f.geom = static_cast<const NdGeom*>(grid->geom);
        f.a4 = grid->a4;
        f.a1 = grid->a1;
        f.cs = grid->cell_start;
        f.L = L;
        f.n_L = n_L;
        f.simp = k == 0 ? nullptr : simplices[k];
        f.fac = k >= 2 ? facets[k] : nullptr;
        f.n = nk;
        f.n_lower = k == 0 ? 0 : (k == 1 ? n_L : n_simplices[k - 1]);
        f.k = k;
        f.m = m;
        f.I = I[k];
        f.lower = k == 0 ? nullptr : vals[k - 1];
        f.vnn = vnn;
        f.vnn_out = vnn;
        f.qmax = qmax;
        f.values = vals[k];
        f.fb = fb;
        f.lam = lam[k];
        f.stats = stats + k * kNdStats;
        f.flags = flags;
        FLOOD_CUDA(cudaMemsetAsync(qmax, 0, sizeof(uint32_t) * nk, s));
        // launches of at most kNdChunk items (the capacity of the fallback list)
        f.fb_cap = static_cast<uint32_t>(kNdChunk);
        const int64_t items = nk * I[k];
        for (int64_t i0 = 0; i0 < items; i0 += kNdChunk) {
            f.item0 = i0;
            f.n_items = std::min<int64_t>(kNdChunk, items - i0);
            f.fb_count = fb_count + chunk_no;
            f.next = next + chunk_no++;
            const unsigned nb = static_cast<unsigned>(std::min<int64_t>(
                ceil_div(f.n_items, int64_t(kNdThreads / 32) * kPool), k == 0 ? resident_v : resident));
            if (k == 0) {
                k_nd_resolve<D, true><<<nb, kNdThreads, 0, s>>>(f);
                k_nd_fallback<D, true><<<fb_blocks, kNdThreads, 0, s>>>(f);
            } else {
                k_nd_resolve<D, false><<<nb, kNdThreads, 0, s>>>(f);
                k_nd_fallback<D, false><<<fb_blocks, kNdThreads, 0, s>>>(f);
            }
            note_launch(2);
        }
        const unsigned nf = static_cast<unsigned>(ceil_div(nk, kNdThreads));
        if (k == 0)
            k_nd_finalize<true><<<nf, kNdThreads, 0, s>>>(f);
        else
            k_nd_finalize<false><<<nf, kNdThreads, 0, s>>>(f);
        note_launch(1);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "flood_filtration_nd kernels");
    // work counters, read back without waiting
    LastNd& last = g_last_nd;
    last.valid = false;
    const size_t sb = sizeof(unsigned long long) * (kNdMaxD + 1) * kNdStats;
    if ((rc = last.buf.reserve(sb))) return rc;
    FLOOD_CUDA(cudaMemcpyAsync(last.buf.host, stats, sb, cudaMemcpyDeviceToHost, s));
    FLOOD_CUDA(cudaEventRecord(last.buf.done, s));
    last.d = D;
    last.valid = true;
    return defer_status(s, flags, "flood_filtration_nd");
}

}  // namespace
}  // namespace flood

using namespace flood;

namespace flood {
// (n, 2) rows to (n, 3) rows at z = 0.
__global__ void __launch_bounds__(256) k_plane_to_space(const float* X, int64_t n, float* X3) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    X3[3 * i + 0] = X[2 * i + 0];
    X3[3 * i + 1] = X[2 * i + 1];
    X3[3 * i + 2] = 0.0f;
}
}  // namespace flood

extern "C" int flood_fps_nd(const float* X, int64_t n_points, int32_t dim, int32_t n_landmarks, int64_t start,
                            int64_t* out_idx, float* out_key, void* stream_) {
    if (!X || !out_idx || dim < 2 || dim > FLOOD_ND_MAX_DIM || n_points < 1 || n_points >= (int64_t(1) << 31) - 1 ||
        n_landmarks < 1 || n_landmarks > n_points || start < 0 || start >= n_points) {
        set_error("flood_fps_nd: need X, out_idx != NULL, 2 <= dim <= 5, 1 <= n_landmarks <= n_points < 2^31 - 1, "
                  "0 <= start < n_points");
        return FLOOD_EINVAL;
    }
    // three coordinates: the three-dimensional FPS (same key, same picks; its chunk skipping is faster there)
    if (dim == 3) return flood_fps(X, n_points, n_landmarks, start, out_idx, out_key, stream_);
    // two coordinates: the same, on the points at z = 0. The key gains the term
    // fl(fl(0 - 0)^2) = 0 and adding 0 is exact, so every key, and every pick,
    // is the two-dimensional one bit for bit.
    if (dim == 2) {
        cudaStream_t s = static_cast<cudaStream_t>(stream_);
        if (int rc = pending_error(s)) return rc;
        float* X3 = nullptr;
        if (cudaMallocAsync(reinterpret_cast<void**>(&X3), sizeof(float) * 3 * size_t(n_points), s) != cudaSuccess) {
            cudaGetLastError();
            set_error("flood_fps_nd: device allocation failed");
            return FLOOD_ENOMEM;
        }
        k_plane_to_space<<<static_cast<unsigned>((n_points + 255) / 256), 256, 0, s>>>(X, n_points, X3);
        note_launch();
        const int rc = flood_fps(X3, n_points, n_landmarks, start, out_idx, out_key, stream_);
        cudaFreeAsync(X3, s);  // after the FPS kernels in stream order
        return rc;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    if (int rc = pending_error(s)) return rc;
    Scratch scr(s);
    uint32_t* flags = nullptr;
    int rc = FLOOD_OK;
    switch (dim) {
        case 2: rc = launch_fps_nd<2>(X, n_points, n_landmarks, start, out_idx, out_key, s, scr, &flags); break;
        case 3: rc = launch_fps_nd<3>(X, n_points, n_landmarks, start, out_idx, out_key, s, scr, &flags); break;
        case 4: rc = launch_fps_nd<4>(X, n_points, n_landmarks, start, out_idx, out_key, s, scr, &flags); break;
        default: rc = launch_fps_nd<5>(X, n_points, n_landmarks, start, out_idx, out_key, s, scr, &flags); break;
    }
    if (rc) {
        if (flags) cudaStreamSynchronize(s);
        return rc;
    }
    return defer_status(s, flags, "flood_fps_nd");
}

extern "C" void flood_grid_nd_destroy(flood_grid_nd* g) {
    if (!g) return;
    if (g->a4) cudaFree(g->a4);
    if (g->a1) cudaFree(g->a1);
    if (g->cell_start) cudaFree(g->cell_start);
    if (g->geom) cudaFree(g->geom);
    if (g->ready) cudaEventDestroy(g->ready);
    free(g);
}

extern "C" int flood_build_grid_nd(const float* X, int64_t n_points, int32_t dim, float cell_size,
                                   flood_grid_nd** out, void* stream_) {
    if (!out) {
        set_error("flood_build_grid_nd: out is NULL");
        return FLOOD_EINVAL;
    }
    *out = nullptr;
    if (!X || dim < 2 || dim > FLOOD_ND_MAX_DIM || n_points < 1 || n_points >= (int64_t(1) << 31) - 1 ||
        !(cell_size >= 0.0f) || !isfinite(cell_size)) {
        set_error("flood_build_grid_nd: need X != NULL, 2 <= dim <= 5, 1 <= n_points < 2^31 - 1, finite cell_size >= 0");
        return FLOOD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    if (int rc = pending_error(s)) return rc;
    flood_grid_nd* g = static_cast<flood_grid_nd*>(calloc(1, sizeof(flood_grid_nd)));
    if (!g) {
        set_error("flood_build_grid_nd: host allocation failed");
        return FLOOD_ENOMEM;
    }
    g->d = dim;
    g->n_points = n_points;
    g->cap_cells = static_cast<int32_t>(std::min<int64_t>(int64_t(1) << 25, std::max<int64_t>(int64_t(1) << 12, 2 * n_points)));
    cudaError_t e1 = cudaMallocAsync(&g->a4, sizeof(float4) * n_points, s);
    cudaError_t e2 = dim > 4 ? cudaMallocAsync(&g->a1, sizeof(float) * n_points, s) : cudaSuccess;
    cudaError_t e3 = cudaMallocAsync(&g->cell_start, sizeof(int32_t) * (int64_t(g->cap_cells) + 1), s);
    cudaError_t e4 = cudaMallocAsync(&g->geom, sizeof(NdGeom), s);
    cudaError_t e5 = cudaEventCreateWithFlags(&g->ready, cudaEventDisableTiming);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess || e5 != cudaSuccess) {
        cudaGetLastError();
        flood_grid_nd_destroy(g);
        set_error("flood_build_grid_nd: device allocation failed");
        return FLOOD_ENOMEM;
    }
    g->device_bytes = int64_t(sizeof(float4) + (dim > 4 ? sizeof(float) : 0)) * n_points +
                      int64_t(sizeof(int32_t)) * (int64_t(g->cap_cells) + 1) + int64_t(sizeof(NdGeom));
    int rc;
    switch (dim) {
        case 2: rc = build_grid_nd<2>(g, X, cell_size, s); break;
        case 3: rc = build_grid_nd<3>(g, X, cell_size, s); break;
        case 4: rc = build_grid_nd<4>(g, X, cell_size, s); break;
        default: rc = build_grid_nd<5>(g, X, cell_size, s); break;
    }
    if (rc != FLOOD_OK) {
        flood_grid_nd_destroy(g);
        return rc;
    }
    *out = g;
    return FLOOD_OK;
}

extern "C" int flood_grid_nd_get_info(const flood_grid_nd* g, flood_grid_nd_info* out) {
    if (!g || !out) {
        set_error("flood_grid_nd_get_info: NULL argument");
        return FLOOD_EINVAL;
    }
    NdGeom h;
    FLOOD_CUDA(cudaEventSynchronize(g->ready));
    FLOOD_CUDA(cudaMemcpy(&h, g->geom, sizeof(h), cudaMemcpyDeviceToHost));
    memset(out, 0, sizeof(*out));
    out->n_points = g->n_points;
    out->n_cells = h.n_cells;
    out->dim = g->d;
    out->cell_size = h.h;
    out->device_bytes = g->device_bytes;
    for (int a = 0; a < g->d; ++a) {
        out->dims[a] = h.dims[a];
        out->bbox_lo[a] = h.lo[a];
        out->bbox_hi[a] = h.hi[a];
    }
    return FLOOD_OK;
}

extern "C" int flood_filtration_nd(const flood_grid_nd* grid, const float* L, int32_t n_landmarks,
                                   const int32_t* const simplices[FLOOD_ND_MAX_DIM + 1],
                                   const int32_t* const facets[FLOOD_ND_MAX_DIM + 1],
                                   const int64_t n_simplices[FLOOD_ND_MAX_DIM + 1], int32_t m,
                                   float* const values[FLOOD_ND_MAX_DIM + 1], void* stream_) {
    if (!grid || !L || !simplices || !facets || !n_simplices || !values || n_landmarks < 1 || m < 1 ||
        m > FLOOD_MAX_M) {
        set_error("flood_filtration_nd: need grid, L, the four arrays != NULL, n_landmarks >= 1, 1 <= m <= %d",
                  FLOOD_MAX_M);
        return FLOOD_EINVAL;
    }
    const int d = grid->d;
    if (n_simplices[0] != 0 && n_simplices[0] != n_landmarks) {
        set_error("flood_filtration_nd: n_simplices[0] must be 0 or n_landmarks");
        return FLOOD_EINVAL;
    }
    for (int k = 1; k <= FLOOD_ND_MAX_DIM; ++k) {
        const int64_t nk = n_simplices[k];
        if (nk < 0 || nk >= (int64_t(1) << 31) || (k > d && nk != 0) || (nk > 0 && !simplices[k]) ||
            (nk > 0 && k >= 2 && !facets[k]) || (nk > 0 && k >= 2 && n_simplices[k - 1] == 0)) {
            set_error("flood_filtration_nd: dimension %d: need 0 <= n_simplices < 2^31 (0 above the grid's "
                      "dimension %d), simplices (and facets for k >= 2) != NULL when n > 0, and faces below",
                      k, d);
            return FLOOD_EINVAL;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    if (int rc = pending_error(s)) return rc;
    switch (d) {
        case 2: return run_filtration_nd<2>(grid, L, n_landmarks, simplices, facets, n_simplices, m, values, s);
        case 3: return run_filtration_nd<3>(grid, L, n_landmarks, simplices, facets, n_simplices, m, values, s);
        case 4: return run_filtration_nd<4>(grid, L, n_landmarks, simplices, facets, n_simplices, m, values, s);
        default: return run_filtration_nd<5>(grid, L, n_landmarks, simplices, facets, n_simplices, m, values, s);
    }
}

extern "C" int flood_last_filtration_nd_stats(flood_nd_stats* out) {
    if (!out) {
        set_error("flood_last_filtration_nd_stats: out is NULL");
        return FLOOD_EINVAL;
    }
    memset(out, 0, sizeof(*out));
    if (!g_last_nd.valid) return FLOOD_OK;
    FLOOD_CUDA(cudaEventSynchronize(g_last_nd.buf.done));
    const unsigned long long* h = static_cast<const unsigned long long*>(g_last_nd.buf.host);
    out->dim = g_last_nd.d;
    for (int k = 0; k <= FLOOD_ND_MAX_DIM; ++k) {
        const unsigned long long* c = h + k * kNdStats;
        out->items[k] = static_cast<int64_t>(c[ST_ITEMS]);
        out->pruned[k] = static_cast<int64_t>(c[ST_PRUNED]);
        out->resolved[k] = static_cast<int64_t>(c[ST_RESOLVED]);
        out->exact[k] = static_cast<int64_t>(c[ST_EXACT]);
        out->fallback[k] = static_cast<int64_t>(c[ST_FALLBACK]);
        out->pairs[k] = static_cast<int64_t>(c[ST_PAIRS]);
        out->pairs_fallback[k] = static_cast<int64_t>(c[ST_PAIRS_FB]);
        out->cells[k] = static_cast<int64_t>(c[ST_CELLS]);
    }
    return FLOOD_OK;
}
