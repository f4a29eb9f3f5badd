// flood_filtration: flood values of every simplex of Del(L) (§4.1).
//
// The value of a k-simplex is the maximum, over its barycentric grid (Lemma
// 1), of the distance to the nearest point of X. Faces are included (the
// discretised complex Flood_r(X,L,P) of §4.1), so the value is
//     f(sigma) = max( max over interior samples p of d(p, X), f(facets) ),
// because P_tau ⊂ P_sigma (App. A.1). Dimensions are processed in increasing
// order, so when a k-simplex is evaluated its facet maximum LB is known, and
// a sample p can only matter if d(p, X) > LB. That gives an exact pruning
// rule (values and attaining samples are identical to the full max-min):
//
//   1. samples   one warp per simplex generates its interior samples and the
//                bound u_p = min_i |p - v_i| >= d(p, X) (v_i ∈ X; the step at
//                the heart of Lemma 2's proof). Samples with u_p <= LB are
//                dropped; the rest are bucketed on a fixed lattice (counting
//                sort, atomics).
//   2. groups    each bucket is cut into groups of up to 32*Q samples.
//   3. flood     a persistent kernel in which every warp pops a group, keeps
//                its samples in registers and scans the cell grid in shells
//                of cells around the group's cells, nearest shell first.
//                Candidate points reach shared memory by 1-D TMA bulk copies
//                (one per row segment, double-buffered, mbarrier-tracked),
//                are shifted to the bucket corner and extended with their
//                squared norm, and every pair costs three FMAs and a min:
//                    |p - x|^2 = |x'|^2 - 2 p'.x' + |p'|^2.
//                After each shell a sample is done when its minimum is below
//                the distance to the next shell (exact) or when it is at most
//                LB (it cannot raise the maximum); the warp stops when all
//                of its samples are done, and at the latest when the shells
//                pass max u_p, beyond which no nearest point can lie.
//   4. finalize  64-bit atomic max of (d^2 bits, ~sample) per simplex gives
//                the own maximum with the lowest sample on ties.
//   5. face-max  f(sigma) = max(sqrt(own), f(facets)).
// Every pair distance depends only on (sample, point, bucket corner), and
// the bucket lattice depends only on X's bounding box, so results do not
// depend on how the work is tiled or batched, nor on the cell size.
#include <algorithm>
#include <climits>
#include <cstring>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "geometry.cuh"
#include "scan.cuh"

namespace flood {

namespace {

constexpr int kThreads = 256;  // flood kernel CTA: 8 independent warps
constexpr int kWarps = kThreads / 32;
constexpr int kWTile = 256;    // candidate points per warp tile (4 KB), two per warp
constexpr int kGroup = 64;     // samples per group (one warp)
constexpr int64_t kMaxBuckets = int64_t(1) << 24;

struct Ctl {
    uint32_t flags;
    uint32_t head[4];
    uint32_t heavy_head[4];
    uint32_t pad[3];
    unsigned long long pairs[4];
    unsigned long long active[4];
    unsigned long long shells[4];
    unsigned long long tiles[4];
};

// Sample lattice: coarse cubes of edge B (a power of two) anchored at the grid
// origin, each split into 2 x 2 x 2 fine buckets (octants). A sample's key is
// coarse id * 8 + octant, so sorting by key keeps the samples of one coarse
// cube together and roughly spatially ordered inside it. (4 x 4 x 4 fine
// buckets, about one sample each, made the per-dimension bucket scan and
// clearing 8x larger for no gain in the flood kernels.)
struct Lattice {
    float ox, oy, oz;
    float B, invB;     // coarse edge
    float invF;        // 2 / B
    int bx, by, bz;    // coarse cubes per axis
};

constexpr int kFine = 8;  // fine buckets per coarse cube

struct SampleRec {
    float x, y, z;  // sample coordinates
    float lb;       // facet maximum of its simplex (LB)
    int32_t sigma;  // simplex row
    int32_t s;      // interior sample rank
    float u;        // vertex bound u_p (rounded up)
    int32_t pad;
};

// Geometry of one job, computed on the device from its grid (no host
// readback): the grid view, the sample lattice and the shell constants.
struct JobGeo {
    GridView g;
    Lattice lat;
    float shell_h;      // cell edge times (1 - 2^-10)
    float shell_slack;  // absolute rounding slack of cell assignment
    int64_t n_coarse;   // coarse cubes of the lattice
};

struct DimArgs {
    int k;
    int I;
    float m;
    int64_t n;
    const int32_t* simplices;
    const int32_t* facets;   // k >= 2
    const float* val_lower;  // final values of dimension k-1
    int64_t n_lower;
    const uint8_t* comp;     // grid samples: interior compositions (I, k+1), or
    const float* lam;        // grid samples: their barycentric coordinates fl(c_j / m) (I, k+1)
    const float* w;          // given samples: barycentric coordinates (n, I, k+1)
    const float* L;
    const float* vbound;     // per landmark: d(v, X) rounded up, 0 for a point of X
    int32_t n_L;
    const JobGeo* geo;       // device: grid view, sample lattice, shell constants
    int64_t n_buckets;      // capacity: n_coarse * kFine sample keys
    int64_t n_coarse;       // capacity: coarse cubes of any lattice this job can get
    int32_t* bucket_count;
    int32_t* bucket_start;  // n_buckets + 1
    int32_t* bucket_fill;
    int32_t* group_off;     // n_coarse + 1
    int2* groups;           // (bucket, index within bucket)
    SampleRec* recs;
    int64_t rec_cap;           // records the sample arrays hold
    int64_t groups_cap;        // groups the group arrays hold
    unsigned long long* best;  // per simplex: (d^2 bits << 32) | ~sample
    const int32_t* n_heavy;    // groups [0, *n_heavy) of the sorted queue go to the CTA kernel
    Ctl* ctl;
};

// ---------------------------------------------------------------- vertices
// f(v) = d(v, X) (P_v = {v}): 0 for a landmark that is a point of X, found in
// its own cell; otherwise the exact nearest point by doubling cull boxes (§3
// allows L ⊄ X). vbound[v] = d(v, X) rounded up with a margin (exactly 0 for a
// point of X) bounds the samples of every coface from above.
// One warp per landmark: its lanes scan the cells together.
__global__ void k_vertices(const float* L, int32_t n_L, const GridView* gp, float* val, int32_t* src, float* vbound,
                           uint32_t* flags) {
    const int v = static_cast<int>((blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (v >= n_L) return;
    const GridView g = *gp;
    const float x = L[3 * v], y = L[3 * v + 1], z = L[3 * v + 2];
    bool found = false;
    if (isfinite(x) && isfinite(y) && isfinite(z)) {
        const int cx = cell_coord(x, g.ox, g.inv_cell, g.dx);
        const int cy = cell_coord(y, g.oy, g.inv_cell, g.dy);
        const int cz = cell_coord(z, g.oz, g.inv_cell, g.dz);
        const int64_t c = (static_cast<int64_t>(cz) * g.dy + cy) * g.dx + cx;
        const bool bad = FLOOD_OOB(c, g.n_cells, flags);
        const int32_t b = bad ? 0 : g.cell_start[c], e = bad ? 0 : g.cell_start[c + 1];
        for (int32_t i0 = b; i0 < e; i0 += 32) {
            bool hit = false;
            if (i0 + lane < e && !FLOOD_OOB(i0 + lane, g.n_pts, flags)) {
                const float4 p = g.pts[i0 + lane];
                hit = __float_as_uint(p.x) == __float_as_uint(x) && __float_as_uint(p.y) == __float_as_uint(y) &&
                      __float_as_uint(p.z) == __float_as_uint(z);
            }
            if (__any_sync(0xffffffffu, hit)) {
                found = true;
                break;
            }
        }
    }
    const bool finite = isfinite(x) && isfinite(y) && isfinite(z);
    float f = 0.0f, bound = 0.0f;
    if (finite && !found) {
        const unsigned long long nn = warp_nearest(g, x, y, z, g.cell, lane);
        if (nn == ~0ull) {
            if (lane == 0) atomicOr(flags, FLAG_INTERNAL);
            f = bound = __int_as_float(0x7fc00000);
        } else {
            const float d2 = __uint_as_float(static_cast<uint32_t>(nn >> 32));
            f = __fsqrt_rn(d2);
            bound = __fmul_ru(__fsqrt_ru(d2), 1.0f + 1.0f / 65536.0f);
        }
    }
    if (lane == 0) {
        if (!finite) atomicOr(flags, FLAG_NONFINITE);
        val[v] = finite ? f : __int_as_float(0x7fc00000);
        vbound[v] = finite ? bound : __int_as_float(0x7fc00000);
        src[2 * v] = v;
        src[2 * v + 1] = 0;
    }
}

// ---------------------------------------------------------------- samples
__device__ __forceinline__ int lattice_coord(float v, float o, float invB, int dim) {
    float t = __fmul_rn(__fsub_rn(v, o), invB);
    t = fminf(fmaxf(t, 0.0f), static_cast<float>(dim - 1));
    return static_cast<int>(t);
}

__device__ __forceinline__ int64_t sample_key(const Lattice& L, float x, float y, float z) {
    const int fx = lattice_coord(x, L.ox, L.invF, 2 * L.bx);
    const int fy = lattice_coord(y, L.oy, L.invF, 2 * L.by);
    const int fz = lattice_coord(z, L.oz, L.invF, 2 * L.bz);
    const int64_t coarse = (static_cast<int64_t>(fz >> 1) * L.by + (fy >> 1)) * L.bx + (fx >> 1);
    const uint32_t fine = (fx & 1) | ((fy & 1) << 1) | ((fz & 1) << 2);
    return coarse * kFine + fine;
}

// Largest binary32 q with sqrt_rn(q) <= lb, for a facet maximum lb >= 0:
// since sqrt_rn is monotone, sqrt_rn(u2) > lb exactly when u2 > q. fl(lb^2)
// is within a few units in the last place of it; should the search not settle
// (it always does), 0 keeps every sample, which only costs time.
__device__ __forceinline__ float sqrt_le_bound(float lb) {
    if (!(lb > 0.0f) || !(lb < INFINITY)) return 0.0f;
    float q = __fmul_rn(lb, lb);
    for (int i = 0; i < 16 && __fsqrt_rn(q) > lb; ++i) q = __uint_as_float(__float_as_uint(q) - 1u);
    if (__fsqrt_rn(q) > lb) return 0.0f;
    for (int i = 0; i < 16; ++i) {
        const float nq = __uint_as_float(__float_as_uint(q) + 1u);
        if (__fsqrt_rn(nq) > lb) return q;
        q = nq;
    }
    return 0.0f;
}

// Pass 1 (SCATTER = false) counts active samples per bucket; pass 2 writes
// them. Both passes evaluate exactly the same arithmetic.
template <bool SCATTER>
__global__ void __launch_bounds__(256) k_samples(DimArgs a) {
    const int64_t w = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= a.n) return;
    const int k = a.k;
    const int32_t* ids = a.simplices + w * (k + 1);
    bool ok = true;
    for (int j = 0; j <= k; ++j) ok &= (ids[j] >= 0 && ids[j] < a.n_L);
    float lb = 0.0f;  // facet maximum (an edge's facets are its vertices)
    if (k >= 2) {
        for (int j = 0; j <= k; ++j) {
            const int32_t t = a.facets[w * (k + 1) + j];
            if (t < 0 || t >= a.n_lower) ok = false;
            else lb = fmaxf(lb, a.val_lower[t]);
        }
    } else if (ok) {
        lb = fmaxf(a.val_lower[ids[0]], a.val_lower[ids[1]]);
    }
    if (!ok) {
        if (!SCATTER && lane == 0) atomicOr(&a.ctl->flags, FLAG_RANGE);
        return;
    }
    Simplex S;
    load_simplex(a.L, ids, k, S);
    // vertices that are points of X keep the plain vertex bound min_j |p - v_j|
    float vb[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    bool members = true;
    for (int j = 0; j <= k; ++j) {
        vb[j] = a.vbound[ids[j]];
        members &= vb[j] == 0.0f;
    }
    // sqrt_rn(u2) > lb exactly when u2 > lbq (one comparison per sample)
    const float lbq = sqrt_le_bound(lb);
    int n_active = 0;
    for (int s = lane; s < a.I; s += 32) {
        float px, py, pz;
        if (a.w) {
            const float* lam = a.w + (w * a.I + s) * (k + 1);
            bool fin = true;
            for (int j = 1; j <= k; ++j) fin &= isfinite(lam[j]);
            if (!fin) {
                if (!SCATTER) atomicOr(&a.ctl->flags, FLAG_NONFINITE);
                continue;
            }
            sample_offset_lambda(S, lam, k, px, py, pz);
        } else {
            sample_offset_lambda(S, a.lam + s * (k + 1), k, px, py, pz);
        }
        float u;
        if (members) {
            const float u2 = vertex_bound_sq(S, k, px, py, pz);
            if (!(u2 > lbq)) continue;  // cannot exceed the facet maximum
            u = __fsqrt_ru(u2);
        } else {
            u = vertex_bound_general(S, k, px, py, pz, vb);
            if (!(u > lb)) continue;
        }
        ++n_active;
        const float x = __fadd_rn(S.v0[0], px), y = __fadd_rn(S.v0[1], py), z = __fadd_rn(S.v0[2], pz);
        const int64_t b = sample_key(a.geo->lat, x, y, z);
        if (FLOOD_OOB(b, a.n_buckets, &a.ctl->flags)) continue;
        if (!SCATTER) {
            atomicAdd(&a.bucket_count[b], 1);
        } else {
            const int32_t pos = a.bucket_start[b] + atomicAdd(&a.bucket_fill[b], 1);
            if (FLOOD_OOB(pos, a.rec_cap, &a.ctl->flags)) continue;
            SampleRec r;
            r.x = x;
            r.y = y;
            r.z = z;
            r.lb = lb;
            r.sigma = static_cast<int32_t>(w);
            r.s = s;
            r.u = u;
            r.pad = 0;
            a.recs[pos] = r;
        }
    }
    if (!SCATTER) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n_active += __shfl_xor_sync(0xffffffffu, n_active, o);
        if (lane == 0 && n_active) atomicAdd(&a.ctl->active[k], static_cast<unsigned long long>(n_active));
    }
}

// Bucket offsets and the group list, from the bucket counts, in two
// launches. Groups never span coarse cubes (their samples share the cube
// corner as the origin of the pair arithmetic): cube c holds
// ceil(samples(c) / kGroup) groups. Both prefix sums (samples over buckets,
// groups over cubes) run over tiles of kCubeTile cubes: the first kernel
// sums each tile, the second adds the sums of the tiles before its own (a
// block reduction over at most a few hundred values) to its block scan.
constexpr int kCubeTile = 1024;  // cubes per block (one per thread)

__device__ __forceinline__ int32_t cube_samples(const int32_t* count, int64_t c, int64_t n_coarse) {
    if (c >= n_coarse) return 0;
    int32_t t = 0;
#pragma unroll
    for (int f = 0; f < kFine; ++f) t += count[c * kFine + f];
    return t;
}

__global__ void __launch_bounds__(kCubeTile) k_cube_sums(const int32_t* count, int64_t n_coarse,
                                                        int32_t* tile_samples, int32_t* tile_groups) {
    const int64_t c = blockIdx.x * int64_t(kCubeTile) + threadIdx.x;
    const int32_t ns = cube_samples(count, c, n_coarse);
    __shared__ int32_t s_red[2][kCubeTile / 32];
    int32_t a = ns, g = (ns + kGroup - 1) / kGroup;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        g += __shfl_xor_sync(0xffffffffu, g, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_red[0][warp] = a;
        s_red[1][warp] = g;
    }
    __syncthreads();
    if (warp == 0) {
        a = s_red[0][lane];
        g = s_red[1][lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        if (lane == 0) {
            tile_samples[blockIdx.x] = a;
            tile_groups[blockIdx.x] = g;
        }
    }
}

// bucket_start[0..n_coarse * kFine] and group_off[0..n_coarse] (the last
// entries are the totals) and groups[] = (cube, index within the cube).
__global__ void __launch_bounds__(kCubeTile) k_cube_scan(const int32_t* count, int64_t n_coarse,
                                                        const int32_t* tile_samples, const int32_t* tile_groups,
                                                        int32_t* bucket_start, int32_t* group_off, int2* groups,
                                                        int64_t groups_cap, uint32_t* flags) {
    __shared__ int32_t s_red[2][kCubeTile / 32];
    __shared__ int32_t s_base[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // sums of the tiles before this one
    int32_t ps = 0, pg = 0;
    for (int t = threadIdx.x; t < static_cast<int>(blockIdx.x); t += kCubeTile) {
        ps += tile_samples[t];
        pg += tile_groups[t];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ps += __shfl_xor_sync(0xffffffffu, ps, o);
        pg += __shfl_xor_sync(0xffffffffu, pg, o);
    }
    if (lane == 0) {
        s_red[0][warp] = ps;
        s_red[1][warp] = pg;
    }
    __syncthreads();
    if (warp == 0) {
        ps = s_red[0][lane];
        pg = s_red[1][lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ps += __shfl_xor_sync(0xffffffffu, ps, o);
            pg += __shfl_xor_sync(0xffffffffu, pg, o);
        }
        if (lane == 0) {
            s_base[0] = ps;
            s_base[1] = pg;
        }
    }
    __syncthreads();
    // block scan of this tile's (samples, groups) per cube
    const int64_t c = blockIdx.x * int64_t(kCubeTile) + threadIdx.x;
    const int32_t ns = cube_samples(count, c, n_coarse), ng = (ns + kGroup - 1) / kGroup;
    int32_t is = ns, ig = ng;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t ys = __shfl_up_sync(0xffffffffu, is, o), yg = __shfl_up_sync(0xffffffffu, ig, o);
        if (lane >= o) {
            is += ys;
            ig += yg;
        }
    }
    __syncthreads();  // s_red is reused
    if (lane == 31) {
        s_red[0][warp] = is;
        s_red[1][warp] = ig;
    }
    __syncthreads();
    if (warp == 0) {
        int32_t ws = s_red[0][lane], wg = s_red[1][lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t ys = __shfl_up_sync(0xffffffffu, ws, o), yg = __shfl_up_sync(0xffffffffu, wg, o);
            if (lane >= o) {
                ws += ys;
                wg += yg;
            }
        }
        s_red[0][lane] = ws;  // inclusive over warps
        s_red[1][lane] = wg;
    }
    __syncthreads();
    const int32_t off_s = s_base[0] + (warp > 0 ? s_red[0][warp - 1] : 0) + is - ns;
    const int32_t off_g = s_base[1] + (warp > 0 ? s_red[1][warp - 1] : 0) + ig - ng;
    if (c < n_coarse) {
        int32_t run = off_s;
#pragma unroll
        for (int f = 0; f < kFine; ++f) {
            bucket_start[c * kFine + f] = run;
            run += count[c * kFine + f];
        }
        group_off[c] = off_g;
        for (int32_t j = 0; j < ng; ++j)
            if (!FLOOD_OOB(off_g + j, groups_cap, flags)) groups[off_g + j] = make_int2(static_cast<int>(c), j);
        if (c == n_coarse - 1) {  // totals
            bucket_start[n_coarse * kFine] = run;
            group_off[n_coarse] = off_g + ng;
        }
    }
}

// Longest-first queue: groups are counting-sorted by the number of shells
// their vertex bound allows (descending), so the groups that may scan far
// start first and the short ones fill in behind them.
constexpr int kClasses = 64;

// Class of group j from the largest vertex bound of its samples (one warp
// per group, grid-stride), stored in gcls; counts per class through a block
// histogram.
__global__ void __launch_bounds__(256) k_group_class_count(DimArgs a, const int32_t* n_groups, int32_t* class_count,
                                                            int32_t* gcls) {
    __shared__ int32_t s_hist[kClasses];
    for (int t = threadIdx.x; t < kClasses; t += blockDim.x) s_hist[t] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int32_t ng = *n_groups;
    const int32_t nw = static_cast<int32_t>(gridDim.x * (blockDim.x >> 5));
    for (int32_t j = static_cast<int32_t>((blockIdx.x * blockDim.x + threadIdx.x) >> 5); j < ng; j += nw) {
        const int2 gb = a.groups[j];
        const int32_t s_begin = a.bucket_start[int64_t(gb.x) * kFine] + gb.y * kGroup;
        const int32_t s_end = min(s_begin + kGroup, a.bucket_start[int64_t(gb.x + 1) * kFine]);
        float R = 0.0f;
        for (int32_t i = s_begin + lane; i < s_end; i += 32)
            if (!FLOOD_OOB(i, a.rec_cap, &a.ctl->flags)) R = fmaxf(R, a.recs[i].u);
        // non-negative floats order like their bit patterns
        R = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(R)));
        const int c = static_cast<int>(ceilf(R / a.geo->shell_h));
        const int cls = kClasses - 1 - min(max(c, 0), kClasses - 1);  // heavier -> smaller class
        if (lane == 0) {
            gcls[j] = cls;
            atomicAdd(&s_hist[cls], 1);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kClasses; t += blockDim.x)
        if (s_hist[t]) atomicAdd(&class_count[t], s_hist[t]);
}

// Every block takes the exclusive scan of the kClasses counts itself (block 0
// also stores it: entry kClasses - heavy_shells is the heavy prefix), then
// places its groups.
__global__ void k_group_class_scatter(DimArgs a, const int32_t* n_groups, const int32_t* class_count,
                                      int32_t* class_start, int32_t* class_fill, int2* sorted,
                                      int32_t* groups_out, const int32_t* gcls) {
    static_assert(kClasses == 64, "two lanes' worth of classes per lane of one warp");
    __shared__ int32_t s_start[kClasses + 1];
    if (blockIdx.x == 0 && threadIdx.x == 32) *groups_out = *n_groups;  // work items of this job (statistics)
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        const int32_t c0 = class_count[2 * l], c1 = class_count[2 * l + 1];
        int32_t incl = c0 + c1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (l >= o) incl += y;
        }
        const int32_t excl = incl - c0 - c1;
        s_start[2 * l] = excl;
        s_start[2 * l + 1] = excl + c0;
        if (l == 31) s_start[kClasses] = incl;
        if (blockIdx.x == 0) {
            class_start[2 * l] = excl;
            class_start[2 * l + 1] = excl + c0;
            if (l == 31) class_start[kClasses] = incl;
        }
    }
    __syncthreads();
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = j < *n_groups;
    const int c = ok ? gcls[j] : -1 - static_cast<int>(threadIdx.x & 31);
    // threads of one class in this warp: the first takes the atomic for all
    const uint32_t peers = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(peers) - 1, lane = threadIdx.x & 31;
    int32_t base = 0;
    if (ok && lane == leader) base = atomicAdd(&class_fill[c], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!ok) return;
    const int32_t at = s_start[c] + base + __popc(peers & ((1u << lane) - 1u));
    if (!FLOOD_OOB(at, a.groups_cap, &a.ctl->flags)) sorted[at] = a.groups[j];
}

// ---------------------------------------------------------------- shell streaming
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Cells at Chebyshev distance exactly s (in cells) from the inner box [lo, hi],
// as rows along x: rows on the y/z faces of the shell are whole x-ranges, the
// others contribute only their two end cells.
struct Shell {
    int lo[3], hi[3];  // inner box (cells, inclusive)
    int s;
    int y0, ny, z0;
    int rows;
    float wlo[3], whi[3];  // bounding box of the group's samples (world)
    float T2;              // squared search radius: no live sample needs points farther away
    float slack;           // absolute rounding slack of cell boundaries
};

__device__ __forceinline__ void shell_setup(const GridView& g, Shell& sh) {
    const int s = sh.s;
    sh.y0 = max(sh.lo[1] - s, 0);
    const int y1 = min(sh.hi[1] + s, g.dy - 1);
    sh.z0 = max(sh.lo[2] - s, 0);
    const int z1 = min(sh.hi[2] + s, g.dz - 1);
    sh.ny = y1 - sh.y0 + 1;
    const int nz = z1 - sh.z0 + 1;
    sh.rows = (sh.ny > 0 && nz > 0) ? sh.ny * nz : 0;
}

// Gap between the samples' box and the cell slab [c, c+1) along one axis.
__device__ __forceinline__ float slab_gap(float o, float h, int c, float lo, float hi, float slack) {
    const float a = __fmaf_rn(static_cast<float>(c), h, o), b = __fmaf_rn(static_cast<float>(c + 1), h, o);
    return fmaxf(fmaxf(a - hi, lo - b) - slack, 0.0f);
}

// Row r of shell s as up to two point ranges. A row (or the part of it along
// x) whose cells lie farther than sqrt(T2) from every sample of the group
// contributes nothing; it cannot change any live sample's nearest distance.
__device__ __forceinline__ void shell_row(const GridView& g, const Shell& sh, int r, int32_t& b1, int32_t& l1,
                                          int32_t& b2, int32_t& l2, uint32_t* flags) {
    const int s = sh.s;
    const int cy = sh.y0 + r % sh.ny;
    const int cz = sh.z0 + r / sh.ny;
    b1 = b2 = 0;
    l1 = l2 = 0;
    const float gy = slab_gap(g.oy, g.cell, cy, sh.wlo[1], sh.whi[1], sh.slack);
    const float gz = slab_gap(g.oz, g.cell, cz, sh.wlo[2], sh.whi[2], sh.slack);
    const float gyz2 = __fmaf_rn(gy, gy, gz * gz);
    if (gyz2 > sh.T2) return;
    // x cells that can hold a point within sqrt(T2) of the samples' box
    const float w = sqrtf(fmaxf(sh.T2 - gyz2, 0.0f)) + sh.slack;
    const int xa = cell_coord(sh.wlo[0] - w, g.ox, g.inv_cell, g.dx);
    const int xb = cell_coord(sh.whi[0] + w, g.ox, g.inv_cell, g.dx);
    const int64_t base = (static_cast<int64_t>(cz) * g.dy + cy) * g.dx;
    const bool face = s == 0 || cy == sh.lo[1] - s || cy == sh.hi[1] + s || cz == sh.lo[2] - s || cz == sh.hi[2] + s;
    // the cell table gives each range directly (empty ones have length 0),
    // in one round of independent loads
    if (face) {
        const int x0 = max(max(sh.lo[0] - s, 0), xa), x1 = min(min(sh.hi[0] + s, g.dx - 1), xb);
        if (x0 <= x1 && !FLOOD_OOB(base + x1 + 1, g.n_cells + 1, flags)) {
            b1 = g.cell_start[base + x0];
            l1 = g.cell_start[base + x1 + 1] - b1;
        }
    } else {
        const int xl = sh.lo[0] - s, xr = sh.hi[0] + s;
        if (xl >= 0 && xl >= xa && xl <= xb && !FLOOD_OOB(base + xl + 1, g.n_cells + 1, flags)) {
            b1 = g.cell_start[base + xl];
            l1 = g.cell_start[base + xl + 1] - b1;
        }
        if (xr < g.dx && xr >= xa && xr <= xb && !FLOOD_OOB(base + xr + 1, g.n_cells + 1, flags)) {
            b2 = g.cell_start[base + xr];
            l2 = g.cell_start[base + xr + 1] - b2;
        }
    }
}

struct Cursor {
    int32_t row;      // first row not yet fully copied
    int32_t row_pos;  // stream position where `row` begins
    int32_t pos;      // next stream position to copy
};

// Copy up to `want` further points of the shell stream into `buf` with bulk
// copies that complete on `bar` (warp-collective; lane 0 arrives once).
// Returns the number of points copied (warp-uniform).
__device__ __noinline__ int produce_shell_tile(const GridView& g, const Shell& sh, Cursor& c, int want, float4* buf,
                                  uint64_t* bar, int lane, uint32_t* flags) {
    int filled = 0;
    while (filled < want && c.row < sh.rows) {
        const int r = c.row + lane;
        int32_t b1 = 0, l1 = 0, b2 = 0, l2 = 0;
        if (r < sh.rows) shell_row(g, sh, r, b1, l1, b2, l2, flags);
        const int32_t len = l1 + l2;
        int32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int32_t seg = c.row_pos + incl - len;
        const int32_t win_lo = c.pos, win_hi = c.pos + (want - filled);
        const int32_t o1lo = max(seg, win_lo), o1hi = min(seg + l1, win_hi);
        const int32_t o2lo = max(seg + l1, win_lo), o2hi = min(seg + len, win_hi);
        const int32_t n1 = (r < sh.rows && o1hi > o1lo) ? o1hi - o1lo : 0;
        const int32_t n2 = (r < sh.rows && o2hi > o2lo) ? o2hi - o2lo : 0;
        int32_t total = n1 + n2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
        if (total > 0) {
            if (lane == 0) mbar_expect_tx(bar, static_cast<uint32_t>(total) * 16u);
            __syncwarp();
            // (checked builds: a copy out of range is skipped; its bytes never arrive and the wait gives up)
            if (n1 > 0 && !FLOOD_OOB(b1 + (o1lo - seg) + n1 - 1, g.n_pts, flags) &&
                !FLOOD_OOB(filled + (o1lo - win_lo) + n1 - 1, want, flags))
                bulk_copy_g2s(buf + filled + (o1lo - win_lo), g.pts + b1 + (o1lo - seg),
                              static_cast<uint32_t>(n1) * 16u, bar);
            if (n2 > 0 && !FLOOD_OOB(b2 + (o2lo - seg - l1) + n2 - 1, g.n_pts, flags) &&
                !FLOOD_OOB(filled + (o2lo - win_lo) + n2 - 1, want, flags))
                bulk_copy_g2s(buf + filled + (o2lo - win_lo), g.pts + b2 + (o2lo - seg - l1),
                              static_cast<uint32_t>(n2) * 16u, bar);
        }
        filled += total;
        c.pos += total;
        const bool done = (r < sh.rows) && (seg + len <= c.pos);
        const int nfull = __popc(__ballot_sync(0xffffffffu, done));
        if (nfull > 0) {
            c.row_pos += __shfl_sync(0xffffffffu, incl, nfull - 1);
            c.row += nfull;
        }
        if (total == 0 && nfull == 0) break;  // nothing left (defensive)
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
    return filled;
}

// ---------------------------------------------------------------- flood kernel
// Warp minimum / maximum of floats with one redux over order-preserving bit
// patterns (a non-negative float keeps its bits with the sign set, a negative
// one is complemented).
__device__ __forceinline__ uint32_t float_order(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float order_float(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ float warp_min_of(float v) {
    return order_float(__reduce_min_sync(0xffffffffu, float_order(v)));
}
__device__ __forceinline__ float warp_max_of(float v) {
    return order_float(__reduce_max_sync(0xffffffffu, float_order(v)));
}

struct WarpCounters {
    unsigned long long pairs = 0ull, shells = 0ull, tiles = 0ull;
};

// One group of samples on one warp. The warp is W sample lanes x 32/W point
// streams: lane (g, l) = (lane / W, lane % W) holds samples q*W + l for
// q < NS and evaluates them on staged points g, g + 32/W, ...; the partial
// minima of the 32/W streams are combined (shuffles over the stream bits)
// whenever a decision needs them. W is the smallest power of two with
// W * NS >= group size, so small groups keep every lane busy.
template <int NS>
__device__ __forceinline__ void process_group(const DimArgs& a, const GridView& g, int W, int32_t s_begin,
                                              int32_t s_end, float ox, float oy, float oz, float4* tiles,
                                              uint64_t* bar, float* s_u, float* s_lb, uint32_t& phases, bool& abort,
                                              WarpCounters& cnt, int lane) {
    static_assert(NS % 2 == 0, "samples are evaluated in pairs");
    const float shell_h = a.geo->shell_h, shell_slack = a.geo->shell_slack;
    // -2 p' per sample, paired over consecutive samples for packed FMAs
    float2 ax[NS / 2], ay[NS / 2], az[NS / 2];
    float pp[NS], mn[NS];
    bool live[NS];
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {-1, -1, -1};
    float wlo[3] = {INFINITY, INFINITY, INFINITY}, whi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float R = 0.0f;
    const int G = 32 / W;  // point streams
    const int gs = lane / W, lw = lane % W;
    __syncwarp();  // the previous group's reads of s_u / s_lb are complete
    auto slot = [&](int q) { return s_begin + q * W + lw; };
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        const int32_t i = slot(q);
        live[q] = i < s_end;
        float* const qx = (q & 1) ? &ax[q >> 1].y : &ax[q >> 1].x;
        float* const qy = (q & 1) ? &ay[q >> 1].y : &ay[q >> 1].x;
        float* const qz = (q & 1) ? &az[q >> 1].y : &az[q >> 1].x;
        *qx = *qy = *qz = pp[q] = 0.0f;
        mn[q] = INFINITY;
        if (live[q]) {
            const SampleRec r = a.recs[i];
            const float px = __fsub_rn(r.x, ox), py = __fsub_rn(r.y, oy), pz = __fsub_rn(r.z, oz);
            *qx = -2.0f * px;
            *qy = -2.0f * py;
            *qz = -2.0f * pz;
            pp[q] = __fmaf_rn(px, px, __fmaf_rn(py, py, __fmul_rn(pz, pz)));
            R = fmaxf(R, r.u);
            wlo[0] = fminf(wlo[0], r.x);
            wlo[1] = fminf(wlo[1], r.y);
            wlo[2] = fminf(wlo[2], r.z);
            whi[0] = fmaxf(whi[0], r.x);
            whi[1] = fmaxf(whi[1], r.y);
            whi[2] = fmaxf(whi[2], r.z);
            const int cx = cell_coord(r.x, g.ox, g.inv_cell, g.dx);
            const int cy = cell_coord(r.y, g.oy, g.inv_cell, g.dy);
            const int cz = cell_coord(r.z, g.oz, g.inv_cell, g.dz);
            lo[0] = min(lo[0], cx);
            lo[1] = min(lo[1], cy);
            lo[2] = min(lo[2], cz);
            hi[0] = max(hi[0], cx);
            hi[1] = max(hi[1], cy);
            hi[2] = max(hi[2], cz);
            if (gs == 0) {  // one lane per sample keeps its bounds in shared memory
                s_u[i - s_begin] = r.u;
                s_lb[i - s_begin] = r.lb;
            }
        }
    }
    R = warp_max_of(R);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = __reduce_min_sync(0xffffffffu, lo[c]);
        hi[c] = __reduce_max_sync(0xffffffffu, hi[c]);
        wlo[c] = warp_min_of(wlo[c]);
        whi[c] = warp_max_of(whi[c]);
    }
    __syncwarp();  // s_u / s_lb written
    const int n_valid = s_end - s_begin;
    // Beyond shell s every point is at least s*h (less rounding slack) from
    // every sample; at max u_p no nearest point can lie farther out.
    const int dmax = max(g.dx, max(g.dy, g.dz));
    const int s_max = min(static_cast<int>(ceilf((R + shell_slack) / shell_h)) + 1, dmax);
    Shell sh;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        sh.lo[c] = lo[c];
        sh.hi[c] = hi[c];
        sh.wlo[c] = wlo[c];
        sh.whi[c] = whi[c];
    }
    sh.slack = shell_slack + g.cell * (1.0f / 1024.0f);
    // combine the partial minima of the point streams
    auto combine = [&]() {
#pragma unroll
        for (int q = 0; q < NS; ++q)
#pragma unroll
            for (int o = W; o < 32; o <<= 1) mn[q] = fminf(mn[q], __shfl_xor_sync(0xffffffffu, mn[q], o));
    };
    // Search radius: the largest current bound of a live sample (its nearest
    // distance so far, or its vertex bound), slightly inflated.
    auto search_radius2 = [&]() {
        combine();
        float t = 0.0f;
#pragma unroll
        for (int q = 0; q < NS; ++q)
            if (live[q]) t = fmaxf(t, fminf(sqrtf(fmaxf(__fadd_rn(mn[q], pp[q]), 0.0f)), s_u[slot(q) - s_begin]));
#pragma unroll
        for (int o = 1; o < W; o <<= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
        const float T = t * (1.0f + 1.0f / 1024.0f) + sh.slack;
        return T * T;
    };
    // shells below s0 hold no point (block distance field)
    const int s0 = min(first_shell(g, lo, hi, lane), s_max);
    // minima to combine since the last combination; while none, the previous
    // radius (an upper bound of a recomputed one) still prunes safely
    bool dirty = true;
    for (int s = s0; s <= s_max; ++s) {
        sh.s = s;
        shell_setup(g, sh);
        if (dirty) {
            sh.T2 = search_radius2();
            dirty = false;
        }
        ++cnt.shells;
        if (sh.rows > 0) {
            Cursor cur{0, 0, 0};
            int nbuf[2];
            nbuf[0] = produce_shell_tile(g, sh, cur, kWTile, tiles, &bar[0], lane, &a.ctl->flags);
            int b = 0;
            for (;;) {
                const int n = nbuf[b];
                if (!mbar_wait(&bar[b], (phases >> b) & 1u, &a.ctl->flags)) abort = true;
                phases ^= 1u << b;
                if (n == 0 || abort) break;
                const bool more = cur.row < sh.rows;
                if (more)
                    nbuf[b ^ 1] = produce_shell_tile(g, sh, cur, kWTile, tiles + (b ^ 1) * kWTile, &bar[b ^ 1], lane, &a.ctl->flags);
                float4* buf = tiles + b * kWTile;
                for (int e = lane; e < n; e += 32) {
                    float4 p = buf[e];
                    p.x = __fsub_rn(p.x, ox);
                    p.y = __fsub_rn(p.y, oy);
                    p.z = __fsub_rn(p.z, oz);
                    p.w = __fmaf_rn(p.x, p.x, __fmaf_rn(p.y, p.y, __fmul_rn(p.z, p.z)));
                    buf[e] = p;
                }
                __syncwarp();
                // two samples per packed FMA chain: the same three rounded
                // FMAs per pair as the scalar form, in the same order
#pragma unroll 4
                for (int j = gs; j < n; j += G) {
                    const float4 x = buf[j];
                    const float2 xx = make_float2(x.x, x.x), xy = make_float2(x.y, x.y), xz = make_float2(x.z, x.z),
                                 xw = make_float2(x.w, x.w);
#pragma unroll
                    for (int q = 0; q < NS / 2; ++q) {
                        const float2 t = __ffma2_rn(ax[q], xx, __ffma2_rn(ay[q], xy, __ffma2_rn(az[q], xz, xw)));
                        mn[2 * q] = fminf(mn[2 * q], t.x);
                        mn[2 * q + 1] = fminf(mn[2 * q + 1], t.y);
                    }
                }
                cnt.pairs += static_cast<unsigned long long>(n) * static_cast<unsigned long long>(n_valid);
                ++cnt.tiles;
                dirty = true;
                // A row's length depends on the radius, so the radius may only
                // tighten between rows, never inside a partly copied one.
                if (cur.pos == cur.row_pos) {
                    sh.T2 = search_radius2();
                    dirty = false;
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (!more) break;
                b ^= 1;
            }
        }
        if (abort) break;
        if (dirty) {
            combine();
            dirty = false;
        }
        const float sl = fmaxf(__fsub_rn(static_cast<float>(s) * shell_h, shell_slack), 0.0f);
        const float sl2 = __fmul_rn(sl, sl);
        bool done = true;
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            if (live[q]) {
                const float d2 = fmaxf(__fadd_rn(mn[q], pp[q]), 0.0f);
                live[q] = !((d2 <= sl2) || (__fsqrt_rn(d2) <= s_lb[slot(q) - s_begin]));
                done &= !live[q];
            }
        }
        if (__all_sync(0xffffffffu, done)) break;
    }
    if (dirty) combine();
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        const int32_t i = slot(q);
        if (i < s_end && gs == 0) {
            const SampleRec r = a.recs[i];
            const float d2 = fmaxf(__fadd_rn(mn[q], pp[q]), 0.0f);
            if (__fsqrt_rn(d2) > r.lb && !FLOOD_OOB(r.sigma, a.n, &a.ctl->flags))
                atomicMax(&a.best[r.sigma], (static_cast<unsigned long long>(__float_as_uint(d2)) << 32) |
                                                (0xffffffffu - static_cast<uint32_t>(r.s)));
        }
    }
}

constexpr int kNS = 4;       // samples per lane (light groups)
constexpr int kHeavyNS = 4;  // samples per thread slot (heavy groups)

// Largest j with off[j] <= item (off has n + 1 non-decreasing entries).
__device__ __forceinline__ int job_of(const int32_t* off, int n, int32_t item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Light groups of every cloud of the batch: the queue is the concatenation of
// each cloud's sorted groups after its heavy prefix (offsets in light_off;
// NULL for a single cloud).
__global__ void __launch_bounds__(kThreads, 2) k_flood(const DimArgs* jobs, int n_jobs, const int32_t* light_off,
                                                       Ctl* ctl, int k) {
    extern __shared__ __align__(128) float4 s_tiles[];  // kWarps x 2 x kWTile
    __shared__ __align__(8) uint64_t s_bar[kWarps][2];
    __shared__ float s_ub[kWarps][2][kGroup];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4* tiles = s_tiles + warp * 2 * kWTile;
    uint64_t* bar = s_bar[warp];
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t phases = 0u;
    bool abort = false;
    WarpCounters cnt;
    // one cloud: its light groups follow its heavy prefix; a batch: offsets per cloud
    const int32_t total = light_off ? light_off[n_jobs] : jobs[0].group_off[jobs[0].n_coarse] - *jobs[0].n_heavy;
    for (;;) {
        int item = 0;
        if (lane == 0) item = static_cast<int>(atomicAdd(&ctl->head[k], 1u));
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total || abort) break;
        const int j = light_off ? job_of(light_off, n_jobs, item) : 0;
        const DimArgs& a = jobs[j];
        const GridView gv = a.geo->g;
        const Lattice lat = a.geo->lat;
        const int2 gb = a.groups[*a.n_heavy + (item - (light_off ? light_off[j] : 0))];
        const int32_t s_begin = a.bucket_start[int64_t(gb.x) * kFine] + gb.y * kGroup;
        const int32_t s_end = min(s_begin + kGroup, a.bucket_start[int64_t(gb.x + 1) * kFine]);
        // coarse cube corner: the origin of the pair arithmetic for this group
        const int bxi = gb.x % lat.bx, byi = (gb.x / lat.bx) % lat.by, bzi = gb.x / (lat.bx * lat.by);
        const float ox = __fadd_rn(lat.ox, static_cast<float>(bxi) * lat.B);
        const float oy = __fadd_rn(lat.oy, static_cast<float>(byi) * lat.B);
        const float oz = __fadd_rn(lat.oz, static_cast<float>(bzi) * lat.B);
        const int n = s_end - s_begin;
        int W = 1;  // sample lanes: the fewest whose slots hold the group
        while (W * kNS < n) W <<= 1;
        process_group<kNS>(a, gv, W, s_begin, s_end, ox, oy, oz, tiles, bar, s_ub[warp][0], s_ub[warp][1], phases,
                           abort, cnt, lane);
    }
    if (lane == 0) {
        atomicAdd(&ctl->pairs[k], cnt.pairs);
        atomicAdd(&ctl->shells[k], cnt.shells);
        atomicAdd(&ctl->tiles[k], cnt.tiles);
    }
}

// ---------------------------------------------------------------- heavy groups
// Groups whose vertex bound allows many shells (samples in empty regions)
// scan far and long; one whole CTA takes each of them. All threads enumerate
// a shell's rows together (the walk over the cell table, not the arithmetic,
// bounds these groups) and fill one shared tile by bulk copies; the layout is the
// warp kernel's (W sample lanes x 256/W point streams) stretched over the CTA,
// and per-sample minima are combined in shared memory.
constexpr int kHeavyTile = 4096;

// Evaluate the NSL used sample slots of one tile (NSL <= kHeavyNS); slots are
// paired for packed FMAs (the same three rounded FMAs per pair, in order).
template <int NSL>
__device__ __forceinline__ void heavy_tile(const float4* buf, int n, int gs, int G, const float2* ax,
                                           const float2* ay, const float2* az, float* mn) {
#pragma unroll 2
    for (int j = gs; j < n; j += G) {
        const float4 x = buf[j];
        if (NSL == 1) {
            const float t = __fmaf_rn(ax[0].x, x.x, __fmaf_rn(ay[0].x, x.y, __fmaf_rn(az[0].x, x.z, x.w)));
            mn[0] = fminf(mn[0], t);
        } else {
            const float2 xx = make_float2(x.x, x.x), xy = make_float2(x.y, x.y), xz = make_float2(x.z, x.z),
                         xw = make_float2(x.w, x.w);
#pragma unroll
            for (int q = 0; q < NSL / 2; ++q) {
                const float2 t = __ffma2_rn(ax[q], xx, __ffma2_rn(ay[q], xy, __ffma2_rn(az[q], xz, xw)));
                mn[2 * q] = fminf(mn[2 * q], t.x);
                mn[2 * q + 1] = fminf(mn[2 * q + 1], t.y);
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads, 2) k_flood_heavy(const DimArgs* jobs, int n_jobs,
                                                             const int32_t* heavy_off, Ctl* ctl, int k) {
    extern __shared__ __align__(128) float4 s_tiles[];  // kHeavyTile points
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_min[kGroup];
    __shared__ int s_live[kGroup];
    __shared__ float s_u[kGroup], s_lb[kGroup];
    __shared__ float s_x[kGroup], s_y[kGroup], s_z[kGroup];
    __shared__ uint32_t s_ub2[kGroup];
    __shared__ int s_item, s_abort;
    __shared__ int32_t s_wsum[kWarps];
    __shared__ float s_T2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    uint32_t phases = 0u;
    unsigned long long pairs = 0ull, n_shells = 0ull, n_tiles = 0ull;
    const int32_t n_heavy = heavy_off ? heavy_off[n_jobs] : *jobs[0].n_heavy;
    for (;;) {
        if (tid == 0) s_item = static_cast<int>(atomicAdd(&ctl->heavy_head[k], 1u));
        __syncthreads();
        const int item = s_item;
        if (item >= n_heavy || s_abort) break;
        const int jb = heavy_off ? job_of(heavy_off, n_jobs, item) : 0;
        const DimArgs& a = jobs[jb];
        const GridView g = a.geo->g;
        const Lattice lat = a.geo->lat;
        const float shell_h = a.geo->shell_h, shell_slack = a.geo->shell_slack;
        const int2 gb = a.groups[item - (heavy_off ? heavy_off[jb] : 0)];
        const int32_t s_begin = a.bucket_start[int64_t(gb.x) * kFine] + gb.y * kGroup;
        const int32_t s_end = min(s_begin + kGroup, a.bucket_start[int64_t(gb.x + 1) * kFine]);
        const int n_valid = s_end - s_begin;
        const int bxi = gb.x % lat.bx, byi = (gb.x / lat.bx) % lat.by, bzi = gb.x / (lat.bx * lat.by);
        const float ox = __fadd_rn(lat.ox, static_cast<float>(bxi) * lat.B);
        const float oy = __fadd_rn(lat.oy, static_cast<float>(byi) * lat.B);
        const float oz = __fadd_rn(lat.oz, static_cast<float>(bzi) * lat.B);
        int W = 1;  // sample threads: the fewest whose slots hold the group
        while (W * kHeavyNS < n_valid) W <<= 1;
        const int G = kThreads / W;
        const int gs = tid / W, lw = tid % W;
        const int nsl = (n_valid + W - 1) / W;  // sample slots in use per thread
        static_assert(kHeavyNS % 2 == 0, "slots are evaluated in pairs");
        float2 ax[kHeavyNS / 2], ay[kHeavyNS / 2], az[kHeavyNS / 2];  // -2 p' per slot, paired
        float pp[kHeavyNS], mn[kHeavyNS];
        bool val[kHeavyNS];
        // the group's records, once, into shared memory
        if (tid < kGroup) {
            s_min[tid] = 0xffffffffu;
            s_live[tid] = tid < n_valid;
            s_ub2[tid] = 0x7f800000u;  // +inf
            if (tid < n_valid) {
                const SampleRec r = a.recs[s_begin + tid];
                s_x[tid] = r.x;
                s_y[tid] = r.y;
                s_z[tid] = r.z;
                s_u[tid] = r.u;
                s_lb[tid] = r.lb;
            }
        }
        __syncthreads();
        // group geometry (every thread reads the same shared records)
        int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {-1, -1, -1};
        float wlo[3] = {INFINITY, INFINITY, INFINITY}, whi[3] = {-INFINITY, -INFINITY, -INFINITY};
        float R = 0.0f;
        for (int i = 0; i < n_valid; ++i) {
            const float rx = s_x[i], ry = s_y[i], rz = s_z[i];
            R = fmaxf(R, s_u[i]);
            wlo[0] = fminf(wlo[0], rx);
            wlo[1] = fminf(wlo[1], ry);
            wlo[2] = fminf(wlo[2], rz);
            whi[0] = fmaxf(whi[0], rx);
            whi[1] = fmaxf(whi[1], ry);
            whi[2] = fmaxf(whi[2], rz);
            const int cx = cell_coord(rx, g.ox, g.inv_cell, g.dx);
            const int cy = cell_coord(ry, g.oy, g.inv_cell, g.dy);
            const int cz = cell_coord(rz, g.oz, g.inv_cell, g.dz);
            lo[0] = min(lo[0], cx);
            lo[1] = min(lo[1], cy);
            lo[2] = min(lo[2], cz);
            hi[0] = max(hi[0], cx);
            hi[1] = max(hi[1], cy);
            hi[2] = max(hi[2], cz);
        }
#pragma unroll
        for (int q = 0; q < kHeavyNS; ++q) {
            const int32_t i = s_begin + q * W + lw;
            val[q] = i < s_end;
            float* const qx = (q & 1) ? &ax[q >> 1].y : &ax[q >> 1].x;
            float* const qy = (q & 1) ? &ay[q >> 1].y : &ay[q >> 1].x;
            float* const qz = (q & 1) ? &az[q >> 1].y : &az[q >> 1].x;
            *qx = *qy = *qz = pp[q] = 0.0f;
            mn[q] = INFINITY;
            if (val[q]) {
                const int li = i - s_begin;
                const float px = __fsub_rn(s_x[li], ox), py = __fsub_rn(s_y[li], oy), pz = __fsub_rn(s_z[li], oz);
                *qx = -2.0f * px;
                *qy = -2.0f * py;
                *qz = -2.0f * pz;
                pp[q] = __fmaf_rn(px, px, __fmaf_rn(py, py, __fmul_rn(pz, pz)));
            }
        }
        // A landmark that is a point of X gives, by its distance, another
        // upper bound of d(p, X), usually far tighter than the simplex's own
        // vertices for samples in empty space; it narrows the search radius.
        // (landmarks farther than R from the samples' box cannot tighten any
        // bound and are skipped; skipping a landmark only loosens a bound)
        const float R2 = R * R;
        for (int l = tid; l < a.n_L; l += kThreads) {
            if (a.vbound[l] != 0.0f) continue;  // not a point of X: no bound from it
            const float lx = a.L[3 * l], ly = a.L[3 * l + 1], lz = a.L[3 * l + 2];
            const float gx = fmaxf(fmaxf(wlo[0] - lx, lx - whi[0]), 0.0f);
            const float gy = fmaxf(fmaxf(wlo[1] - ly, ly - whi[1]), 0.0f);
            const float gz = fmaxf(fmaxf(wlo[2] - lz, lz - whi[2]), 0.0f);
            if (!(gx * gx + gy * gy + gz * gz < R2)) continue;
            for (int i = 0; i < n_valid; ++i) {
                const float dx = __fsub_rn(lx, s_x[i]), dy = __fsub_rn(ly, s_y[i]), dz = __fsub_rn(lz, s_z[i]);
                const float d2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
                if (d2 < s_u[i] * s_u[i]) atomicMin(reinterpret_cast<unsigned int*>(&s_ub2[i]), __float_as_uint(d2));
            }
        }
        __syncthreads();
        // A sample whose tightened bound cannot exceed the facet maximum (with a
        // margin far above the rounding of the distances the scan would
        // compute) can neither raise the simplex's value nor attain it, so it
        // leaves the group before the scan: s_min = 0 marks it dominated.
        if (tid < n_valid) {
            const float u = fminf(s_u[tid], __fsqrt_ru(__uint_as_float(s_ub2[tid])) * (1.0f + 1.0f / 65536.0f));
            s_u[tid] = u;
            if (__fadd_rn(__fmul_rn(u, 1.0f + 1.0f / 4096.0f), shell_slack) <= s_lb[tid]) {
                s_live[tid] = 0;
                s_min[tid] = 0u;
            }
        }
        __syncthreads();
        R = 0.0f;
        bool any_live = false;
        for (int i = 0; i < n_valid; ++i)
            if (s_live[i]) {
                R = fmaxf(R, s_u[i]);
                any_live = true;
            }
        const int dmax = max(g.dx, max(g.dy, g.dz));
        const int s_max = any_live ? min(static_cast<int>(ceilf((R + shell_slack) / shell_h)) + 1, dmax) : -1;
        Shell sh;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sh.lo[c] = lo[c];
            sh.hi[c] = hi[c];
            sh.wlo[c] = wlo[c];
            sh.whi[c] = whi[c];
        }
        sh.slack = shell_slack + g.cell * (1.0f / 1024.0f);
        // Fold the threads' partial minima into s_min (squared distances >= 0
        // order like their bit patterns) and recompute the search radius.
        auto fold = [&]() {
#pragma unroll
            for (int q = 0; q < kHeavyNS; ++q) {
                float m = mn[q];
                for (int o = W; o < 32; o <<= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (val[q] && gs % (32 / W) == 0 && m < INFINITY)
                    atomicMin(&s_min[q * W + lw], __float_as_uint(fmaxf(__fadd_rn(m, pp[q]), 0.0f)));
            }
            __syncthreads();
            if (warp == 0) {
                float t = 0.0f;
                for (int i = lane; i < n_valid; i += 32)
                    if (s_live[i]) {
                        const float d = s_min[i] == 0xffffffffu ? INFINITY : sqrtf(__uint_as_float(s_min[i]));
                        t = fmaxf(t, fminf(d, s_u[i]));
                    }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
                if (lane == 0) {
                    const float T = t * (1.0f + 1.0f / 1024.0f) + sh.slack;
                    s_T2 = T * T;
                }
            }
            __syncthreads();
        };
        // shells below s0 hold no point; a group with no live sample scans none
        const int s0 = any_live ? min(first_shell(g, lo, hi, lane), s_max) : 0;
        // fold only after tiles were evaluated: otherwise s_min is current and
        // the previous radius (an upper bound of the new one) still prunes safely
        bool dirty = any_live;
        for (int s = s0; s <= s_max; ++s) {
            sh.s = s;
            shell_setup(g, sh);
            if (dirty) {
                fold();
                dirty = false;
            }
            sh.T2 = s_T2;
            ++n_shells;
            // All threads enumerate the shell's rows, 256 at a time: each
            // thread finds its row's point ranges, a block scan places them,
            // and the owners bulk-copy them into the tile window by window.
            for (int row0 = 0; row0 < sh.rows && !s_abort; row0 += kThreads) {
                int32_t b1 = 0, l1 = 0, b2 = 0, l2 = 0;
                if (row0 + tid < sh.rows) shell_row(g, sh, row0 + tid, b1, l1, b2, l2, &a.ctl->flags);
                const int32_t len = l1 + l2;
                int32_t incl = len;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (lane == 31) s_wsum[warp] = incl;
                __syncthreads();
                int32_t before = 0, total = 0;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) {
                    const int32_t v = s_wsum[w];
                    before += w < warp ? v : 0;
                    total += v;
                }
                const int32_t off = before + incl - len;  // stream position of this row
                for (int32_t w0 = 0; w0 < total; w0 += kHeavyTile) {
                    const int32_t cnt = min(kHeavyTile, total - w0);
                    if (tid == 0) mbar_arrive_expect_tx(&s_bar[0], static_cast<uint32_t>(cnt) * 16u);
                    __syncthreads();
                    const int32_t o1lo = max(off, w0), o1hi = min(off + l1, w0 + cnt);
                    const int32_t o2lo = max(off + l1, w0), o2hi = min(off + len, w0 + cnt);
                    if (o1hi > o1lo && !FLOOD_OOB(b1 + (o1hi - off) - 1, g.n_pts, &a.ctl->flags) &&
                        !FLOOD_OOB(o1hi - w0 - 1, kHeavyTile, &a.ctl->flags))
                        bulk_copy_g2s(s_tiles + (o1lo - w0), g.pts + b1 + (o1lo - off),
                                      static_cast<uint32_t>(o1hi - o1lo) * 16u, &s_bar[0]);
                    if (o2hi > o2lo && !FLOOD_OOB(b2 + (o2hi - off - l1) - 1, g.n_pts, &a.ctl->flags) &&
                        !FLOOD_OOB(o2hi - w0 - 1, kHeavyTile, &a.ctl->flags))
                        bulk_copy_g2s(s_tiles + (o2lo - w0), g.pts + b2 + (o2lo - off - l1),
                                      static_cast<uint32_t>(o2hi - o2lo) * 16u, &s_bar[0]);
                    if (!mbar_wait(&s_bar[0], phases & 1u, &a.ctl->flags)) s_abort = 1;
                    phases ^= 1u;
                    __syncthreads();  // any timeout is visible to every thread
                    if (s_abort) break;
                    for (int e = tid; e < cnt; e += kThreads) {
                        float4 p = s_tiles[e];
                        p.x = __fsub_rn(p.x, ox);
                        p.y = __fsub_rn(p.y, oy);
                        p.z = __fsub_rn(p.z, oz);
                        p.w = __fmaf_rn(p.x, p.x, __fmaf_rn(p.y, p.y, __fmul_rn(p.z, p.z)));
                        s_tiles[e] = p;
                    }
                    __syncthreads();
                    if (nsl == 1)
                        heavy_tile<1>(s_tiles, cnt, gs, G, ax, ay, az, mn);
                    else if (nsl == 2)
                        heavy_tile<2>(s_tiles, cnt, gs, G, ax, ay, az, mn);
                    else if (nsl <= 4)
                        heavy_tile<4>(s_tiles, cnt, gs, G, ax, ay, az, mn);
                    else
                        heavy_tile<kHeavyNS>(s_tiles, cnt, gs, G, ax, ay, az, mn);
                    pairs += tid == 0 ? static_cast<unsigned long long>(cnt) * n_valid : 0ull;
                    n_tiles += tid == 0;
                    dirty = true;
                    fence_proxy_async_smem();
                    __syncthreads();  // the tile is free for the next window's copies
                }
                __syncthreads();  // s_wsum is free for the next rows
            }
            if (s_abort) break;
            if (dirty) {
                fold();
                dirty = false;
            }
            // termination: every sample exact (below the next shell) or dominated
            const float sl = fmaxf(__fsub_rn(static_cast<float>(s) * shell_h, shell_slack), 0.0f);
            const float sl2 = __fmul_rn(sl, sl);
            int live = 0;
            if (tid < n_valid && s_live[tid]) {
                const float d2 = s_min[tid] == 0xffffffffu ? INFINITY : __uint_as_float(s_min[tid]);
                const bool fin = (d2 <= sl2) || (__fsqrt_rn(d2) <= s_lb[tid]);
                s_live[tid] = !fin;
                live = !fin;
            }
            if (!__syncthreads_or(live)) break;
        }
        if (dirty) fold();
        if (tid < n_valid) {
            const SampleRec r = a.recs[s_begin + tid];
            const float d2 = __uint_as_float(s_min[tid]);
            if (s_min[tid] != 0xffffffffu && __fsqrt_rn(d2) > r.lb && !FLOOD_OOB(r.sigma, a.n, &a.ctl->flags))
                atomicMax(&a.best[r.sigma], (static_cast<unsigned long long>(s_min[tid]) << 32) |
                                                (0xffffffffu - static_cast<uint32_t>(r.s)));
        }
        __syncthreads();
    }
    if (tid == 0) {
        atomicAdd(&ctl->pairs[k], pairs);
        atomicAdd(&ctl->shells[k], n_shells);
        atomicAdd(&ctl->tiles[k], n_tiles);
    }
}

// Prefix offsets of the heavy and light queues over the clouds of a batch.
__global__ void k_queue_offsets(const DimArgs* jobs, int n_jobs, int32_t* heavy_off, int32_t* light_off) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int32_t h = 0, l = 0;
    for (int j = 0; j < n_jobs; ++j) {
        heavy_off[j] = h;
        light_off[j] = l;
        const int32_t nh = *jobs[j].n_heavy;
        const int32_t ng = jobs[j].group_off[jobs[j].n_coarse];
        h += nh;
        l += ng - nh;
    }
    heavy_off[n_jobs] = h;
    light_off[n_jobs] = l;
}

// Own maximum per simplex from the packed atomic maxima (0 when no sample can
// exceed the facet maximum).
// ---------------------------------------------------------------- face-max
// f(sigma) = max(sqrt(g2), f(facets)), g2 and its sample from the simplex's
// packed maximum (squared distance bits << 32 | ~sample; 0: no sample above
// the facets); the source of the maximum is the lowest (dim << 28 | row,
// sample) among those attaining it.
__global__ void k_facemax(int k, int64_t n, const int32_t* simplices, const int32_t* facets, int64_t n_lower,
                          const unsigned long long* own, const float* val_lower, const int32_t* src_lower,
                          float* val, int32_t* src, uint32_t* flags) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const unsigned long long b = own[i];
    float best = b ? __fsqrt_rn(__uint_as_float(static_cast<uint32_t>(b >> 32))) : 0.0f;
    int32_t s0 = (k << 28) | static_cast<int32_t>(i), s1 = b ? static_cast<int32_t>(0xffffffffu - static_cast<uint32_t>(b)) : 0;
    for (int j = 0; j <= k; ++j) {
        const int32_t t = (k == 1) ? simplices[i * 2 + (1 - j)] : facets[i * (k + 1) + j];
        if (t < 0 || t >= n_lower) {
            atomicOr(flags, FLAG_RANGE);
            continue;
        }
        const float fv = val_lower[t];
        const int32_t f0 = src_lower[2 * t], f1 = src_lower[2 * t + 1];
        if (fv > best || (fv == best && (f0 < s0 || (f0 == s0 && f1 < s1)))) {
            best = fv;
            s0 = f0;
            s1 = f1;
        }
    }
    val[i] = best;
    src[2 * i] = s0;
    src[2 * i + 1] = s1;
}

// ---------------------------------------------------------------- host side
// Resident CTAs per SM of a flood kernel at its shared-memory size, set up
// once per device (the attribute call and the occupancy query are host
// round trips worth skipping on every call).
template <class K>
int flood_kernel_per_sm(K kernel, size_t smem, int* cache) {
    int dev = 0;
    FLOOD_CUDA(cudaGetDevice(&dev));
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && cache[dev] > 0) return cache[dev];
    FLOOD_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int per_sm = 0;
    FLOOD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem));
    per_sm = std::max(per_sm, 1);
    if (dev >= 0 && dev < 64) cache[dev] = per_sm;
    return per_sm;
}

int launch_flood_heavy(const DimArgs* jobs, int n_jobs, const int32_t* heavy_off, Ctl* ctl, int k,
                       cudaStream_t s) {
    const size_t smem = size_t(kHeavyTile) * sizeof(float4);
    static int cache[64] = {};
    const int per_sm = flood_kernel_per_sm(k_flood_heavy, smem, cache);
    if (per_sm < 0) return per_sm;
    k_flood_heavy<<<static_cast<unsigned>(device_sm_count() * per_sm), kThreads, smem, s>>>(jobs, n_jobs, heavy_off,
                                                                                          ctl, k);
    note_launch();
    FLOOD_CUDA(cudaGetLastError());
    return FLOOD_OK;
}

int launch_flood(const DimArgs* jobs, int n_jobs, const int32_t* light_off, Ctl* ctl, int k, cudaStream_t s) {
    const size_t smem = size_t(kWarps) * 2 * kWTile * sizeof(float4);
    static int cache[64] = {};
    const int per_sm = flood_kernel_per_sm(k_flood, smem, cache);
    if (per_sm < 0) return per_sm;
    const int64_t grid = int64_t(device_sm_count()) * per_sm;
    k_flood<<<static_cast<unsigned>(grid), kThreads, smem, s>>>(jobs, n_jobs, light_off, ctl, k);
    note_launch();
    FLOOD_CUDA(cudaGetLastError());
    return FLOOD_OK;
}

// Sample lattice: coarse edge B = a power of two near extent / c, anchored at
// the grid origin, with c = cbrt(samples / 64) clamped to [4, 40] so that a
// coarse cube holds enough samples for full groups. It depends only on X's
// bounding box and the size of the complex, never on the cell size or on
// how clouds are batched. Computed on the device from the grid's box (one
// thread per job); the host sizes the bucket arrays for the largest lattice
// any box can give: ext / B <= sqrt(2) c per axis, so at most cap_axis =
// floor(1.5 c) + 2 cubes per axis (B doubles should rounding exceed it).
float lattice_divisions(int64_t n_samples) {
    return std::min(40.0f, std::max(4.0f, std::cbrt(static_cast<float>(n_samples) / 64.0f)));
}
int lattice_cap_axis(float div) { return static_cast<int>(std::floor(1.5f * div)) + 2; }

__global__ void k_job_geometry(const GridGeom* gg, float div, int cap_axis, JobGeo* out) {
    JobGeo J;
    J.g = gg->v;
    float ext[3], emax = 0.0f;
    for (int c = 0; c < 3; ++c) {
        ext[c] = gg->bbox_hi[c] - gg->bbox_lo[c];
        emax = fmaxf(emax, ext[c]);
    }
    Lattice& L = J.lat;
    L.ox = J.g.ox;
    L.oy = J.g.oy;
    L.oz = J.g.oz;
    float B = emax > 0.0f ? exp2f(rintf(log2f(emax / div))) : 1.0f;
    for (;;) {
        L.bx = static_cast<int>(floorf(ext[0] / B)) + 1;
        L.by = static_cast<int>(floorf(ext[1] / B)) + 1;
        L.bz = static_cast<int>(floorf(ext[2] / B)) + 1;
        if (L.bx <= cap_axis && L.by <= cap_axis && L.bz <= cap_axis) break;
        B *= 2.0f;
    }
    L.B = B;
    L.invB = 1.0f / B;
    L.invF = 2.0f / B;
    J.n_coarse = int64_t(L.bx) * L.by * L.bz;
    J.shell_h = J.g.cell * (1.0f - 1.0f / 1024.0f);
    const float amax = fmaxf(fabsf(J.g.ox), fmaxf(fabsf(J.g.oy), fabsf(J.g.oz)));
    J.shell_slack = (amax + emax) * (1.0f / 262144.0f);
    *out = J;
}

// The calling thread's last filtration: its counters are copied back without
// waiting (pinned buffer: Ctl, then int32 work items per job and dimension)
// and read by flood_last_filtration_stats once the call's stream is done.
struct LastFiltration {
    HostStats buf;
    cudaEvent_t ev[4][2] = {};  // flood kernels of each dimension (timing events, this thread's device)
    int ev_device = -1;
    bool timed[4] = {false, false, false, false};
    int n_jobs = 0;
    int64_t simplices[4] = {0, 0, 0, 0}, samples[4] = {0, 0, 0, 0};
    bool valid = false;
    ~LastFiltration() {
        for (auto& p : ev)
            for (auto& e : p)
                if (e) cudaEventDestroy(e);
    }
    int events() {  // timing events on the current device
        int dev = 0;
        FLOOD_CUDA(cudaGetDevice(&dev));
        if (ev_device != dev) {
            for (auto& p : ev)
                for (auto& e : p) {
                    if (e) cudaEventDestroy(e);
                    e = nullptr;
                }
            for (auto& p : ev)
                for (auto& e : p) FLOOD_CUDA(cudaEventCreate(&e));
            ev_device = dev;
        }
        return FLOOD_OK;
    }
};
thread_local LastFiltration g_last;

// CUDA events around the flood kernel of each dimension, destroyed on scope exit.
// A second stream per host thread and device, with a pair of fork/join
// events, for the light-group kernel: launched beside the heavy-group kernel,
// its CTAs take SM slots as the heavy CTAs run out of groups.
struct SideStream {
    int dev = -1;
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

// The streams and events of one host thread, released when the thread ends.
struct SideStreams {
    SideStream x[8];
    ~SideStreams() {
        for (SideStream& y : x)
            if (y.s) {
                cudaStreamDestroy(y.s);
                cudaEventDestroy(y.fork);
                cudaEventDestroy(y.join);
            }
    }
};

int side_stream(SideStream** out) {
    thread_local SideStreams holder;
    SideStream* side = holder.x;
    int dev = 0;
    FLOOD_CUDA(cudaGetDevice(&dev));
    SideStream& x = side[dev & 7];
    if (x.dev != dev) {
        if (x.s) {
            cudaStreamDestroy(x.s);
            cudaEventDestroy(x.fork);
            cudaEventDestroy(x.join);
        }
        x = SideStream{};
        FLOOD_CUDA(cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking));
        FLOOD_CUDA(cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming));
        FLOOD_CUDA(cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming));
        x.dev = dev;
    }
    *out = &x;
    return FLOOD_OK;
}

}  // namespace

// Vertex values d(v, X) and bounds (k_vertices), for the backward pass.
int launch_vertices(const float* L, int32_t n_L, const flood_grid* grid, float* val, int32_t* src, float* vbound,
                    uint32_t* flags, cudaStream_t s) {
    const unsigned blocks = static_cast<unsigned>(ceil_div(int64_t(n_L) * 32, 256));  // a warp per landmark
    k_vertices<<<blocks, 256, 0, s>>>(L, n_L, view_of(grid), val, src, vbound, flags);
    note_launch();
    FLOOD_CUDA(cudaGetLastError());
    return FLOOD_OK;
}

std::vector<uint8_t> interior_table(int m, int k) {
    // compositions of m into k+1 parts >= 1, lexicographic in (c_0, ..., c_k)
    std::vector<uint8_t> out;
    int c[4];
    if (k == 1) {
        for (c[0] = 1; c[0] <= m - 1; ++c[0]) {
            c[1] = m - c[0];
            out.push_back(uint8_t(c[0]));
            out.push_back(uint8_t(c[1]));
        }
    } else if (k == 2) {
        for (c[0] = 1; c[0] <= m - 2; ++c[0])
            for (c[1] = 1; c[1] <= m - 1 - c[0]; ++c[1]) {
                c[2] = m - c[0] - c[1];
                for (int j = 0; j < 3; ++j) out.push_back(uint8_t(c[j]));
            }
    } else if (k == 3) {
        for (c[0] = 1; c[0] <= m - 3; ++c[0])
            for (c[1] = 1; c[1] <= m - 2 - c[0]; ++c[1])
                for (c[2] = 1; c[2] <= m - 1 - c[0] - c[1]; ++c[2]) {
                    c[3] = m - c[0] - c[1] - c[2];
                    for (int j = 0; j < 4; ++j) out.push_back(uint8_t(c[j]));
                }
    }
    return out;
}

// Device copy of interior_table(m, k), uploaded once per device and kept for
// the life of the process (at most C(63, 3) x 4 bytes per (m, k)).
int device_interior_table(int m, int k, const std::vector<uint8_t>& host, const uint8_t** out) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int>, uint8_t*> cache;
    int dev = 0;
    FLOOD_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    uint8_t*& p = cache[std::make_tuple(dev, m, k)];
    if (!p) {
        uint8_t* q = nullptr;
        FLOOD_CUDA(cudaMalloc(&q, host.size()));
        const cudaError_t e = cudaMemcpy(q, host.data(), host.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(q);
            return cuda_fail(e, "interior table upload");
        }
        p = q;
    }
    *out = p;
    return FLOOD_OK;
}

// Barycentric coordinates of the interior grid, fl(c_j / m) in binary32 (the
// rounding of sample_offset's division), uploaded once per (device, m, k).
int device_lambda_table(int m, int k, const std::vector<uint8_t>& comp, const float** out) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int>, float*> cache;
    int dev = 0;
    FLOOD_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    float*& p = cache[std::make_tuple(dev, m, k)];
    if (!p) {
        std::vector<float> lam(comp.size());
        const volatile float fm = static_cast<float>(m);  // binary32 division, rounded to nearest
        for (size_t i = 0; i < comp.size(); ++i) lam[i] = static_cast<float>(comp[i]) / fm;
        float* q = nullptr;
        FLOOD_CUDA(cudaMalloc(&q, sizeof(float) * std::max<size_t>(lam.size(), 1)));
        const cudaError_t e = cudaMemcpy(q, lam.data(), sizeof(float) * lam.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(q);
            return cuda_fail(e, "barycentric table upload");
        }
        p = q;
    }
    *out = p;
    return FLOOD_OK;
}


}  // namespace flood

using namespace flood;

extern "C" int flood_last_filtration_stats(flood_filtration_stats* out) {
    if (!out) {
        set_error("flood_last_filtration_stats: out is NULL");
        return FLOOD_EINVAL;
    }
    flood_filtration_stats st{};
    if (g_last.valid) {
        FLOOD_CUDA(cudaEventSynchronize(g_last.buf.done));
        Ctl c;
        const unsigned char* hb = static_cast<const unsigned char*>(g_last.buf.host);
        memcpy(&c, hb, sizeof(Ctl));
        const int32_t* items = reinterpret_cast<const int32_t*>(hb + sizeof(Ctl));
        for (int k = 0; k <= 3; ++k) {
            st.simplices[k] = g_last.simplices[k];
            st.samples[k] = g_last.samples[k];
            for (int i = 0; i < g_last.n_jobs; ++i) st.work_items[k] += items[i * 4 + k];
            st.pairs[k] = static_cast<int64_t>(c.pairs[k]);
            st.active_samples[k] = static_cast<int64_t>(c.active[k]);
            st.shells[k] = static_cast<int64_t>(c.shells[k]);
            st.tiles[k] = static_cast<int64_t>(c.tiles[k]);
            if (g_last.timed[k]) cudaEventElapsedTime(&st.flood_kernel_ms[k], g_last.ev[k][0], g_last.ev[k][1]);
        }
    }
    *out = st;
    return FLOOD_OK;
}

namespace flood {
namespace {

// Per-cloud state of one batched filtration call.
struct JobState {
    flood_filtration_job in;
    float* val[4];
    int32_t* src[4];
    int64_t nk[4];
    int I[4];
    JobGeo* geo;  // device
    int64_t n_coarse, n_buckets, max_samples, max_n, max_groups;  // capacities
    std::vector<uint8_t> tables[4];
    const uint8_t* comp[4];
    const float* lam[4];
    const float* w[4];
    float* vbound;
    // per dimension, carved from one region zeroed by a single memset
    int32_t *bcount[4], *bfill[4], *cls[4];
    unsigned long long* best[4];
    int32_t *bstart, *goff;
    int32_t* tile_sums;  // per tile of kCubeTile cubes: samples, then groups
    int2 *groups, *groups_sorted;
    int32_t* gcls;  // class of each group (cube order)
    SampleRec* recs;
    int heavy_shells;  // groups with at least this many shells go to the CTA kernel
};

int check_job(const flood_filtration_job& j, int idx) {
    if (!j.grid || !j.L || j.n_landmarks < 1 || j.m < 1 || j.m > FLOOD_MAX_M) {
        set_error("flood_filtration: job %d needs grid, L, n_landmarks >= 1 and 1 <= m <= %d", idx, FLOOD_MAX_M);
        return FLOOD_EINVAL;
    }
    if (j.n_simplices[0] != 0 && j.n_simplices[0] != j.n_landmarks) {
        set_error("flood_filtration: job %d: n_simplices[0] must be 0 or n_landmarks", idx);
        return FLOOD_EINVAL;
    }
    for (int k = 1; k <= 3; ++k) {
        if (j.n_simplices[k] < 0 || j.n_simplices[k] >= (int64_t(1) << 28)) {
            set_error("flood_filtration: job %d: n_simplices[%d] out of range", idx, k);
            return FLOOD_EINVAL;
        }
        if (j.n_simplices[k] > 0 && (!j.simplices[k] || (k >= 2 && !j.facets[k]))) {
            set_error("flood_filtration: job %d: simplices[%d] (and facets for k >= 2) must be given", idx, k);
            return FLOOD_EINVAL;
        }
        if (j.n_simplices[k] > 0 && k >= 2 && j.n_simplices[k - 1] == 0) {
            set_error("flood_filtration: job %d: dimension %d present without dimension %d", idx, k, k - 1);
            return FLOOD_EINVAL;
        }
    }
    return FLOOD_OK;
}

// Caller-given sample sets of one job (random P_sigma): per dimension k >= 1,
// S[k] points per simplex as barycentric coordinates (n_k, S[k], k+1).
struct GivenSets {
    const float* w[4];
    int32_t S[4];
};

int check_given(const flood_filtration_job& j, const GivenSets& g) {
    for (int k = 1; k <= 3; ++k) {
        if (g.S[k] < 0 || g.S[k] > FLOOD_MAX_GIVEN_SAMPLES) {
            set_error("flood_filtration_given: n_samples[%d] must be in [0, %d]", k, FLOOD_MAX_GIVEN_SAMPLES);
            return FLOOD_EINVAL;
        }
        if (j.n_simplices[k] > 0 && g.S[k] > 0) {
            if (!g.w[k]) {
                set_error("flood_filtration_given: weights[%d] is NULL", k);
                return FLOOD_EINVAL;
            }
            if (j.n_simplices[k] * g.S[k] >= (int64_t(1) << 31)) {
                set_error("flood_filtration_given: n_simplices[%d] * n_samples[%d] must be below 2^31", k, k);
                return FLOOD_EINVAL;
            }
        }
    }
    return FLOOD_OK;
}

int filtration_batch(const flood_filtration_job* in, int n_jobs, cudaStream_t s,
                     const GivenSets* given = nullptr) {
    if (n_jobs < 0 || (n_jobs > 0 && !in)) {
        set_error("flood_filtration_batch: bad job array");
        return FLOOD_EINVAL;
    }
    for (int i = 0; i < n_jobs; ++i) {
        if (int rc = check_job(in[i], i)) return rc;
        if (given)
            if (int rc = check_given(in[i], given[i])) return rc;
    }
    if (int rc = pending_error(s)) return rc;
    Scratch scr(s);
    Ctl* ctl;
    int rc;
    if ((rc = scr.alloc(&ctl, 1))) return rc;
    FLOOD_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    std::vector<JobState> js(n_jobs);
    for (int i = 0; i < n_jobs; ++i) {
        JobState& J = js[i];
        J.in = in[i];
        const flood_grid* grid = J.in.grid;
        J.nk[0] = J.in.n_landmarks;
        for (int k = 1; k <= 3; ++k) J.nk[k] = J.in.n_simplices[k];
        for (int k = 0; k <= 3; ++k) {
            J.val[k] = J.in.values[k];
            J.src[k] = J.in.src[k];
            if (!J.val[k] && (rc = scr.alloc(&J.val[k], J.nk[k]))) return rc;
            if (!J.src[k] && (rc = scr.alloc(&J.src[k], 2 * J.nk[k]))) return rc;
        }
        if ((rc = scr.alloc(&J.vbound, J.nk[0]))) return rc;
        const unsigned vblocks = static_cast<unsigned>(ceil_div(J.nk[0] * int64_t(32), 256));  // a warp per landmark
        k_vertices<<<vblocks, 256, 0, s>>>(J.in.L, J.in.n_landmarks, view_of(grid), J.val[0], J.src[0], J.vbound,
                                           &ctl->flags);
        note_launch();
        FLOOD_CUDA(cudaGetLastError());
        J.max_samples = 1;
        J.max_n = 1;
        int64_t total_samples = 0;
        for (int k = 1; k <= 3; ++k) {
            J.I[k] = 0;
            J.comp[k] = nullptr;
            J.lam[k] = nullptr;
            J.w[k] = nullptr;
            if (J.nk[k] == 0) continue;
            if (given) {
                J.I[k] = given[i].S[k];
                J.w[k] = given[i].w[k];
            } else {
                J.tables[k] = interior_table(J.in.m, k);
                J.I[k] = static_cast<int>(J.tables[k].size() / (k + 1));
            }
            J.max_samples = std::max(J.max_samples, J.nk[k] * J.I[k]);
            J.max_n = std::max(J.max_n, J.nk[k]);
            total_samples += J.nk[k] * J.I[k];
            if (!given && J.I[k] > 0 && ((rc = device_interior_table(J.in.m, k, J.tables[k], &J.comp[k])) ||
                                         (rc = device_lambda_table(J.in.m, k, J.tables[k], &J.lam[k]))))
                return rc;
        }
        const float div = lattice_divisions(total_samples);
        const int cap_axis = lattice_cap_axis(div);
        J.n_coarse = int64_t(cap_axis) * cap_axis * cap_axis;
        J.n_buckets = J.n_coarse * kFine;
        if ((rc = scr.alloc(&J.geo, 1))) return rc;
        k_job_geometry<<<1, 1, 0, s>>>(grid->geom, div, cap_axis, J.geo);
        note_launch();
        J.max_groups = J.max_samples / kGroup + J.n_coarse + 1;
        if ((rc = scr.alloc(&J.bstart, J.n_buckets + 1)) || (rc = scr.alloc(&J.goff, J.n_coarse + 1)) ||
            (rc = scr.alloc(&J.tile_sums, 2 * ceil_div(J.n_coarse, kCubeTile))) ||
            (rc = scr.alloc(&J.groups, J.max_groups)) || (rc = scr.alloc(&J.groups_sorted, J.max_groups)) ||
            (rc = scr.alloc(&J.gcls, J.max_groups)) ||
            (rc = scr.alloc(&J.recs, J.max_samples)))
            return rc;
        // bucket counts and fills, class table and per-simplex maxima of every
        // dimension in 8-byte words of one region, cleared by one memset
        const int64_t w_buckets = (J.n_buckets * 4 + 7) / 8, w_cls = ((3 * kClasses + 1) * 4 + 7) / 8;
        int64_t words = 0;
        for (int k = 1; k <= 3; ++k)
            if (J.nk[k] > 0) words += 2 * w_buckets + w_cls + J.nk[k];
        unsigned long long* zr;
        if ((rc = scr.alloc(&zr, std::max<int64_t>(words, 1)))) return rc;
        FLOOD_CUDA(cudaMemsetAsync(zr, 0, sizeof(unsigned long long) * std::max<int64_t>(words, 1), s));
        for (int k = 1; k <= 3; ++k) {
            J.bcount[k] = J.bfill[k] = J.cls[k] = nullptr;
            J.best[k] = nullptr;
            if (J.nk[k] == 0) continue;
            J.bcount[k] = reinterpret_cast<int32_t*>(zr);
            J.bfill[k] = reinterpret_cast<int32_t*>(zr + w_buckets);
            J.cls[k] = reinterpret_cast<int32_t*>(zr + 2 * w_buckets);
            J.best[k] = zr + 2 * w_buckets + w_cls;
            zr += 2 * w_buckets + w_cls + J.nk[k];
        }
        J.heavy_shells = tuning_for(grid->n_points, J.in.n_landmarks, J.in.m).heavy_shells;
    }
    int32_t* d_counts;  // work items per (job, dimension), for the statistics
    if ((rc = scr.alloc(&d_counts, 4 * std::max(n_jobs, 1)))) return rc;
    FLOOD_CUDA(cudaMemsetAsync(d_counts, 0, sizeof(int32_t) * 4 * std::max(n_jobs, 1), s));
    g_last.valid = false;
    if ((rc = g_last.events())) return rc;
    for (int k = 0; k < 4; ++k) g_last.timed[k] = false;
    // every dimension's job table, built and uploaded at once (all pointers are known now)
    std::vector<DimArgs> h_jobs;
    std::vector<int> job_of_entry;
    int first[5] = {0, 0, 0, 0, 0};
    for (int k = 1; k <= 3; ++k) {
        first[k] = static_cast<int>(h_jobs.size());
        for (int i = 0; i < n_jobs; ++i) {
            JobState& J = js[i];
            if (J.nk[k] == 0 || J.I[k] == 0) continue;
            DimArgs a{};
            a.k = k;
            a.I = J.I[k];
            a.m = static_cast<float>(J.in.m);
            a.n = J.nk[k];
            a.simplices = J.in.simplices[k];
            a.facets = k >= 2 ? J.in.facets[k] : nullptr;
            a.val_lower = J.val[k - 1];
            a.n_lower = J.nk[k - 1];
            a.comp = J.comp[k];
            a.lam = J.lam[k];
            a.w = J.w[k];
            a.L = J.in.L;
            a.vbound = J.vbound;
            a.n_L = J.in.n_landmarks;
            a.geo = J.geo;
            a.n_buckets = J.n_buckets;
            a.n_coarse = J.n_coarse;
            a.bucket_count = J.bcount[k];
            a.bucket_start = J.bstart;
            a.bucket_fill = J.bfill[k];
            a.group_off = J.goff;
            a.groups = J.groups_sorted;  // the flood kernels read the longest-first order
            a.recs = J.recs;
            a.rec_cap = J.max_samples;
            a.groups_cap = J.max_groups;
            a.best = J.best[k];
            a.ctl = ctl;
            // heavy groups: shell bound >= heavy_shells, i.e. classes [0, kClasses - heavy_shells)
            a.n_heavy = J.cls[k] + 2 * kClasses + (kClasses - J.heavy_shells);
            h_jobs.push_back(a);
            job_of_entry.push_back(i);
        }
    }
    first[4] = static_cast<int>(h_jobs.size());
    DimArgs* d_jobs = nullptr;
    int32_t* d_off = nullptr;  // queue offsets (batches of several clouds)
    if (!h_jobs.empty()) {
        if ((rc = scr.alloc(&d_jobs, h_jobs.size())) || (rc = scr.alloc(&d_off, 2 * (n_jobs + 1)))) return rc;
        FLOOD_CUDA(cudaMemcpyAsync(d_jobs, h_jobs.data(), sizeof(DimArgs) * h_jobs.size(), cudaMemcpyHostToDevice, s));
    }
    for (int k = 1; k <= 3; ++k) {
        const int nj = first[k + 1] - first[k];
        for (int e = first[k]; e < first[k + 1]; ++e) {
            DimArgs a = h_jobs[e];
            JobState& J = js[job_of_entry[e]];
            a.groups = J.groups;  // preparation kernels fill the cube order; the class scatter sorts it
            const unsigned wb = static_cast<unsigned>(ceil_div(a.n * 32, 256));
            k_samples<false><<<wb, 256, 0, s>>>(a);
            const unsigned tiles = static_cast<unsigned>(ceil_div(J.n_coarse, kCubeTile));
            k_cube_sums<<<tiles, kCubeTile, 0, s>>>(J.bcount[k], J.n_coarse, J.tile_sums, J.tile_sums + tiles);
            k_cube_scan<<<tiles, kCubeTile, 0, s>>>(J.bcount[k], J.n_coarse, J.tile_sums, J.tile_sums + tiles,
                                                    J.bstart, J.goff, J.groups, J.max_groups, &ctl->flags);
            k_samples<true><<<wb, 256, 0, s>>>(a);
            // longest-first order of this cloud's groups; the count stays on the device
            const int32_t* n_groups = J.goff + J.n_coarse;
            // cls: counts [0, kClasses), fill [kClasses, 2 kClasses), starts [2 kClasses, 3 kClasses + 1)
            const unsigned gbk = static_cast<unsigned>(ceil_div(J.max_groups, 256));
            const unsigned gwk = static_cast<unsigned>(std::min<int64_t>(ceil_div(J.max_groups, 8), 148 * 8));
            int32_t* cls = J.cls[k];
            k_group_class_count<<<gwk, 256, 0, s>>>(a, n_groups, cls, J.gcls);
            k_group_class_scatter<<<gbk, 256, 0, s>>>(a, n_groups, cls, cls + 2 * kClasses, cls + kClasses,
                                                      J.groups_sorted, d_counts + job_of_entry[e] * 4 + k, J.gcls);
            note_launch(6);
            FLOOD_CUDA(cudaGetLastError());
        }
        if (nj > 0) {
            const DimArgs* dj = d_jobs + first[k];
            // a batch needs the queue offsets of its clouds; one cloud's queues start at 0
            int32_t* heavy_off = nullptr;
            int32_t* light_off = nullptr;
            if (nj > 1) {
                heavy_off = d_off;
                light_off = d_off + (nj + 1);
                if (k > 1 && (rc = scr.alloc(&heavy_off, 2 * (nj + 1)))) return rc;  // earlier launches may read d_off
                if (k > 1) light_off = heavy_off + (nj + 1);
                k_queue_offsets<<<1, 32, 0, s>>>(dj, nj, heavy_off, light_off);
                note_launch();
            }
            FLOOD_CUDA(cudaEventRecord(g_last.ev[k][0], s));
            SideStream* side;
            if ((rc = side_stream(&side))) return rc;
            FLOOD_CUDA(cudaEventRecord(side->fork, s));
            FLOOD_CUDA(cudaStreamWaitEvent(side->s, side->fork, 0));
            if ((rc = launch_flood_heavy(dj, nj, heavy_off, ctl, k, s))) return rc;
            if ((rc = launch_flood(dj, nj, light_off, ctl, k, side->s))) return rc;
            FLOOD_CUDA(cudaEventRecord(side->join, side->s));
            FLOOD_CUDA(cudaStreamWaitEvent(s, side->join, 0));
            FLOOD_CUDA(cudaEventRecord(g_last.ev[k][1], s));
            g_last.timed[k] = true;
        }
        for (int i = 0; i < n_jobs; ++i) {
            JobState& J = js[i];
            const int64_t n = J.nk[k];
            if (n == 0) continue;
            k_facemax<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, s>>>(
                k, n, J.in.simplices[k], J.in.facets[k], J.nk[k - 1], J.best[k], J.val[k - 1], J.src[k - 1],
                J.val[k], J.src[k], &ctl->flags);
            note_launch();
            FLOOD_CUDA(cudaGetLastError());
        }
    }
    // counters back without waiting; the status word is reported by flood_check
    const size_t stat_bytes = sizeof(Ctl) + sizeof(int32_t) * 4 * std::max(n_jobs, 1);
    if ((rc = g_last.buf.reserve(stat_bytes))) return rc;
    unsigned char* hb = static_cast<unsigned char*>(g_last.buf.host);
    FLOOD_CUDA(cudaMemcpyAsync(hb, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    if (n_jobs > 0)
        FLOOD_CUDA(cudaMemcpyAsync(hb + sizeof(Ctl), d_counts, sizeof(int32_t) * 4 * n_jobs, cudaMemcpyDeviceToHost, s));
    FLOOD_CUDA(cudaEventRecord(g_last.buf.done, s));
    g_last.n_jobs = n_jobs;
    for (int k = 0; k <= 3; ++k) {
        g_last.simplices[k] = g_last.samples[k] = 0;
        for (int i = 0; i < n_jobs; ++i) {
            g_last.simplices[k] += js[i].nk[k];
            g_last.samples[k] += k == 0 ? 0 : js[i].nk[k] * js[i].I[k];
        }
    }
    g_last.valid = true;
    return defer_status(s, &ctl->flags, "flood_filtration");
}

}  // namespace
}  // namespace flood

extern "C" int flood_filtration_batch(const flood_filtration_job* jobs, int32_t n_jobs, void* stream) {
    return filtration_batch(jobs, n_jobs, static_cast<cudaStream_t>(stream));
}

extern "C" int flood_filtration(const flood_grid* grid, const float* L, int32_t n_landmarks,
                                const int32_t* const simplices[4], const int32_t* const facets[4],
                                const int64_t n_simplices[4], int32_t m, float* const values[4],
                                int32_t* const src[4], void* stream) {
    if (!simplices || !n_simplices || !values) {
        set_error("flood_filtration: simplices, n_simplices and values must be given");
        return FLOOD_EINVAL;
    }
    flood_filtration_job j{};
    j.grid = grid;
    j.L = L;
    j.n_landmarks = n_landmarks;
    j.m = m;
    for (int k = 0; k < 4; ++k) {
        j.simplices[k] = simplices[k];
        j.facets[k] = facets ? facets[k] : nullptr;
        j.n_simplices[k] = n_simplices[k];
        j.values[k] = values[k];
        j.src[k] = src ? src[k] : nullptr;
    }
    return filtration_batch(&j, 1, static_cast<cudaStream_t>(stream));
}

extern "C" int flood_filtration_given(const flood_grid* grid, const float* L, int32_t n_landmarks,
                                      const int32_t* const simplices[4], const int32_t* const facets[4],
                                      const int64_t n_simplices[4], const float* const weights[4],
                                      const int32_t n_samples[4], float* const values[4], int32_t* const src[4],
                                      void* stream) {
    if (!simplices || !n_simplices || !values || !weights || !n_samples) {
        set_error("flood_filtration_given: simplices, n_simplices, weights, n_samples and values must be given");
        return FLOOD_EINVAL;
    }
    flood_filtration_job j{};
    GivenSets g{};
    j.grid = grid;
    j.L = L;
    j.n_landmarks = n_landmarks;
    j.m = 1;  // unused: the samples are given
    for (int k = 0; k < 4; ++k) {
        j.simplices[k] = simplices[k];
        j.facets[k] = facets ? facets[k] : nullptr;
        j.n_simplices[k] = n_simplices[k];
        j.values[k] = values[k];
        j.src[k] = src ? src[k] : nullptr;
        g.w[k] = k ? weights[k] : nullptr;
        g.S[k] = k ? n_samples[k] : 0;
    }
    return filtration_batch(&j, 1, static_cast<cudaStream_t>(stream), &g);
}
