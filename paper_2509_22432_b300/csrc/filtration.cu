// flood_filtration: flood values of every simplex of Del(L) (§4.1).
//
// Per dimension k = 1..3:
//   prep     one warp per simplex: interior samples (Lemma 1, parts >= 1),
//            R = max_p min_i |p - v_i| (a bound on each sample's nearest
//            distance since v_i ∈ X, the step behind Lemma 2), the cull box
//            in cells, its candidate count, and how many work items it needs.
//   scan     work-item offsets.
//   flood    a persistent kernel pops (simplex, candidate chunk) items from a
//            device queue. Candidates stream through shared memory in tiles
//            filled by 1-D TMA bulk copies (one per row segment of the cull
//            box, double-buffered, mbarrier-tracked), are shifted to the
//            simplex's first vertex and extended with their squared norm,
//            then every lane evaluates its register-resident samples p with
//                |p - x|^2 = |x'|^2 - 2 p'.x' + |p'|^2   (x' = x - v0)
//            as three FMAs and a min per pair.
//   finalize maximum over samples of simplices split over several items.
// Then the face-max pass runs by increasing dimension (§4.1's discretised
// complex; P_tau ⊂ P_sigma, App. A.1): f(sigma) = max(own, facets).
#include <algorithm>
#include <vector>

#include "geometry.cuh"
#include "scan.cuh"

namespace flood {

namespace {

constexpr int kThreads = 256;  // flood kernel CTA: 8 warps
constexpr int kWarps = kThreads / 32;
constexpr int kTile = 1536;    // candidate points per shared-memory tile (24 KB)
constexpr int kQMax = 8;       // samples per lane held in registers
constexpr int kSRMax = kWarps * 32 * kQMax;
constexpr int64_t kChunkPairs = int64_t(1) << 20;  // target pairs per work item

struct Ctl {
    uint32_t flags;
    uint32_t head[4];
    uint32_t split[4];
    uint32_t pad;
    unsigned long long pairs[4];
};

struct SimplexPlan {
    CellBox box;
    int32_t n_cand;
    int32_t n_chunks;
};

// Thread layout of the flood kernel for one dimension.
struct Layout {
    int W;   // lanes sharing one point stream (distinct samples), power of two
    int Q;   // samples per lane
    int NW;  // warps per sample set
    int P;   // point partitions (warps with the same samples)
};

struct DimArgs {
    int k;
    int I;  // interior samples per simplex
    float m;
    int64_t n;
    const int32_t* simplices;
    const uint8_t* comp;  // I x (k+1) interior compositions, lexicographic
    const float* L;
    int32_t n_L;
    GridView g;
    SimplexPlan* plan;
    int32_t* chunks;
    int32_t* item_off;
    int32_t chunk_pts;
    float* g2;      // own squared value (max over interior samples of the min squared distance)
    int32_t* arg;   // interior sample rank attaining g2
    uint32_t* slots;  // n x I, per-sample min squared distance bits of split simplices
    Ctl* ctl;
};

// ---------------------------------------------------------------- vertices
// f(v) = d(v, X) = 0 for a landmark that is a point of X; anything else is an
// input error (the cull bound relies on L ⊂ X).
__global__ void k_vertices(const float* L, int32_t n_L, GridView g, float* val, int32_t* src, uint32_t* flags) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_L) return;
    const float x = L[3 * v], y = L[3 * v + 1], z = L[3 * v + 2];
    bool found = false;
    if (isfinite(x) && isfinite(y) && isfinite(z)) {
        const int cx = cell_coord(x, g.ox, g.inv_cell, g.dx);
        const int cy = cell_coord(y, g.oy, g.inv_cell, g.dy);
        const int cz = cell_coord(z, g.oz, g.inv_cell, g.dz);
        const int64_t c = (static_cast<int64_t>(cz) * g.dy + cy) * g.dx + cx;
        const int32_t b = g.cell_start[c], e = g.cell_start[c + 1];
        for (int32_t i = b; i < e && !found; ++i) {
            const float4 p = g.pts[i];
            found = __float_as_uint(p.x) == __float_as_uint(x) && __float_as_uint(p.y) == __float_as_uint(y) &&
                    __float_as_uint(p.z) == __float_as_uint(z);
        }
    }
    if (!found) atomicOr(flags, FLAG_NOT_SUBSET);
    val[v] = found ? 0.0f : __int_as_float(0x7fc00000);
    src[2 * v] = v;
    src[2 * v + 1] = 0;
}

// ---------------------------------------------------------------- prep
__global__ void __launch_bounds__(256) k_prep(DimArgs a) {
    const int64_t w = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= a.n) return;
    const int k = a.k;
    const int32_t* ids = a.simplices + w * (k + 1);
    bool ok = true;
    for (int j = 0; j <= k; ++j) ok &= (ids[j] >= 0 && ids[j] < a.n_L);
    if (!ok) {
        if (lane == 0) {
            atomicOr(&a.ctl->flags, FLAG_RANGE);
            a.plan[w] = SimplexPlan{};
            a.chunks[w] = 0;
            a.g2[w] = 0.0f;
            a.arg[w] = 0;
        }
        return;
    }
    Simplex S;
    load_simplex(a.L, ids, k, S);
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float umax = 0.0f;
    for (int s = lane; s < a.I; s += 32) {
        float px, py, pz;
        sample_offset(S, a.comp + s * (k + 1), k, a.m, px, py, pz);
        umax = fmaxf(umax, vertex_bound_sq(S, k, px, py, pz));
        lo[0] = fminf(lo[0], px);
        lo[1] = fminf(lo[1], py);
        lo[2] = fminf(lo[2], pz);
        hi[0] = fmaxf(hi[0], px);
        hi[1] = fmaxf(hi[1], py);
        hi[2] = fmaxf(hi[2], pz);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    }
    const CellBox b = cull_box(a.g, S.v0, lo, hi, __fsqrt_ru(umax));
    const int rows = b.n[1] * b.n[2];
    long long cnt = 0;
    for (int r = lane; r < rows; r += 32) {
        int32_t rb, re;
        box_row(a.g, b, r, rb, re);
        cnt += re - rb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) {
        const int32_t n_chunks = static_cast<int32_t>(cnt > 0 ? (cnt + a.chunk_pts - 1) / a.chunk_pts : 1);
        a.plan[w] = SimplexPlan{b, static_cast<int32_t>(cnt), n_chunks};
        a.chunks[w] = n_chunks;
        atomicAdd(&a.ctl->pairs[k], static_cast<unsigned long long>(cnt) * static_cast<unsigned long long>(a.I));
        if (n_chunks > 1) atomicAdd(&a.ctl->split[k], 1u);
    }
}

// ---------------------------------------------------------------- flood kernel
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Row cursor over the concatenated candidate stream of one cull box (warp 0).
struct Cursor {
    int32_t row;      // first row not yet fully consumed
    int32_t row_pos;  // stream position where `row` begins
    int32_t pos;      // next stream position to copy
};

// Advance `c` so that c.row contains stream position c.pos (warp-collective).
__device__ void cursor_seek(const GridView& g, const CellBox& b, int rows, Cursor& c, int lane) {
    while (c.row < rows) {
        const int r = c.row + lane;
        int32_t len = 0;
        if (r < rows) {
            int32_t rb, re;
            box_row(g, b, r, rb, re);
            len = re - rb;
        }
        int32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        // rows whose end is at or before pos are skipped
        const bool done = (r < rows) && (c.row_pos + incl <= c.pos);
        const unsigned m = __ballot_sync(0xffffffffu, done);
        const int nfull = __popc(m);  // done rows form a prefix
        if (nfull == 0) return;
        const int32_t adv = __shfl_sync(0xffffffffu, incl, nfull - 1);
        c.row += nfull;
        c.row_pos += adv;
        if (nfull < 32) return;
    }
}

// Copy the next `want` stream points into `buf` with bulk copies completing on
// `bar` (warp-collective; lane 0 arrives on the barrier once at the end).
__device__ void produce_tile(const GridView& g, const CellBox& b, int rows, Cursor& c, int want, float4* buf,
                             uint64_t* bar, int lane) {
    int filled = 0;
    while (filled < want && c.row < rows) {
        const int r = c.row + lane;
        int32_t rb = 0, len = 0;
        if (r < rows) {
            int32_t re;
            box_row(g, b, r, rb, re);
            len = re - rb;
        }
        int32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int32_t seg_lo = c.row_pos + incl - len, seg_hi = c.row_pos + incl;
        const int32_t win_lo = c.pos, win_hi = c.pos + (want - filled);
        const int32_t ov_lo = max(seg_lo, win_lo), ov_hi = min(seg_hi, win_hi);
        const int32_t n = (r < rows && ov_hi > ov_lo) ? ov_hi - ov_lo : 0;
        int32_t total = n;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
        if (total > 0) {
            if (lane == 0) mbar_expect_tx(bar, static_cast<uint32_t>(total) * 16u);
            __syncwarp();
            if (n > 0)
                bulk_copy_g2s(buf + filled + (ov_lo - win_lo), g.pts + rb + (ov_lo - seg_lo),
                              static_cast<uint32_t>(n) * 16u, bar);
        }
        filled += total;
        c.pos += total;
        // retire rows that are now fully copied
        const bool done = (r < rows) && (seg_hi <= c.pos);
        const unsigned m = __ballot_sync(0xffffffffu, done);
        const int nfull = __popc(m);
        if (nfull > 0) {
            c.row_pos += __shfl_sync(0xffffffffu, incl, nfull - 1);
            c.row += nfull;
        }
        if (total == 0 && nfull == 0) break;  // nothing left in range (defensive)
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
}

template <int Q>
__global__ void __launch_bounds__(kThreads) k_flood(DimArgs a, Layout lay) {
    extern __shared__ __align__(128) float4 s_tiles[];  // 2 x kTile
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_min[kSRMax];
    __shared__ unsigned long long s_red[kWarps];
    __shared__ unsigned long long s_best;
    __shared__ int s_item, s_sigma, s_chunk, s_abort;
    __shared__ float s_geo[12];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = lay.W, G = 32 / W, NW = lay.NW, P = lay.P;
    const int ss = warp % NW, pp = warp / NW;
    const bool computes = pp < P;
    const int gsub = lane / W, lig = lane % W;
    const int SR = NW * W * Q;
    const int k = a.k, I = a.I;

    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    uint32_t phases = 0u;  // bit b: parity of the next completion of s_bar[b]
    const int32_t total_items = a.item_off[a.n];

    for (;;) {
        if (tid == 0) {
            int item = static_cast<int>(atomicAdd(&a.ctl->head[k], 1u));
            if (s_abort) item = total_items;
            s_item = item;
            if (item < total_items) {
                // simplex owning this item: largest sigma with item_off[sigma] <= item
                int64_t lo = 0, hi = a.n - 1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi + 1) >> 1;
                    if (a.item_off[mid] <= item) lo = mid;
                    else hi = mid - 1;
                }
                s_sigma = static_cast<int>(lo);
                s_chunk = item - a.item_off[lo];
                Simplex S;
                load_simplex(a.L, a.simplices + lo * (k + 1), k, S);
                for (int c = 0; c < 3; ++c) {
                    s_geo[c] = S.v0[c];
                    s_geo[3 + c] = S.e[0][c];
                    s_geo[6 + c] = S.e[1][c];
                    s_geo[9 + c] = S.e[2][c];
                }
            }
        }
        __syncthreads();
        const int item = s_item;
        if (item >= total_items) break;
        const int sigma = s_sigma, chunk = s_chunk;
        const SimplexPlan pl = a.plan[sigma];
        Simplex S;
        for (int c = 0; c < 3; ++c) {
            S.v0[c] = s_geo[c];
            S.e[0][c] = s_geo[3 + c];
            S.e[1][c] = s_geo[6 + c];
            S.e[2][c] = s_geo[9 + c];
        }
        const int rows = pl.box.n[1] * pl.box.n[2];
        const int32_t pos_begin = chunk * a.chunk_pts;
        const int32_t pos_end = min(pos_begin + a.chunk_pts, pl.n_cand);
        const int n_tiles = static_cast<int>((max(pos_end - pos_begin, 0) + kTile - 1) / kTile);
        const bool single = pl.n_chunks == 1;
        if (tid == 0) s_best = 0ull;

        for (int round = 0; round * SR < I; ++round) {
            // ---- samples of this lane: a = -2 p', min accumulator
            float ax[Q], ay[Q], az[Q], mn[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int s = round * SR + ss * (W * Q) + q * W + lig;
                float px = 0.0f, py = 0.0f, pz = 0.0f;
                if (s < I) sample_offset(S, a.comp + s * (k + 1), k, a.m, px, py, pz);
                ax[q] = -2.0f * px;
                ay[q] = -2.0f * py;
                az[q] = -2.0f * pz;
                mn[q] = INFINITY;
            }
            for (int i = tid; i < SR; i += kThreads) s_min[i] = 0xffffffffu;
            __syncthreads();

            // ---- stream candidate tiles
            Cursor cur{0, 0, pos_begin};
            if (warp == 0) {
                cursor_seek(a.g, pl.box, rows, cur, lane);
                if (n_tiles > 0)
                    produce_tile(a.g, pl.box, rows, cur, min(kTile, pos_end - pos_begin), s_tiles, &s_bar[0], lane);
            }
            for (int t = 0; t < n_tiles; ++t) {
                const int bsel = t & 1;
                float4* buf = s_tiles + bsel * kTile;
                const int32_t t_lo = pos_begin + t * kTile;
                const int n_tile = min(kTile, pos_end - t_lo);
                if (warp == 0 && t + 1 < n_tiles)
                    produce_tile(a.g, pl.box, rows, cur, min(kTile, pos_end - (t_lo + kTile)),
                                 s_tiles + (bsel ^ 1) * kTile, &s_bar[bsel ^ 1], lane);
                if (!mbar_wait(&s_bar[bsel], (phases >> bsel) & 1u, &a.ctl->flags)) s_abort = 1;
                phases ^= 1u << bsel;
                // shift to the simplex origin and append |x'|^2
                for (int e = tid; e < n_tile; e += kThreads) {
                    float4 p = buf[e];
                    p.x = __fsub_rn(p.x, S.v0[0]);
                    p.y = __fsub_rn(p.y, S.v0[1]);
                    p.z = __fsub_rn(p.z, S.v0[2]);
                    p.w = __fmaf_rn(p.x, p.x, __fmaf_rn(p.y, p.y, __fmul_rn(p.z, p.z)));
                    buf[e] = p;
                }
                __syncthreads();
                if (computes) {
                    const int step = G * P;
#pragma unroll 2
                    for (int j = pp * G + gsub; j < n_tile; j += step) {
                        const float4 x = buf[j];
#pragma unroll
                        for (int q = 0; q < Q; ++q) {
                            const float t2 = __fmaf_rn(ax[q], x.x, __fmaf_rn(ay[q], x.y, __fmaf_rn(az[q], x.z, x.w)));
                            mn[q] = fminf(mn[q], t2);
                        }
                    }
                }
                fence_proxy_async_smem();
                __syncthreads();
            }

            // ---- per-sample minimum over all streams of the CTA
            if (computes) {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    for (int o = W; o < 32; o <<= 1) mn[q] = fminf(mn[q], __shfl_xor_sync(0xffffffffu, mn[q], o));
                    if (gsub == 0) {
                        const int l = ss * (W * Q) + q * W + lig;
                        const float pp2 = 0.25f * __fmaf_rn(ax[q], ax[q], __fmaf_rn(ay[q], ay[q], __fmul_rn(az[q], az[q])));
                        const float d2 = fmaxf(__fadd_rn(mn[q], pp2), 0.0f);
                        atomicMin(&s_min[l], __float_as_uint(d2));
                    }
                }
            }
            __syncthreads();
            if (single) {
                unsigned long long best = 0ull;
                for (int l = tid; l < SR; l += kThreads) {
                    const int s = round * SR + l;
                    if (s < I) {
                        const unsigned long long key = (static_cast<unsigned long long>(s_min[l]) << 32) |
                                                       (0xffffffffu - static_cast<uint32_t>(s));
                        best = max(best, key);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) best = max(best, static_cast<unsigned long long>(shfl_xor_u64(best, o)));
                if (lane == 0) s_red[warp] = best;
                __syncthreads();
                if (tid == 0) {
                    unsigned long long b = s_best;
                    for (int w2 = 0; w2 < kWarps; ++w2) b = max(b, s_red[w2]);
                    s_best = b;
                }
            } else {
                uint32_t* slot = a.slots + static_cast<int64_t>(sigma) * I;
                for (int l = tid; l < SR; l += kThreads) {
                    const int s = round * SR + l;
                    if (s < I && s_min[l] != 0xffffffffu) atomicMin(&slot[s], s_min[l]);
                }
            }
            __syncthreads();
        }
        if (single && tid == 0) {
            const unsigned long long b = s_best;
            a.g2[sigma] = __uint_as_float(static_cast<uint32_t>(b >> 32));
            a.arg[sigma] = static_cast<int32_t>(0xffffffffu - static_cast<uint32_t>(b));
        }
        __syncthreads();
    }
}

// Max over the per-sample minima of simplices split over several items.
__global__ void k_finalize(DimArgs a) {
    const int64_t w = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= a.n || a.chunks[w] <= 1) return;
    const uint32_t* slot = a.slots + w * a.I;
    unsigned long long best = 0ull;
    for (int s = lane; s < a.I; s += 32)
        best = max(best, (static_cast<unsigned long long>(slot[s]) << 32) | (0xffffffffu - static_cast<uint32_t>(s)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, static_cast<unsigned long long>(shfl_xor_u64(best, o)));
    if (lane == 0) {
        a.g2[w] = __uint_as_float(static_cast<uint32_t>(best >> 32));
        a.arg[w] = static_cast<int32_t>(0xffffffffu - static_cast<uint32_t>(best));
    }
}

// ---------------------------------------------------------------- face-max
// f(sigma) = max(sqrt(g2), f(facets)); the source of the maximum is the
// lowest (dim << 28 | row, sample) among those attaining it.
__global__ void k_facemax(int k, int64_t n, const int32_t* simplices, const int32_t* facets, int64_t n_lower,
                          const float* g2, const int32_t* arg, const float* val_lower, const int32_t* src_lower,
                          float* val, int32_t* src, uint32_t* flags) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    float best = __fsqrt_rn(g2[i]);
    int32_t s0 = (k << 28) | static_cast<int32_t>(i), s1 = arg[i];
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
// Pick (W, Q, NW) minimising the modelled per-lane instruction count per
// candidate point: rounds * (4 Q + 3 + bank-conflict replays) / (G * P).
Layout choose_layout(int I) {
    Layout best{32, 1, 8, 1};
    double best_cost = 1e30;
    for (int W = 1; W <= 32; W <<= 1)
        for (int Q = 1; Q <= kQMax; ++Q)
            for (int NW = 1; NW <= kWarps; NW <<= 1) {
                const int P = kWarps / NW, G = 32 / W;
                const int SR = NW * W * Q;
                const int rounds = (I + SR - 1) / SR;
                const double replay = G > 8 ? 2.0 * (G / 8 - 1) : 0.0;
                const double cost = rounds * (4.0 * Q + 3.0 + replay) / (G * P);
                if (cost < best_cost - 1e-12) {
                    best_cost = cost;
                    best = Layout{W, Q, NW, P};
                }
            }
    return best;
}

template <int Q>
int launch_flood_q(const DimArgs& a, const Layout& lay, cudaStream_t s) {
    const size_t smem = size_t(2) * kTile * sizeof(float4);
    FLOOD_CUDA(cudaFuncSetAttribute(k_flood<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int per_sm = 0;
    FLOOD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_flood<Q>, kThreads, smem));
    per_sm = std::max(per_sm, 1);
    const int64_t grid = int64_t(device_sm_count()) * per_sm;
    k_flood<Q><<<static_cast<unsigned>(grid), kThreads, smem, s>>>(a, lay); note_launch();
    FLOOD_CUDA(cudaGetLastError());
    return FLOOD_OK;
}

int launch_flood(const DimArgs& a, const Layout& lay, cudaStream_t s) {
    switch (lay.Q) {
        case 1: return launch_flood_q<1>(a, lay, s);
        case 2: return launch_flood_q<2>(a, lay, s);
        case 3: return launch_flood_q<3>(a, lay, s);
        case 4: return launch_flood_q<4>(a, lay, s);
        case 5: return launch_flood_q<5>(a, lay, s);
        case 6: return launch_flood_q<6>(a, lay, s);
        case 7: return launch_flood_q<7>(a, lay, s);
        default: return launch_flood_q<8>(a, lay, s);
    }
}

thread_local flood_filtration_stats g_stats;

// CUDA events around the flood kernel of each dimension, destroyed on scope exit.
struct EventPairs {
    cudaEvent_t e[4][2] = {};
    cudaEvent_t* operator[](int k) { return e[k]; }
    ~EventPairs() {
        for (auto& p : e)
            for (auto& x : p)
                if (x) cudaEventDestroy(x);
    }
};

}  // namespace

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


}  // namespace flood

using namespace flood;

extern "C" int flood_last_filtration_stats(flood_filtration_stats* out) {
    if (!out) {
        set_error("flood_last_filtration_stats: out is NULL");
        return FLOOD_EINVAL;
    }
    *out = g_stats;
    return FLOOD_OK;
}

extern "C" int flood_filtration(const flood_grid* grid, const float* L, int32_t n_landmarks,
                                const int32_t* const simplices[4], const int32_t* const facets[4],
                                const int64_t n_simplices[4], int32_t m, float* const values[4],
                                int32_t* const src[4], void* stream_) {
    if (!grid || !L || n_landmarks < 1 || !simplices || !n_simplices || !values || m < 1 || m > FLOOD_MAX_M) {
        set_error("flood_filtration: need grid, L, simplices, n_simplices, values and 1 <= m <= %d", FLOOD_MAX_M);
        return FLOOD_EINVAL;
    }
    if (n_simplices[0] != 0 && n_simplices[0] != n_landmarks) {
        set_error("flood_filtration: n_simplices[0] must be 0 or n_landmarks");
        return FLOOD_EINVAL;
    }
    for (int k = 1; k <= 3; ++k) {
        if (n_simplices[k] < 0 || n_simplices[k] >= (int64_t(1) << 28)) {
            set_error("flood_filtration: n_simplices[%d] out of range", k);
            return FLOOD_EINVAL;
        }
        if (n_simplices[k] > 0 && (!simplices[k] || (k >= 2 && (!facets || !facets[k])))) {
            set_error("flood_filtration: simplices[%d] (and facets for k >= 2) must be given", k);
            return FLOOD_EINVAL;
        }
        if (n_simplices[k] > 0 && k >= 2 && n_simplices[k - 1] == 0) {
            set_error("flood_filtration: dimension %d present without its facets (dimension %d)", k, k - 1);
            return FLOOD_EINVAL;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    Scratch scr(s);
    GridView gv = view_of(grid);
    Ctl* ctl;
    int rc;
    if ((rc = scr.alloc(&ctl, 1))) return rc;
    FLOOD_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));

    float* val[4];
    int32_t* sr[4];
    const int64_t nk[4] = {n_landmarks, n_simplices[1], n_simplices[2], n_simplices[3]};
    for (int k = 0; k <= 3; ++k) {
        val[k] = values[k];
        sr[k] = src ? src[k] : nullptr;
        if (!val[k] && (rc = scr.alloc(&val[k], nk[k]))) return rc;
        if (!sr[k] && (rc = scr.alloc(&sr[k], 2 * nk[k]))) return rc;
    }
    k_vertices<<<static_cast<unsigned>(ceil_div(n_landmarks, 256)), 256, 0, s>>>(L, n_landmarks, gv, val[0], sr[0],
                                                                                 &ctl->flags); note_launch();
    FLOOD_CUDA(cudaGetLastError());

    std::vector<uint8_t> tables[4];
    EventPairs ev;
    float* g2[4] = {};
    int32_t* arg[4] = {};
    int32_t* item_off[4] = {};
    for (int k = 1; k <= 3; ++k) {
        const int64_t n = nk[k];
        if (n == 0) continue;
        tables[k] = interior_table(m, k);
        const int I = static_cast<int>(tables[k].size() / (k + 1));
        if (I == 0) {
            // m <= k: no interior samples; the value is the face maximum alone.
            if ((rc = scr.alloc(&g2[k], n)) || (rc = scr.alloc(&arg[k], n))) return rc;
            FLOOD_CUDA(cudaMemsetAsync(g2[k], 0, sizeof(float) * n, s));
            FLOOD_CUDA(cudaMemsetAsync(arg[k], 0, sizeof(int32_t) * n, s));
            continue;
        }
        uint8_t* comp;
        SimplexPlan* plan;
        int32_t* chunks;
        uint32_t* slots;
        if ((rc = scr.alloc(&comp, tables[k].size())) || (rc = scr.alloc(&plan, n)) || (rc = scr.alloc(&chunks, n)) ||
            (rc = scr.alloc(&item_off[k], n + 1)) || (rc = scr.alloc(&g2[k], n)) || (rc = scr.alloc(&arg[k], n)) ||
            (rc = scr.alloc(&slots, n * I)))
            return rc;
        FLOOD_CUDA(cudaMemcpyAsync(comp, tables[k].data(), tables[k].size(), cudaMemcpyHostToDevice, s));
        FLOOD_CUDA(cudaMemsetAsync(slots, 0xff, sizeof(uint32_t) * n * I, s));
        DimArgs a{};
        a.k = k;
        a.I = I;
        a.m = static_cast<float>(m);
        a.n = n;
        a.simplices = simplices[k];
        a.comp = comp;
        a.L = L;
        a.n_L = n_landmarks;
        a.g = gv;
        a.plan = plan;
        a.chunks = chunks;
        a.item_off = item_off[k];
        a.chunk_pts = static_cast<int32_t>(std::max<int64_t>(kTile, kChunkPairs / I));
        a.g2 = g2[k];
        a.arg = arg[k];
        a.slots = slots;
        a.ctl = ctl;
        k_prep<<<static_cast<unsigned>(ceil_div(n * 32, 256)), 256, 0, s>>>(a); note_launch();
        FLOOD_CUDA(cudaGetLastError());
        if ((rc = exclusive_scan(chunks, item_off[k], n, s, scr))) return rc;
        const Layout lay = choose_layout(I);
        if (cudaEventCreate(&ev[k][0]) == cudaSuccess && cudaEventCreate(&ev[k][1]) == cudaSuccess)
            cudaEventRecord(ev[k][0], s);
        if ((rc = launch_flood(a, lay, s))) return rc;
        if (ev[k][1]) cudaEventRecord(ev[k][1], s);
        k_finalize<<<static_cast<unsigned>(ceil_div(n * 32, 256)), 256, 0, s>>>(a); note_launch();
        FLOOD_CUDA(cudaGetLastError());
    }
    for (int k = 1; k <= 3; ++k) {
        const int64_t n = nk[k];
        if (n == 0) continue;
        k_facemax<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, s>>>(
            k, n, simplices[k], facets ? facets[k] : nullptr, nk[k - 1], g2[k], arg[k], val[k - 1], sr[k - 1], val[k],
            sr[k], &ctl->flags); note_launch();
        FLOOD_CUDA(cudaGetLastError());
    }
    Ctl h_ctl{};
    int32_t h_items[4] = {0, 0, 0, 0};
    FLOOD_CUDA(cudaMemcpyAsync(&h_ctl, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    for (int k = 1; k <= 3; ++k)
        if (item_off[k]) FLOOD_CUDA(cudaMemcpyAsync(&h_items[k], item_off[k] + nk[k], sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FLOOD_CUDA(cudaStreamSynchronize(s));
    rc = status_from_flags(h_ctl.flags, "flood_filtration");
    if (rc) return rc;
    flood_filtration_stats st{};
    for (int k = 0; k <= 3; ++k) {
        st.simplices[k] = nk[k];
        const int I = k == 0 ? 1 : static_cast<int>(tables[k].size() / (k + 1));
        st.samples[k] = nk[k] * (k == 0 ? 0 : I);
        st.pairs[k] = static_cast<int64_t>(h_ctl.pairs[k]);
        st.work_items[k] = h_items[k];
        st.split_simplices[k] = h_ctl.split[k];
        st.flood_kernel_ms[k] = 0.0f;
        if (ev[k][0] && ev[k][1]) cudaEventElapsedTime(&st.flood_kernel_ms[k], ev[k][0], ev[k][1]);
    }
    g_stats = st;
    return FLOOD_OK;
}
