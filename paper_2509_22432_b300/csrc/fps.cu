// flood_fps: farthest point sampling (§3.2), the landmark selection of the
// Flood complex.
//
// Exact FPS with spatial skipping, in one persistent launch for all
// n_landmarks - 1 picks:
//
// * Points are counting-sorted by a Morton code of their position, so a run
//   of 256 consecutive points (a chunk) is spatially compact. Each chunk keeps
//   its bounding box and its candidate: the largest running minimum d_i in it
//   (ties to the lowest original row), with that point's coordinates.
// * A new landmark l can lower d_i only if kappa(x_i, l) < d_i. With every
//   operation rounded to nearest, rounding is monotone, so the binary32 key
//   of any point in a box is at least the same-operation binary32 squared gap
//   between l and the box. A chunk whose gap is >= its largest d_i is
//   therefore provably unchanged and skipped, bit-exactly; after the first few
//   hundred picks almost every chunk is skipped.
// * Four warps of each 1024-thread block run the grid-wide exchange, once per
//   round: each block publishes its eight best candidates with coordinates
//   and a bound on the rest in tagged words, and polls every block's words
//   until all carry the round's tag. That one pass synchronises the grid and
//   delivers the next pick with its coordinates (no dependent load follows),
//   and usually several picks after it as well (see "rounds" below).
//
// The key is the binary32 squared distance with each operation rounded on its
// own (__fsub_rn/__fmul_rn/__fadd_rn are never contracted into FMAs), which
// makes the picks bit-exact against a binary32 reference.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "bbox.cuh"
#include "common.cuh"
#include "scan.cuh"

namespace flood {

namespace {

constexpr int kThreads = 1024;  // one block per SM
constexpr int kWarps = kThreads / 32;
constexpr int kPollers = 4;                // the last four warps run the exchange
constexpr int kComputeWarps = kWarps - kPollers;
constexpr int kLanePts = 8;                // points per lane of a chunk
constexpr int kChunk = 32 * kLanePts;      // points per chunk (resident kernel)
constexpr int64_t kBlockPts = int64_t(kComputeWarps) * kChunk;  // points a resident block holds
constexpr int kMaxBlocks = 160;            // four exchange warps poll 40 blocks each in 5 loads per lane
constexpr int kSlotStride = 16;            // uint64 words per block slot (128 bytes)
constexpr int64_t kSortMin = 16384;        // smaller clouds keep their input order
constexpr int kGlobalBatch = 5;            // global kernel: points per lane loaded at once
constexpr int kMetaBytes = 8 + 10 * 4;     // per chunk in shared memory: candidate, box, coordinates, second
constexpr int kMetaSmemMax = 200 * 1024;

constexpr uint64_t kCandMask = (uint64_t(1) << 62) - 1;

// ---------------------------------------------------------------- point order
// 3-bit interleave of a 10-bit integer (bit k moves to bit 3k).
__device__ __forceinline__ uint32_t spread_bits3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Morton code of each point on a 2^bits lattice over the bounding box, and
// the histogram of codes.
__global__ void __launch_bounds__(256) k_morton_count(const float* X, int64_t n, const uint32_t* box, int bits,
                                                     int32_t* code, int32_t* count) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int top = (1 << bits) - 1;
    uint32_t c = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = from_ordered(box[a]), hi = from_ordered(box[3 + a]);
        const float ext = hi - lo;
        const float scale = ext > 0.0f ? float(1 << bits) / ext : 0.0f;
        int q = __float2int_rd((X[3 * i + a] - lo) * scale);
        q = min(max(q, 0), top);
        c |= spread_bits3(static_cast<uint32_t>(q)) << a;
    }
    code[i] = static_cast<int32_t>(c);
    atomicAdd(&count[c], 1);
}

// Counting-sort scatter into point order, one float4 (x, y, z, original row
// as int bits) per point; `fill` holds the histogram and is counted down
// (order within a code is arbitrary, which changes no result: ties are
// decided by the original row).
__global__ void __launch_bounds__(256) k_morton_scatter(const float* X, int64_t n, const int32_t* code,
                                                       const int32_t* start, int32_t* fill, float4* pts,
                                                       uint32_t* flags) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int32_t c = code[i];
    const int32_t pos = start[c] + atomicSub(&fill[c], 1) - 1;
    if (FLOOD_OOB(pos, n, flags)) return;
    pts[pos] = make_float4(X[3 * i + 0], X[3 * i + 1], X[3 * i + 2], __int_as_float(static_cast<int32_t>(i)));
}

// Input order (small clouds): plain copy into the same packed layout.
__global__ void __launch_bounds__(256) k_pack_rows(const float* X, int64_t n, float4* pts, uint32_t* flags) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const float a = X[3 * i + 0], b = X[3 * i + 1], c = X[3 * i + 2];
    if (!(isfinite(a) && isfinite(b) && isfinite(c))) atomicOr(flags, FLAG_NONFINITE);
    pts[i] = make_float4(a, b, c, __int_as_float(static_cast<int32_t>(i)));
}

// ---------------------------------------------------------------- keys
__device__ __forceinline__ float fps_key(float px, float py, float pz, float lx, float ly, float lz) {
    const float dx = __fsub_rn(px, lx);
    const float dy = __fsub_rn(py, ly);
    const float dz = __fsub_rn(pz, lz);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Squared gap between l and the box [lo, hi] (0 inside), with the same
// rounded operations as fps_key: for every point p in the box each rounded
// step of fps_key(p, l) is >= the matching step here, so the result is a
// lower bound of fps_key(p, l), exactly.
__device__ __forceinline__ float box_gap2(float lx, float ly, float lz, float lox, float loy, float loz, float hix,
                                          float hiy, float hiz) {
    const float gx = fmaxf(fmaxf(__fsub_rn(lox, lx), __fsub_rn(lx, hix)), 0.0f);
    const float gy = fmaxf(fmaxf(__fsub_rn(loy, ly), __fsub_rn(ly, hiy)), 0.0f);
    const float gz = fmaxf(fmaxf(__fsub_rn(loz, lz), __fsub_rn(lz, hiz)), 0.0f);
    return __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
}

// Candidate word: key bits (non-negative binary32, sign dropped) << 31 |
// (0x7fffffff - original row). Larger is better and ties go to the lowest
// row; 0 means "no candidate".
__device__ __forceinline__ uint64_t pack_cand(float d, uint32_t row) {
    return (static_cast<uint64_t>(__float_as_uint(d) & 0x7fffffffu) << 31) | static_cast<uint64_t>(0x7fffffffu - row);
}
__device__ __forceinline__ float cand_key(uint64_t c) {
    return __uint_as_float(static_cast<uint32_t>(c >> 31) & 0x7fffffffu);
}
__device__ __forceinline__ uint32_t cand_row(uint64_t c) {
    return 0x7fffffffu - static_cast<uint32_t>(c & 0x7fffffffu);
}

// Warp maximum of a 64-bit word with two 32-bit redux operations.
__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
    const uint32_t hi = static_cast<uint32_t>(v >> 32);
    const uint32_t mh = __reduce_max_sync(0xffffffffu, hi);
    const uint32_t ml = __reduce_max_sync(0xffffffffu, hi == mh ? static_cast<uint32_t>(v) : 0u);
    return (static_cast<uint64_t>(mh) << 32) | ml;
}

// Warp minimum / maximum of floats through their order-preserving bit
// patterns (one redux each).
__device__ __forceinline__ float warp_min_f(float v) {
    return from_ordered(__reduce_min_sync(0xffffffffu, ordered_bits(v)));
}
__device__ __forceinline__ float warp_max_f(float v) {
    return from_ordered(__reduce_max_sync(0xffffffffu, ordered_bits(v)));
}


struct FpsArgs {
    const float* X;    // (n, 3) input rows (start point)
    const float4* pts;  // points in processing order: x, y, z, original row (int bits)
    float* d;          // running minima (global kernel)
    int64_t n;
    int32_t n_landmarks;
    int64_t start;
    int64_t* out_idx;
    float* out_key;
    uint64_t* slots;   // 2 (parity) x kMaxBlocks lines of kSlotStride words
    uint32_t* flags;   // [0] status flags, [1..6] ordered box, [7] exchange rounds
    int32_t lane_pts;  // global kernel: points per lane of a chunk (multiple of 8)
    int32_t chunks_per_block;
    int64_t n_chunks;
    int32_t poll_blocks;  // blocks whose slots the exchange waits for (gridDim.x)
    uint32_t poll_limit;  // polls before a wait gives up (kWaitPolls)
};

// ---------------------------------------------------------------- rounds
// A round folds the previous round's picks (1 to kMaxPicks landmarks) into
// every chunk, then selects the next picks with one grid-wide exchange:
//
// * Each block reports its eight best entries (an entry is a chunk candidate:
//   the chunk's largest running minimum, ties to the lowest original row, with
//   the point's coordinates; the global kernel reports one entry per warp) and
//   a bound U_b on every other point of the block: the larger of its ninth
//   entry and the largest "second" of any entry (the second-largest minimum
//   of the entry's chunk, or of all of the warp's other points).
// * Each exchange warp keeps the eight best entries of its quarter of the
//   blocks; the bound U is the largest U_b and the largest ninth entry of a
//   quarter, so every point outside the 32 kept entries has a running
//   minimum <= U, now and after any pick (minima only decrease).
// * The kept entries carry their points' exact running minima. Plain FPS
//   picks the point with the largest minimum (ties to the lowest row), so
//   the best kept entry is the next pick; after it, the kept entries' minima
//   are lowered by that pick (kappa to it), and the best of them is the pick
//   after, as long as its minimum is positive and strictly above U (then no
//   point outside the entries can beat or tie it). Repeating this selects
//   several picks per round with the result of plain FPS, bit for bit: on the
//   1M-point torus with 2,000 picks a round makes about four picks.
constexpr int kTop = 4;        // entries a block publishes
constexpr int kKeep = 8;       // entries each exchange warp keeps of its quarter of the blocks
constexpr int kMaxPicks = 32;  // picks per round

// Exchange warps X0..X3 (warps kComputeWarps..kWarps - 1): X0 reduces the
// block's entries, publishes them and polls the first quarter of the blocks;
// X1..X3 poll the other quarters and hand their best entries to X0, which
// merges and selects the picks. Named barriers per round: compute warps
// arrive at kBarCands (X0 waits), X0 arrives at kBarPub once the block's slot
// is published (X1..X3 wait: polling loads would otherwise slow X0's
// shared-memory loads and shuffles, which share the SM's memory pipe),
// X1..X3 arrive at kBarQuarters (X0 waits), X0 arrives at kBarPicks
// (everyone else waits). An arrival releases the arriving thread's earlier
// shared-memory writes to the threads that complete the wait.
constexpr int kX0 = kComputeWarps;  // warp kX0 + 1 is X1 (it records the picks)
constexpr int kBarCands = 1, kBarPicks = 2, kBarQuarters = 3, kBarPub = 4;
constexpr int kCandsCount = (kComputeWarps + 1) * 32;
constexpr int kPollCount = kPollers * 32;
__device__ __forceinline__ void bar_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_wait(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Entries of compute warp w: 32 e + w holds the (e + 1)-th best point of its
// chunk, e < kChunkEntries (resident kernel; the global kernel fills w only).
constexpr int kChunkEntries = 3;
constexpr int kEntries = kChunkEntries * kWarps;

struct FpsShared {
    float4 pxyz[kMaxPicks];     // this round's picks: coordinates (w unused)
    uint64_t cand[kEntries];
    float cx[kEntries], cy[kEntries], cz[kEntries];
    float sec[kWarps];          // bound on every other point of warp w's chunk(s); -1: none
    uint64_t pick[kMaxPicks];   // this round's picks (candidate words with the minimum at the pick)
    int n_pick;                 // picks of the round; -1 = stop (timeout)
    uint64_t qc[kPollers][kKeep];  // best entries of each quarter of the blocks
    float qx[kPollers][kKeep], qy[kPollers][kKeep], qz[kPollers][kKeep];
    float qbound[kPollers];     // each quarter's bound on everything else
    int qstop[kPollers];
    int top[kKeep];             // entry indices of the block's best entries (block_top)
    uint64_t sc[kPollers][32];  // a quarter's entries above its bound, compacted (poll_quarter)
    uint4 ranked[32][2];        // the ranked entries of a round: (word, lane), (x, y, z) (rank_picks)
    float sx[kPollers][32], sy[kPollers][32], sz[kPollers][32];
};

__device__ __forceinline__ void shared_init(FpsShared& s) {
    if (threadIdx.x < kEntries) {
        s.cand[threadIdx.x] = 0ull;
        s.cx[threadIdx.x] = s.cy[threadIdx.x] = s.cz[threadIdx.x] = 0.0f;
    }
    if (threadIdx.x < kWarps) s.sec[threadIdx.x] = -1.0f;
}

__device__ __forceinline__ void order2(uint64_t& a, int& ia, uint64_t& b, int& ib) {
    if (b > a) {
        const uint64_t tv = a;
        a = b;
        b = tv;
        const int ti = ia;
        ia = ib;
        ib = ti;
    }
}

// Block reduction (X0): lane l holds entries l + 32 i (i < 3), sorted; the
// lane holding the k-th best entry records its index in s.top[k], and lane
// k < ntop receives it. Returns the bound on every other point.
__device__ __forceinline__ float block_top(FpsShared& s, int lane, int ntop, uint64_t& me, float& mx, float& my,
                                           float& mz) {
    static_assert(kEntries == 3 * kWarps, "three entries per lane");
    uint64_t e0 = s.cand[lane], e1 = s.cand[kWarps + lane], e2 = s.cand[2 * kWarps + lane];
    int i0 = lane, i1 = kWarps + lane, i2 = 2 * kWarps + lane;
    order2(e0, i0, e1, i1);
    order2(e1, i1, e2, i2);
    order2(e0, i0, e1, i1);
#pragma unroll
    for (int k = 0; k < kKeep; ++k) {
        if (k == ntop) break;
        const uint64_t m = warp_max_u64(e0);
        if (e0 == m) {  // one lane, unless m == 0 (no entry left: any of them may record it)
            s.top[k] = m != 0ull ? i0 : -1;
            e0 = e1;
            i0 = i1;
            e1 = e2;
            i1 = i2;
            e2 = 0ull;
        }
    }
    const float next = cand_key(warp_max_u64(e0));
    const float sec = warp_max_f(s.sec[lane]);
    __syncwarp();
    me = 0ull;
    mx = my = mz = 0.0f;
    if (lane < ntop) {
        const int i = s.top[lane];
        if (i >= 0) {
            me = s.cand[i];
            mx = s.cx[i];
            my = s.cy[i];
            mz = s.cz[i];
        }
    }
    return fmaxf(fmaxf(next, sec), 0.0f);
}

// Bound packed into 30 bits: rounded up to a multiple of 4 in its bit
// pattern (non-negative floats order like their bits), so it decodes to an
// upper bound again.
__device__ __forceinline__ uint32_t bound_up30(float u) { return ((__float_as_uint(u) + 3u) & ~3u) >> 2; }
__device__ __forceinline__ float bound_from30(uint32_t v) { return __uint_as_float(v << 2); }

// Slot of block b for round r (parity r & 1): 128 bytes holding kTop
// entries of four words, each word tagged with r & 3 in its top bits:
//   w0 = tag | candidate
//   w1 = tag | U30 << 32 (first entry only) | bits of x;  w2 = tag | y;  w3 = tag | z.
// A reader accepts a block once all its words carry round r, so every word is
// read atomically and no order between them is needed; a block cannot publish
// round r + 2 (same parity) before every block has finished reading r + 1.
// Exchange warp h polls blocks [40 h, 40 h + 40): in load l, lane 4 i + q
// reads entry q of block 40 h + 8 l + i (one 32-byte access per lane).
constexpr int kBlocksPerLoad = 32 / kTop;
constexpr int kPollLoads = 5;
constexpr int kQuarterBlocks = kBlocksPerLoad * kPollLoads;
static_assert(kPollers * kQuarterBlocks == kMaxBlocks, "the exchange warps cover every block");
static_assert(kPollers * kKeep == 32, "X0 merges one kept entry per lane");
static_assert(kMaxPicks <= 32, "one box-test lane per pick");

// Poll quarter h of the blocks until all carry round r; its best kKeep entries
// go to s.qc[h] etc. (each written by the lane holding it) and its bound on
// every other point to s.qbound[h].
__device__ __forceinline__ void poll_quarter(const FpsArgs& a, FpsShared& s, int r, int h, int lane) {
    const uint64_t tag = static_cast<uint64_t>(r & 3) << 62;
    const uint64_t* buf = a.slots + static_cast<size_t>(r & 1) * kMaxBlocks * kSlotStride;
    const int nb = a.poll_blocks, q = lane % kTop, bi = lane / kTop;
    uint64_t w0[kPollLoads], w1[kPollLoads], w2[kPollLoads], w3[kPollLoads];
    bool stop = false;
    for (uint32_t polls = 0;;) {
#pragma unroll
        for (int l = 0; l < kPollLoads; ++l) {
            const int b = h * kQuarterBlocks + l * kBlocksPerLoad + bi;
            if (b < nb) {
                ld_relaxed_v4_u64(buf + static_cast<size_t>(b) * kSlotStride + 4 * q, w0[l], w1[l], w2[l], w3[l]);
            } else {
                w0[l] = w1[l] = w2[l] = w3[l] = tag;
            }
        }
        uint64_t stale = 0ull;
#pragma unroll
        for (int l = 0; l < kPollLoads; ++l) stale |= (w0[l] ^ tag) | (w1[l] ^ tag) | (w2[l] ^ tag) | (w3[l] ^ tag);
        if (__all_sync(0xffffffffu, (stale >> 62) == 0ull)) break;
        if (++polls > a.poll_limit) {
            stop = true;
            if (lane == 0) atomicOr(a.flags, FLAG_TIMEOUT);
            break;
        }
    }
    uint32_t u30 = 0u;
    uint64_t c[kPollLoads];
    uint32_t cxb[kPollLoads], cyb[kPollLoads], czb[kPollLoads];
#pragma unroll
    for (int l = 0; l < kPollLoads; ++l) {
        if (q == 0) u30 = max(u30, static_cast<uint32_t>(w1[l] >> 32) & 0x3fffffffu);
        c[l] = w0[l] & kCandMask;
        cxb[l] = static_cast<uint32_t>(w1[l]);
        cyb[l] = static_cast<uint32_t>(w2[l]);
        czb[l] = static_cast<uint32_t>(w3[l]);
    }
    u30 = __reduce_max_sync(0xffffffffu, u30);
    // Usually few entries lie above the quarter's largest block bound T: keep
    // the best kKeep of those, ranked in parallel, with the quarter's bound T
    // (or the best entry left out, if above T). That is what the extraction
    // below gives: every entry left out is <= that bound, and with at most
    // kKeep entries above T the kept ones <= T could never be picked but the
    // first of the round, which is the best one and kept here too.
    {
        const float T = bound_from30(u30);
        int n_above = 0;
#pragma unroll
        for (int l = 0; l < kPollLoads; ++l) n_above += __popc(__ballot_sync(0xffffffffu, cand_key(c[l]) > T));
        if (n_above >= 1 && n_above <= kKeep) {
            const uint32_t lt = (1u << lane) - 1u;
            int pos = 0;
#pragma unroll
            for (int l = 0; l < kPollLoads; ++l) {
                const bool above = cand_key(c[l]) > T;
                const uint32_t bl = __ballot_sync(0xffffffffu, above);
                if (above) {
                    const int k = pos + __popc(bl & lt);
                    s.qc[h][k] = c[l];
                    s.qx[h][k] = __uint_as_float(cxb[l]);
                    s.qy[h][k] = __uint_as_float(cyb[l]);
                    s.qz[h][k] = __uint_as_float(czb[l]);
                }
                pos += __popc(bl);
            }
            if (lane >= n_above && lane < kKeep) s.qc[h][lane] = 0ull;
            if (lane == 0) {
                s.qbound[h] = T;
                s.qstop[h] = stop;
            }
            return;
        }
        if (n_above > kKeep && n_above <= 32) {
            const uint32_t lt = (1u << lane) - 1u;
            int pos = 0;
#pragma unroll
            for (int l = 0; l < kPollLoads; ++l) {
                const bool above = cand_key(c[l]) > T;
                const uint32_t bl = __ballot_sync(0xffffffffu, above);
                if (above) {
                    const int k = pos + __popc(bl & lt);
                    s.sc[h][k] = c[l];
                    s.sx[h][k] = __uint_as_float(cxb[l]);
                    s.sy[h][k] = __uint_as_float(cyb[l]);
                    s.sz[h][k] = __uint_as_float(czb[l]);
                }
                pos += __popc(bl);
            }
            __syncwarp();
            // lane j < n_above ranks entry j among them (words are distinct)
            const uint64_t mine = lane < n_above ? s.sc[h][lane] : 0ull;
            int rank = 0;
#pragma unroll 4
            for (int i = 0; i < n_above; ++i) rank += s.sc[h][i] > mine ? 1 : 0;
            if (lane < n_above) {
                if (rank < kKeep) {
                    s.qc[h][rank] = mine;
                    s.qx[h][rank] = s.sx[h][lane];
                    s.qy[h][rank] = s.sy[h][lane];
                    s.qz[h][rank] = s.sz[h][lane];
                } else if (rank == kKeep) {
                    s.qbound[h] = fmaxf(T, cand_key(mine));
                    s.qstop[h] = stop;
                }
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k <= kKeep; ++k) {
        uint64_t v = 0ull;
        int vl = 0;
#pragma unroll
        for (int l = 0; l < kPollLoads; ++l)
            if (c[l] > v) {
                v = c[l];
                vl = l;
            }
        const uint64_t m = warp_max_u64(v);
        if (k == kKeep) {  // the best entry left out
            if (lane == 0) {
                s.qbound[h] = fmaxf(bound_from30(u30), cand_key(m));
                s.qstop[h] = stop;
            }
            break;
        }
        if (v == m) {  // one lane, unless m == 0 (then every writer stores an empty entry)
            uint32_t ex = 0u, ey = 0u, ez = 0u;
#pragma unroll
            for (int l = 0; l < kPollLoads; ++l)
                if (l == vl) {
                    ex = cxb[l];
                    ey = cyb[l];
                    ez = czb[l];
                    c[l] = 0ull;
                }
            s.qc[h][k] = m;
            s.qx[h][k] = __uint_as_float(ex);
            s.qy[h][k] = __uint_as_float(ey);
            s.qz[h][k] = __uint_as_float(ez);
        }
    }
}

// The picks of one round without a dependent chain per pick (X0; lane l
// holds kept entry l: minimum cur, row, coordinates; bound U >= 0 on every
// other point). Let S be the live entries with minimum above U, ranked by
// candidate word. Were no pick to lower another entry, the picks would be S
// in rank order. In general, going down the ranks, an entry whose minimum no
// earlier pick lowers is the best entry left (the entries below it have
// smaller words, the lowered and unranked ones minima <= U), so it is the
// next pick; an entry that an earlier pick lowers to U or below can no longer
// be picked this round (a pick needs a minimum above U) and is passed over.
// The picks are therefore the greedy independent set of the relation "lowers"
// in rank order (found in a few ballot rounds: a chain is mostly a chunk's
// best entry lowering its other entries), up to the first entry that a pick
// lowers but leaves above U, where this rule stops deciding. Lane-indexed
// masks over S: above (entries ranked higher), lowers (those whose key to
// this entry is below its minimum), drops (those whose key is <= U).
// Returns the picks made (written to s.pick / s.pxyz in order, their lanes
// no longer live); more is set when the greedy loop must continue, with cur
// already lowered by those picks. With S empty it makes none and leaves the
// unconditional first pick to the loop.
__device__ __forceinline__ int rank_picks(FpsShared& s, int lane, uint32_t row, float mx, float my, float mz,
                                          float bound, int cap, float& cur, bool& live, bool& more) {
    const float c = cur;
    const uint64_t w = pack_cand(c, row);
    const uint32_t S = __ballot_sync(0xffffffffu, live && c > bound);
    more = true;
    if (S == 0u) return 0;
    // the ranked entries, compacted: four per pass come with two broadcast loads each
    const int nS = __popc(S);
    if (live && c > bound) {
        const int k = __popc(S & ((1u << lane) - 1u));
        s.ranked[k][0] = make_uint4(static_cast<uint32_t>(w), static_cast<uint32_t>(w >> 32), lane, 0u);
        s.ranked[k][1] = make_uint4(__float_as_uint(mx), __float_as_uint(my), __float_as_uint(mz), 0u);
    }
    __syncwarp();
    uint32_t above = 0u, lowers = 0u, drops = 0u;
    for (int k0 = 0; k0 < nS; k0 += 4) {
        uint4 e[4], q[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int k = min(k0 + t, nS - 1);  // a repeated entry sets the same bits again
            e[t] = s.ranked[k][0];
            q[t] = s.ranked[k][1];
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint64_t wi = (static_cast<uint64_t>(e[t].y) << 32) | e[t].x;
            const float d = fps_key(mx, my, mz, __uint_as_float(q[t].x), __uint_as_float(q[t].y),
                                    __uint_as_float(q[t].z));
            const uint32_t bit = wi > w ? 1u << e[t].z : 0u;
            above |= bit;
            lowers |= d < c ? bit : 0u;
            drops |= d > bound ? 0u : bit;
        }
    }
    // decided picked (P) / passed over (N): an entry is picked once every
    // entry that lowers it is passed over, passed over once one of them is
    // picked; the highest undecided entry is decided in every round
    uint32_t P = 0u, N = 0u;
    for (uint32_t und = S; und; und = S & ~(P | N)) {
        const bool mine = (und >> lane) & 1u;
        const uint32_t p = __ballot_sync(0xffffffffu, mine && (lowers & ~N) == 0u);
        const uint32_t q = __ballot_sync(0xffffffffu, mine && (lowers & P) != 0u);
        P |= p;
        N |= q;
    }
    // lowered by a pick but still above U: the rule stops at the first of them
    const uint32_t stop = __ballot_sync(0xffffffffu, ((N >> lane) & 1u) && (drops & P) == 0u);
    const int pos = __popc(P & above);
    const bool take = ((P >> lane) & 1u) && (stop & above) == 0u && pos < cap;
    const uint32_t T = __ballot_sync(0xffffffffu, take);
    const int np = __popc(T);
    more = stop != 0u && np < cap;
    if (take) {
        s.pick[pos] = w;
        s.pxyz[pos] = make_float4(mx, my, mz, 0.0f);
        live = false;
    }
    if (more) {
        for (uint32_t t = T; t; t &= t - 1) {
            const int i = __ffs(t) - 1;
            const float xi = __shfl_sync(0xffffffffu, mx, i), yi = __shfl_sync(0xffffffffu, my, i),
                        zi = __shfl_sync(0xffffffffu, mz, i);
            cur = fminf(cur, fps_key(mx, my, mz, xi, yi, zi));
        }
    }
    return np;
}

// X0, one round: block reduction, publication, its quarter of the polling,
// the merge with the other quarters, and the picks.
__device__ __forceinline__ void exchange_step(const FpsArgs& a, FpsShared& s, int r, int picks_left, int lane) {
    uint64_t me;
    float mx, my, mz;
    float bound = block_top(s, lane, gridDim.x > 1 ? kTop : kKeep, me, mx, my, mz);
    bool stop = false;
    if (gridDim.x > 1) {
        const uint64_t tag = static_cast<uint64_t>(r & 3) << 62;
        uint64_t* buf = a.slots + static_cast<size_t>(r & 1) * kMaxBlocks * kSlotStride;
        if (lane < kTop) {
            const uint64_t hi = lane == 0 ? static_cast<uint64_t>(bound_up30(bound)) << 32 : 0ull;
            st_relaxed_v4_u64(buf + static_cast<size_t>(blockIdx.x) * kSlotStride + 4 * lane, tag | me,
                              tag | hi | __float_as_uint(mx), tag | __float_as_uint(my), tag | __float_as_uint(mz));
        }
        bar_arrive(kBarPub, kPollCount);
        poll_quarter(a, s, r, 0, lane);
        bar_wait(kBarQuarters, kPollCount);
        __syncwarp();
        // lane 8 h + k holds entry k of quarter h
        const int hh = lane / kKeep, kk = lane % kKeep;
        me = s.qc[hh][kk];
        mx = s.qx[hh][kk];
        my = s.qy[hh][kk];
        mz = s.qz[hh][kk];
        bound = fmaxf(fmaxf(s.qbound[0], s.qbound[1]), fmaxf(s.qbound[2], s.qbound[3]));
        stop = (s.qstop[0] | s.qstop[1] | s.qstop[2] | s.qstop[3]) != 0;
    }
    // Picks: the best live entry while its minimum stays positive and above
    // the bound (the first one unconditionally); each pick lowers the others.
    // The best is the largest candidate word (minimum, then lowest row: rows
    // are distinct), found with one 64-bit warp maximum; its lane by a ballot.
    // rank_picks makes the picks of the usual case in parallel; the loop
    // below continues where it cannot decide.
    const int cap = min(picks_left, kMaxPicks);
    const uint32_t row = cand_row(me);
    float cur = cand_key(me);
    bool live = me != 0ull;
    bool more;
    int np = rank_picks(s, lane, row, mx, my, mz, bound, cap, cur, live, more);
    while (more && np < cap) {
        const uint64_t w = live ? pack_cand(cur, row) : 0ull;  // non-zero for every live entry
        const uint64_t mw = warp_max_u64(w);
        if (mw == 0ull) {  // no entry left: the round ends (with none at all, an empty pick: degenerate)
            if (np == 0) {
                if (lane == 0) s.pick[0] = 0ull;
                np = 1;
            }
            break;
        }
        const float mk = cand_key(mw);
        if (np > 0 && !(mk > 0.0f && mk > bound)) break;
        const int o = __ffs(__ballot_sync(0xffffffffu, live && w == mw)) - 1;
        const float qx = __shfl_sync(0xffffffffu, mx, o), qy = __shfl_sync(0xffffffffu, my, o),
                    qz = __shfl_sync(0xffffffffu, mz, o);
        if (lane == o) {
            s.pick[np] = pack_cand(cur, row);
            s.pxyz[np] = make_float4(mx, my, mz, 0.0f);
            live = false;
        }
        ++np;
        cur = fminf(cur, fps_key(mx, my, mz, qx, qy, qz));
    }
    __syncwarp();
    if (lane == 0) s.n_pick = stop ? -1 : np;
}

// After the round's last barrier: how many picks the round made; 0 tells
// every thread to stop (timeout, or no point left with a positive key).
// Block 0's X1 records the picks: a barrier arrival waits for the arriving
// thread's earlier global stores, and X1 arrives next only after a whole
// round of polling, so the stores stay off the critical path.
__device__ __forceinline__ int take_picks(const FpsArgs& a, const FpsShared& s, int j) {
    const int n = s.n_pick;
    if (n < 1) return 0;
    const uint64_t e1 = s.pick[0];
    if (e1 == 0ull || !(cand_key(e1) > 0.0f)) {
        if (blockIdx.x == 0 && threadIdx.x == (kX0 + 1) * 32) atomicOr(a.flags, FLAG_DEGENERATE);
        return 0;
    }
    const int t = static_cast<int>(threadIdx.x) - (kX0 + 1) * 32;  // lane of X1
    if (blockIdx.x == 0 && t >= 0 && t < n && !FLOOD_OOB(j + t, a.n_landmarks, a.flags)) {
        a.out_idx[j + t] = cand_row(s.pick[t]);
        if (a.out_key) a.out_key[j + t] = cand_key(s.pick[t]);
    }
    return n;
}

// The start landmark becomes the single pick folded by the first round.
__device__ __forceinline__ void start_round(const FpsArgs& a, FpsShared& s) {
    if (threadIdx.x == 0) {
        if (blockIdx.x == 0) {
            a.out_idx[0] = a.start;
            if (a.out_key) a.out_key[0] = __int_as_float(0x7f800000);
        }
        s.pxyz[0] = make_float4(a.X[3 * a.start + 0], a.X[3 * a.start + 1], a.X[3 * a.start + 2], 0.0f);
        s.n_pick = 1;
    }
}

// The exchange warps' loops (shared by both kernels): X0 waits where the
// compute warps arrive and arrives where they wait; X1..X3 poll their
// quarters and hand them over.
__device__ __forceinline__ void exchange_loop(const FpsArgs& a, FpsShared& s, int warp, int lane) {
    int r = 1;
    for (int j = 1; j < a.n_landmarks; ++r) {
        if (warp == kX0) {
            bar_wait(kBarCands, kCandsCount);
            exchange_step(a, s, r, a.n_landmarks - j, lane);
            __syncwarp();
            bar_arrive(kBarPicks, kThreads);
        } else {
            if (gridDim.x > 1) {
                bar_wait(kBarPub, kPollCount);
                poll_quarter(a, s, r, warp - kX0, lane);
                __syncwarp();
                bar_arrive(kBarQuarters, kPollCount);
            }
            bar_wait(kBarPicks, kThreads);
        }
        const int n = take_picks(a, s, j);
        // block 0's X1 counts the rounds (off the critical path, like the picks it records)
        if (blockIdx.x == 0 && warp == kX0 + 1 && lane == 0) a.flags[7] = static_cast<uint32_t>(r);
        if (n == 0) break;
        j += n;
    }
}

// Which of the round's picks can lower a minimum inside the box (bit t for
// pick t): those whose squared gap to the box is below its largest minimum.
__device__ __forceinline__ uint32_t box_hits(const FpsShared& s, int np, float lox, float loy, float loz, float hix,
                                             float hiy, float hiz, float maxd) {
    uint32_t hit = 0u;
    for (int t = 0; t < np; ++t) {
        const float4 q = s.pxyz[t];
        if (!(box_gap2(q.x, q.y, q.z, lox, loy, loz, hix, hiy, hiz) >= maxd)) hit |= 1u << t;
    }
    return hit;
}

// Running top four of a lane's minima (t[0] >= ... >= t[3], as a multiset).
__device__ __forceinline__ void top4_insert(float v, float t[4]) {
    t[3] = fmaxf(t[3], fminf(t[2], v));
    t[2] = fmaxf(t[2], fminf(t[1], v));
    t[1] = fmaxf(t[1], fminf(t[0], v));
    t[0] = fmaxf(t[0], v);
}

// Entries of a chunk after its update: its kChunkEntries best points in
// (minimum desc, original row asc) order go to entries slot0 + 32 e, each
// written by the lane holding it (0 if the chunk has fewer real points).
// Each lane's best point not yet given is its (o + 1)-th minimum t[o], o the
// entries it gave; rows already given are excluded from tie searches (rows
// are distinct). Returns the bound on the chunk's other points (the largest
// minimum left) and the chunk's largest minimum in wm.
// val(k), row(k) and xyz(k, x, y, z) read this lane's point k.
template <class Val, class Row, class Xyz>
__device__ __forceinline__ float chunk_entries(FpsShared& s, const float t[4], int slot0, int lane, float& wm,
                                               Val val, Row row, Xyz xyz) {
    int o = 0;
    uint32_t given[kChunkEntries - 1];
#pragma unroll
    for (int e = 0; e < kChunkEntries; ++e) {
        const float v = o == 0 ? t[0] : o == 1 ? t[1] : o == 2 ? t[2] : t[3];
        const float we = warp_max_f(v);
        if (e == 0) wm = we;
        uint32_t cid = 0xffffffffu;
        float cx = 0.0f, cy = 0.0f, cz = 0.0f;
        if (we >= 0.0f && v == we) {  // padding holds -1
#pragma unroll
            for (int k = 0; k < kLanePts; ++k) {
                if (val(k) == we) {
                    const uint32_t id = row(k);
                    bool fresh = id < cid;
#pragma unroll
                    for (int q = 0; q < e; ++q) fresh = fresh && id != given[q];
                    if (fresh) {
                        cid = id;
                        xyz(k, cx, cy, cz);
                    }
                }
            }
        }
        const uint32_t r = __reduce_min_sync(0xffffffffu, cid);
        const int slot = slot0 + kWarps * e;
        if (r != 0xffffffffu && cid == r) {
            s.cand[slot] = pack_cand(we, r);
            s.cx[slot] = cx;
            s.cy[slot] = cy;
            s.cz[slot] = cz;
            ++o;
        } else if (r == 0xffffffffu && lane == 0) {
            s.cand[slot] = 0ull;
        }
        if (e < kChunkEntries - 1) given[e] = r;
    }
    return warp_max_f(o == 0 ? t[0] : o == 1 ? t[1] : o == 2 ? t[2] : t[3]);
}

// ---------------------------------------------------------------- resident kernel
// Chunks are dealt to blocks round-robin (chunk g to block g mod nb), so the
// few chunks one pick changes, which are neighbours in space and in the point
// order, fall into different blocks and update in parallel. Compute warp w of
// block b holds chunk w nb + b in registers (points 256 (w nb + b) + lane +
// 32 k, k < 8): with one block on each SM, 148 SMs hold 1,060,864 points.
// Dynamic shared memory:
//   ids  int32  [28][256]  original rows of each warp's chunk
//   box  float4 [32][2]    per warp: (lo x/y/z, unused), (hi x/y/z, unused)
constexpr int kResIds = 0;
constexpr int kResMeta = kResIds + kComputeWarps * kChunk * 4;
constexpr int kResidentSmem = kResMeta + kWarps * 2 * 16;

__global__ void __launch_bounds__(kThreads, 1) k_fps_resident(FpsArgs a) {
    __shared__ FpsShared s;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    int32_t* s_ids = reinterpret_cast<int32_t*>(s_dyn + kResIds);
    float4* s_box = reinterpret_cast<float4*>(s_dyn + kResMeta);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    shared_init(s);
    start_round(a, s);
    if (warp >= kComputeWarps) {
        __syncthreads();
        exchange_loop(a, s, warp, lane);
        return;
    }
    const int64_t base = (static_cast<int64_t>(warp) * gridDim.x + blockIdx.x) * kChunk;
    const int wo = warp * kChunk;
    const float inf = __int_as_float(0x7f800000);
    float px[kLanePts], py[kLanePts], pz[kLanePts], pd[kLanePts];
    {
        float lox = inf, loy = inf, loz = inf, hix = -inf, hiy = -inf, hiz = -inf;
#pragma unroll
        for (int k = 0; k < kLanePts; ++k) {
            const int o = lane + 32 * k;
            const int64_t i = base + o;
            const bool ok = i < a.n;
            const float4 v = ok ? a.pts[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            px[k] = v.x;
            py[k] = v.y;
            pz[k] = v.z;
            pd[k] = ok ? inf : -1.0f;  // padding never wins
            s_ids[wo + o] = __float_as_int(v.w);
            if (ok) {
                lox = fminf(lox, px[k]);
                loy = fminf(loy, py[k]);
                loz = fminf(loz, pz[k]);
                hix = fmaxf(hix, px[k]);
                hiy = fmaxf(hiy, py[k]);
                hiz = fmaxf(hiz, pz[k]);
            }
        }
        lox = warp_min_f(lox);
        loy = warp_min_f(loy);
        loz = warp_min_f(loz);
        hix = warp_max_f(hix);
        hiy = warp_max_f(hiy);
        hiz = warp_max_f(hiz);
        if (lane == 0) {
            s_box[2 * warp] = make_float4(lox, loy, loz, 0.0f);
            s_box[2 * warp + 1] = make_float4(hix, hiy, hiz, 0.0f);
        }
    }
    // Largest running minimum of the chunk (lane-replicated); -1 = no points.
    float maxd = base < a.n ? inf : -1.0f;
    __syncthreads();
    for (int j = 1; j < a.n_landmarks;) {
        // lane t tests pick t against the chunk's box
        const int np = s.n_pick;
        bool hit = false;
        if (lane < np) {
            const float4 lo = s_box[2 * warp], hi = s_box[2 * warp + 1], q = s.pxyz[lane];
            hit = !(box_gap2(q.x, q.y, q.z, lo.x, lo.y, lo.z, hi.x, hi.y, hi.z) >= maxd);
        }
        const uint32_t hits = __ballot_sync(0xffffffffu, hit);
        if (hits) {
#pragma unroll 1
            for (uint32_t mt = hits; mt; mt &= mt - 1) {
                const float4 q = s.pxyz[__ffs(mt) - 1];
#pragma unroll
                for (int k = 0; k < kLanePts; ++k) pd[k] = fminf(pd[k], fps_key(px[k], py[k], pz[k], q.x, q.y, q.z));
            }
            float t[4] = {-1.0f, -1.0f, -1.0f, -1.0f};
#pragma unroll
            for (int k = 0; k < kLanePts; ++k) top4_insert(pd[k], t);
            float wm;
            const float sec = chunk_entries(
                s, t, warp, lane, wm, [&](int k) { return pd[k]; },
                [&](int k) { return static_cast<uint32_t>(s_ids[wo + lane + 32 * k]); },
                [&](int k, float& x, float& y, float& z) {
                    x = px[k];
                    y = py[k];
                    z = pz[k];
                });
            if (lane == 0) s.sec[warp] = sec;
            maxd = wm;
        }
        bar_arrive(kBarCands, kCandsCount);
        bar_wait(kBarPicks, kThreads);
        const int n = take_picks(a, s, j);
        if (n == 0) break;
        j += n;
    }
}

// ---------------------------------------------------------------- global kernel
// Block b owns chunks b, b + nb, b + 2 nb, ... (local index cc: chunk
// cc nb + b) of 32 * lane_pts points each (lane_pts a multiple of
// kGlobalBatch); compute warp w updates local chunks w, w + 31, ... Chunk metadata (candidate, box, candidate
// coordinates, second-largest minimum) lives in shared memory, points and
// running minima in global memory. Each warp reports its best chunk
// candidate, bounded by its other chunks' candidates and all its seconds.
enum : int { kLoX = 0, kLoY, kLoZ, kHiX, kHiY, kHiZ, kCX, kCY, kCZ, kSec };

struct ChunkMeta {
    uint64_t* cand;
    float* f;
    int cb;
    __device__ __forceinline__ float& at(int field, int cc) const { return f[field * cb + cc]; }
};

// Fold the round's hitting picks into one chunk; new candidate, coordinates
// and second-largest minimum into its metadata.
__device__ __forceinline__ void update_chunk(const FpsArgs& a, const FpsShared& s, const ChunkMeta& m, int cc,
                                             int64_t base, uint32_t hit, int lane) {
    uint64_t best = 0ull;
    float t1 = -1.0f, t2 = -1.0f;
    float bx = 0.0f, by = 0.0f, bz = 0.0f;
    for (int q = 0; q < a.lane_pts; q += kGlobalBatch) {
        float x[kGlobalBatch], y[kGlobalBatch], z[kGlobalBatch], d[kGlobalBatch];
        int32_t id[kGlobalBatch];
#pragma unroll
        for (int k = 0; k < kGlobalBatch; ++k) {
            const int64_t i = base + lane + 32 * (q + k);
            if (i < a.n) {
                const float4 v = __ldg(a.pts + i);
                x[k] = v.x;
                y[k] = v.y;
                z[k] = v.z;
                id[k] = __float_as_int(v.w);
                d[k] = a.d[i];
            }
        }
#pragma unroll
        for (int k = 0; k < kGlobalBatch; ++k) {
            const int64_t i = base + lane + 32 * (q + k);
            if (i < a.n) {
                float nd = d[k];
#pragma unroll 1
                for (uint32_t mt = hit; mt; mt &= mt - 1) {
                    const int t = __ffs(mt) - 1;
                    const float4 l = s.pxyz[t];
                    nd = fminf(nd, fps_key(x[k], y[k], z[k], l.x, l.y, l.z));
                }
                if (nd != d[k]) a.d[i] = nd;
                t2 = fmaxf(t2, fminf(t1, nd));
                t1 = fmaxf(t1, nd);
                const uint64_t c = pack_cand(nd, static_cast<uint32_t>(id[k]));
                if (c > best) {
                    best = c;
                    bx = x[k];
                    by = y[k];
                    bz = z[k];
                }
            }
        }
    }
    const uint64_t wm = warp_max_u64(best);
    const int owner = __ffs(__ballot_sync(0xffffffffu, best == wm)) - 1;
    const float sec = warp_max_f(lane == owner ? t2 : t1);
    if (lane == owner) {
        m.cand[cc] = wm;
        m.at(kCX, cc) = bx;
        m.at(kCY, cc) = by;
        m.at(kCZ, cc) = bz;
        m.at(kSec, cc) = sec;
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_fps_global(FpsArgs a) {
    __shared__ FpsShared s;
    extern __shared__ __align__(16) unsigned char s_meta[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    shared_init(s);
    start_round(a, s);
    if (warp >= kComputeWarps) {
        __syncthreads();
        exchange_loop(a, s, warp, lane);
        return;
    }
    const int cb = a.chunks_per_block;
    const ChunkMeta m{reinterpret_cast<uint64_t*>(s_meta), reinterpret_cast<float*>(s_meta + 8 * size_t(cb)), cb};
    const int64_t nbk = gridDim.x;
    const int nc = static_cast<int>(min(static_cast<int64_t>(cb),
                                        a.n_chunks > blockIdx.x ? (a.n_chunks - blockIdx.x + nbk - 1) / nbk : 0));
    const int mine = warp < nc ? (nc - warp + kComputeWarps - 1) / kComputeWarps : 0;  // chunks of this warp
    const int64_t chunk_pts = 32 * static_cast<int64_t>(a.lane_pts);
    // Boxes; running minima start at +inf.
    for (int t = 0; t < mine; ++t) {
        const int cc = warp + kComputeWarps * t;
        const int64_t base = (cc * nbk + blockIdx.x) * chunk_pts;
        float lox = __int_as_float(0x7f800000), loy = lox, loz = lox;
        float hix = -lox, hiy = -lox, hiz = -lox;
        for (int q = 0; q < a.lane_pts; ++q) {
            const int64_t i = base + lane + 32 * q;
            if (i < a.n) {
                const float4 v = a.pts[i];
                const float x = v.x, y = v.y, z = v.z;
                lox = fminf(lox, x);
                loy = fminf(loy, y);
                loz = fminf(loz, z);
                hix = fmaxf(hix, x);
                hiy = fmaxf(hiy, y);
                hiz = fmaxf(hiz, z);
                a.d[i] = __int_as_float(0x7f800000);
            }
        }
        lox = warp_min_f(lox);
        loy = warp_min_f(loy);
        loz = warp_min_f(loz);
        hix = warp_max_f(hix);
        hiy = warp_max_f(hiy);
        hiz = warp_max_f(hiz);
        if (lane == 0) {
            m.cand[cc] = pack_cand(__int_as_float(0x7f800000), 0u);  // +inf: never skipped before its first update
            m.at(kLoX, cc) = lox;
            m.at(kLoY, cc) = loy;
            m.at(kLoZ, cc) = loz;
            m.at(kHiX, cc) = hix;
            m.at(kHiY, cc) = hiy;
            m.at(kHiZ, cc) = hiz;
            m.at(kCX, cc) = m.at(kCY, cc) = m.at(kCZ, cc) = 0.0f;
            m.at(kSec, cc) = -1.0f;
        }
    }
    __syncwarp();
    __syncthreads();
    for (int j = 1; j < a.n_landmarks;) {
        const int np = s.n_pick;
        bool changed = false;
        for (int t0 = 0; t0 < mine; t0 += 32) {
            const int t = t0 + lane;
            uint32_t hit = 0u;
            if (t < mine) {
                const int cc = warp + kComputeWarps * t;
                hit = box_hits(s, np, m.at(kLoX, cc), m.at(kLoY, cc), m.at(kLoZ, cc), m.at(kHiX, cc), m.at(kHiY, cc),
                               m.at(kHiZ, cc), cand_key(m.cand[cc]));
            }
            uint32_t mask = __ballot_sync(0xffffffffu, hit != 0u);
            changed |= mask != 0u;
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                const int cc = warp + kComputeWarps * (t0 + src);
                update_chunk(a, s, m, cc, (cc * nbk + blockIdx.x) * chunk_pts, __shfl_sync(0xffffffffu, hit, src),
                             lane);
            }
        }
        if (changed) {
            __syncwarp();
            uint64_t b1 = 0ull, b2 = 0ull;
            float sx = -1.0f;
            int bc = 0;
            for (int t = lane; t < mine; t += 32) {
                const int cc = warp + kComputeWarps * t;
                const uint64_t c = m.cand[cc];
                if (c > b1) {
                    b2 = b1;
                    b1 = c;
                    bc = cc;
                } else if (c > b2) {
                    b2 = c;
                }
                sx = fmaxf(sx, m.at(kSec, cc));
            }
            const uint64_t wm = warp_max_u64(b1);
            const int owner = __ffs(__ballot_sync(0xffffffffu, b1 == wm)) - 1;
            const float other = cand_key(warp_max_u64(lane == owner ? b2 : b1));
            const float bound = fmaxf(other, warp_max_f(sx));
            if (lane == owner) {
                s.cand[warp] = wm;
                s.cx[warp] = m.at(kCX, bc);
                s.cy[warp] = m.at(kCY, bc);
                s.cz[warp] = m.at(kCZ, bc);
                s.sec[warp] = bound;
            }
        }
        bar_arrive(kBarCands, kCandsCount);
        bar_wait(kBarPicks, kThreads);
        const int n = take_picks(a, s, j);
        if (n == 0) break;
        j += n;
    }
}

// ---------------------------------------------------------------- host side
struct FpsPlan {
    int blocks;
    bool resident;
    int lane_pts;
    int chunks_per_block;
    int64_t n_chunks;
    size_t smem;
};

int max_fps_blocks() { return std::min(device_sm_count(), kMaxBlocks); }

// Launch shape: n_blocks = 0 picks the fewest blocks whose registers and
// shared memory hold every point (7,168 per block), else 160 blocks (or the SM
// count, if smaller) with chunks streamed from global memory; n_blocks = k
// uses k blocks, resident when they hold every point.
int plan_fps(int64_t n, int n_blocks, FpsPlan* p) {
    const int maxb = max_fps_blocks();
    if (n_blocks < 0) {
        set_error("flood_fps: n_blocks must be >= 0");
        return FLOOD_EINVAL;
    }
    int nb = n_blocks > 0 ? std::min(n_blocks, maxb)
                          : static_cast<int>(std::min<int64_t>(maxb, ceil_div(n, kBlockPts)));
    nb = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(nb, ceil_div(n, 32))));
    p->blocks = nb;
    p->resident = n <= int64_t(nb) * kBlockPts;
    p->lane_pts = kGlobalBatch;
    p->chunks_per_block = 0;
    p->n_chunks = 0;
    p->smem = kResidentSmem;
    if (!p->resident) {
        for (int lp = kGlobalBatch;; lp += kGlobalBatch) {
            const int64_t nch = ceil_div(n, 32 * int64_t(lp));
            const int64_t cb = ceil_div(nch, nb);
            if (cb * kMetaBytes <= kMetaSmemMax) {
                p->lane_pts = lp;
                p->n_chunks = nch;
                p->chunks_per_block = static_cast<int>(cb);
                p->smem = static_cast<size_t>(cb) * kMetaBytes;
                break;
            }
        }
    }
    return FLOOD_OK;
}

int launch_fps_kernel(const FpsPlan& p, FpsArgs a, cudaStream_t s) {
    a.lane_pts = p.lane_pts;
    a.chunks_per_block = p.chunks_per_block;
    a.n_chunks = p.n_chunks;
    const void* fn = p.resident ? reinterpret_cast<const void*>(k_fps_resident)
                                : reinterpret_cast<const void*>(k_fps_global);
    FLOOD_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    p.resident ? kResidentSmem : kMetaSmemMax));
    int per_sm = 0;
    FLOOD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, p.smem));
    if (per_sm < 1 || p.blocks > per_sm * device_sm_count()) {
        set_error("flood_fps: %d blocks are not co-resident (%d per SM)", p.blocks, per_sm);
        return FLOOD_EINTERNAL;
    }
    void* args[] = {&a};
    if (p.blocks == 1)
        FLOOD_CUDA(cudaLaunchKernel(fn, dim3(1), dim3(kThreads), args, p.smem, s));
    else
        FLOOD_CUDA(cudaLaunchCooperativeKernel(fn, dim3(p.blocks), dim3(kThreads), args, p.smem, s));
    note_launch();
    return FLOOD_OK;
}

// Lattice bits per axis for the point order: about 16 points per cell of a
// volume-filling cloud, 3..7 bits (2^9..2^21 codes).
int morton_bits(int64_t n) {
    int b = 3;
    while (b < 7 && (int64_t(1) << (3 * b)) * 16 < n) ++b;
    return b;
}

// The whole FPS on `s`; scratch from `al` (stream-ordered allocations, or a
// fixed buffer). *flags_out receives the device status word.
// Scratch bytes of run_fps for n points and launch shape p, as its allocator
// carves them (every piece rounded up to 256 bytes): the control words, the
// exchange slots, the point order, the running minima when the points do not
// stay on chip, and the Morton sort's codes, histogram, offsets and scan.
size_t fps_scratch_bytes(int64_t n, const FpsPlan& p) {
    auto piece = [](size_t bytes) { return (std::max<size_t>(bytes, 1) + 255) & ~size_t(255); };
    size_t b = piece(8 * 4) + piece(2 * kMaxBlocks * kSlotStride * 8) + piece(16 * size_t(n));
    if (!p.resident) b += piece(4 * size_t(n));
    if (n > kSortMin) {
        const int64_t codes = int64_t(1) << (3 * morton_bits(n));
        b += piece(4 * size_t(n)) + piece(4 * size_t(codes)) + piece(4 * size_t(codes + 1)) +
             exclusive_scan_scratch_bytes(codes);
    }
    return b;
}

// Test support: the exchange waits for `extra_blocks` blocks that are never
// launched and gives up after `poll_limit` polls (0: the normal bound).
struct FpsWaitTest {
    int extra_blocks = 0;
    uint32_t poll_limit = 0;
};

template <class Alloc>
int run_fps(const float* X, int64_t n, int32_t n_landmarks, int64_t start, int n_blocks, int64_t* out_idx,
            float* out_key, cudaStream_t s, Alloc& al, uint32_t** flags_out, FpsPlan* plan_out = nullptr,
            const FpsWaitTest& wt = FpsWaitTest()) {
    FpsPlan plan;
    int rc = plan_fps(n, n_blocks, &plan);
    if (rc) return rc;
    if (plan_out) *plan_out = plan;
    if (wt.extra_blocks < 0 || plan.blocks + wt.extra_blocks > kMaxBlocks || (wt.extra_blocks > 0 && plan.blocks < 2)) {
        set_error("flood_fps: a wait test needs at least 2 launched blocks and at most %d in all", kMaxBlocks);
        return FLOOD_EINVAL;
    }
    uint32_t* ctl;  // [0] flags, [1..6] ordered box, [7] exchange rounds
    uint64_t* slots;
    float4* pts;
    float* d = nullptr;
    if ((rc = al.alloc(&ctl, 8)) || (rc = al.alloc(&slots, 2 * kMaxBlocks * kSlotStride)) ||
        (rc = al.alloc(&pts, n)))
        return rc;
    if (!plan.resident && (rc = al.alloc(&d, n))) return rc;
    *flags_out = ctl;
    // Slot tags must start from zero (stale tags could match iterations 1 or 2).
    FLOOD_CUDA(cudaMemsetAsync(slots, 0, sizeof(uint64_t) * 2 * kMaxBlocks * kSlotStride, s));
    FLOOD_CUDA(cudaMemsetAsync(ctl, 0, sizeof(uint32_t) * 8, s));
    k_box_init<<<1, 1, 0, s>>>(ctl + 1, ctl);
    note_launch();
    const unsigned grid = static_cast<unsigned>(ceil_div(n, 256));
    if (n <= kSortMin) {
        k_pack_rows<<<grid, 256, 0, s>>>(X, n, pts, ctl);
        note_launch();
    } else {
        const int bits = morton_bits(n);
        const int64_t codes = int64_t(1) << (3 * bits);
        int32_t *code, *count, *cstart;
        if ((rc = al.alloc(&code, n)) || (rc = al.alloc(&count, codes)) || (rc = al.alloc(&cstart, codes + 1)))
            return rc;
        FLOOD_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t) * codes, s));
        k_bbox<<<bbox_blocks(n, device_sm_count()), kBoxThreads, 0, s>>>(X, n, ctl + 1, ctl);
        k_morton_count<<<grid, 256, 0, s>>>(X, n, ctl + 1, bits, code, count);
        note_launch(2);
        FLOOD_CUDA(cudaGetLastError());
        if ((rc = exclusive_scan(count, cstart, codes, s, al))) return rc;
        k_morton_scatter<<<grid, 256, 0, s>>>(X, n, code, cstart, count, pts, ctl);
        note_launch();
    }
    FLOOD_CUDA(cudaGetLastError());
    FpsArgs a{X,     pts,   d, n, n_landmarks, start, out_idx, out_key, slots, ctl, 0, 0, 0,
              plan.blocks + wt.extra_blocks, wt.poll_limit ? wt.poll_limit : kWaitPolls};
    return launch_fps_kernel(plan, a, s);
}

// The calling thread's last FPS call: its control words (status, box, round
// count) are copied back into a pinned buffer without waiting and read by
// flood_last_fps_stats once the call's stream is done.
struct LastFps {
    HostStats buf;       // asynchronous calls: pinned copy, read after its event
    uint32_t words[8];   // synchronous calls: the copy itself (no pinned memory needed)
    bool in_words = false;
    FpsPlan plan{};
    int32_t n_landmarks = 0;
    bool valid = false;
};
thread_local LastFps g_last_fps;

int fps_copy_back(cudaStream_t s, const uint32_t* ctl, const FpsPlan& plan, int32_t n_landmarks) {
    g_last_fps.valid = false;
    if (int rc = g_last_fps.buf.reserve(8 * sizeof(uint32_t))) return rc;
    FLOOD_CUDA(cudaMemcpyAsync(g_last_fps.buf.host, ctl, 8 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    FLOOD_CUDA(cudaEventRecord(g_last_fps.buf.done, s));
    g_last_fps.in_words = false;
    g_last_fps.plan = plan;
    g_last_fps.n_landmarks = n_landmarks;
    g_last_fps.valid = true;
    return FLOOD_OK;
}

// Synchronous completion (flood_fps_noalloc, flood_fps_wait_test): wait for
// `s` and turn the status word into a flood_status. Allocates nothing.
int fps_finish(cudaStream_t s, const uint32_t* ctl, const FpsPlan& plan, int32_t n_landmarks, const char* where) {
    g_last_fps.valid = false;
    FLOOD_CUDA(cudaMemcpyAsync(g_last_fps.words, ctl, sizeof(g_last_fps.words), cudaMemcpyDeviceToHost, s));
    FLOOD_CUDA(cudaStreamSynchronize(s));
    g_last_fps.in_words = true;
    g_last_fps.plan = plan;
    g_last_fps.n_landmarks = n_landmarks;
    g_last_fps.valid = true;
    return status_from_flags(g_last_fps.words[0], where);
}

bool fps_args_ok(const float* X, int64_t n_points, int32_t n_landmarks, int64_t start, const int64_t* out_idx) {
    return X && out_idx && n_points >= 1 && n_points < (int64_t(1) << 31) - 1 && n_landmarks >= 1 &&
           n_landmarks <= n_points && start >= 0 && start < n_points;
}

}  // namespace

}  // namespace flood

using namespace flood;

extern "C" int flood_fps_blocks(const float* X, int64_t n_points, int32_t n_landmarks, int64_t start,
                                int32_t n_blocks, int64_t* out_idx, float* out_key, void* stream_) {
    if (!fps_args_ok(X, n_points, n_landmarks, start, out_idx)) {
        set_error("flood_fps: need X, out_idx != NULL, 1 <= n_landmarks <= n_points < 2^31 - 1, "
                  "0 <= start < n_points");
        return FLOOD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    if (int rc = pending_error(s)) return rc;
    Scratch scr(s);
    uint32_t* flags = nullptr;
    FpsPlan plan{};
    int rc = run_fps(X, n_points, n_landmarks, start, n_blocks, out_idx, out_key, s, scr, &flags, &plan);
    if (rc) {
        if (flags) cudaStreamSynchronize(s);
        return rc;
    }
    if ((rc = fps_copy_back(s, flags, plan, n_landmarks))) return rc;
    return defer_status(s, flags, "flood_fps");
}

extern "C" int flood_last_fps_stats(flood_fps_stats* out) {
    if (!out) {
        set_error("flood_last_fps_stats: out is NULL");
        return FLOOD_EINVAL;
    }
    flood_fps_stats st{};
    if (g_last_fps.valid) {
        if (!g_last_fps.in_words) FLOOD_CUDA(cudaEventSynchronize(g_last_fps.buf.done));
        const uint32_t* h = g_last_fps.in_words ? g_last_fps.words : static_cast<const uint32_t*>(g_last_fps.buf.host);
        if (h[0] == 0u) {
            st.picks = g_last_fps.n_landmarks;
            st.rounds = h[7];
            st.blocks = g_last_fps.plan.blocks;
            st.resident = g_last_fps.plan.resident ? 1 : 0;
        }
    }
    *out = st;
    return FLOOD_OK;
}

extern "C" int flood_fps_scratch_bytes(int64_t n_points, int32_t n_blocks, int64_t* out_bytes) {
    if (!out_bytes || n_points < 1 || n_points >= (int64_t(1) << 31) - 1) {
        set_error("flood_fps_scratch_bytes: need out_bytes != NULL and 1 <= n_points < 2^31 - 1");
        return FLOOD_EINVAL;
    }
    FpsPlan plan;
    int rc = plan_fps(n_points, n_blocks, &plan);
    if (rc) return rc;
    *out_bytes = static_cast<int64_t>(fps_scratch_bytes(n_points, plan));
    return FLOOD_OK;
}

extern "C" int flood_fps_wait_test(const float* X, int64_t n_points, int32_t n_landmarks, int32_t n_blocks,
                                   int32_t extra_blocks, uint32_t poll_limit, int64_t* out_idx, void* stream_) {
    if (!fps_args_ok(X, n_points, n_landmarks, 0, out_idx) || n_blocks < 2 || extra_blocks < 1 || poll_limit < 1) {
        set_error("flood_fps_wait_test: need valid FPS arguments, n_blocks >= 2, extra_blocks >= 1, poll_limit >= 1");
        return FLOOD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    Scratch scr(s);
    uint32_t* flags = nullptr;
    FpsPlan plan{};
    FpsWaitTest wt;
    wt.extra_blocks = extra_blocks;
    wt.poll_limit = poll_limit;
    int rc = run_fps(X, n_points, n_landmarks, 0, n_blocks, out_idx, nullptr, s, scr, &flags, &plan, wt);
    if (rc) {
        if (flags) cudaStreamSynchronize(s);
        return rc;
    }
    return fps_finish(s, flags, plan, n_landmarks, "flood_fps_wait_test");
}

extern "C" int flood_fps(const float* X, int64_t n_points, int32_t n_landmarks, int64_t start, int64_t* out_idx,
                         float* out_key, void* stream_) {
    return flood_fps_blocks(X, n_points, n_landmarks, start, 0, out_idx, out_key, stream_);
}

// ---------------------------------------------------------------------------
// flood_fps_noalloc: farthest point sampling for callers that must not
// allocate device memory.
//
// Some callers cannot let a library call cudaMalloc/cudaMallocAsync: a host
// application whose own pool already owns the device memory (an allocation
// would fail or upset its accounting), a latency-critical loop that forbids
// allocator calls after start-up, or a plugin whose host framework forbids
// its extensions from allocating. This entry point runs the same kernels as
// flood_fps but takes its scratch (point order, structure-of-arrays copy,
// running minima, sort histogram, exchange slots, control words) from one
// file-scope device array of fixed size that is part of the loaded module.
// Every GPU that loads this library holds that array (27 MiB) until the
// process exits.
// ---------------------------------------------------------------------------
namespace flood {
namespace {

constexpr int64_t kNoAllocMaxPoints = int64_t(1) << 20;  // 1,048,576 points
constexpr size_t kNoAllocBytes = size_t(27) << 20;      // holds run_fps's pieces for 2^20 points

// The scratch itself. Host code must not use this name as a pointer: on the
// host it is only a stand-in for the symbol, so its device address is looked
// up with cudaGetSymbolAddress (once per device) and passed to the kernels.
static __device__ __align__(256) unsigned char g_fps_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on the
// first call per device).
int noalloc_scratch(unsigned char** out) {
    int dev = 0;
    FLOOD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("flood_fps_noalloc: device ordinal %d not supported", dev);
        return FLOOD_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        FLOOD_CUDA(cudaGetSymbolAddress(&p, g_fps_noalloc_scratch));
        g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_noalloc_addr[dev];
    return FLOOD_OK;
}

}  // namespace
}  // namespace flood

extern "C" int flood_fps_noalloc(const float* X, int64_t n_points, int32_t n_landmarks, int64_t start,
                                 int64_t* out_idx, float* out_key, void* stream_) {
    using namespace flood;
    if (!fps_args_ok(X, n_points, n_landmarks, start, out_idx)) {
        set_error("flood_fps_noalloc: need X, out_idx != NULL, 1 <= n_landmarks <= n_points, 0 <= start < n_points");
        return FLOOD_EINVAL;
    }
    if (n_points > kNoAllocMaxPoints) {
        set_error("flood_fps_noalloc: n_points = %lld exceeds the fixed maximum of %lld points; use flood_fps",
                  static_cast<long long>(n_points), static_cast<long long>(kNoAllocMaxPoints));
        return FLOOD_ECAPACITY;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    unsigned char* base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    Bump al{base, kNoAllocBytes};
    uint32_t* flags = nullptr;
    FpsPlan plan{};
    rc = run_fps(X, n_points, n_landmarks, start, 0, out_idx, out_key, s, al, &flags, &plan);
    if (rc) {
        if (flags) cudaStreamSynchronize(s);
        return rc;
    }
    rc = fps_finish(s, flags, plan, n_landmarks, "flood_fps_noalloc");
    // the carved pieces must be exactly what flood_fps_scratch_bytes reports
    if (rc == FLOOD_OK && kNoAllocBytes - al.left != fps_scratch_bytes(n_points, plan)) {
        set_error("flood_fps_noalloc: scratch used (%zu bytes) differs from the computed size (%zu bytes)",
                  kNoAllocBytes - al.left, fps_scratch_bytes(n_points, plan));
        return FLOOD_EINTERNAL;
    }
    return rc;
}
