// flood_fps: farthest point sampling (§3.2), the landmark selection of the
// Flood complex.
//
// Exact FPS with spatial skipping, in one persistent launch for all
// n_landmarks - 1 iterations:
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
// * One warp of each 1024-thread block runs the grid-wide argmax exchange:
//   per iteration each block publishes four tagged 64-bit words (candidate,
//   x, y, z) and polls every block's words until all carry this iteration's
//   tag. That one pass both synchronises the grid and delivers the winner
//   with its coordinates, so no dependent load of the new landmark follows.
//
// Two kernels: k_fps_resident keeps a block's points on chip (62 chunks per
// block, two per compute warp: one in registers, one in shared memory), so a
// cloud of up to 15,872 points runs on one block with no grid exchange at all;
// k_fps_global streams chunks from global memory for clouds larger than all
// SMs hold (or launches narrower than the cloud needs).
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
constexpr int kComputeWarps = kWarps - 1;  // the last warp runs the exchange
constexpr int kLanePts = 8;                // points per lane of a chunk
constexpr int kChunk = 32 * kLanePts;      // points per chunk (resident kernel)
constexpr int64_t kBlockPts = 2 * int64_t(kComputeWarps) * kChunk;  // points a resident block holds
constexpr int kMaxBlocks = 160;            // the exchange polls at most 5 rounds of 32 blocks
constexpr int kPollRounds = kMaxBlocks / 32;
constexpr int kSlotStride = 16;            // uint64 words per slot line (128 bytes; 4 used)
constexpr int64_t kSortMin = 16384;        // smaller clouds keep their input order
constexpr int kGlobalBatch = 5;            // global kernel: points per lane loaded at once
constexpr int kMetaBytes = 8 + 9 * 4;      // per chunk in shared memory: candidate, box, coordinates
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

// Counting-sort scatter into structure-of-arrays order; `fill` holds the
// histogram and is counted down (order within a code is arbitrary, which
// changes no result: ties are decided by the original row).
__global__ void __launch_bounds__(256) k_morton_scatter(const float* X, int64_t n, const int32_t* code,
                                                       const int32_t* start, int32_t* fill, float* x, float* y,
                                                       float* z, int32_t* ids) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int32_t c = code[i];
    const int32_t pos = start[c] + atomicSub(&fill[c], 1) - 1;
    x[pos] = X[3 * i + 0];
    y[pos] = X[3 * i + 1];
    z[pos] = X[3 * i + 2];
    ids[pos] = static_cast<int32_t>(i);
}

// Input order (small clouds): plain structure-of-arrays copy.
__global__ void __launch_bounds__(256) k_soa_ids(const float* X, int64_t n, float* x, float* y, float* z,
                                                int32_t* ids, uint32_t* flags) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const float a = X[3 * i + 0], b = X[3 * i + 1], c = X[3 * i + 2];
    if (!(isfinite(a) && isfinite(b) && isfinite(c))) atomicOr(flags, FLAG_NONFINITE);
    x[i] = a;
    y[i] = b;
    z[i] = c;
    ids[i] = static_cast<int32_t>(i);
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
    const float* x;    // points in processing order, structure of arrays
    const float* y;
    const float* z;
    const int32_t* ids;  // original row of each point
    float* d;          // running minima (global kernel)
    int64_t n;
    int32_t n_landmarks;
    int64_t start;
    int64_t* out_idx;
    float* out_key;
    uint64_t* slots;   // 2 (parity) x kMaxBlocks lines of kSlotStride words
    uint32_t* flags;
    int32_t lane_pts;  // global kernel: points per lane of a chunk (multiple of 8)
    int32_t chunks_per_block;
    int64_t n_chunks;
};

// Block-shared state of one iteration. Candidates: entry w for the first
// chunk of compute warp w, entry 32 + w for its second chunk (resident kernel).
struct FpsShared {
    uint64_t cand[2 * kWarps];
    float cx[2 * kWarps], cy[2 * kWarps], cz[2 * kWarps];
    uint64_t win;
    float wx, wy, wz;
    int stop;
};

__device__ __forceinline__ void shared_init(FpsShared& s) {
    if (threadIdx.x < 2 * kWarps) {
        s.cand[threadIdx.x] = 0ull;
        s.cx[threadIdx.x] = s.cy[threadIdx.x] = s.cz[threadIdx.x] = 0.0f;
    }
}

// Exchange warp, one iteration: the block's candidate from its chunks' ones,
// then (more than one block) the grid-wide exchange. Leaves the winner in s.
//
// Slot of block b for iteration j: its own 128-byte line (parity j & 1), so
// that the polls of all blocks spread over many L2 slices, written and read
// as one 32-byte access of four words:
//   w0 = (j & 3) << 62 | candidate     w1..w3 = j << 32 | bits of x, y, z.
// A reader accepts block b once all four words carry iteration j, so each
// word is read atomically and no ordering between them is needed. A block
// cannot publish j + 2 (same parity) before every block has finished reading
// j + 1, hence before every reader is done with j.
__device__ __forceinline__ void exchange_step(const FpsArgs& a, FpsShared& s, int j, int lane) {
    const uint64_t va = s.cand[lane], vb = s.cand[kWarps + lane];
    const uint64_t v = vb > va ? vb : va;
    const int vi = vb > va ? kWarps + lane : lane;
    uint64_t win = warp_max_u64(v);
    const int oi = __shfl_sync(0xffffffffu, vi, __ffs(__ballot_sync(0xffffffffu, v == win)) - 1);
    float wx = s.cx[oi], wy = s.cy[oi], wz = s.cz[oi];
    int stop = 0;
    const int nb = gridDim.x;
    if (nb > 1) {
        const uint32_t tj = static_cast<uint32_t>(j & 3);
        const uint32_t jj = static_cast<uint32_t>(j);
        const uint64_t jt = static_cast<uint64_t>(jj) << 32;
        uint64_t* buf = a.slots + static_cast<size_t>(j & 1) * kMaxBlocks * kSlotStride;
        if (lane == 0) {
            st_relaxed_v4_u64(buf + static_cast<size_t>(blockIdx.x) * kSlotStride,
                              (static_cast<uint64_t>(tj) << 62) | win, jt | __float_as_uint(wx),
                              jt | __float_as_uint(wy), jt | __float_as_uint(wz));
        }
        uint64_t v0[kPollRounds], v1[kPollRounds], v2[kPollRounds], v3[kPollRounds];
        for (uint32_t polls = 0;;) {
#pragma unroll
            for (int r = 0; r < kPollRounds; ++r) {
                const int b = lane + 32 * r;
                if (b < nb) {
                    ld_relaxed_v4_u64(buf + static_cast<size_t>(b) * kSlotStride, v0[r], v1[r], v2[r], v3[r]);
                } else {
                    v0[r] = static_cast<uint64_t>(tj) << 62;
                    v1[r] = v2[r] = v3[r] = jt;
                }
            }
            uint32_t stale = 0u;
#pragma unroll
            for (int r = 0; r < kPollRounds; ++r)
                stale |= (static_cast<uint32_t>(v0[r] >> 62) ^ tj) | (static_cast<uint32_t>(v1[r] >> 32) ^ jj) |
                         (static_cast<uint32_t>(v2[r] >> 32) ^ jj) | (static_cast<uint32_t>(v3[r] >> 32) ^ jj);
            if (__all_sync(0xffffffffu, stale == 0u)) break;
            if (++polls > kWaitPolls) {
                stop = 1;
                if (lane == 0) atomicOr(a.flags, FLAG_TIMEOUT);
                break;
            }
        }
        uint64_t best = 0ull;
        uint32_t bx = 0u, by = 0u, bz = 0u;
#pragma unroll
        for (int r = 0; r < kPollRounds; ++r) {
            const uint64_t c = v0[r] & kCandMask;
            if (c > best) {
                best = c;
                bx = static_cast<uint32_t>(v1[r]);
                by = static_cast<uint32_t>(v2[r]);
                bz = static_cast<uint32_t>(v3[r]);
            }
        }
        win = warp_max_u64(best);
        const int o = __ffs(__ballot_sync(0xffffffffu, best == win)) - 1;
        wx = __uint_as_float(__shfl_sync(0xffffffffu, bx, o));
        wy = __uint_as_float(__shfl_sync(0xffffffffu, by, o));
        wz = __uint_as_float(__shfl_sync(0xffffffffu, bz, o));
    }
    if (lane == 0) {
        s.win = win;
        s.wx = wx;
        s.wy = wy;
        s.wz = wz;
        s.stop = stop;
    }
}

// After the second barrier of iteration j: record the pick, or tell every
// thread to stop (timeout, or no point left with a positive key).
__device__ __forceinline__ bool accept_winner(const FpsArgs& a, const FpsShared& s, int j, float& lx, float& ly,
                                              float& lz) {
    if (s.stop) return false;
    const uint64_t win = s.win;
    const float key = cand_key(win);
    if (win == 0ull || !(key > 0.0f)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.flags, FLAG_DEGENERATE);
        return false;
    }
    lx = s.wx;
    ly = s.wy;
    lz = s.wz;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.out_idx[j] = cand_row(win);
        if (a.out_key) a.out_key[j] = key;
    }
    return true;
}

__device__ __forceinline__ void record_start(const FpsArgs& a, float& lx, float& ly, float& lz) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.out_idx[0] = a.start;
        if (a.out_key) a.out_key[0] = __int_as_float(0x7f800000);
    }
    lx = a.X[3 * a.start + 0];
    ly = a.X[3 * a.start + 1];
    lz = a.X[3 * a.start + 2];
}

// The exchange warp's loop (shared by both kernels): the same barriers as
// the compute warps, the exchange in between.
__device__ __forceinline__ void exchange_loop(const FpsArgs& a, FpsShared& s, int lane) {
    float lx, ly, lz;
    record_start(a, lx, ly, lz);
    for (int j = 1; j < a.n_landmarks; ++j) {
        __syncthreads();
        exchange_step(a, s, j, lane);
        __syncthreads();
        if (!accept_winner(a, s, j, lx, ly, lz)) break;
    }
}

// ---------------------------------------------------------------- resident kernel
// Compute warp w of block b holds two adjacent chunks of the point order,
// base = (b * 31 + w) * 512: chunk A (points base + lane + 32 k, k < 8) in
// registers and chunk B (the next 256 points) in shared memory; boxes and
// chunk B's largest minimum in shared memory, chunk A's in a register.
// Dynamic shared memory:
//   ids  int32 [2][31][256]  original rows of chunks A and B
//   pts  float [4][31][256]  chunk B: x, y, z, running minimum
//   meta float [13][32]      chunk B: box lo x/y/z, hi x/y/z, largest minimum;
//                            chunk A: box lo x/y/z, hi x/y/z
constexpr int kResIds = 0;
constexpr int kResPts = kResIds + 2 * kComputeWarps * kChunk * 4;
constexpr int kResMeta = kResPts + 4 * kComputeWarps * kChunk * 4;
constexpr int kResidentSmem = kResMeta + 13 * kWarps * 4;

// Candidate of a chunk after its update: warp maximum of the minima, ties to
// the lowest original row; written to s.cand[slot] by one lane.
__device__ __forceinline__ void publish_chunk(FpsShared& s, int slot, float wm, uint32_t cid, float cx, float cy,
                                              float cz, int lane) {
    uint32_t have = __ballot_sync(0xffffffffu, cid != 0xffffffffu);
    if (__popc(have) > 1) {
        const uint32_t m = __reduce_min_sync(0xffffffffu, cid);
        have = __ballot_sync(0xffffffffu, cid == m);
    }
    if (have && lane == __ffs(have) - 1) {
        s.cand[slot] = pack_cand(wm, cid);
        s.cx[slot] = cx;
        s.cy[slot] = cy;
        s.cz[slot] = cz;
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_fps_resident(FpsArgs a) {
    __shared__ FpsShared s;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    int32_t* s_ids = reinterpret_cast<int32_t*>(s_dyn + kResIds);
    float* s_pts = reinterpret_cast<float*>(s_dyn + kResPts);
    float* s_bm = reinterpret_cast<float*>(s_dyn + kResMeta);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    shared_init(s);
    if (warp == kComputeWarps) {
        __syncthreads();
        exchange_loop(a, s, lane);
        return;
    }
    const int64_t base = (static_cast<int64_t>(blockIdx.x) * kComputeWarps + warp) * (2 * kChunk);
    // shared-memory rows of this warp: index field * kPlane + wo + lane + 32 k
    constexpr int kPlane = kComputeWarps * kChunk;
    const int wo = warp * kChunk;
    // chunk A into registers, chunk B into shared memory; boxes of both
    float px[kLanePts], py[kLanePts], pz[kLanePts], pd[kLanePts];
    const float inf = __int_as_float(0x7f800000);
    float lox = inf, loy = inf, loz = inf, hix = -inf, hiy = -inf, hiz = -inf;
    float blox = inf, bloy = inf, bloz = inf, bhix = -inf, bhiy = -inf, bhiz = -inf;
#pragma unroll
    for (int k = 0; k < kLanePts; ++k) {
        const int o = lane + 32 * k;
        const int64_t i = base + o;
        const bool ok = i < a.n;
        px[k] = ok ? a.x[i] : 0.0f;
        py[k] = ok ? a.y[i] : 0.0f;
        pz[k] = ok ? a.z[i] : 0.0f;
        pd[k] = ok ? inf : -1.0f;  // padding never wins
        s_ids[wo + o] = ok ? a.ids[i] : 0;
        if (ok) {
            lox = fminf(lox, px[k]);
            loy = fminf(loy, py[k]);
            loz = fminf(loz, pz[k]);
            hix = fmaxf(hix, px[k]);
            hiy = fmaxf(hiy, py[k]);
            hiz = fmaxf(hiz, pz[k]);
        }
        const int64_t ib = i + kChunk;
        const bool okb = ib < a.n;
        const float qx = okb ? a.x[ib] : 0.0f, qy = okb ? a.y[ib] : 0.0f, qz = okb ? a.z[ib] : 0.0f;
        s_pts[wo + o] = qx;
        s_pts[kPlane + wo + o] = qy;
        s_pts[2 * kPlane + wo + o] = qz;
        s_pts[3 * kPlane + wo + o] = okb ? inf : -1.0f;
        s_ids[kPlane + wo + o] = okb ? a.ids[ib] : 0;
        if (okb) {
            blox = fminf(blox, qx);
            bloy = fminf(bloy, qy);
            bloz = fminf(bloz, qz);
            bhix = fmaxf(bhix, qx);
            bhiy = fmaxf(bhiy, qy);
            bhiz = fmaxf(bhiz, qz);
        }
    }
    lox = warp_min_f(lox);
    loy = warp_min_f(loy);
    loz = warp_min_f(loz);
    hix = warp_max_f(hix);
    hiy = warp_max_f(hiy);
    hiz = warp_max_f(hiz);
    if (lane == 0) {
        s_bm[7 * kWarps + warp] = lox;
        s_bm[8 * kWarps + warp] = loy;
        s_bm[9 * kWarps + warp] = loz;
        s_bm[10 * kWarps + warp] = hix;
        s_bm[11 * kWarps + warp] = hiy;
        s_bm[12 * kWarps + warp] = hiz;
    }
    blox = warp_min_f(blox);
    bloy = warp_min_f(bloy);
    bloz = warp_min_f(bloz);
    bhix = warp_max_f(bhix);
    bhiy = warp_max_f(bhiy);
    bhiz = warp_max_f(bhiz);
    if (lane == 0) {
        s_bm[0 * kWarps + warp] = blox;
        s_bm[1 * kWarps + warp] = bloy;
        s_bm[2 * kWarps + warp] = bloz;
        s_bm[3 * kWarps + warp] = bhix;
        s_bm[4 * kWarps + warp] = bhiy;
        s_bm[5 * kWarps + warp] = bhiz;
        s_bm[6 * kWarps + warp] = base + kChunk < a.n ? inf : -1.0f;
    }
    // Largest running minimum of chunk A (lane-replicated); -1 = no points.
    float maxd = base < a.n ? inf : -1.0f;
    float lx, ly, lz;
    record_start(a, lx, ly, lz);
    __syncthreads();
    for (int j = 1; j < a.n_landmarks; ++j) {
        if (!(box_gap2(lx, ly, lz, s_bm[7 * kWarps + warp], s_bm[8 * kWarps + warp], s_bm[9 * kWarps + warp],
                       s_bm[10 * kWarps + warp], s_bm[11 * kWarps + warp], s_bm[12 * kWarps + warp]) >= maxd)) {
            float tmax = -1.0f;
#pragma unroll
            for (int k = 0; k < kLanePts; ++k) {
                pd[k] = fminf(pd[k], fps_key(px[k], py[k], pz[k], lx, ly, lz));
                tmax = fmaxf(tmax, pd[k]);
            }
            const float wm = warp_max_f(tmax);
            uint32_t cid = 0xffffffffu;
            float cx = 0.0f, cy = 0.0f, cz = 0.0f;
            if (tmax == wm) {
#pragma unroll
                for (int k = 0; k < kLanePts; ++k) {
                    if (pd[k] == wm) {
                        const uint32_t id = static_cast<uint32_t>(s_ids[wo + lane + 32 * k]);
                        if (id < cid) {
                            cid = id;
                            cx = px[k];
                            cy = py[k];
                            cz = pz[k];
                        }
                    }
                }
            }
            publish_chunk(s, warp, wm, cid, cx, cy, cz, lane);
            maxd = wm;
        }
        const float bmax = s_bm[6 * kWarps + warp];
        if (!(box_gap2(lx, ly, lz, s_bm[warp], s_bm[kWarps + warp], s_bm[2 * kWarps + warp], s_bm[3 * kWarps + warp],
                       s_bm[4 * kWarps + warp], s_bm[5 * kWarps + warp]) >= bmax)) {
            float tmax = -1.0f;
#pragma unroll 4
            for (int k = 0; k < kLanePts; ++k) {
                const int o = lane + 32 * k;
                const float d = fminf(s_pts[3 * kPlane + wo + o],
                                      fps_key(s_pts[wo + o], s_pts[kPlane + wo + o], s_pts[2 * kPlane + wo + o], lx,
                                              ly, lz));
                s_pts[3 * kPlane + wo + o] = d;
                tmax = fmaxf(tmax, d);
            }
            const float wm = warp_max_f(tmax);
            uint32_t cid = 0xffffffffu;
            float cx = 0.0f, cy = 0.0f, cz = 0.0f;
            if (tmax == wm) {
                for (int k = 0; k < kLanePts; ++k) {
                    const int o = lane + 32 * k;
                    if (s_pts[3 * kPlane + wo + o] == wm) {
                        const uint32_t id = static_cast<uint32_t>(s_ids[kPlane + wo + o]);
                        if (id < cid) {
                            cid = id;
                            cx = s_pts[wo + o];
                            cy = s_pts[kPlane + wo + o];
                            cz = s_pts[2 * kPlane + wo + o];
                        }
                    }
                }
            }
            publish_chunk(s, kWarps + warp, wm, cid, cx, cy, cz, lane);
            if (lane == 0) s_bm[6 * kWarps + warp] = wm;
        }
        __syncthreads();
        __syncthreads();
        if (!accept_winner(a, s, j, lx, ly, lz)) break;
    }
}

// ---------------------------------------------------------------- global kernel
// Block b owns chunks [b * CB, (b + 1) * CB) of 32 * lane_pts points each
// (lane_pts a multiple of kGlobalBatch);
// compute warp w updates chunks w, w + 31, ... of its block. Chunk metadata
// (candidate, box, candidate coordinates) lives in shared memory, points and
// running minima in global memory.
// Chunk metadata in shared memory: cand[cb] (uint64), then nine float fields
// of cb entries each (box lo x/y/z, hi x/y/z, candidate x/y/z).
enum : int { kLoX = 0, kLoY, kLoZ, kHiX, kHiY, kHiZ, kCX, kCY, kCZ };

struct ChunkMeta {
    uint64_t* cand;
    float* f;
    int cb;
    __device__ __forceinline__ float& at(int field, int cc) const { return f[field * cb + cc]; }
};

// Fold l into one chunk; new candidate and coordinates into its metadata.
__device__ __forceinline__ void update_chunk(const FpsArgs& a, const ChunkMeta& m, int cc, int64_t base, float lx,
                                             float ly, float lz, int lane) {
    uint64_t best = 0ull;
    float bx = 0.0f, by = 0.0f, bz = 0.0f;
    for (int q = 0; q < a.lane_pts; q += kGlobalBatch) {
        float x[kGlobalBatch], y[kGlobalBatch], z[kGlobalBatch], d[kGlobalBatch];
        int32_t id[kGlobalBatch];
#pragma unroll
        for (int k = 0; k < kGlobalBatch; ++k) {
            const int64_t i = base + lane + 32 * (q + k);
            if (i < a.n) {
                x[k] = __ldg(a.x + i);
                y[k] = __ldg(a.y + i);
                z[k] = __ldg(a.z + i);
                id[k] = __ldg(a.ids + i);
                d[k] = a.d[i];
            }
        }
#pragma unroll
        for (int k = 0; k < kGlobalBatch; ++k) {
            const int64_t i = base + lane + 32 * (q + k);
            if (i < a.n) {
                const float nd = fminf(d[k], fps_key(x[k], y[k], z[k], lx, ly, lz));
                if (nd != d[k]) a.d[i] = nd;
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
    if (lane == owner) {
        m.cand[cc] = wm;
        m.at(kCX, cc) = bx;
        m.at(kCY, cc) = by;
        m.at(kCZ, cc) = bz;
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_fps_global(FpsArgs a) {
    __shared__ FpsShared s;
    extern __shared__ __align__(16) unsigned char s_meta[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    shared_init(s);
    if (warp == kComputeWarps) {
        __syncthreads();
        exchange_loop(a, s, lane);
        return;
    }
    const int cb = a.chunks_per_block;
    const ChunkMeta m{reinterpret_cast<uint64_t*>(s_meta), reinterpret_cast<float*>(s_meta + 8 * size_t(cb)), cb};
    const int64_t c0 = static_cast<int64_t>(blockIdx.x) * cb;
    const int nc = static_cast<int>(max(min(static_cast<int64_t>(cb), a.n_chunks - c0), int64_t(0)));
    const int mine = warp < nc ? (nc - warp + kComputeWarps - 1) / kComputeWarps : 0;  // chunks of this warp
    const int64_t chunk_pts = 32 * static_cast<int64_t>(a.lane_pts);
    // Boxes; running minima start at +inf.
    for (int t = 0; t < mine; ++t) {
        const int cc = warp + kComputeWarps * t;
        const int64_t base = (c0 + cc) * chunk_pts;
        float lox = __int_as_float(0x7f800000), loy = lox, loz = lox;
        float hix = -lox, hiy = -lox, hiz = -lox;
        for (int q = 0; q < a.lane_pts; ++q) {
            const int64_t i = base + lane + 32 * q;
            if (i < a.n) {
                const float x = a.x[i], y = a.y[i], z = a.z[i];
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
        }
    }
    __syncwarp();
    float lx, ly, lz;
    record_start(a, lx, ly, lz);
    __syncthreads();
    for (int j = 1; j < a.n_landmarks; ++j) {
        bool changed = false;
        for (int t0 = 0; t0 < mine; t0 += 32) {
            const int t = t0 + lane;
            bool hit = false;
            if (t < mine) {
                const int cc = warp + kComputeWarps * t;
                hit = !(box_gap2(lx, ly, lz, m.at(kLoX, cc), m.at(kLoY, cc), m.at(kLoZ, cc), m.at(kHiX, cc),
                                 m.at(kHiY, cc), m.at(kHiZ, cc)) >= cand_key(m.cand[cc]));
            }
            uint32_t mask = __ballot_sync(0xffffffffu, hit);
            changed |= mask != 0u;
            while (mask) {
                const int tt = t0 + __ffs(mask) - 1;
                mask &= mask - 1;
                const int cc = warp + kComputeWarps * tt;
                update_chunk(a, m, cc, (c0 + cc) * chunk_pts, lx, ly, lz, lane);
            }
        }
        if (changed) {
            __syncwarp();
            uint64_t best = 0ull;
            int bc = 0;
            for (int t = lane; t < mine; t += 32) {
                const int cc = warp + kComputeWarps * t;
                const uint64_t c = m.cand[cc];
                if (c > best) {
                    best = c;
                    bc = cc;
                }
            }
            const uint64_t wm = warp_max_u64(best);
            const int owner = __ffs(__ballot_sync(0xffffffffu, best == wm)) - 1;
            if (lane == owner) {
                s.cand[warp] = wm;
                s.cx[warp] = m.at(kCX, bc);
                s.cy[warp] = m.at(kCY, bc);
                s.cz[warp] = m.at(kCZ, bc);
            }
        }
        __syncthreads();
        __syncthreads();
        if (!accept_winner(a, s, j, lx, ly, lz)) break;
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
// shared memory hold every point (15,872 per block), else every SM with
// chunks streamed from global memory; n_blocks = k uses k blocks, resident
// when they hold every point.
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
template <class Alloc>
int run_fps(const float* X, int64_t n, int32_t n_landmarks, int64_t start, int n_blocks, int64_t* out_idx,
            float* out_key, cudaStream_t s, Alloc& al, uint32_t** flags_out) {
    FpsPlan plan;
    int rc = plan_fps(n, n_blocks, &plan);
    if (rc) return rc;
    uint32_t* ctl;  // [0] flags, [1..6] ordered box
    uint64_t* slots;
    float *x, *y, *z, *d = nullptr;
    int32_t* ids;
    if ((rc = al.alloc(&ctl, 8)) || (rc = al.alloc(&slots, 2 * kMaxBlocks * kSlotStride)) ||
        (rc = al.alloc(&x, n)) || (rc = al.alloc(&y, n)) || (rc = al.alloc(&z, n)) || (rc = al.alloc(&ids, n)))
        return rc;
    if (!plan.resident && (rc = al.alloc(&d, n))) return rc;
    *flags_out = ctl;
    // Slot tags must start from zero (stale tags could match iterations 1 or 2).
    FLOOD_CUDA(cudaMemsetAsync(slots, 0, sizeof(uint64_t) * 2 * kMaxBlocks * kSlotStride, s));
    k_box_init<<<1, 1, 0, s>>>(ctl + 1, ctl);
    note_launch();
    const unsigned grid = static_cast<unsigned>(ceil_div(n, 256));
    if (n <= kSortMin) {
        k_soa_ids<<<grid, 256, 0, s>>>(X, n, x, y, z, ids, ctl);
        note_launch();
    } else {
        const int bits = morton_bits(n);
        const int64_t codes = int64_t(1) << (3 * bits);
        int32_t *code, *count, *cstart;
        if ((rc = al.alloc(&code, n)) || (rc = al.alloc(&count, codes)) || (rc = al.alloc(&cstart, codes + 1)))
            return rc;
        FLOOD_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t) * codes, s));
        const int64_t bb = std::min<int64_t>(ceil_div(n, kBoxThreads), int64_t(device_sm_count()) * 8);
        k_bbox<<<static_cast<unsigned>(bb), kBoxThreads, 0, s>>>(X, n, ctl + 1, ctl);
        k_morton_count<<<grid, 256, 0, s>>>(X, n, ctl + 1, bits, code, count);
        note_launch(2);
        FLOOD_CUDA(cudaGetLastError());
        if ((rc = exclusive_scan(count, cstart, codes, s, al))) return rc;
        k_morton_scatter<<<grid, 256, 0, s>>>(X, n, code, cstart, count, x, y, z, ids);
        note_launch();
    }
    FLOOD_CUDA(cudaGetLastError());
    FpsArgs a{X, x, y, z, ids, d, n, n_landmarks, start, out_idx, out_key, slots, ctl, 0, 0, 0};
    return launch_fps_kernel(plan, a, s);
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
    Scratch scr(s);
    uint32_t* flags = nullptr;
    int rc = run_fps(X, n_points, n_landmarks, start, n_blocks, out_idx, out_key, s, scr, &flags);
    if (rc) {
        if (flags) cudaStreamSynchronize(s);
        return rc;
    }
    return finish(s, flags, "flood_fps");
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
// Every GPU that loads this library holds that array (26 MiB) until the
// process exits.
// ---------------------------------------------------------------------------
namespace flood {
namespace {

constexpr int64_t kNoAllocMaxPoints = int64_t(1) << 20;  // 1,048,576 points
constexpr size_t kNoAllocBytes = size_t(26) << 20;      // holds run_fps's pieces for 2^20 points

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
    rc = run_fps(X, n_points, n_landmarks, start, 0, out_idx, out_key, s, al, &flags);
    if (rc) {
        if (flags) cudaStreamSynchronize(s);
        return rc;
    }
    return finish(s, flags, "flood_fps_noalloc");
}
