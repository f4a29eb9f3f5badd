// flood_fps: farthest point sampling (§3.2), the landmark selection of the
// Flood complex.
//
// One persistent cooperative kernel runs all n_landmarks - 1 iterations.
// Every thread owns a fixed, strided set of points; per iteration it folds the
// newest landmark into its points' running minima and keeps its local argmax.
// Block results go to a per-iteration slot array, one grid-wide arrival
// counter (bounded spin) orders the iteration, and every block then reduces
// all slots itself, so a single barrier per iteration suffices. The argmax is
// a 64-bit max over (key bits << 32 | ~index): non-negative binary32 keys
// order like their bit patterns, and ~index makes ties go to the lowest index.
//
// The key is the binary32 squared distance with each operation rounded on its
// own (__fsub_rn/__fmul_rn/__fadd_rn are never contracted into FMAs), which
// makes the picks bit-exact against a binary32 reference.
#include <algorithm>

#include "common.cuh"

namespace flood {

namespace {


__global__ void __launch_bounds__(256) k_aos_to_soa(const float* X, int64_t n, float* x, float* y, float* z,
                                                   uint32_t* flags) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const float a = X[3 * i + 0], b = X[3 * i + 1], c = X[3 * i + 2];
    if (!(isfinite(a) && isfinite(b) && isfinite(c))) atomicOr(flags, FLAG_NONFINITE);
    x[i] = a;
    y[i] = b;
    z[i] = c;
}

__device__ __forceinline__ float fps_key(float px, float py, float pz, float lx, float ly, float lz) {
    const float dx = __fsub_rn(px, lx);
    const float dy = __fsub_rn(py, ly);
    const float dz = __fsub_rn(pz, lz);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

__device__ __forceinline__ uint64_t pack_key(float d, uint32_t i) {
    return (static_cast<uint64_t>(__float_as_uint(d)) << 32) | static_cast<uint64_t>(0xffffffffu - i);
}

// Per-block candidate of one iteration, in one 64-bit word that is written
// and read atomically (naturally aligned):
//   bits 63..62  iteration tag (j mod 4)
//   bits 61..31  key bits (non-negative binary32, sign bit dropped)
//   bits 30..0   0x7fffffff - index (ties go to the lowest index)
// Readers poll the slots of iteration j until every tag matches, which both
// synchronises the grid and delivers the candidates in one pass. Slots are
// double-buffered by parity; a block cannot run two iterations ahead of a
// reader because it needs that reader's next slot first.
using FpsSlot = unsigned long long;

__device__ __forceinline__ uint64_t pack_slot(float d, uint32_t i, int j) {
    return (static_cast<uint64_t>(j & 3) << 62) | (static_cast<uint64_t>(__float_as_uint(d) & 0x7fffffffu) << 31) |
           static_cast<uint64_t>(0x7fffffffu - i);
}

struct FpsArgs {
    const float* x;
    const float* y;
    const float* z;
    float* dmin;  // streaming variant only
    int64_t n;
    int32_t n_landmarks;
    int64_t start;
    int64_t* out_idx;
    float* out_key;
    FpsSlot* slots;  // 2 * gridDim.x
    uint32_t* counter;
    uint32_t* flags;
};

constexpr uint64_t kSlotValue = (uint64_t(1) << 62) - 1;

// K points per thread live in registers when RESIDENT; otherwise coordinates
// and running minima stream from global memory every iteration.
template <int K, bool RESIDENT, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) k_fps(FpsArgs a) {
    constexpr int kWarpsPerBlock = THREADS / 32;
    __shared__ unsigned long long s_key[kWarpsPerBlock];
    __shared__ unsigned long long s_win;
    __shared__ int s_stop;
    const int nb = gridDim.x;
    const uint32_t n = static_cast<uint32_t>(a.n);
    const uint32_t stride = static_cast<uint32_t>(nb) * THREADS;
    const uint32_t gt = blockIdx.x * THREADS + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    float px[RESIDENT ? K : 1], py[RESIDENT ? K : 1], pz[RESIDENT ? K : 1], pd[RESIDENT ? K : 1];
    if (RESIDENT) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint32_t i = gt + k * stride;
            const bool ok = i < n;
            px[k] = ok ? a.x[i] : 0.0f;
            py[k] = ok ? a.y[i] : 0.0f;
            pz[k] = ok ? a.z[i] : 0.0f;
            pd[k] = ok ? __int_as_float(0x7f800000) : -1.0f;  // padding never wins
        }
    }
    if (gt == 0) {
        a.out_idx[0] = a.start;
        if (a.out_key) a.out_key[0] = __int_as_float(0x7f800000);
    }
    float lx = a.x[a.start], ly = a.y[a.start], lz = a.z[a.start];
    for (int j = 1; j < a.n_landmarks; ++j) {
        float best = -1.0f;
        uint32_t bi = 0;
        if (RESIDENT) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                pd[k] = fminf(pd[k], fps_key(px[k], py[k], pz[k], lx, ly, lz));
                if (pd[k] > best) {
                    best = pd[k];
                    bi = gt + k * stride;
                }
            }
        } else {
            for (uint32_t i = gt; i < n; i += stride) {
                const float d = fminf(a.dmin[i], fps_key(a.x[i], a.y[i], a.z[i], lx, ly, lz));
                a.dmin[i] = d;
                if (d > best) {
                    best = d;
                    bi = i;
                }
            }
        }
        uint64_t key = best >= 0.0f ? (pack_slot(best, bi, 0) & kSlotValue) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) key = umax64(key, shfl_xor_u64(key, o));
        if (lane == 0) s_key[warp] = key;
        __syncthreads();
        if (warp == 0) {
            uint64_t bk = lane < kWarpsPerBlock ? s_key[lane] : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bk = umax64(bk, shfl_xor_u64(bk, o));
            const uint64_t tag = static_cast<uint64_t>(j & 3) << 62;
            FpsSlot* buf = a.slots + (j & 1) * nb;
            if (lane == 0) __stcg(buf + blockIdx.x, tag | bk);
            // Poll every block's slot of iteration j (bounded); the maximum of
            // the values is the winner.
            uint64_t w = 0ull;
            uint32_t polls = 0;
            int stop = 0;
            for (;;) {
                bool ready = true;
                uint64_t m = 0ull;
                for (int b = lane; b < nb; b += 32) {
                    const uint64_t v = __ldcg(buf + b);
                    ready &= (v & ~kSlotValue) == tag;
                    m = umax64(m, v & kSlotValue);
                }
                if (__all_sync(0xffffffffu, ready)) {
                    w = m;
                    break;
                }
                if (++polls > kWaitPolls) {
                    stop = 1;
                    if (lane == 0) atomicOr(a.flags, FLAG_TIMEOUT);
                    break;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w = umax64(w, shfl_xor_u64(w, o));
            if (lane == 0) {
                s_win = w;
                s_stop = stop;
            }
        }
        __syncthreads();
        const uint64_t w = s_win;
        const int stop = s_stop;
        __syncthreads();
        if (stop) break;
        const float wkey = __uint_as_float(static_cast<uint32_t>(w >> 31));
        const uint32_t widx = 0x7fffffffu - static_cast<uint32_t>(w & 0x7fffffffu);
        if (!(wkey > 0.0f) || w == 0ull) {
            if (gt == 0) atomicOr(a.flags, FLAG_DEGENERATE);
            break;
        }
        lx = a.x[widx];
        ly = a.y[widx];
        lz = a.z[widx];
        if (gt == 0) {
            a.out_idx[j] = widx;
            if (a.out_key) a.out_key[j] = wkey;
        }
    }
}

constexpr int kResidentThreads = 1024;
constexpr int kStreamThreads = 512;

// The grid holds just enough blocks for the points (at most all co-resident
// blocks): small clouds synchronise fewer blocks and leave the rest of the
// GPU to other work.
template <int K, bool RESIDENT, int THREADS>
int launch_fps(const FpsArgs& a, cudaStream_t s) {
    int per_sm = 0;
    FLOOD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fps<K, RESIDENT, THREADS>, THREADS, 0));
    if (per_sm < 1) {
        set_error("flood_fps: kernel does not fit on an SM");
        return FLOOD_EINTERNAL;
    }
    const int64_t needed = ceil_div(a.n, int64_t(THREADS) * K);
    const int nb = static_cast<int>(std::min<int64_t>(int64_t(device_sm_count()) * per_sm, std::max<int64_t>(needed, 1)));
    if (nb > 4096) {
        set_error("flood_fps: too many co-resident blocks (%d)", nb);
        return FLOOD_EINTERNAL;
    }
    FpsArgs b = a;
    void* args[] = {&b};
    FLOOD_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_fps<K, RESIDENT, THREADS>), dim3(nb),
                                           dim3(THREADS), args, 0, s));
    note_launch();
    return FLOOD_OK;
}

// Points per thread that the register-resident variants cover at full occupancy.
template <int K>
int64_t resident_capacity() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fps<K, true, kResidentThreads>, kResidentThreads,
                                                      0) != cudaSuccess)
        return 0;
    return int64_t(per_sm) * device_sm_count() * kResidentThreads * K;
}

// Launch the register-resident variant that covers n points, else the streaming one.
int launch_fps_any(FpsArgs a, float* dmin, cudaStream_t s) {
    const int64_t n = a.n;
    // Slot tags must start from zero (stale tags could match iteration 1 or 2).
    FLOOD_CUDA(cudaMemsetAsync(a.slots, 0, sizeof(FpsSlot) * 2 * 4096, s));
    if (n <= resident_capacity<1>()) return launch_fps<1, true, kResidentThreads>(a, s);
    if (n <= resident_capacity<2>()) return launch_fps<2, true, kResidentThreads>(a, s);
    if (n <= resident_capacity<4>()) return launch_fps<4, true, kResidentThreads>(a, s);
    if (n <= resident_capacity<8>()) return launch_fps<8, true, kResidentThreads>(a, s);
    // 0xffffffff is a NaN, and fminf(NaN, key) = key: the first update installs the key.
    FLOOD_CUDA(cudaMemsetAsync(dmin, 0xff, sizeof(float) * n, s));
    a.dmin = dmin;
    return launch_fps<1, false, kStreamThreads>(a, s);
}

}  // namespace

}  // namespace flood

using namespace flood;

extern "C" int flood_fps(const float* X, int64_t n_points, int32_t n_landmarks, int64_t start, int64_t* out_idx,
                         float* out_key, void* stream_) {
    if (!X || !out_idx || n_points < 1 || n_points >= (int64_t(1) << 31) || n_landmarks < 1 ||
        n_landmarks > n_points || start < 0 || start >= n_points) {
        set_error("flood_fps: need X, out_idx != NULL, 1 <= n_landmarks <= n_points < 2^31, 0 <= start < n_points");
        return FLOOD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    Scratch scr(s);
    float *x, *y, *z, *dmin = nullptr;
    FpsSlot* slots;
    uint32_t* ctl;  // [0] counter, [1] flags
    int rc;
    if ((rc = scr.alloc(&x, n_points)) || (rc = scr.alloc(&y, n_points)) || (rc = scr.alloc(&z, n_points)) ||
        (rc = scr.alloc(&slots, 2 * 4096)) || (rc = scr.alloc(&ctl, 2)))
        return rc;
    FLOOD_CUDA(cudaMemsetAsync(ctl, 0, 2 * sizeof(uint32_t), s));
    k_aos_to_soa<<<static_cast<unsigned>(ceil_div(n_points, 256)), 256, 0, s>>>(X, n_points, x, y, z, ctl + 1); note_launch();
    FLOOD_CUDA(cudaGetLastError());

    if (n_points > resident_capacity<8>() && (rc = scr.alloc(&dmin, n_points))) return rc;
    FpsArgs a{x, y, z, nullptr, n_points, n_landmarks, start, out_idx, out_key, slots, ctl, ctl + 1};
    rc = launch_fps_any(a, dmin, s);
    if (rc) return rc;
    return finish(s, ctl + 1, "flood_fps");
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
// flood_fps but takes its scratch (the structure-of-arrays copy of X, running
// minima, per-block slots and control words) from one file-scope device array
// of fixed size that is part of the loaded module. Every GPU that loads this
// library holds that array (about 16 MiB) until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace flood {
namespace {

constexpr int64_t kNoAllocMaxPoints = int64_t(1) << 20;  // 1,048,576 points
constexpr int kNoAllocMaxBlocks = 4096;
constexpr size_t kNoAllocCtlBytes = 256;
constexpr size_t kNoAllocSlotBytes = sizeof(FpsSlot) * 2 * kNoAllocMaxBlocks;
constexpr size_t kNoAllocArrayBytes = sizeof(float) * kNoAllocMaxPoints;
constexpr size_t kNoAllocBytes = kNoAllocCtlBytes + kNoAllocSlotBytes + 4 * kNoAllocArrayBytes;

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
    if (!X || !out_idx || n_points < 1 || n_landmarks < 1 || n_landmarks > n_points || start < 0 ||
        start >= n_points) {
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
    uint32_t* ctl = reinterpret_cast<uint32_t*>(base);  // [0] barrier counter, [1] flags
    FpsSlot* slots = reinterpret_cast<FpsSlot*>(base + kNoAllocCtlBytes);
    float* arrays = reinterpret_cast<float*>(base + kNoAllocCtlBytes + kNoAllocSlotBytes);
    float* x = arrays;
    float* y = arrays + kNoAllocMaxPoints;
    float* z = arrays + 2 * kNoAllocMaxPoints;
    float* dmin = arrays + 3 * kNoAllocMaxPoints;
    // The array keeps whatever the previous call left: clear the counter and flags.
    FLOOD_CUDA(cudaMemsetAsync(ctl, 0, 2 * sizeof(uint32_t), s));
    k_aos_to_soa<<<static_cast<unsigned>(ceil_div(n_points, 256)), 256, 0, s>>>(X, n_points, x, y, z, ctl + 1);
    note_launch();
    FLOOD_CUDA(cudaGetLastError());
    FpsArgs a{x, y, z, nullptr, n_points, n_landmarks, start, out_idx, out_key, slots, ctl, ctl + 1};
    rc = launch_fps_any(a, dmin, s);
    if (rc) return rc;
    return finish(s, ctl + 1, "flood_fps_noalloc");
}
