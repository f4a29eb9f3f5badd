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

constexpr int kFpsThreads = 512;

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
    unsigned long long* slots;  // 2 * gridDim.x
    uint32_t* counter;
    uint32_t* flags;
};

// K points per thread live in registers when RESIDENT; otherwise coordinates
// and running minima stream from global memory every iteration.
template <int K, bool RESIDENT>
__global__ void __launch_bounds__(kFpsThreads) k_fps(FpsArgs a) {
    __shared__ unsigned long long s_red[kFpsThreads / 32];
    __shared__ unsigned long long s_win;
    __shared__ int s_stop;
    const int nb = gridDim.x;
    const int64_t stride = int64_t(nb) * blockDim.x;
    const int64_t gt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    float px[RESIDENT ? K : 1], py[RESIDENT ? K : 1], pz[RESIDENT ? K : 1], pd[RESIDENT ? K : 1];
    if (RESIDENT) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int64_t i = gt + k * stride;
            const bool ok = i < a.n;
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
    int64_t cur = a.start;
    for (int j = 1; j < a.n_landmarks; ++j) {
        const float lx = a.x[cur], ly = a.y[cur], lz = a.z[cur];
        float best = -1.0f;
        uint32_t bi = 0;
        if (RESIDENT) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                pd[k] = fminf(pd[k], fps_key(px[k], py[k], pz[k], lx, ly, lz));
                if (pd[k] > best) {
                    best = pd[k];
                    bi = static_cast<uint32_t>(gt + k * stride);
                }
            }
        } else {
            for (int64_t i = gt; i < a.n; i += stride) {
                const float d = fminf(a.dmin[i], fps_key(a.x[i], a.y[i], a.z[i], lx, ly, lz));
                a.dmin[i] = d;
                if (d > best) {
                    best = d;
                    bi = static_cast<uint32_t>(i);
                }
            }
        }
        uint64_t key = best >= 0.0f ? pack_key(best, bi) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) key = umax64(key, shfl_xor_u64(key, o));
        if (lane == 0) s_red[warp] = key;
        __syncthreads();
        if (warp == 0) {
            key = lane < (kFpsThreads / 32) ? s_red[lane] : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) key = umax64(key, shfl_xor_u64(key, o));
            if (lane == 0) {
                unsigned long long* slot = a.slots + (j & 1) * nb;
                __stcg(slot + blockIdx.x, static_cast<unsigned long long>(key));
                __threadfence();
                atomicAdd(a.counter, 1u);
                // Grid barrier: every block has published iteration j.
                const uint32_t target = static_cast<uint32_t>(j) * static_cast<uint32_t>(nb);
                uint32_t polls = 0;
                int stop = 0;
                while (ld_acquire_u32(a.counter) < target) {
                    if (++polls > kWaitPolls) {
                        atomicOr(a.flags, FLAG_TIMEOUT);
                        stop = 1;
                        break;
                    }
                }
                s_stop = stop;
            }
            __syncwarp();
            const unsigned long long* slot = a.slots + (j & 1) * nb;
            uint64_t w = 0;
            for (int b = lane; b < nb; b += 32) w = umax64(w, __ldcg(slot + b));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w = umax64(w, shfl_xor_u64(w, o));
            if (lane == 0) s_win = w;
        }
        __syncthreads();
        const uint64_t w = s_win;
        const int stop = s_stop;
        __syncthreads();
        if (stop) break;
        const float wkey = __uint_as_float(static_cast<uint32_t>(w >> 32));
        const int64_t widx = static_cast<int64_t>(0xffffffffu - static_cast<uint32_t>(w));
        if (!(wkey > 0.0f) || w == 0ull) {
            if (gt == 0) atomicOr(a.flags, FLAG_DEGENERATE);
            break;
        }
        cur = widx;
        if (gt == 0) {
            a.out_idx[j] = widx;
            if (a.out_key) a.out_key[j] = wkey;
        }
    }
}

template <int K, bool RESIDENT>
int launch_fps(const FpsArgs& a, cudaStream_t s) {
    int per_sm = 0;
    FLOOD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fps<K, RESIDENT>, kFpsThreads, 0));
    if (per_sm < 1) {
        set_error("flood_fps: kernel does not fit on an SM");
        return FLOOD_EINTERNAL;
    }
    const int nb = device_sm_count() * per_sm;
    if (nb > 4096) {
        set_error("flood_fps: too many co-resident blocks (%d)", nb);
        return FLOOD_EINTERNAL;
    }
    FpsArgs b = a;
    void* args[] = {&b};
    FLOOD_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_fps<K, RESIDENT>), dim3(nb),
                                           dim3(kFpsThreads), args, 0, s));
    note_launch();
    return FLOOD_OK;
}

// Points per thread that the register-resident variants cover at full occupancy.
template <int K>
int64_t resident_capacity() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fps<K, true>, kFpsThreads, 0) != cudaSuccess)
        return 0;
    return int64_t(per_sm) * device_sm_count() * kFpsThreads * K;
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
    unsigned long long* slots;
    uint32_t* ctl;  // [0] counter, [1] flags
    int rc;
    if ((rc = scr.alloc(&x, n_points)) || (rc = scr.alloc(&y, n_points)) || (rc = scr.alloc(&z, n_points)) ||
        (rc = scr.alloc(&slots, 2 * 4096)) || (rc = scr.alloc(&ctl, 2)))
        return rc;
    FLOOD_CUDA(cudaMemsetAsync(ctl, 0, 2 * sizeof(uint32_t), s));
    k_aos_to_soa<<<static_cast<unsigned>(ceil_div(n_points, 256)), 256, 0, s>>>(X, n_points, x, y, z, ctl + 1); note_launch();
    FLOOD_CUDA(cudaGetLastError());

    FpsArgs a{x, y, z, nullptr, n_points, n_landmarks, start, out_idx, out_key, slots, ctl, ctl + 1};
    if (n_points <= resident_capacity<1>())
        rc = launch_fps<1, true>(a, s);
    else if (n_points <= resident_capacity<2>())
        rc = launch_fps<2, true>(a, s);
    else if (n_points <= resident_capacity<4>())
        rc = launch_fps<4, true>(a, s);
    else if (n_points <= resident_capacity<8>())
        rc = launch_fps<8, true>(a, s);
    else if (n_points <= resident_capacity<16>())
        rc = launch_fps<16, true>(a, s);
    else {
        if ((rc = scr.alloc(&dmin, n_points))) return rc;
        // 0x7f = +inf bit pattern per byte would not give +inf; fill with a kernel-free memset of 0xff:
        // 0xffffffff is a NaN, and fminf(NaN, key) = key, so the first update installs the key.
        FLOOD_CUDA(cudaMemsetAsync(dmin, 0xff, sizeof(float) * n_points, s));
        a.dmin = dmin;
        rc = launch_fps<1, false>(a, s);
    }
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
constexpr size_t kNoAllocSlotBytes = sizeof(unsigned long long) * 2 * kNoAllocMaxBlocks;
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
    unsigned long long* slots = reinterpret_cast<unsigned long long*>(base + kNoAllocCtlBytes);
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
    if (n_points <= resident_capacity<1>())
        rc = launch_fps<1, true>(a, s);
    else if (n_points <= resident_capacity<2>())
        rc = launch_fps<2, true>(a, s);
    else if (n_points <= resident_capacity<4>())
        rc = launch_fps<4, true>(a, s);
    else if (n_points <= resident_capacity<8>())
        rc = launch_fps<8, true>(a, s);
    else if (n_points <= resident_capacity<16>())
        rc = launch_fps<16, true>(a, s);
    else {
        FLOOD_CUDA(cudaMemsetAsync(dmin, 0xff, sizeof(float) * n_points, s));
        a.dmin = dmin;
        rc = launch_fps<1, false>(a, s);
    }
    if (rc) return rc;
    return finish(s, ctl + 1, "flood_fps_noalloc");
}
