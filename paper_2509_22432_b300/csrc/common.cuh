// Internal helpers shared by the libflood translation units: status plumbing,
// device status flags, scratch allocation and inline-PTX wrappers for the
// mbarrier / bulk-copy (TMA) instructions of sm_90+ used on sm_103a.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/flood.h"

namespace flood {

// ---------------------------------------------------------------- device status flags
// Kernels OR these into a device status word instead of trapping; the host
// maps them to a flood_status after the stream has completed.
enum : uint32_t {
    FLAG_NONFINITE = 1u << 0,
    FLAG_RANGE = 1u << 1,       // vertex / facet id out of range
    FLAG_NOT_SUBSET = 1u << 2,  // a landmark is not a point of X
    FLAG_TIMEOUT = 1u << 3,     // a bounded wait gave up
    FLAG_DEGENERATE = 1u << 4,  // FPS ran out of distinct points
    FLAG_INTERNAL = 1u << 5,    // internal capacity / consistency check
    FLAG_BOUNDS = 1u << 6,      // bounds-checked build: an index was out of range (the access was skipped)
};

// Bounds-checked builds (compiled with -DFLOOD_BOUNDS_CHECK, the library
// libflood_checked.so): every data-dependent index of the kernels is tested
// before use; an index outside [0, n) skips the access and raises FLAG_BOUNDS
// in the call's status word (reported as FLOOD_EINTERNAL) instead of reading
// or writing out of range. In the normal build the test compiles away.
#ifdef FLOOD_BOUNDS_CHECK
#define FLOOD_OOB(i, n, flags) (::flood::index_out_of_range(static_cast<long long>(i), static_cast<long long>(n), (flags)))
#else
#define FLOOD_OOB(i, n, flags) false
#endif

// Bound on polls of a device-side wait (mbarrier phase, grid barrier). Each
// poll is at least a round trip to L2 or a try_wait time slice, so the bound
// is seconds, far above any legitimate wait.
constexpr uint32_t kWaitPolls = 1u << 22;

// ---------------------------------------------------------------- host-side status
void set_error(const char* fmt, ...);
int status_from_flags(uint32_t flags, const char* where);
int cuda_fail(cudaError_t e, const char* what);

#define FLOOD_CUDA(call)                                  \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return ::flood::cuda_fail(e_, #call); \
    } while (0)

// Keep the device's default memory pool from returning freed memory to the
// driver at every synchronisation (up to 4 GiB stays cached; once per device).
void keep_pool_warm();

// Stream-ordered scratch that is returned on scope exit. Pieces (256-byte
// aligned) are carved from chunks of at least 16 MiB taken from the
// stream-ordered pool, so a call makes one or two pool requests instead of
// one per buffer.
struct Scratch {
    static constexpr size_t kChunk = size_t(16) << 20;
    cudaStream_t stream;
    std::vector<void*> ptrs;  // chunks
    unsigned char* cur = nullptr;
    size_t left = 0;
    explicit Scratch(cudaStream_t s) : stream(s) { keep_pool_warm(); }
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, stream);
    }
    template <class T>
    int alloc(T** out, size_t count) {
        *out = nullptr;
        if (count == 0) count = 1;
        const size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (bytes > left) {
            const size_t size = bytes > kChunk ? bytes : kChunk;
            void* p = nullptr;
            cudaError_t e = cudaMallocAsync(&p, size, stream);
            if (e != cudaSuccess) {
                cudaGetLastError();
                set_error("device allocation of %zu bytes failed: %s", size, cudaGetErrorString(e));
                return FLOOD_ENOMEM;
            }
            ptrs.push_back(p);
            cur = static_cast<unsigned char*>(p);
            left = size;
        }
        *out = reinterpret_cast<T*>(cur);
        cur += bytes;
        left -= bytes;
        return FLOOD_OK;
    }
};

// Scratch carved from a caller-owned device buffer (no allocation): the same
// alloc() interface as Scratch, 256-byte aligned pieces, FLOOD_ECAPACITY when
// the buffer is exhausted.
struct Bump {
    unsigned char* p;
    size_t left;
    template <class T>
    int alloc(T** out, size_t count) {
        if (count == 0) count = 1;
        const size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (bytes > left) {
            *out = nullptr;
            set_error("fixed scratch exhausted (%zu bytes requested, %zu left)", bytes, left);
            return FLOOD_ECAPACITY;
        }
        *out = reinterpret_cast<T*>(p);
        p += bytes;
        left -= bytes;
        return FLOOD_OK;
    }
};

// Wait for `stream`, then turn the device status word into a flood_status.
int finish(cudaStream_t stream, const uint32_t* d_flags, const char* where);

// Deferred status of the asynchronous entry points. defer_status enqueues a
// copy of the call's device status word into a pinned host slot and returns
// at once; flood_check(stream) synchronises the stream and reports the first
// error of its calls. pending_error returns, without waiting, an error that
// an earlier call on `stream` has already delivered (every asynchronous
// entry point calls it first, so an error is reported by the next call at
// the latest). A status that arrives while the slot table is full is
// waited for on the spot.
int defer_status(cudaStream_t stream, const uint32_t* d_flags, const char* where);
int pending_error(cudaStream_t stream);

// Pinned host buffer and a completion event of the calling thread, for
// statistics that calls copy back without waiting (one per purpose and thread).
struct HostStats {
    void* host = nullptr;
    size_t bytes = 0;
    cudaEvent_t done = nullptr;
    int device = -1;
    bool valid = false;
    ~HostStats();
    int reserve(size_t n);  // pinned buffer of at least n bytes and an event on the current device
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int device_sm_count();

// Tuned launch parameters for a workload bucket (tuning table, or defaults).
flood_tuning tuning_for(int64_t n_points, int32_t n_landmarks, int32_t m);

// Process-wide count of kernels this library has launched (reported by
// flood_kernel_launches for launch accounting).
void note_launch(int n = 1);

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order earlier generic-proxy accesses of shared memory before later
// async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase. Returns false (and raises FLAG_TIMEOUT)
// if the phase did not complete within kWaitPolls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* flags) {
    for (uint32_t i = 0; i < kWaitPolls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(flags, FLAG_TIMEOUT);
    return false;
}

// 1-D bulk copy global -> shared through the TMA unit; completion is counted
// in bytes on `bar`. dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Four relaxed 64-bit words at a 32-byte aligned address (one 256-bit access);
// each word is single-copy atomic on its own (no atomicity across words).
__device__ __forceinline__ void ld_relaxed_v4_u64(const uint64_t* p, uint64_t& a, uint64_t& b, uint64_t& c,
                                                  uint64_t& d) {
    asm volatile("ld.relaxed.gpu.global.v4.u64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(a), "=l"(b), "=l"(c), "=l"(d)
                 : "l"(p)
                 : "memory");
}

__device__ __forceinline__ void st_relaxed_v4_u64(uint64_t* p, uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
    asm volatile("st.relaxed.gpu.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d)
                 : "memory");
}

#ifdef FLOOD_BOUNDS_CHECK
__device__ __forceinline__ bool index_out_of_range(long long i, long long n, uint32_t* flags) {
    if (i >= 0 && i < n) return false;
    if (flags) atomicOr(flags, FLAG_BOUNDS);
    return true;
}
#endif

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int mask) {
    uint32_t lo = static_cast<uint32_t>(v), hi = static_cast<uint32_t>(v >> 32);
    lo = __shfl_xor_sync(0xffffffffu, lo, mask);
    hi = __shfl_xor_sync(0xffffffffu, hi, mask);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

}  // namespace flood
