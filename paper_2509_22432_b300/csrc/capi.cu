// Status plumbing shared by every entry point of libflood.
#include <stdarg.h>
#include <atomic>
#include <mutex>
#include <stdio.h>

#include "common.cuh"

namespace flood {

static thread_local char g_error[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_error, sizeof(g_error), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a sticky-free error so later calls start clean
    set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return FLOOD_ENOMEM;
    return FLOOD_ECUDA;
}

int status_from_flags(uint32_t flags, const char* where) {
    if (flags == 0) return FLOOD_OK;
    if (flags & FLAG_NONFINITE) {
        set_error("%s: input coordinates or sample weights contain NaN or Inf", where);
        return FLOOD_EINVAL;
    }
    if (flags & FLAG_RANGE) {
        set_error("%s: a vertex or facet id is out of range", where);
        return FLOOD_EINVAL;
    }
    if (flags & FLAG_NOT_SUBSET) {
        set_error("%s: a landmark is not (bitwise) a point of X; L must be a subset of X", where);
        return FLOOD_EINVAL;
    }
    if (flags & FLAG_TIMEOUT) {
        set_error("%s: a bounded device-side wait timed out", where);
        return FLOOD_ETIMEOUT;
    }
    if (flags & FLAG_DEGENERATE) {
        set_error("%s: fewer distinct points than requested landmarks", where);
        return FLOOD_EDEGENERATE;
    }
    set_error("%s: internal consistency check failed (flags 0x%x)", where, flags);
    return FLOOD_EINTERNAL;
}

int finish(cudaStream_t stream, const uint32_t* d_flags, const char* where) {
    uint32_t flags = 0;
    FLOOD_CUDA(cudaMemcpyAsync(&flags, d_flags, sizeof(flags), cudaMemcpyDeviceToHost, stream));
    FLOOD_CUDA(cudaStreamSynchronize(stream));
    return status_from_flags(flags, where);
}

static std::atomic<long long> g_launches{0};

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

// Stream-ordered allocations come from the device's default memory pool. With
// the pool's default release threshold of 0, every synchronisation hands
// freed memory back to the driver and the next allocation maps it again; the
// library keeps up to 4 GiB cached instead (once per device, process-wide).
void keep_pool_warm() {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static bool done[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return;
    done[dev] = true;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    uint64_t threshold = uint64_t(4) << 30;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold) != cudaSuccess) cudaGetLastError();
}

}  // namespace flood

extern "C" const char* flood_last_error(void) { return flood::g_error; }

extern "C" const char* flood_version(void) { return "0.1.0"; }

extern "C" int64_t flood_kernel_launches(void) { return flood::g_launches.load(); }
