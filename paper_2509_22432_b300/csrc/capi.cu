// Status plumbing shared by every entry point of libflood.
#include <stdarg.h>
#include <atomic>
#include <mutex>
#include <stdio.h>
#include <vector>

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
    if (flags & FLAG_BOUNDS) {
        set_error("%s: an index was out of range (bounds-checked build; the access was skipped)", where);
        return FLOOD_EINTERNAL;
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

// ---------------------------------------------------------------- deferred status
namespace {

constexpr int kStatusSlots = 4096;
constexpr int kMaxPendingPerStream = 1024;

struct Pending {
    cudaStream_t stream;
    int device;
    int slot;
    char where[48];
};

std::mutex g_pend_mu;
volatile uint32_t* g_slot_words = nullptr;  // pinned host memory, written by stream-ordered copies
std::vector<int> g_free_slots;
std::vector<Pending> g_pending;

int slots_ready_locked() {
    if (g_slot_words) return FLOOD_OK;
    void* p = nullptr;
    cudaError_t e = cudaHostAlloc(&p, sizeof(uint32_t) * kStatusSlots, cudaHostAllocPortable);
    if (e != cudaSuccess) return cuda_fail(e, "status slots (cudaHostAlloc)");
    g_slot_words = static_cast<volatile uint32_t*>(p);
    for (int i = kStatusSlots - 1; i >= 0; --i) g_free_slots.push_back(i);
    return FLOOD_OK;
}

// Remove the entries of (stream, device) that are final (all of them, or
// those whose word already arrived non-zero) and return the first error.
int collect_locked(cudaStream_t s, int dev, bool all) {
    int rc = FLOOD_OK;
    size_t keep = 0;
    for (size_t i = 0; i < g_pending.size(); ++i) {
        Pending& p = g_pending[i];
        const bool mine = p.stream == s && p.device == dev;
        const uint32_t w = mine ? g_slot_words[p.slot] : 0u;
        if (mine && (all || w != 0u)) {
            if (rc == FLOOD_OK && w != 0u) rc = status_from_flags(w, p.where);
            g_free_slots.push_back(p.slot);
        } else {
            g_pending[keep++] = p;
        }
    }
    g_pending.resize(keep);
    return rc;
}

size_t count_locked(cudaStream_t s, int dev) {
    size_t n = 0;
    for (const Pending& p : g_pending) n += p.stream == s && p.device == dev;
    return n;
}

}  // namespace

int pending_error(cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return FLOOD_OK;
    }
    std::lock_guard<std::mutex> lock(g_pend_mu);
    if (g_pending.empty()) return FLOOD_OK;
    return collect_locked(s, dev, false);
}

static int check_stream(cudaStream_t s) {
    int dev = 0;
    FLOOD_CUDA(cudaGetDevice(&dev));
    FLOOD_CUDA(cudaStreamSynchronize(s));
    std::lock_guard<std::mutex> lock(g_pend_mu);
    if (g_pending.empty()) return FLOOD_OK;
    return collect_locked(s, dev, true);
}

int defer_status(cudaStream_t s, const uint32_t* d_flags, const char* where) {
    int dev = 0;
    FLOOD_CUDA(cudaGetDevice(&dev));
    int slot = -1;
    size_t n_mine = 0;
    {
        std::lock_guard<std::mutex> lock(g_pend_mu);
        if (int rc = slots_ready_locked()) return rc;
        if (!g_free_slots.empty()) {
            slot = g_free_slots.back();
            g_free_slots.pop_back();
            g_slot_words[slot] = 0u;
            Pending p{s, dev, slot, {0}};
            snprintf(p.where, sizeof(p.where), "%s", where);
            g_pending.push_back(p);
            n_mine = count_locked(s, dev);
        }
    }
    if (slot < 0) return finish(s, d_flags, where);  // table full: wait for this call's status now
    FLOOD_CUDA(cudaMemcpyAsync(const_cast<uint32_t*>(g_slot_words + slot), d_flags, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
    if (n_mine > static_cast<size_t>(kMaxPendingPerStream)) return check_stream(s);  // bound the table per stream
    return FLOOD_OK;
}

HostStats::~HostStats() {
    if (host) cudaFreeHost(host);
    if (done) cudaEventDestroy(done);
}

int HostStats::reserve(size_t n) {
    int dev = 0;
    FLOOD_CUDA(cudaGetDevice(&dev));
    if (done && device != dev) {
        cudaEventDestroy(done);
        done = nullptr;
    }
    if (!done) {
        FLOOD_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
        device = dev;
    }
    if (bytes < n) {
        if (host) cudaFreeHost(host);
        host = nullptr;
        bytes = 0;
        FLOOD_CUDA(cudaHostAlloc(&host, n, cudaHostAllocPortable));
        bytes = n;
    }
    return FLOOD_OK;
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

extern "C" int flood_check(void* stream) { return flood::check_stream(static_cast<cudaStream_t>(stream)); }

extern "C" const char* flood_version(void) { return "0.1.0"; }

extern "C" int64_t flood_kernel_launches(void) { return flood::g_launches.load(); }
