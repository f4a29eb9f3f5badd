// Serving runtime: continuous batching of many point clouds on one GPU.
//
// The paper evaluates one cloud at a time; this is the request loop around
// the same computation. Stages of one request:
//   admission  FIFO; a request is admitted when an in-flight slot is free and
//              its estimated device memory fits the budget (no overtaking).
//   gpu        a GPU worker thread copies X to the device, runs FPS and the
//              grid build on its own stream (these overlap across requests).
//   host       a triangulation worker calls the user's callback on the
//              landmarks (Del(L) is input to the method, computed on the host).
//              A callback may return the tetrahedra alone; the worker then
//              builds the triangles, edges and facet incidence on the device
//              (flood_complex_faces) on its own stream.
//   flood      one flood thread takes every request that is ready (up to
//              max_batch) and runs them through a single batched filtration
//              (one persistent flood launch per dimension over all of them),
//              then copies the values back and frees the request's device
//              memory, which admits queued requests.
// While a batch is on the device, later requests keep flowing through the
// gpu and host stages, so their work overlaps. A failing batch is retried one
// request at a time, so a bad request fails alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace flood {
void grid_release_async(flood_grid* g, cudaStream_t s);  // grid.cu: stream-ordered release

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kFloodWorkers = 2;  // threads running batched filtrations

struct Request {
    uint64_t ticket = 0;
    std::vector<float> X;
    int64_t N = 0;
    int32_t n_L = 0;
    int32_t m = 0;
    int64_t bytes = 0;
    Clock::time_point t_submit, t_done;
    // device state (owned while in flight)
    float* X_dev = nullptr;
    int64_t* idx_dev = nullptr;
    float* key_dev = nullptr;
    float* L_dev = nullptr;
    flood_grid* grid = nullptr;
    int32_t* simp_dev[4] = {};
    int32_t* fac_dev[4] = {};
    float* val_dev[4] = {};
    // host state
    std::vector<int64_t> idx;
    std::vector<float> L;
    int64_t nk[4] = {0, 0, 0, 0};
    std::vector<int32_t> simp[4], fac[4];
    std::vector<float> values[4];
    int status = FLOOD_OK;
    bool done = false;
};

}  // namespace
}  // namespace flood

struct flood_server {
    flood_serve_config cfg;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_gpu, cv_tri, cv_flood, cv_done;
    std::deque<flood::Request*> queue, gpu_q, tri_q, ready;
    std::unordered_map<uint64_t, std::unique_ptr<flood::Request>> all;
    uint64_t next_ticket = 1;
    int inflight = 0;
    int64_t bytes_in_use = 0, bytes_peak = 0;
    bool stop = false;
    std::vector<std::thread> threads;
    // statistics
    int64_t submitted = 0, completed = 0, failed = 0, batches = 0, batched_clouds = 0;
    std::vector<double> latencies_ms;
    bool have_first = false;
    flood::Clock::time_point first_submit, last_done;
};

namespace flood {
namespace {

// Device memory a request is expected to hold: X, FPS scratch and grid
// (~64 B per point) plus the filtration's sample records and buckets
// (~20 KB per landmark at moderate m) and a fixed allowance.
int64_t estimate_bytes(int64_t N, int32_t n_L, int32_t m) {
    const double per_landmark = 20000.0 * std::max(1.0, std::pow(m / 8.0, 3.0));
    return static_cast<int64_t>(64.0 * N + per_landmark * n_L) + (int64_t(8) << 20);
}

void admit_locked(flood_server* s) {
    while (!s->queue.empty()) {
        Request* r = s->queue.front();
        if (s->inflight >= s->cfg.max_inflight) break;
        if (s->bytes_in_use + r->bytes > s->cfg.device_budget_bytes) break;
        s->queue.pop_front();
        ++s->inflight;
        s->bytes_in_use += r->bytes;
        s->bytes_peak = std::max(s->bytes_peak, s->bytes_in_use);
        s->gpu_q.push_back(r);
        s->cv_gpu.notify_one();
    }
}

void free_device(Request* r, cudaStream_t st) {
    for (int k = 0; k < 4; ++k) {
        if (r->simp_dev[k]) cudaFreeAsync(r->simp_dev[k], st);
        if (r->fac_dev[k]) cudaFreeAsync(r->fac_dev[k], st);
        if (r->val_dev[k]) cudaFreeAsync(r->val_dev[k], st);
        r->simp_dev[k] = r->fac_dev[k] = nullptr;
        r->val_dev[k] = nullptr;
    }
    if (r->X_dev) cudaFreeAsync(r->X_dev, st);
    if (r->idx_dev) cudaFreeAsync(r->idx_dev, st);
    if (r->key_dev) cudaFreeAsync(r->key_dev, st);
    if (r->L_dev) cudaFreeAsync(r->L_dev, st);
    r->X_dev = r->L_dev = r->key_dev = nullptr;
    r->idx_dev = nullptr;
    // every use of the grid has completed (the stages wait for their streams);
    // a stream-ordered release keeps the other workers' streams running
    if (r->grid) grid_release_async(r->grid, st);
    r->grid = nullptr;
    cudaStreamSynchronize(st);
}

// Mark a request finished (successfully or not) and admit queued ones.
void finish_request(flood_server* s, Request* r, int status, cudaStream_t st) {
    free_device(r, st);
    std::lock_guard<std::mutex> lock(s->mu);
    r->status = status;
    r->done = true;
    r->t_done = Clock::now();
    s->last_done = r->t_done;
    if (status == FLOOD_OK) {
        ++s->completed;
        s->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    } else {
        ++s->failed;
    }
    --s->inflight;
    s->bytes_in_use -= r->bytes;
    admit_locked(s);
    s->cv_done.notify_all();
}

template <class T>
int dev_alloc(T** p, size_t n, cudaStream_t st) {
    return cudaMallocAsync(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T), st) == cudaSuccess
               ? FLOOD_OK
               : FLOOD_ENOMEM;
}

// gpu stage: H2D, FPS, landmarks to the host, grid.
int gpu_stage(flood_server* s, Request* r, cudaStream_t st) {
    int rc;
    if ((rc = dev_alloc(&r->X_dev, 3 * r->N, st)) || (rc = dev_alloc(&r->idx_dev, r->n_L, st)) ||
        (rc = dev_alloc(&r->key_dev, r->n_L, st)) || (rc = dev_alloc(&r->L_dev, 3 * r->n_L, st)))
        return rc;
    if (cudaMemcpyAsync(r->X_dev, r->X.data(), sizeof(float) * 3 * r->N, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "serve: copy X");
    if ((rc = flood_fps(r->X_dev, r->N, r->n_L, 0, r->idx_dev, r->key_dev, st))) return rc;
    r->idx.resize(r->n_L);
    float last_key = 0.0f;
    if (cudaMemcpyAsync(r->idx.data(), r->idx_dev, sizeof(int64_t) * r->n_L, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(&last_key, r->key_dev + (r->n_L - 1), sizeof(float), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
        return cuda_fail(cudaGetLastError(), "serve: copy landmarks");
    if ((rc = flood_check(st))) return rc;  // waits for the landmarks; FPS's own status
    // L = X[idx], taken from the host copy: the same floats bit for bit
    r->L.resize(3 * static_cast<size_t>(r->n_L));
    for (int32_t i = 0; i < r->n_L; ++i)
        for (int c = 0; c < 3; ++c) r->L[3 * i + c] = r->X[3 * r->idx[i] + c];
    if (cudaMemcpyAsync(r->L_dev, r->L.data(), sizeof(float) * 3 * r->n_L, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return cuda_fail(cudaGetLastError(), "serve: copy L");
    const float cover = (r->n_L > 1 && std::isfinite(last_key)) ? std::sqrt(last_key) : 0.0f;
    const float factor = s->cfg.cell_factor > 0.0f ? s->cfg.cell_factor : tuning_for(r->N, r->n_L, r->m).cell_factor;
    const float cell = cover > 0.0f ? factor * cover : 0.0f;
    if ((rc = flood_build_grid(r->X_dev, r->N, cell, &r->grid, st))) return rc;
    return flood_check(st);  // the grid is complete before another stream uses it
}

void gpu_worker(flood_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    for (;;) {
        Request* r;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv_gpu.wait(lock, [&] { return s->stop || !s->gpu_q.empty(); });
            if (s->gpu_q.empty()) break;
            r = s->gpu_q.front();
            s->gpu_q.pop_front();
        }
        const int rc = gpu_stage(s, r, st);
        if (rc) {
            finish_request(s, r, rc, st);
            continue;
        }
        std::lock_guard<std::mutex> lock(s->mu);
        s->tri_q.push_back(r);
        s->cv_tri.notify_one();
    }
    if (st) cudaStreamDestroy(st);
}

// Faces of a tetrahedra-only complex on the device; the host copies of the
// edges and triangles go into the result (their row order is the device's).
int device_faces(Request* r, cudaStream_t st) {
    const int64_t n3 = r->nk[3];
    if (dev_alloc(&r->simp_dev[3], n3 * 4, st) || dev_alloc(&r->simp_dev[2], 4 * n3 * 3, st) ||
        dev_alloc(&r->simp_dev[1], 6 * n3 * 2, st) || dev_alloc(&r->fac_dev[3], n3 * 4, st) ||
        dev_alloc(&r->fac_dev[2], 4 * n3 * 3, st))
        return FLOOD_ENOMEM;
    if (cudaMemcpyAsync(r->simp_dev[3], r->simp[3].data(), sizeof(int32_t) * n3 * 4, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return FLOOD_ECUDA;
    int64_t n2 = 0, n1 = 0;
    int rc = flood_complex_faces(r->simp_dev[3], n3, r->n_L, r->simp_dev[2], r->simp_dev[1], r->fac_dev[3],
                                 r->fac_dev[2], nullptr, &n2, &n1, st);
    if (rc) return rc;
    r->nk[2] = n2;
    r->nk[1] = n1;
    r->simp[2].resize(static_cast<size_t>(n2 * 3));
    r->simp[1].resize(static_cast<size_t>(n1 * 2));
    if (cudaMemcpyAsync(r->simp[2].data(), r->simp_dev[2], sizeof(int32_t) * n2 * 3, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(r->simp[1].data(), r->simp_dev[1], sizeof(int32_t) * n1 * 2, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FLOOD_ECUDA;
    return FLOOD_OK;
}

void tri_worker(flood_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t fst = nullptr;  // this worker's stream for device face builds
    if (cudaStreamCreateWithFlags(&fst, cudaStreamNonBlocking) != cudaSuccess) fst = nullptr;
    for (;;) {
        Request* r;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv_tri.wait(lock, [&] { return s->stop || !s->tri_q.empty(); });
            if (s->tri_q.empty()) break;
            r = s->tri_q.front();
            s->tri_q.pop_front();
        }
        flood_host_complex hc;
        std::memset(&hc, 0, sizeof(hc));
        int rc = s->cfg.triangulate(s->cfg.user, r->L.data(), r->n_L, &hc);
        // tetrahedra alone: the faces are built on the device below
        const bool tets_only = rc == 0 && hc.n_simplices[3] > 0 && hc.n_simplices[1] == 0 && hc.n_simplices[2] == 0;
        if (rc == 0) {
            for (int k = 0; k < 4; ++k) {
                r->nk[k] = hc.n_simplices[k];
                if (r->nk[k] < 0 || (k >= 1 && r->nk[k] > 0 && !hc.simplices[k]) ||
                    (k >= 2 && r->nk[k] > 0 && !tets_only && !hc.facets[k])) {
                    rc = FLOOD_EINVAL;
                    break;
                }
                if (k >= 1 && r->nk[k] > 0) {
                    r->simp[k].assign(hc.simplices[k], hc.simplices[k] + r->nk[k] * (k + 1));
                    if (k >= 2 && !tets_only) r->fac[k].assign(hc.facets[k], hc.facets[k] + r->nk[k] * (k + 1));
                }
            }
            if (rc == 0 && r->nk[0] != 0 && r->nk[0] != r->n_L) rc = FLOOD_EINVAL;
        } else {
            rc = FLOOD_EINVAL;
        }
        if (s->cfg.release && hc.owner) s->cfg.release(s->cfg.user, hc.owner);
        if (rc == 0 && tets_only) rc = fst ? device_faces(r, fst) : FLOOD_ECUDA;
        if (rc) {
            cudaStream_t st = nullptr;
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
            finish_request(s, r, rc, st);
            if (st) cudaStreamDestroy(st);
            continue;
        }
        std::lock_guard<std::mutex> lock(s->mu);
        s->ready.push_back(r);
        s->cv_flood.notify_one();
    }
    if (fst) cudaStreamDestroy(fst);
}

// Upload the complexes of a batch, run the batched filtration and copy values back.
int run_batch(std::vector<Request*>& batch, cudaStream_t st) {
    std::vector<flood_filtration_job> jobs(batch.size());
    for (size_t i = 0; i < batch.size(); ++i) {
        Request* r = batch[i];
        flood_filtration_job& j = jobs[i];
        std::memset(&j, 0, sizeof(j));
        j.grid = r->grid;
        j.L = r->L_dev;
        j.n_landmarks = r->n_L;
        j.m = r->m;
        j.n_simplices[0] = r->n_L;
        for (int k = 0; k < 4; ++k) {
            const int64_t n = k == 0 ? r->n_L : r->nk[k];
            if (k >= 1) j.n_simplices[k] = n;
            if (!r->val_dev[k] && dev_alloc(&r->val_dev[k], n, st)) return FLOOD_ENOMEM;
            j.values[k] = r->val_dev[k];
            if (k >= 1 && n > 0) {
                if (!r->simp_dev[k]) {
                    if (dev_alloc(&r->simp_dev[k], n * (k + 1), st)) return FLOOD_ENOMEM;
                    cudaMemcpyAsync(r->simp_dev[k], r->simp[k].data(), sizeof(int32_t) * n * (k + 1),
                                    cudaMemcpyHostToDevice, st);
                }
                j.simplices[k] = r->simp_dev[k];
                if (k >= 2) {
                    if (!r->fac_dev[k]) {
                        if (dev_alloc(&r->fac_dev[k], n * (k + 1), st)) return FLOOD_ENOMEM;
                        cudaMemcpyAsync(r->fac_dev[k], r->fac[k].data(), sizeof(int32_t) * n * (k + 1),
                                        cudaMemcpyHostToDevice, st);
                    }
                    j.facets[k] = r->fac_dev[k];
                }
            }
        }
    }
    int rc = flood_filtration_batch(jobs.data(), static_cast<int32_t>(jobs.size()), st);
    if (rc) return rc;
    for (Request* r : batch)
        for (int k = 0; k < 4; ++k) {
            const int64_t n = k == 0 ? r->n_L : r->nk[k];
            r->values[k].resize(static_cast<size_t>(n));
            if (n > 0)
                cudaMemcpyAsync(r->values[k].data(), r->val_dev[k], sizeof(float) * n, cudaMemcpyDeviceToHost, st);
        }
    return flood_check(st);  // waits for the values; the filtration's own status
}

void flood_worker(flood_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    for (;;) {
        std::vector<Request*> batch;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv_flood.wait(lock, [&] { return s->stop || !s->ready.empty(); });
            if (s->ready.empty()) break;
            while (!s->ready.empty() && static_cast<int>(batch.size()) < s->cfg.max_batch) {
                batch.push_back(s->ready.front());
                s->ready.pop_front();
            }
            ++s->batches;
            s->batched_clouds += static_cast<int64_t>(batch.size());
        }
        int rc = run_batch(batch, st);
        if (rc && batch.size() > 1) {
            // isolate the failing request(s): one at a time
            for (Request* r : batch) {
                std::vector<Request*> one{r};
                finish_request(s, r, run_batch(one, st), st);
            }
            continue;
        }
        for (Request* r : batch) finish_request(s, r, rc, st);
    }
    if (st) cudaStreamDestroy(st);
}

}  // namespace
}  // namespace flood

using namespace flood;

extern "C" int flood_serve_create(const flood_serve_config* cfg, flood_server** out) {
    if (!cfg || !out || cfg->device_budget_bytes <= 0 || cfg->max_inflight < 1 || cfg->max_batch < 1 ||
        cfg->gpu_workers < 1 || cfg->triangulation_workers < 1 || !(cfg->cell_factor >= 0.0f) ||
        !(cfg->landmark_fraction > 0.0f) || !cfg->triangulate) {
        set_error("flood_serve_create: invalid configuration");
        return FLOOD_EINVAL;
    }
    flood_server* s = new (std::nothrow) flood_server();
    if (!s) {
        set_error("flood_serve_create: host allocation failed");
        return FLOOD_ENOMEM;
    }
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    for (int i = 0; i < cfg->gpu_workers; ++i) s->threads.emplace_back(gpu_worker, s);
    for (int i = 0; i < cfg->triangulation_workers; ++i) s->threads.emplace_back(tri_worker, s);
    // two batch threads on their own streams: one batch's host work and
    // copies overlap the other's kernels
    for (int i = 0; i < kFloodWorkers; ++i) s->threads.emplace_back(flood_worker, s);
    *out = s;
    return FLOOD_OK;
}

extern "C" int flood_serve_submit(flood_server* s, const float* X, int64_t N, int32_t n_L, int32_t m,
                                  uint64_t* ticket) {
    if (!s || !X || !ticket || N < 4 || N >= (int64_t(1) << 31) || m < 1 || m > FLOOD_MAX_M || n_L < 0) {
        set_error("flood_serve_submit: need server, X, ticket, 4 <= N < 2^31, 1 <= m <= %d", FLOOD_MAX_M);
        return FLOOD_EINVAL;
    }
    if (n_L == 0) n_L = static_cast<int32_t>(std::lround(s->cfg.landmark_fraction * static_cast<double>(N)));
    n_L = static_cast<int32_t>(std::min<int64_t>(std::max<int32_t>(n_L, 4), N));
    const int64_t bytes = estimate_bytes(N, n_L, m);
    if (bytes > s->cfg.device_budget_bytes) {
        set_error("flood_serve_submit: cloud needs about %lld bytes, budget is %lld", static_cast<long long>(bytes),
                  static_cast<long long>(s->cfg.device_budget_bytes));
        return FLOOD_ECAPACITY;
    }
    auto r = std::make_unique<Request>();
    r->X.assign(X, X + 3 * N);
    r->N = N;
    r->n_L = n_L;
    r->m = m;
    r->bytes = bytes;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lock(s->mu);
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    if (!s->have_first) {
        s->have_first = true;
        s->first_submit = r->t_submit;
    }
    ++s->submitted;
    s->queue.push_back(r.get());
    s->all.emplace(r->ticket, std::move(r));
    admit_locked(s);
    return FLOOD_OK;
}

extern "C" int flood_serve_poll(flood_server* s, uint64_t ticket, int32_t timeout_ms, flood_result* out) {
    if (!s || !out) {
        set_error("flood_serve_poll: NULL argument");
        return FLOOD_EINVAL;
    }
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        set_error("flood_serve_poll: unknown ticket %llu", static_cast<unsigned long long>(ticket));
        return FLOOD_EINVAL;
    }
    Request* r = it->second.get();
    auto pred = [&] { return r->done; };
    if (timeout_ms < 0)
        s->cv_done.wait(lock, pred);
    else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), pred)) {
        set_error("flood_serve_poll: request %llu not finished", static_cast<unsigned long long>(ticket));
        return FLOOD_ETIMEOUT;
    }
    std::memset(out, 0, sizeof(*out));
    out->status = r->status;
    out->n_landmarks = r->n_L;
    out->landmarks = r->idx.data();
    for (int k = 0; k < 4; ++k) {
        out->n_simplices[k] = k == 0 ? r->n_L : r->nk[k];
        out->values[k] = r->values[k].empty() ? nullptr : r->values[k].data();
        out->simplices[k] = (k == 0 || r->simp[k].empty()) ? nullptr : r->simp[k].data();
    }
    out->latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    return FLOOD_OK;
}

extern "C" int flood_serve_release(flood_server* s, uint64_t ticket) {
    if (!s) return FLOOD_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end() || !it->second->done) {
        set_error("flood_serve_release: ticket %llu is unknown or still running", static_cast<unsigned long long>(ticket));
        return FLOOD_EINVAL;
    }
    s->all.erase(it);
    return FLOOD_OK;
}

extern "C" int flood_serve_stats(flood_server* s, flood_serve_stats_t* out) {
    if (!s || !out) return FLOOD_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->inflight = s->inflight;
    out->batches = s->batches;
    out->mean_batch = s->batches ? static_cast<double>(s->batched_clouds) / s->batches : 0.0;
    out->device_bytes_in_use = s->bytes_in_use;
    out->device_bytes_peak = s->bytes_peak;
    if (!s->latencies_ms.empty()) {
        std::vector<double> v = s->latencies_ms;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[std::min(v.size() - 1, static_cast<size_t>(f * (v.size() - 1) + 0.5))]; };
        out->p50_ms = q(0.5);
        out->p99_ms = q(0.99);
        double sum = 0.0;
        for (double x : v) sum += x;
        out->mean_ms = sum / v.size();
        const double span = std::chrono::duration<double>(s->last_done - s->first_submit).count();
        out->clouds_per_s = span > 0 ? s->completed / span : 0.0;
    }
    return FLOOD_OK;
}

extern "C" void flood_serve_destroy(flood_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        // requests never admitted are dropped
        s->queue.clear();
    }
    s->cv_gpu.notify_all();
    s->cv_tri.notify_all();
    s->cv_flood.notify_all();
    for (auto& t : s->threads) t.join();
    // requests caught between stages still hold device memory
    cudaSetDevice(s->device);
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) {
        for (auto& kv : s->all)
            if (!kv.second->done) free_device(kv.second.get(), st);
        cudaStreamDestroy(st);
    }
    delete s;
}
