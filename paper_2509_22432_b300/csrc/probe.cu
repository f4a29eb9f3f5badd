// flood_fp32_peak_probe: the FP32 FMA throughput of this GPU, measured.
//
// The flood kernels are bound by the FP32 pipe when they are dense (three
// FMAs and a min per sample-point pair), so their roofline is the rate at
// which this GPU retires FP32 FMAs. This kernel issues nothing else: every
// thread runs 16 independent FMA chains (8 packed pairs in the packed form),
// enough to cover the pipe latency at full occupancy, and keeps the results
// alive with one conditional store. The caller times the launch with CUDA
// events on `stream` and divides the flop count by the elapsed time.
#include "common.cuh"

namespace flood {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;
constexpr int kChains = 16;

__global__ void __launch_bounds__(kProbeThreads) k_ffma_peak(float* sink, int64_t iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = static_cast<float>(threadIdx.x) * 1e-7f + static_cast<float>(i);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = __fmaf_rn(x[i], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.0f) sink[blockIdx.x * kProbeThreads + threadIdx.x] = s;  // never true; keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) k_ffma2_peak(float* sink, int64_t iters, float a, float b) {
    float2 x[kChains / 2];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i)
        x[i] = make_float2(static_cast<float>(threadIdx.x) * 1e-7f + static_cast<float>(2 * i),
                           static_cast<float>(threadIdx.x) * 1e-7f + static_cast<float>(2 * i + 1));
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains / 2; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i) s += x[i].x + x[i].y;
    if (s == -1.0f) sink[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace flood

using namespace flood;

extern "C" int flood_fp32_peak_probe(int32_t packed, int64_t iterations, double* flops_out, void* stream_) {
    if (!flops_out || iterations < 1 || iterations > (int64_t(1) << 30)) {
        set_error("flood_fp32_peak_probe: need flops_out != NULL and 1 <= iterations <= 2^30");
        return FLOOD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    const int blocks = device_sm_count() * kProbeBlocksPerSm;
    Scratch scr(s);
    float* sink;
    int rc = scr.alloc(&sink, size_t(blocks) * kProbeThreads);
    if (rc) return rc;
    const float a = 0.99999994f, b = 1e-7f;  // contracting: chains stay finite and normal
    if (packed)
        k_ffma2_peak<<<blocks, kProbeThreads, 0, s>>>(sink, iterations, a, b);
    else
        k_ffma_peak<<<blocks, kProbeThreads, 0, s>>>(sink, iterations, a, b);
    note_launch();
    FLOOD_CUDA(cudaGetLastError());
    *flops_out = 2.0 * kChains * static_cast<double>(iterations) * blocks * kProbeThreads;
    return FLOOD_OK;
}
