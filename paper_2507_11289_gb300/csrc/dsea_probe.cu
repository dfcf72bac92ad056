// dsea_probe.cu -- arithmetic peak probes of this GPU, for the roofline
// denominators of the benchmark (no counterpart in the paper).
//
// Each probe launches 8 CTAs of 256 threads per SM; every thread runs 8
// independent fused-multiply-add chains (enough independent work to hide the
// pipe latency) for a fixed number of trips, unrolled so that loop overhead
// is a few percent of the issued instructions.  The rate is the counted
// flops (2 per FMA, 4 per packed two-lane FMA) over the CUDA-event time of
// the fastest of three launches, after one untimed warm-up launch.
#include "dsea_host.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;
constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kTrips = 2048;

__global__ void __launch_bounds__(kProbeThreads) k_probe_f32(float seed, float *sink)
{
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
    const float m = 0.999f, k = 1.0e-3f;
    for (int t = 0; t < kTrips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, k);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.678f) sink[blockIdx.x] = s;   // keeps the chains alive; never true in practice
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2,%3};\n\tmov.b64 rb, {%4,%5};\n\t"
        "mov.b64 rc, {%6,%7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0,%1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_f32x2(float seed, float *sink)
{
    float2 a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = make_float2(seed + (float)(threadIdx.x + c), seed - (float)c);
    const float2 m = make_float2(0.999f, 0.998f), k = make_float2(1.0e-3f, 2.0e-3f);
    for (int t = 0; t < kTrips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fma2(a[c], m, k);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c].x + a[c].y;
    if (s == 12345.678f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_f64(double seed, float *sink)
{
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (double)(threadIdx.x + c);
    const double m = 0.999, k = 1.0e-3;
    for (int t = 0; t < kTrips / 16; ++t) {   // the FP64 pipe is far slower: fewer trips
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, k);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.678) sink[blockIdx.x] = (float)s;
}

}  // namespace

extern "C" int dsea_probe_peak(int kind, void *cuda_stream, double *tflops)
{
    if (!tflops || kind < DSEA_PROBE_FP32 || kind > DSEA_PROBE_FP64) return DSEA_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return DSEA_ERR_NO_DEVICE;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int blocks = sms * kProbeBlocksPerSm;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(float) * (size_t)blocks);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // a warm-up, then three timed launches
        if (rep > 0) e = cudaEventRecord(e0, st);
        if (kind == DSEA_PROBE_FP32) k_probe_f32<<<blocks, kProbeThreads, 0, st>>>(1.0f, sink);
        else if (kind == DSEA_PROBE_FP32X2) k_probe_f32x2<<<blocks, kProbeThreads, 0, st>>>(1.0f, sink);
        else k_probe_f64<<<blocks, kProbeThreads, 0, st>>>(1.0, sink);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (rep > 0 && e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (rep > 0 && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (rep > 0 && e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0 && e == cudaSuccess && (ms == 0.f || t < ms)) ms = t;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess || !(ms > 0.f)) {
        cudaGetLastError();
        return DSEA_ERR_CUDA;
    }
    const double threads = (double)blocks * kProbeThreads;
    const double fmas = kind == DSEA_PROBE_FP64 ? (double)(kTrips / 16) * kUnroll * kChains
                                                : (double)kTrips * kUnroll * kChains;
    const double flops_per_fma = kind == DSEA_PROBE_FP32X2 ? 4.0 : 2.0;
    *tflops = threads * fmas * flops_per_fma / ((double)ms * 1e-3) / 1e12;
    return DSEA_OK;
}
