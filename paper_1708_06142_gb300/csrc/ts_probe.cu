// Arithmetic peak probe: achieved FMA throughput of this GPU with many independent dependency
// chains per thread, for the roofline denominators of the walk kernels (a measurement utility; no
// counterpart in the paper).  Kinds: FP32 scalar FMA, FP32 packed f32x2 FMA (sm_100+), FP64 FMA.
#include "ts_internal.cuh"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_fma_probe(float* out, int iters, float a, float b) {
    const float t = (float)threadIdx.x * 1e-7f;
    if constexpr (KIND == 0) {
        float x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = t + (float)c;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
        }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += x[c];
        if (s == -1.2345f) out[0] = s;   // keeps the chains alive; never true for the inputs used
    } else if constexpr (KIND == 1) {
        float2 x[kChains / 2];
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) x[c] = make_float2(t + (float)c, t - (float)c);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains / 2; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
        }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) s += x[c].x + x[c].y;
        if (s == -1.2345f) out[0] = s;
    } else {
        double x[kChains / 2];
        const double ad = a, bd = b;
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) x[c] = (double)t + c;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains / 2; ++c) x[c] = fma(x[c], ad, bd);
        }
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) s += x[c];
        if (s == -1.2345) out[0] = (float)s;
    }
}

}  // namespace

extern "C" ts_status ts_peak_probe(int32_t device, int32_t kind, double* tflops) {
    FaultSite fault_site("probe");
    if (!tflops || kind < 0 || kind > 2) return ts_fail(TS_ERR_INVALID_ARG, "ts_peak_probe: kind in [0, 2], tflops not NULL");
    DeviceGuard g(device);
    int nsm = 0;
    TS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float* d_out = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = ts_malloc((void**)&d_out, sizeof(float));
    const int grid = nsm * 8;
    // flops per iteration and thread: FP32 scalar 2 per chain, packed 2 per lane of a pair, FP64 2 per chain
    const double flop_it = kind == 2 ? 2.0 * (kChains / 2) : 2.0 * kChains;
    const int iters = kind == 2 ? 4000 : 100000;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // first run warms up, second is timed
        e = cudaEventRecord(e0, st);
        if (kind == 0) k_fma_probe<0><<<grid, kThreads, 0, st>>>(d_out, iters, 0.999999f, 1e-7f);
        else if (kind == 1) k_fma_probe<1><<<grid, kThreads, 0, st>>>(d_out, iters, 0.999999f, 1e-7f);
        else k_fma_probe<2><<<grid, kThreads, 0, st>>>(d_out, iters, 0.999999f, 1e-7f);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (d_out) cudaFree(d_out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return ts_cuda_fail(e, "ts_peak_probe");
    *tflops = flop_it * iters * (double)grid * kThreads / (ms * 1e-3) / 1e12;
    return TS_OK;
}
