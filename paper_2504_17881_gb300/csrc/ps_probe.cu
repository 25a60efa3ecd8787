// Arithmetic-throughput probes (include/ps.h, ps_measure_fma_rate).
//
// The complex128 tile pass does two FP64 fused multiply-adds per amplitude
// and rotation and, on GB300, is bound by the FP64 pipe rather than by HBM.
// Its roofline needs the pipe's peak on this device, measured the same way
// the kernel runs: independent fused multiply-add chains in every thread of
// a full grid, timed with CUDA events.  The FP32 variant gives the same
// figure for the complex64 pass's arithmetic.
#include <cuda_runtime.h>

#include <string>

#include "ps_internal.h"

namespace ps {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;  // independent accumulators per thread (hides the FMA latency)

// Every thread runs kProbeChains chains of `iters` fused multiply-adds
// acc <- acc * a + b; |a| < 1 keeps the values bounded.  The sum of the
// accumulators is written so that no chain can be removed.
template <typename R>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(R a, R b, int iters, R *sink) {
    R acc[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc[c] = (R)(threadIdx.x + c) * (R)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) acc[c] = fma(acc[c], a, b);
    }
    R s = 0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += acc[c];
    if (s == (R)12345.678) sink[blockIdx.x] = s;  // practically never true, but not provably false
}

template <typename R>
int run_probe(int blocks_per_sm, int iters, double *tflops_out, std::string *err) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    R *sink = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&sink, sizeof(R) * (size_t)sms * blocks_per_sm);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_ms = 0.f;
    const unsigned grid = (unsigned)(sms * blocks_per_sm);
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first launch is warm-up
        cudaEventRecord(e0, nullptr);
        k_fma_probe<R><<<grid, kProbeThreads>>>((R)0.999999, (R)1e-7, iters, sink);
        cudaEventRecord(e1, nullptr);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) {
        *err = std::string("fma probe: ") + cudaGetErrorString(e);
        return PS_ERR_CUDA;
    }
    const double flops = 2.0 * kProbeChains * (double)iters * (double)grid * kProbeThreads;
    *tflops_out = flops / (best_ms * 1e-3) / 1e12;
    return PS_OK;
}

}  // namespace
}  // namespace ps

extern "C" int ps_measure_fma_rate(int dtype, double *tflops_out) {
    using namespace ps;
    if (!tflops_out) {
        set_error("null output pointer");
        return PS_ERR_ARG;
    }
    std::string err;
    int rc;
    // 2e11 FP64 / 3e12 FP32 flops: about 0.1 s per launch at either rate
    if (dtype == PS_C128)
        rc = run_probe<double>(8, 1 << 12, tflops_out, &err);
    else if (dtype == PS_C64)
        rc = run_probe<float>(8, 1 << 16, tflops_out, &err);
    else {
        set_error("dtype must be PS_C64 or PS_C128");
        return PS_ERR_ARG;
    }
    if (rc) set_error(err);
    return rc;
}
