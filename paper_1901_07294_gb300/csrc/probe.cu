// Device probe: measured FMA throughput in FP64 and FP32.
//
// The FP64 operator is bounded by the FP64 units rather than by HBM; its
// roofline needs the machine's FP64 rate, which this probe measures: every
// thread runs 8 independent FMA chains (enough to cover the pipeline
// latency), the grid fills every SM, and the time comes from CUDA events.
#include "wd_internal.h"

namespace wd {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T *sink, int iters, T a, T b)
{
    T c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) c[k] = fma(c[k], a, b);
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += c[k];
    if (s == (T)-1.2345) sink[0] = s;   // keeps the chains alive; never true for these inputs
}

template <typename T> int run_probe(wd_ctx *ctx, double *tflops)
{
    DeviceGuard dg(ctx->device);
    T *sink = nullptr;
    WD_CUDA_TRY(cudaMalloc(&sink, sizeof(T)));
    cudaStream_t s;
    WD_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = ctx->num_sms * 8, threads = 256;
    const int iters = sizeof(T) == 8 ? 4096 : 65536;
    const T a = (T)0.999999, b = (T)1e-7;
    fma_probe_kernel<T><<<blocks, threads, 0, s>>>(sink, iters / 16, a, b);   // warm-up
    cudaEventRecord(e0, s);
    fma_probe_kernel<T><<<blocks, threads, 0, s>>>(sink, iters, a, b);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(sink);
    if (e != cudaSuccess) return set_error(WD_ECUDA, "FMA probe failed: %s", cudaGetErrorString(e));
    const double fmas = (double)blocks * threads * iters * 8;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return WD_OK;
}

} // namespace
} // namespace wd

using namespace wd;

extern "C" int wd_probe_fma(wd_ctx *ctx, int prec, double *tflops)
{
    clear_error();
    if (!ctx || !tflops) return set_error(WD_EINVAL, "NULL argument");
    if (prec == WD_F64) return run_probe<double>(ctx, tflops);
    if (prec == WD_F32) return run_probe<float>(ctx, tflops);
    return set_error(WD_EINVAL, "the FMA probe measures WD_F64 or WD_F32");
}

extern "C" int wd_device_info(const wd_ctx *ctx, wd_device_props *out)
{
    clear_error();
    if (!ctx || !out) return set_error(WD_EINVAL, "NULL argument");
    int v[6] = {0, 0, 0, 0, 0, 0};
    const cudaDeviceAttr attrs[6] = {cudaDevAttrMultiProcessorCount, cudaDevAttrMemoryClockRate,
                                     cudaDevAttrGlobalMemoryBusWidth, cudaDevAttrL2CacheSize,
                                     cudaDevAttrComputeCapabilityMajor, cudaDevAttrComputeCapabilityMinor};
    for (int k = 0; k < 6; ++k) WD_CUDA_TRY(cudaDeviceGetAttribute(&v[k], attrs[k], ctx->device));
    out->sm_count = v[0];
    out->mem_clock_khz = v[1];
    out->mem_bus_bits = v[2];
    out->l2_bytes = v[3];
    out->cc_major = v[4];
    out->cc_minor = v[5];
    // double data rate: two transfers per memory clock
    out->nominal_hbm_gbs = 2.0 * (double)v[1] * 1e3 * (double)v[2] / 8.0 / 1e9;
    int pageable = 0;
    WD_CUDA_TRY(cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, ctx->device));
    out->pageable_memory_access = pageable;
    return WD_OK;
}

extern "C" int wd_device_status(wd_ctx *ctx, int *code)
{
    clear_error();
    if (!ctx || !code) return set_error(WD_EINVAL, "NULL argument");
    DeviceGuard dg(ctx->device);
    WD_CUDA_TRY(cudaDeviceSynchronize());
    int *w = ctx_status_word(ctx);
    int v = 0;
    WD_CUDA_TRY(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) WD_CUDA_TRY(cudaMemset(w, 0, sizeof(int)));
    *code = v;
    return WD_OK;
}
