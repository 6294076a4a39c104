// FP32-pipe throughput probe: the denominator of the pair kernels' roofline is
// measured on the device at hand rather than derived from a data sheet.  Each
// thread advances 8 independent FMA chains for `iters` steps, either as scalar FMAs
// or as packed two-lane FMAs (f32x2); the result is written so nothing is elided.
#include <cuda_runtime.h>

#include "plan.cuh"

namespace tpcf {

__global__ void __launch_bounds__(256) fma_probe_scalar(float* out, int iters, float a, float b) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 123.456f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma_probe_packed(float* out, int iters, float a, float b) {
    float2 x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = make_float2((float)(threadIdx.x + j) * 1e-3f, (float)j * 1e-3f);
    const float2 A = make_float2(a, a), B = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = __ffma2_rn(x[j], A, B);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j].x + x[j].y;
    if (s == 123.456f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace tpcf

using namespace tpcf;

extern "C" tpcf_status tpcf_probe_fp32_peak(double* tflops2, void* stream) {
    if (!tflops2) return TPCF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    TRY_CUDA(cudaGetDevice(&dev));
    TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256, iters = 1 << 16;
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = dev_malloc((void**)&out, sizeof(float) * blocks * threads);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
        float best = 1e30f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
            cudaEventRecord(e0, s);
            if (kind == 0)
                fma_probe_scalar<<<blocks, threads, 0, s>>>(out, iters, 0.999f, 1e-3f);
            else
                fma_probe_packed<<<blocks, threads, 0, s>>>(out, iters, 0.999f, 1e-3f);
            cudaEventRecord(e1, s);
            e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;  // the first launch warms up
        }
        const double lanes = kind == 0 ? 1.0 : 2.0;
        const double flops = (double)blocks * threads * iters * 8.0 * lanes * 2.0;
        tflops2[kind] = flops / (best * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(out);
    if (e != cudaSuccess) return cuda_fail(e, "tpcf_probe_fp32_peak");
    return TPCF_OK;
}
