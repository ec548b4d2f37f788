// FMA issue-rate probe: the ALU roofline denominators of the FP64 and FP32
// stencil kernels, measured on the device the library runs on.  Diagnostic
// only; no part of the integrator uses it.
#include <cuda_runtime.h>

#include "et.h"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_chain_kernel(T* out, int iters, T a, T b) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(tid % 97) * (T)1e-3 + (T)c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[tid] = s;
}

template <typename T>
cudaError_t time_chain(T* out, int blocks, int iters, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                       double* tflops) {
    fma_chain_kernel<T><<<blocks, kProbeThreads, 0, st>>>(out, 16, (T)0.999999, (T)1e-7);
    cudaEventRecord(e0, st);
    fma_chain_kernel<T><<<blocks, kProbeThreads, 0, st>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return e;
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * (double)blocks * kProbeThreads * (double)iters * kChains;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return cudaGetLastError();
}

}  // namespace

extern "C" ET_API et_status et_probe_alu(void* scratch, size_t scratch_bytes, void* cuda_stream,
                                         double* fp64_tflops, double* fp32_tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ET_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ET_ERR_CUDA;
    const int blocks = sms * 8;
    const size_t need = (size_t)blocks * kProbeThreads * sizeof(double);
    if (!scratch || scratch_bytes < need || !fp64_tflops || !fp32_tflops) return ET_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return ET_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return ET_ERR_CUDA;
    }
    cudaError_t e = time_chain<double>((double*)scratch, blocks, 4000, st, e0, e1, fp64_tflops);
    if (e == cudaSuccess) e = time_chain<float>((float*)scratch, blocks, 100000, st, e0, e1, fp32_tflops);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e == cudaSuccess ? ET_OK : ET_ERR_CUDA;
}

extern "C" ET_API size_t et_probe_alu_scratch_bytes(void) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return (size_t)sms * 8 * kProbeThreads * sizeof(double);
}
