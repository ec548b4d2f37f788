// FMA issue-rate probe: the ALU roofline denominators of the FP64 and FP32
// stencil kernels, measured on the device the library runs on.  Diagnostic
// only; no part of the integrator uses it.
#include <cuda_runtime.h>

#include <cstdint>

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

// ---- streaming-bandwidth probe ----------------------------------------------
// A plain device stream: dst[i] = sum of nin input buffers at i (16-byte loads
// and stores, four in flight per input, grid-stride over all SMs).  nin = 1 is
// a copy; nin = 6 reads six fields for one written, the mix of a stencil term
// (z, three weights, the diagonal, b in; one term out).  With every buffer far
// larger than the L2 it measures HBM; with all of them inside the L2 (the FP32
// chain of a 128^3 grid keeps its fields there) it measures the L2.

namespace {

constexpr int kStreamUnroll = 4;
constexpr int kStreamMaxIn = 8;

template <int NIN>
__global__ void stream_probe_kernel(const float4* __restrict__ src, float4* __restrict__ dst, long long n4) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (kStreamUnroll - 1) * stride < n4; i += kStreamUnroll * stride) {
        float4 v[kStreamUnroll];
#pragma unroll
        for (int u = 0; u < kStreamUnroll; ++u) v[u] = src[i + u * stride];
#pragma unroll
        for (int f = 1; f < NIN; ++f) {
#pragma unroll
            for (int u = 0; u < kStreamUnroll; ++u) {
                const float4 w = src[f * n4 + i + u * stride];
                v[u].x += w.x;
                v[u].y += w.y;
                v[u].z += w.z;
                v[u].w += w.w;
            }
        }
#pragma unroll
        for (int u = 0; u < kStreamUnroll; ++u) dst[i + u * stride] = v[u];
    }
    for (; i < n4; i += stride) {
        float4 v = src[i];
        for (int f = 1; f < NIN; ++f) {
            const float4 w = src[f * n4 + i];
            v.x += w.x;
            v.y += w.y;
            v.z += w.z;
            v.w += w.w;
        }
        dst[i] = v;
    }
}

template <int NIN>
void launch_stream(int blocks, int threads, cudaStream_t st, const float4* src, float4* dst, long long n4) {
    stream_probe_kernel<NIN><<<blocks, threads, 0, st>>>(src, dst, n4);
}

void launch_stream_n(int nin, int blocks, int threads, cudaStream_t st, const float4* src, float4* dst,
                     long long n4) {
    switch (nin) {
        case 1: launch_stream<1>(blocks, threads, st, src, dst, n4); break;
        case 2: launch_stream<2>(blocks, threads, st, src, dst, n4); break;
        case 3: launch_stream<3>(blocks, threads, st, src, dst, n4); break;
        case 4: launch_stream<4>(blocks, threads, st, src, dst, n4); break;
        case 5: launch_stream<5>(blocks, threads, st, src, dst, n4); break;
        case 6: launch_stream<6>(blocks, threads, st, src, dst, n4); break;
        case 7: launch_stream<7>(blocks, threads, st, src, dst, n4); break;
        default: launch_stream<8>(blocks, threads, st, src, dst, n4); break;
    }
}

}  // namespace

extern "C" ET_API et_status et_probe_stream(const void* src, void* dst, size_t bytes, int nin, int reps,
                                            void* cuda_stream, double* gbs) {
    if (!src || !dst || !gbs || reps < 1 || nin < 1 || nin > kStreamMaxIn || bytes < 16 || (bytes & 15u) ||
        ((uintptr_t)src & 15u) || ((uintptr_t)dst & 15u))
        return ET_ERR_ARG;
    const char* s = (const char*)src;
    char* d = (char*)dst;
    const size_t in_bytes = bytes * (size_t)nin;
    if (!(s + in_bytes <= d || d + bytes <= s)) return ET_ERR_ARG;  // the output must not overlap the inputs
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ET_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ET_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return ET_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return ET_ERR_CUDA;
    }
    const long long n4 = (long long)(bytes / 16);
    // launch shapes: threads per block x blocks per SM; the best one counts
    const int shapes[][2] = {{256, 4}, {256, 8}, {512, 4}, {1024, 2}};
    double best = 0.0;
    cudaError_t e = cudaSuccess;
    for (const auto& sh : shapes) {
        const int blocks = sms * sh[1];
        for (int w = 0; w < 3; ++w) launch_stream_n(nin, blocks, sh[0], st, (const float4*)src, (float4*)dst, n4);
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) launch_stream_n(nin, blocks, sh[0], st, (const float4*)src, (float4*)dst, n4);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        const double rate = (double)(nin + 1) * (double)bytes * reps / (ms * 1e-3) / 1e9;
        if (rate > best) best = rate;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return ET_ERR_CUDA;
    *gbs = best;
    return ET_OK;
}
