// Arithmetic-throughput probe: sustained fused multiply-add rate of the plain
// (non-tensor) FP64 or FP32 pipes of the device, used as the roofline peak of
// kernels bound by ordinary arithmetic.  Every thread runs independent FMA
// chains long enough to hide latency; one launch fills every SM.
#include <cuda_runtime.h>

#include "vof_internal.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T *out, int iters, T a, T b)
{
    T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)12345.678) out[0] = s;  // keeps the chains alive
}

template <typename T>
int run_probe(int device, double *flops, cudaStream_t s, int iters)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return VOF_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int blocks = sms * 8, threads = 256;
    k_fma_probe<T><<<blocks, threads, 0, s>>>(out, 4, (T)0.999, (T)1e-3);  // warm-up
    cudaEventRecord(e0, s);
    k_fma_probe<T><<<blocks, threads, 0, s>>>(out, iters, (T)0.999, (T)1e-3);
    cudaEventRecord(e1, s);
    int rc = VOF_OK;
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = VOF_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *flops = 2.0 * 8.0 * 16.0 * (double)iters * blocks * threads / (ms * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}

}  // namespace

extern "C" int vof_probe_fma(int device, int precision, double *flops_per_s, void *stream)
{
    if (!flops_per_s || (precision != VOF_FP64 && precision != VOF_MIXED)) return VOF_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return VOF_ERR_NO_DEVICE;
    cudaStream_t s = (cudaStream_t)stream;
    return precision == VOF_FP64 ? run_probe<double>(device, flops_per_s, s, 256)
                                 : run_probe<float>(device, flops_per_s, s, 4096);
}
