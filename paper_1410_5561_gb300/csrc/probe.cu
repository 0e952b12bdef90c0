// Vector FMA throughput probe: the FP32 / FP64 ALU peak the roofline divides by.
//
// Every thread runs 8 independent dependent-FMA chains (enough instruction-level
// parallelism to keep the pipe busy) for `iters` iterations; the grid fills
// every SM several times over. The result is written out so the chains are not
// removed by the compiler. Not an operation of the paper: measurement support.
#include "../../include/stencil_gb300.h"
#include "internal.h"

namespace stg {

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            x0 = Ar<T>::fma(x0, a, b);
            x1 = Ar<T>::fma(x1, a, b);
            x2 = Ar<T>::fma(x2, a, b);
            x3 = Ar<T>::fma(x3, a, b);
            x4 = Ar<T>::fma(x4, a, b);
            x5 = Ar<T>::fma(x5, a, b);
            x6 = Ar<T>::fma(x6, a, b);
            x7 = Ar<T>::fma(x7, a, b);
        }
    }
    T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == (T)-12345.0) out[blockIdx.x] = s;  // practically never taken
}

}  // namespace stg

extern "C" int stencil_probe_fma(int dtype, int iters, void* scratch, void* cuda_stream, double* seconds,
                                 double* flops) {
    using namespace stg;
    if (!scratch || !seconds || !flops || iters < 1) return STENCIL_EINVAL;
    if (dtype != STENCIL_F32 && dtype != STENCIL_F64) return STENCIL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return STENCIL_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return STENCIL_ECUDA;
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return STENCIL_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return STENCIL_ECUDA;
    }
    // warm-up launch, then the timed one
    for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1) cudaEventRecord(e0, s);
        if (dtype == STENCIL_F32)
            fma_probe_kernel<float><<<blocks, threads, 0, s>>>((float*)scratch, iters, 0.999f, 1e-3f);
        else
            fma_probe_kernel<double><<<blocks, threads, 0, s>>>((double*)scratch, iters, 0.999, 1e-3);
    }
    cudaEventRecord(e1, s);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return STENCIL_ECUDA;
    *seconds = ms * 1e-3;
    *flops = 2.0 * 8.0 * 16.0 * (double)iters * (double)blocks * (double)threads;
    return STENCIL_OK;
}
