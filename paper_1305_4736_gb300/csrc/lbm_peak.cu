// lbm_peak.cu -- float64 FMA-chain kernel: the measured ALU peak that the
// float64 mode's roofline divides by.  Eight independent chains per thread,
// a grid of 8 blocks of 256 threads per SM, timed with CUDA events after a
// warm-up launch.  Each thread writes one result (bounds: grid * block).
#include "lbm_internal.h"

namespace lbm {

constexpr int kPeakIters = 4096;

__global__ void __launch_bounds__(256) k_fma_chain(double *out, double a, double b)
{
    double x0 = threadIdx.x * 1e-9, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < kPeakIters; i++) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

cudaError_t measure_fp64_fma(double *flops)
{
    int dev = 0, sms = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) return ce;
    const int grid = sms * 8, block = 256, reps = 5;
    double *buf = nullptr;
    ce = cudaMalloc(&buf, sizeof(double) * grid * block);
    if (ce != cudaSuccess) return ce;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_chain<<<grid, block>>>(buf, 0.999999, 1e-7);
    cudaEventRecord(e0);
    for (int r = 0; r < reps; r++) k_fma_chain<<<grid, block>>>(buf, 0.999999, 1e-7);
    cudaEventRecord(e1);
    ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (ce == cudaSuccess) ce = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (ce != cudaSuccess) return ce;
    *flops = 2.0 * 8.0 * kPeakIters * (double)grid * block * reps / (ms * 1e-3);
    return cudaSuccess;
}

}  // namespace lbm
