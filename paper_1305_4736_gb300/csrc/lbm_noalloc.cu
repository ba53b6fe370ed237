// lbm_noalloc.cu -- conserved totals of a population field with no device allocation.
//
// For callers that cannot allocate device memory: their device memory is owned
// by another allocator (a framework's caching pool, a serving engine with a
// fixed memory plan), or they must not call cudaMalloc / cudaFree, which can
// synchronise the whole device and stall other work.  The reduction's scratch
// (one partial per grid row plus the result) lives in a file-scope device
// array, so every GPU that loads this library holds it until the process exits.
//
// The first call on a device looks up the array's device address on that
// device (cudaGetSymbolAddress, with the device current); make that first call
// before any stream capture.  The address is kept for the life of the process:
// after a cudaDeviceReset of that device it is no longer valid, so the entry
// point must not be called on a device that was reset.  All calls share the array and each call
// overwrites the rows it uses and the result slot, so nothing needs clearing;
// calls whose work overlaps on the GPU (different streams, or different host
// threads on one device) race on it and must be serialised by the caller.
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace {

constexpr int kRows = LBM_TOTALS_NOALLOC_MAX_ROWS;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// [kRows][4] row partials followed by the 4 results.
static __device__ __align__(256) double g_totals_scratch[(kRows + 1) * 4];

std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {};

__device__ __forceinline__ double block_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int j = 0; j < kThreads / 32; j++) s += red[j];
    return s;
}

// One block per row (grid-stride over rows): rho, j_x, j_y, e of the row in a fixed order.
__global__ void __launch_bounds__(kThreads) k_rows(const double *__restrict__ f, int nx, int ny, double *scratch)
{
    __shared__ double red[kThreads / 32];
    const long long plane = (long long)nx * ny;
    for (int y = blockIdx.x; y < ny; y += gridDim.x) {
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        for (int x = threadIdx.x; x < nx; x += kThreads) {
            double g[lbm::NQ];
            const long long c = (long long)y * nx + x;
#pragma unroll
            for (int q = 0; q < lbm::NQ; q++) g[q] = f[q * plane + c];
            const lbm::Shells<double> s = lbm::shells_of(g);
            double rho, jx, jy, e;
            lbm::conserved_of(s, rho, jx, jy, e);
            a[0] += rho;
            a[1] += jx;
            a[2] += jy;
            a[3] += e;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const double t = block_sum(a[k], red);
            if (threadIdx.x == 0) scratch[4 * y + k] = t;
        }
    }
}

// One block: the row partials in a fixed order, times the cell area dx dy, into the result slot.
__global__ void __launch_bounds__(kThreads) k_final(int ny, double scale, double *scratch)
{
    __shared__ double red[kThreads / 32];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int y = threadIdx.x; y < ny; y += kThreads)
#pragma unroll
        for (int k = 0; k < 4; k++) a[k] += scratch[4 * y + k];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const double t = block_sum(a[k], red);
        if (threadIdx.x == 0) scratch[4 * kRows + k] = t * scale;
    }
}

}  // namespace

extern "C" int lbm_totals_noalloc(const double *f, int nx, int ny, double dx, double dy, void *stream,
                                  double out[4])
{
    if (!f || !out) return LBM_ERR_ARG;
    if (nx < 1 || ny < 1 || !(dx > 0.0) || !(dy > 0.0)) return LBM_ERR_ARG;
    if (ny > kRows) return LBM_ERR_ARG;   // the row partials are sized for LBM_TOTALS_NOALLOC_MAX_ROWS rows
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ERR_CUDA;
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_totals_scratch) != cudaSuccess || !p) return LBM_ERR_CUDA;
            g_scratch_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = ny < 1024 ? ny : 1024;
    k_rows<<<grid, kThreads, 0, st>>>(f, nx, ny, scratch);
    k_final<<<1, kThreads, 0, st>>>(ny, dx * dy, scratch);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaMemcpyAsync(out, scratch + 4 * kRows, 4 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LBM_ERR_CUDA;
    return LBM_OK;
}
