// FP64 fused multiply-add throughput of the CUDA cores (measurement probe).
//
// Every thread runs CHAINS independent FMA chains x <- x * a + b for `iters`
// iterations (a slightly below 1 and b small keep x bounded), so the FP64 pipe,
// not the dependency latency, sets the rate.  The grid is a multiple of the SM
// count.  The result is written to out so the compiler keeps the work.
#include <cuda_runtime.h>

namespace {

constexpr int CHAINS = 8;

__global__ void __launch_bounds__(256) dfma_kernel(double a, double b, int iters, double *out)
{
    double x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// Measures the FP64 FMA rate of `device` over about `seconds` of work and writes
// it (TFLOP/s, 2 flops per FMA) to *tflops.  `scratch` must hold blocks_per_sm x
// SMs x 256 doubles of device memory (the caller's).  Returns 0 or a CUDA error code.
extern "C" int probe_dfma_tflops(int device, int blocks_per_sm, double seconds, double *scratch, double *tflops)
{
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return (int)e;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return (int)e;
    const int grid = sms * blocks_per_sm;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int iters = 1 << 14;
    double best = 0.0;
    for (int rep = 0; rep < 8; ++rep) {
        cudaEventRecord(e0);
        dfma_kernel<<<grid, 256>>>(0.999999, 1e-6, iters, scratch);
        cudaEventRecord(e1);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * CHAINS * (double)iters * grid * 256.0;
        const double rate = flops / (ms * 1e-3) / 1e12;
        if (rate > best) best = rate;
        // grow the launch until one takes about seconds / 4
        if (ms < 250.0 * seconds && iters < (1 << 26)) iters *= 2;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    *tflops = best;
    return (int)e;
}
