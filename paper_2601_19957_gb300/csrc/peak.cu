// peak.cu -- FP64 FMA throughput of the GPU the library runs on, for the
// roofline of the FP64 kernels (the FP64 units, not memory, bound the Newton
// polish, the Hessian and its Cholesky factor, and the plain FP64 path).
//
// Every thread runs kChains independent FMA chains x <- x * m + c (no
// dependence between chains, so the FP64 pipe, not the FMA latency, limits the
// rate); the grid puts kBlocksPerSM CTAs on every SM. Each FMA is two flops.
#include "sb_internal.cuh"

namespace sb {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;
constexpr int kIters = 8192;

__device__ double g_fma_sink;

__global__ void __launch_bounds__(kThreads) k_fma_loop(int iters, double m, double c) {
    double x[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = 1.0 + 1e-3 * q + 1e-9 * threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) x[q] = fma(x[q], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += x[q];
    if (s == -1.0) g_fma_sink = s;  // never true; keeps the chains live
}

}  // namespace
}  // namespace sb

extern "C" double sb_fp64_fma_peak(void *stream) {
    using namespace sb;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return -1.0;
    const int grid = sms * kBlocksPerSM;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.0;
    }
    float best = -1.f;
    for (int rep = 0; rep < 6; ++rep) {
        cudaEventRecord(e0, s);
        note_launch();
        k_fma_loop<<<grid, kThreads, 0, s>>>(kIters, 0.9999999, 1e-7);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best < 0.f || ms < best)) best = ms;  // the first launch warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best <= 0.f || cudaGetLastError() != cudaSuccess) return -1.0;
    const double flop = 2.0 * kChains * (double)kIters * (double)grid * kThreads;
    return flop / (best * 1e-3) / 1e12;
}
