// FP64 fused multiply-add throughput of the current device (a diagnostic for the FP64
// evaluation path's roofline: every kernel of that path does its arithmetic in FP64).
#include "../../include/ofdft.h"
#include "common.cuh"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread
constexpr int kIter = 4096;     // FMAs per chain

__global__ void __launch_bounds__(256) fp64_fma_kernel(double b, double c, double *out) {
    double acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) acc[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < kIter; i++)
#pragma unroll
        for (int k = 0; k < kChains; k++) acc[k] = fma(acc[k], b, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += acc[k];
    if (s == 12345.678) *out = s;          // never true: keeps the chains alive
}

}  // namespace

extern "C" int ofdft_fp64_fma_rate(void *cuda_stream, double *gflops) {
    if (!gflops) return OFDFT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return OFDFT_ERR_CUDA;
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return OFDFT_ERR_OOM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = OFDFT_OK;
    const dim3 grid(nsm * 8), block(256);
    const int reps = 3;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = OFDFT_ERR_CUDA;
    if (rc == OFDFT_OK) {
        fp64_fma_kernel<<<grid, block, 0, s>>>(0.999999, 1e-7, out);        // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; r++) fp64_fma_kernel<<<grid, block, 0, s>>>(0.999999, 1e-7, out);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
            rc = OFDFT_ERR_CUDA;
        else
            *gflops = 2.0 * kChains * (double)kIter * grid.x * block.x * reps / (ms * 1e-3) / 1e9;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}
