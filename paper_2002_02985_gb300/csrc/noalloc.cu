// Thomas-Fermi energy and potential without any device allocation.
//
// The regular entry points keep their reduction partials in a workspace that
// the library allocates with cudaMalloc on first use.  Some callers cannot let
// a library allocate: a host program whose own allocator owns all device
// memory (a pool it sized up front, or memory shared with another runtime),
// where an allocation behind its back can fail or fragment that pool, or code
// that must not pay for cudaMalloc's device-wide synchronisation.  For them this
// variant of the density reduction keeps its partials in a fixed file-scope
// device array.
//
// The array is a static __device__ symbol: every GPU that loads the library
// holds it until the process exits.  Host code must not pass the symbol itself
// to a kernel (on the host it is only a stand-in, not a device address): its
// device address is looked up once per device with cudaGetSymbolAddress and
// that pointer is passed instead.  The first call on a device does that
// look-up; make that first call before any stream capture.  All calls share
// the array and it keeps the last call's contents (the completion ticket is
// cleared on every call), so two calls that overlap on the GPU (different
// streams, no ordering between them) race on it.
//
// A density with NaN, Inf or negative values gives E = NaN: the regular entry
// point returns OFDFT_ERR_BAD_DENSITY instead, which this one cannot do without
// synchronising its stream.
#include <atomic>

#include "../../include/ofdft.h"
#include "common.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int kPerThread = 8;
constexpr int kPerBlock = kBlock * kPerThread;                 // points per block
constexpr int kMaxBlocks = OFDFT_NOALLOC_MAX_POINTS / kPerBlock; // 4096

// [0, kMaxBlocks): per-block partial sums of rho^(5/3); slot kMaxBlocks holds the
// completion ticket (an unsigned int in the first 4 bytes of that double).
static __device__ __align__(256) double noalloc_scratch[kMaxBlocks + 2];

// per-device address of the array (host threads may race on a first call: each one
// stores the same value, atomically)
constexpr int kMaxDevices = 64;
std::atomic<double *> g_scratch_ptr[kMaxDevices];

template <typename T>
__global__ void __launch_bounds__(kBlock)
tf_noalloc_kernel(const T *rho, long long n, double c_dV, T *V, double *E, double *scratch) {
    __shared__ double sd[32];
    __shared__ int last;
    const long long base = (long long)blockIdx.x * kPerBlock;
    double acc = 0.0;
    int bad = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; k++) {
        const long long i = base + (long long)k * kBlock + threadIdx.x;
        if (i < n) {
            const T x = rho[i];
            if (!(x >= (T)0) || x - x != (T)0) bad = 1;                // NaN, negative or Inf
            const T c = ofdft::dcbrt(x > (T)0 ? x : (T)0);
            acc += (double)(x * c * c);                               // rho^(5/3)
            if (V) V[i] = (T)(5.0 / 3.0 * ofdft::kCTF) * c * c;       // (5/3) C_TF rho^(2/3)
        }
    }
    // a bad value anywhere in the block makes its partial, hence E, NaN
    if (__syncthreads_or(bad)) acc = __longlong_as_double(0x7ff8000000000000LL);
    acc = ofdft::block_sum(acc, sd);
    unsigned int *ticket = (unsigned int *)(scratch + kMaxBlocks);
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = acc;
        __threadfence();
        last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    // the last block to finish sums the partials in block order (deterministic)
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kBlock) s += __ldcg(scratch + b);
    s = ofdft::block_sum(s, sd);
    if (threadIdx.x == 0) {
        *E = c_dV * s;
        *ticket = 0u;
    }
}

}  // namespace

extern "C" int ofdft_tf_energy_potential_noalloc(const void *rho_dev, long long n, double dV, int precision,
                                                 double *E_dev, void *V_dev, void *cuda_stream) {
    if (!rho_dev || !E_dev || n < 1 || !(dV > 0.0)) return OFDFT_ERR_INVALID_ARG;
    if (n > OFDFT_NOALLOC_MAX_POINTS) return OFDFT_ERR_INVALID_ARG;     // beyond the static scratch
    if (precision != OFDFT_FP64 && precision != OFDFT_FP32_MIXED) return OFDFT_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OFDFT_ERR_CUDA;
    double *scratch = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!scratch) {
        // once per device, with that device current: the device address of the array
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, noalloc_scratch) != cudaSuccess || !p) return OFDFT_ERR_CUDA;
        scratch = (double *)p;
        g_scratch_ptr[dev].store(scratch, std::memory_order_release);
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the completion ticket must start at zero
    if (cudaMemsetAsync(scratch + kMaxBlocks, 0, sizeof(double), s) != cudaSuccess) return OFDFT_ERR_CUDA;
    const unsigned blocks = (unsigned)((n + kPerBlock - 1) / kPerBlock);
    const double c_dV = ofdft::kCTF * dV;
    if (precision == OFDFT_FP64)
        tf_noalloc_kernel<double><<<blocks, kBlock, 0, s>>>((const double *)rho_dev, n, c_dV, (double *)V_dev,
                                                            E_dev, scratch);
    else
        tf_noalloc_kernel<float><<<blocks, kBlock, 0, s>>>((const float *)rho_dev, n, c_dV, (float *)V_dev,
                                                           E_dev, scratch);
    return cudaGetLastError() == cudaSuccess ? OFDFT_OK : OFDFT_ERR_CUDA;
}
