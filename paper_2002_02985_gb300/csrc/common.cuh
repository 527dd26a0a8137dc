// Shared device/host definitions of the OFDFT CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define OFDFT_MAX_KNOTS 64
#define OFDFT_MAX_PASS 12

namespace ofdft {

// Allow a kernel the largest dynamic shared memory the device permits next to
// its own static shared memory.
template <typename K> inline cudaError_t allow_max_dynamic_smem(K kernel) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

// --------------------------------------------------------------- physical constants
// C_TF = (3/10)(3 pi^2)^(2/3) and C_WT = (6/25)(3 pi^2)^(2/3) (Sec. 2.3, Eq. WT).
constexpr double kPi = 3.14159265358979323846;
constexpr double kThreePi2 = 29.608813203268074;     // 3 pi^2
constexpr double kCbrtThreePi2 = 3.0936677262801355;  // (3 pi^2)^(1/3)
constexpr double kCTF = 2.871234000188191;           // 0.3 (3 pi^2)^(2/3)
constexpr double kCWT = 2.2969872001505527;          // 0.24 (3 pi^2)^(2/3)

// --------------------------------------------------------------- bulk (TMA) copies
// One-dimensional bulk copies between global and shared memory done by the
// tensor memory accelerator: both addresses 16-byte aligned, size a multiple of
// 16 bytes (callers check this and fall back to element copies otherwise).
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make generic-proxy shared-memory writes (and the barrier init) visible to the async proxy
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// true once the phase with the given parity has completed (the hardware may suspend
// the thread for a bounded time inside one call)
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false if the phase did not complete within `limit` polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, unsigned limit) {
    for (unsigned i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *smem_dst, const void *gmem_src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_s2g(void *gmem_dst, const void *smem_src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gmem_dst),
                 "r"(smem_u32(smem_src)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// wait until the committed bulk stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// wait until the committed bulk stores are complete (visible in global memory)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// --------------------------------------------------------------- async copies
// Asynchronous global -> shared copies (one 8- or 16-byte element per call).
// src_bytes = 0 fills the destination with zeros (used for ragged tiles).
template <int BYTES> __device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    const int n = valid ? BYTES : 0;
    if (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem_src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem_src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// --------------------------------------------------------------- complex helpers
template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };

template <typename C> __host__ __device__ __forceinline__ C cmake(decltype(C::x) a, decltype(C::x) b) {
    C c; c.x = a; c.y = b; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmake<C>(a.x * s, a.y * s); }
// FP32 complex values: both components in one packed two-wide FP32 instruction (sm_100 and
// later); each component is rounded exactly as the scalar operation rounds it (a - b is
// fma(b, -1, a), a single rounding of the exact difference)
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
template <> __device__ __forceinline__ float2 cscale<float2>(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
// multiply by (s i) with s = -1 (forward) or +1 (inverse)
template <int DIR, typename C> __device__ __forceinline__ C cmul_si(C a) {
    return DIR < 0 ? cmake<C>(a.y, -a.x) : cmake<C>(-a.y, a.x);
}

// --------------------------------------------------------------- math wrappers
// four consecutive values from a 16-byte (float) / 32-byte (double) aligned address
__device__ __forceinline__ void load4(const float *p, float v[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double *p, double v[4]) {
    const double2 q0 = reinterpret_cast<const double2 *>(p)[0], q1 = reinterpret_cast<const double2 *>(p)[1];
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dcbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ double dcbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float dpow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double dpow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float dlog(float x) { return logf(x); }
__device__ __forceinline__ double dlog(double x) { return log(x); }
__device__ __forceinline__ float dabs(float x) { return fabsf(x); }
__device__ __forceinline__ double dabs(double x) { return fabs(x); }

// --------------------------------------------------------------- reductions
// Deterministic block sum of a double: warp shuffles, then warp 0 over the
// per-warp partials.  Every thread of the block must call it; result valid in
// thread 0.  scratch: >= 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
    if (warp == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// K sums at once (same shuffle tree per value as block_sum, one pair of barriers for
// all): the totals are valid in thread 0.  scratch: 32 K doubles.
template <int K> __device__ __forceinline__ void block_sum_n(double (&v)[K], double *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < K; k++) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) scratch[k * 32 + warp] = v[k];
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = (threadIdx.x < nw) ? scratch[k * 32 + threadIdx.x] : 0.0;
    if (warp == 0)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < K; k++) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
}

// K sums where the per-thread values need only FP32 within a warp (the FP32-mixed
// path): warp sums in FP32, the warps' sums in FP64 by thread 0 (GB300 does two FP64
// operations per clock per SM, so FP64 shuffle trees dominate small kernels).  The
// totals are valid in thread 0.  scratch: 32 K doubles.
template <int K> __device__ __forceinline__ void block_sum_n_f32warp(double (&v)[K], double *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float f[K];
#pragma unroll
    for (int k = 0; k < K; k++) f[k] = (float)v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < K; k++) f[k] += __shfl_down_sync(0xffffffffu, f[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) scratch[k * 32 + warp] = (double)f[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int k = 0; k < K; k++) {
            double t = 0.0;
            for (int w = 0; w < nw; w++) t += scratch[k * 32 + w];
            v[k] = t;
        }
    }
}

template <typename T> __device__ __forceinline__ T block_min(T v, T *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) { T w = __shfl_down_sync(0xffffffffu, v, o); v = w < v ? w : v; }
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? scratch[threadIdx.x] : scratch[0];
    if (warp == 0)
        for (int o = 16; o > 0; o >>= 1) { T w = __shfl_down_sync(0xffffffffu, v, o); v = w < v ? w : v; }
    return v;
}
template <typename T> __device__ __forceinline__ T block_max(T v, T *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) { T w = __shfl_down_sync(0xffffffffu, v, o); v = w > v ? w : v; }
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? scratch[threadIdx.x] : scratch[0];
    if (warp == 0)
        for (int o = 16; o > 0; o >>= 1) { T w = __shfl_down_sync(0xffffffffu, v, o); v = w > v ? w : v; }
    return v;
}

}  // namespace ofdft
