// Grouped launches of a batch: one launch per pass over the evaluations of the snapshots
// that share a launch geometry (same grid shape, same compiled kernels and tiles).  Each
// evaluation keeps the blocks, partial sums and reduction order of its single launch.
#include "recip.cuh"

namespace ofdft {

template <typename T> void generic_group_kernels(LaunchSet &ks) {
    ks.row_fwd_g = (const void *)row_fwd_group<T, RtPolicy<T, 2>>;
    ks.row_inv_g = (const void *)row_inv_group<T, RtPolicy<T, 2>>;
    ks.pen_fwd_g = (const void *)pencil1_group<T, -1, RtPolicy<T, 1>>;
    ks.pen_inv_g = (const void *)pencil1_group<T, +1, RtPolicy<T, 1>>;
    ks.axis0_g = (const void *)axis0_group<T, RtPolicy<T, 0>, false>;
    ks.axis0_mgp_g = (const void *)axis0_group<T, RtPolicy<T, 0>, true>;
}

template <typename T> bool grouped_ok(const LaunchSet &ks, const EvalArgs<T> &a) {
    if (a.exact_sums) return false;
    if (a.nfwd > 0 && !ks.row_fwd_g) return false;
    if ((a.ncol > 0 && !ks.pen_fwd_g) || (a.ncol_inv > 0 && !ks.pen_inv_g) || !ks.row_inv_g) return false;
    if (ks.recip.k) return (a.mgp_tab ? ks.recip.g_mgp : ks.recip.g) != nullptr;
    return (a.mgp_tab ? ks.axis0_mgp_g : ks.axis0_g) != nullptr;
}

// Clears the per-evaluation flags (bad density, the WT kF, the device-wait counters): the
// grouped form of the single evaluation's flag memset.
template <typename T> __global__ void group_clear_kernel(const EvalArgs<T> *__restrict__ ga, int K) {
    const int k = threadIdx.x >> 2, i = threadIdx.x & 3;
    if (k < K) ga[k].scal[S_BAD + i] = 0.0;
}

template <typename T>
cudaError_t launch_group(const EvalArgs<T> &a, const EvalArgs<T> *ga, int K, const LaunchSet &ks, cudaStream_t s,
                         const RecipMaps *maps) {
    if (K < 1 || K > kGroupMax || !grouped_ok(ks, a)) return cudaErrorInvalidValue;
    const long long R = (long long)a.n0 * a.n1;
    const int nrt = (int)(((R + 1) / 2 + a.Brow - 1) / a.Brow);
    auto launch = [&](const void *k, int bps, int nt, size_t smem) {
        void *args[] = {(void *)&ga, (void *)&bps};
        return cudaLaunchKernel(k, dim3((unsigned)(K * bps)), dim3(nt), args, smem, s);
    };
    group_clear_kernel<T><<<1, 4 * kGroupMax, 0, s>>>(ga, K);
    stats_group<T><<<K * a.nb_stats, 256, 0, s>>>(ga, a.nb_stats);   // (each evaluation's last block: knots)
    cudaError_t e = cudaSuccess;
    if (a.nfwd > 0 && (e = launch(ks.row_fwd_g, nrt, a.thr_rowf, rowf_smem<T>(a)))) return e;
    if (a.ncol > 0 &&
        (e = launch(ks.pen_fwd_g, (int)pencil_tiles(a, a.ncol), a.thr_p1, pencil_smem_bytes<T>(a.n1, a.TW1))))
        return e;
    if (ks.recip.k) {
        if (!maps) return cudaErrorInvalidValue;
        RecipMapsGroup mg;
        for (int k = 0; k < K; k++) mg.m[k] = maps[k];
        int bps = a.nb_ax0;
        void *args[] = {(void *)&ga, (void *)&bps, (void *)&mg};
        e = cudaLaunchKernel(a.mgp_tab ? ks.recip.g_mgp : ks.recip.g, dim3((unsigned)(K * bps)), dim3(ks.recip.nt),
                             args, ks.recip.smem, s);
    } else {
        e = launch(a.mgp_tab ? ks.axis0_mgp_g : ks.axis0_g, a.nb_ax0, a.thr_ax0,
                   axis0_smem_bytes<T>(a.n0, a.TW0, a.ax0_scr));
    }
    if (e) return e;
    if (a.ncol_inv > 0 &&
        (e = launch(ks.pen_inv_g, (int)pencil_tiles(a, a.ncol_inv), a.thr_p1, pencil_smem_bytes<T>(a.n1, a.TW1))))
        return e;
    if ((e = launch(ks.row_inv_g, nrt, a.thr_rowi, rowi_smem<T>(a)))) return e;
    finalize_group<T><<<K * 5, 256, 0, s>>>(ga, 5);
    return cudaGetLastError();
}

// Gathers the energies and the scalar slots of evaluations ga[0..n) into out[k (E_NUM + S_NSCAL) ...]
// (one copy to the host for a whole batch).
template <typename T> __global__ void collect_kernel(const EvalArgs<T> *__restrict__ ga, int n, double *out) {
    constexpr int W = E_NUM + S_NSCAL;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * W; i += gridDim.x * blockDim.x) {
        const int k = i / W, j = i - k * W;
        out[i] = j < E_NUM ? __ldcg(ga[k].energies + j) : __ldcg(ga[k].scal + (j - E_NUM));
    }
}
template <typename T> cudaError_t launch_collect(const EvalArgs<T> *ga, int n, double *out, cudaStream_t s) {
    const int W = E_NUM + S_NSCAL;
    collect_kernel<T><<<(n * W + 255) / 256, 256, 0, s>>>(ga, n, out);
    return cudaGetLastError();
}

#define INST(T)                                                                                                  \
    template void generic_group_kernels<T>(LaunchSet &);                                                       \
    template bool grouped_ok<T>(const LaunchSet &, const EvalArgs<T> &);                                        \
    template cudaError_t launch_group<T>(const EvalArgs<T> &, const EvalArgs<T> *, int, const LaunchSet &,      \
                                         cudaStream_t, const RecipMaps *);                                      \
    template cudaError_t launch_collect<T>(const EvalArgs<T> *, int, double *, cudaStream_t);
INST(float)
INST(double)

}  // namespace ofdft
