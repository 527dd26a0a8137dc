// Generic (runtime-size) instantiations, the size registry and the launcher.
#include "kernels.cuh"

namespace ofdft {

// size-specialised instantiations live in the inst_*.cu translation units
template <typename T> void candidates_a(int, int, std::vector<KernelCand> &);
template <typename T> void candidates_b(int, int, std::vector<KernelCand> &);
template <typename T> void candidates_c(int, int, std::vector<KernelCand> &);
template <typename T> void candidates_d(int, int, std::vector<KernelCand> &);

template <typename T> void kernel_candidates(int role, int n, std::vector<KernelCand> &out) {
    out.clear();
    if (role == ROLE_AXIS0) recip_candidates<T>(n, out);
    candidates_a<T>(role, n, out);
    candidates_b<T>(role, n, out);
    candidates_c<T>(role, n, out);
    candidates_d<T>(role, n, out);
}

template <typename T> bool find_specialised(int role, int n, const void **k1, const void **k2, int *B, int *nt) {
    std::vector<KernelCand> c;
    kernel_candidates<T>(role, n, c);
    for (const KernelCand &k : c)
        if (!k.recip.k) {
            *k1 = k.k1;
            *k2 = k.k2;
            *B = k.B;
            *nt = k.nt;
            return true;
        }
    return false;
}

template <typename T> LaunchSet generic_kernels(bool exact_sums) {
    LaunchSet ks;
    ks.row_fwd = (const void *)row_fwd_kernel<T, RtPolicy<T, 2>>;
    ks.pen_fwd = (const void *)pencil1_kernel<T, -1, RtPolicy<T, 1>>;
    ks.pen_inv = (const void *)pencil1_kernel<T, +1, RtPolicy<T, 1>>;
    if (!exact_sums) generic_group_kernels<T>(ks);
    if (exact_sums) {
        ks.row_inv = (const void *)row_inv_kernel<T, RtPolicy<T, 2>, true>;
        ks.axis0 = (const void *)axis0_kernel<T, RtPolicy<T, 0>, false, true>;
        ks.axis0_mgp = (const void *)axis0_kernel<T, RtPolicy<T, 0>, true, true>;
    } else {
        ks.row_inv = (const void *)row_inv_kernel<T, RtPolicy<T, 2>>;
        ks.axis0 = (const void *)axis0_kernel<T, RtPolicy<T, 0>, false>;
        ks.axis0_mgp = (const void *)axis0_kernel<T, RtPolicy<T, 0>, true>;
    }
    return ks;
}

cudaError_t prepare_kernels(const LaunchSet &ks) {
    const void *k[16] = {ks.row_fwd,   ks.row_inv,   ks.pen_fwd,   ks.pen_inv,   ks.axis0,     ks.axis0_mgp,
                         ks.recip.k,   ks.recip.k_mgp, ks.recip.g, ks.recip.g_mgp, ks.row_fwd_g, ks.row_inv_g,
                         ks.pen_fwd_g, ks.pen_inv_g, ks.axis0_g,   ks.axis0_mgp_g};
    for (int i = 0; i < 16; i++) {
        if (!k[i]) continue;
        cudaError_t e = allow_max_dynamic_smem(k[i]);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}


template <typename T>
static cudaError_t launch(const void *k, dim3 g, int nt, size_t smem, const EvalArgs<T> &a, cudaStream_t s) {
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(k, g, dim3(nt), args, smem, s);
}

template <typename T>
cudaError_t launch_eval(const EvalArgs<T> &a, const LaunchSet &ks, cudaStream_t s, const ProfHook *ph,
                        const RecipMaps *maps) {
    const long long R = (long long)a.n0 * a.n1;
    const long long pairs = (R + 1) / 2;
    const int nrt = (int)((pairs + a.Brow - 1) / a.Brow);
    cudaError_t e = cudaSuccess;
    auto mark = [&](int id, int phase) {
        if (ph) ph->record(ph->ctx, id, phase, s);
    };
    mark(K_STATS, 0);
    if (a.exact_sums) stats_kernel<T, true><<<a.nb_stats, 256, 0, s>>>(a);   // (its last block makes the knots)
    else stats_kernel<T><<<a.nb_stats, 256, 0, s>>>(a);
    mark(K_STATS, 1);
    if (a.nfwd > 0) {
        mark(K_ROW_FWD, 0);
        e = launch(ks.row_fwd, dim3(nrt), a.thr_rowf, rowf_smem<T>(a), a, s);
        if (e) return e;
        mark(K_ROW_FWD, 1);
    }
    if (a.ncol > 0) {
        mark(K_PENCIL_FWD, 0);
        e = launch(ks.pen_fwd, dim3(pencil_tiles(a, a.ncol)), a.thr_p1, pencil_smem_bytes<T>(a.n1, a.TW1), a, s);
        if (e) return e;
        mark(K_PENCIL_FWD, 1);
    }
    mark(K_AXIS0, 0);
    if (ks.recip.k && maps) {
        void *args[] = {(void *)&a, (void *)maps};
        e = cudaLaunchKernel(a.mgp_tab ? ks.recip.k_mgp : ks.recip.k, dim3(a.nb_ax0), dim3(ks.recip.nt), args,
                             ks.recip.smem, s);
    } else {
        e = launch(a.mgp_tab ? ks.axis0_mgp : ks.axis0, dim3(a.nb_ax0), a.thr_ax0,
                   axis0_smem_bytes<T>(a.n0, a.TW0, a.ax0_scr), a, s);
    }
    if (e) return e;
    mark(K_AXIS0, 1);
    if (a.ncol_inv > 0) {
        mark(K_PENCIL_INV, 0);
        e = launch(ks.pen_inv, dim3(pencil_tiles(a, a.ncol_inv)), a.thr_p1, pencil_smem_bytes<T>(a.n1, a.TW1),
                   a, s);
        if (e) return e;
        mark(K_PENCIL_INV, 1);
    }
    mark(K_ROW_INV, 0);
    e = launch(ks.row_inv, dim3(nrt), a.thr_rowi, rowi_smem<T>(a), a, s);
    if (e) return e;
    mark(K_ROW_INV, 1);
    mark(K_FINALIZE, 0);
    finalize_kernel<T><<<5, 256, 0, s>>>(a);
    mark(K_FINALIZE, 1);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_forward_rows_cols(const EvalArgs<T> &a, const LaunchSet &ks, cudaStream_t s) {
    const long long R = (long long)a.n0 * a.n1;
    const long long pairs = (R + 1) / 2;
    const int nrt = (int)((pairs + a.Brow - 1) / a.Brow);
    stats_kernel<T><<<a.nb_stats, 256, 0, s>>>(a);
    cudaError_t e = launch(ks.row_fwd, dim3(nrt), a.thr_rowf, rowf_smem<T>(a), a, s);
    if (e) return e;
    e = launch(ks.pen_fwd, dim3(pencil_tiles(a, a.ncol)), a.thr_p1, pencil_smem_bytes<T>(a.n1, a.TW1), a, s);
    if (e) return e;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_inverse_cols_rows(const EvalArgs<T> &a, const LaunchSet &ks, cudaStream_t s) {
    const long long R = (long long)a.n0 * a.n1;
    const long long pairs = (R + 1) / 2;
    const int nrt = (int)((pairs + a.Brow - 1) / a.Brow);
    cudaError_t e = launch(ks.pen_inv, dim3(pencil_tiles(a, a.ncol_inv)), a.thr_p1,
                           pencil_smem_bytes<T>(a.n1, a.TW1), a, s);
    if (e) return e;
    e = launch(ks.row_inv, dim3(nrt), a.thr_rowi, rowi_smem<T>(a), a, s);
    if (e) return e;
    return cudaGetLastError();
}

// ---------------------------------------------------------------- MGP correction table
// J_y(eta) = 2 int_0^1 r^p G_NL(eta / r^2) dr, p = 6y - 1 (the t-integral of Eq. MGP after
// t = r^6 and an integration by parts).  G_NL has a logarithmic kink at r = sqrt(eta); each
// piece between 0, the kink and 1 is split at its middle and each half is cut into panels
// shrinking geometrically (by halves) toward its outer end, 8-point Gauss-Legendre on each.
struct Gl8 {
    double x[8], w[8];
};
constexpr int kMgpGrade = 24;

__device__ __forceinline__ double mgp_panel(double a, double b, double eta, double p, const Gl8 &q) {
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const double r = c + h * q.x[k];
        s += q.w[k] * pow(r, p) * gnl<double>(eta / (r * r));
    }
    return 2.0 * h * s;
}
__device__ double mgp_graded(double a, double b, double eta, double p, const Gl8 &q) {
    const double m = 0.5 * (a + b);
    double s = mgp_panel(a, a + (m - a) * ldexp(1.0, -kMgpGrade), eta, p, q) +
               mgp_panel(b - (b - m) * ldexp(1.0, -kMgpGrade), b, eta, p, q);
    for (int j = 0; j < kMgpGrade; j++) {
        s += mgp_panel(a + (m - a) * ldexp(1.0, -(j + 1)), a + (m - a) * ldexp(1.0, -j), eta, p, q);
        s += mgp_panel(b - (b - m) * ldexp(1.0, -j), b - (b - m) * ldexp(1.0, -(j + 1)), eta, p, q);
    }
    return s;
}
template <typename T> __global__ void mgp_table_kernel(T *tab, int n, double y, Gl8 q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double p = 6.0 * y - 1.0;
    double J;
    if (i == 0) {
        J = 0.0;                                   // eta = 0: G_NL(0) = 0
    } else if (i == n - 1) {
        J = -8.0 / (15.0 * y);                     // eta -> infinity: G_NL -> -8/5
    } else {
        const double u = (double)i / (double)(n - 1), eta = u / (1.0 - u);
        if (eta < 1.0) {
            const double rk = sqrt(eta);
            J = mgp_graded(0.0, rk, eta, p, q) + mgp_graded(rk, 1.0, eta, p, q);
        } else {
            J = mgp_graded(0.0, 1.0, eta, p, q);
        }
    }
    tab[i] = (T)J;
}
template <typename T> cudaError_t launch_mgp_table(T *tab, int n, double y, const double *gl, cudaStream_t s) {
    Gl8 q;
    for (int k = 0; k < 8; k++) {
        q.x[k] = gl[k];
        q.w[k] = gl[8 + k];
    }
    mgp_table_kernel<T><<<(n + 127) / 128, 128, 0, s>>>(tab, n, y, q);
    return cudaGetLastError();
}

#define INST(T)                                                                                              \
    template cudaError_t launch_mgp_table<T>(T *, int, double, const double *, cudaStream_t);               \
    template bool find_specialised<T>(int, int, const void **, const void **, int *, int *);                 \
    template void kernel_candidates<T>(int, int, std::vector<KernelCand> &);                                 \
    template LaunchSet generic_kernels<T>(bool);                                                             \
    template cudaError_t launch_eval<T>(const EvalArgs<T> &, const LaunchSet &, cudaStream_t, const ProfHook *,   \
                                        const RecipMaps *);                                                  \
    template cudaError_t launch_forward_rows_cols<T>(const EvalArgs<T> &, const LaunchSet &, cudaStream_t); \
    template cudaError_t launch_inverse_cols_rows<T>(const EvalArgs<T> &, const LaunchSet &, cudaStream_t);
INST(float)
INST(double)

}  // namespace ofdft
