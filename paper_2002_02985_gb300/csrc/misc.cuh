// Per-geometry kernels (structure factor, forces) and optimiser vector kernels.
#pragma once

#include "fft.cuh"

namespace ofdft {

// V_ext(G) = (1/Omega) sum_s v_s(|G|) S_s(G), S_s(G) = sum_{I in s} e^{-iG.R_I}
// (with charge_ff: S_Z(G) = sum_s Z_s S_s(G) instead, for the ion-ion Ewald sum)
// with the phase of each ion factorised per axis: e^{-iG.R} = P0[k0] P1[k1] P2[k2],
// P_a[k] = e^{-2 pi i m_a(k) f_a} (f = fractional coordinates).  FP64 throughout.
struct IonArgs {
    int n0, n1, n2, n2h, n_ions, n_species;
    double omega;
    double bvec[9];                  // 2 pi b_i
    const double2 *ph0, *ph1, *ph2;  // [n_ions][n0], [n_ions][n1], [n_ions][n2h]
    const int *species;              // [n_ions]
    const double *Z, *rc;            // [n_species]
    int charge_ff = 0;               // 1: form factor Z_s instead of v_s (Ewald: S_Z(G) and its forces)
};

// vext64 != null: FP64 build; otherwise the FP32 copy from FP32 phase products
// (ph32 = FP32 copy of the phase tables) with FP64 accumulation of 8-ion groups
cudaError_t launch_vext(const IonArgs &a, double2 *vext64, float2 *vext32, cudaStream_t s,
                        const float2 *ph32 = nullptr);
cudaError_t launch_round_phases(const double2 *in, float2 *out, long long n, cudaStream_t s);
// FP32-mixed forces (separable form): gf = the per-species tables of launch_force_tables
// ([n_species][NH] floats: -w v_s(|G|)); sp_ions = the ions grouped by species, sp_off (HOST)
// the groups' offsets; partials [n_ions][nrb][3] (the S_a sums per row-tile block), then
// launch_reduce_force_sep assembles F_I = sum_a b_a S_a(I)
cudaError_t launch_force_tables(const IonArgs &a, float *gf, cudaStream_t st);
int forces_sep_blocks(const IonArgs &a, int nsm);
cudaError_t launch_forces_sep(const IonArgs &a, const float2 *rhohat, const float2 *ph32, const float *gf,
                              const int *sp_ions, const int *sp_off, int nrb, double *partials, cudaStream_t st);
cudaError_t launch_reduce_force_sep(const IonArgs &a, const double *part, int nrb, double *F, cudaStream_t s);

// forces from the normalised half spectrum rho_hat (FP64 or FP32 complex)
template <typename C>
cudaError_t launch_forces(const IonArgs &a, const C *rhohat, double *partials, int nchunk, cudaStream_t s);

// F = the partials [n_ions][nchunk][3] summed over the chunks in order
cudaError_t launch_reduce_force_partials(const double *part, int n_ions, int nchunk, double *F, cudaStream_t s);

// plain forward FFT along n0 of a half spectrum (in place), used by forces
template <typename T>
cudaError_t launch_axis0_fft(typename Vec2<T>::type *data, int n0, long long P, const FFTPlan &p,
                             const typename Vec2<T>::type *tw, int TW, int thr, double scale, cudaStream_t s,
                             int dir = -1);

// ---- optimiser vector kernels (all reductions FP64, fixed order) ----------
// out[slot] = sum_i a_i b_i (c_i if c != null)
// (exact: every FP32 product converted and summed in FP64, for tests of the default grouping)
template <typename T>
cudaError_t launch_dot(const T *a, const T *b, const T *c, long long N, double *partials, int nblk,
                       double *out, cudaStream_t s, bool exact = false);
// y = alpha * x + beta * y (scalars read from device double pointers when given)
template <typename T>
cudaError_t launch_axpby(T *y, const T *x, double alpha, double beta, long long N, cudaStream_t s);
// psi_l = psi cos(l) + p sin(l);  rho = psi_l^2
template <typename T>
cudaError_t launch_rotate(T *psi_l, T *rho, const T *psi, const T *p, double c, double sn, long long N,
                          cudaStream_t s);
// g = 2 psi (V - mu) dV
template <typename T>
cudaError_t launch_grad(T *g, const T *psi, const T *V, double mu, double dV, long long N, cudaStream_t s);
// rho = psi^2 (and optional scale of psi)
template <typename T>
cudaError_t launch_square(T *rho, T *psi, double scale, long long N, cudaStream_t s);
// d = -g + beta d ; dot partial <d, g> computed by launch_dot afterwards
template <typename T> cudaError_t launch_copy(T *dst, const T *src, long long N, cudaStream_t s);
// Fourier interpolation between two grids of one cell on normalised half spectra (layouts
// [k0][k1][k2], k2 <= n2/2): frequencies present on both grids are copied; a Nyquist term
// of the smaller grid is shared between +-n/2 of the larger (up) or made of both (down).
template <typename C>
cudaError_t launch_spectral_map(const C *src, int f0, int f1, int f2, C *dst, int t0, int t1, int t2,
                                cudaStream_t s);
// Hq = 2 dV (q (Vq - mu) + psi (Vq - V) / e): the Hessian of E[psi^2] - mu int psi^2 applied
// to q by a forward difference, Vq = V[(psi + e q)^2]
template <typename T>
cudaError_t launch_hvp(T *Hq, const T *psi, const T *q, const T *V, const T *Vq, double e, double mu, double dV,
                       long long N, cudaStream_t s);
// ---- real-time TD-OFDFT
struct TdCell {
    double a[9];      // lattice vectors (rows), bohr
};
// h(G) *= G^2/2 (mode 0) or 1 / (1 + tau^2 (G^2/2 + vbar)^2) (mode 1), normalised half spectrum
template <typename C>
cudaError_t launch_spectral_factor(C *h, int n0, int n1, int n2, const double *bvec, int mode, double tau, double vbar,
                                   cudaStream_t s);
// out = a out + b v u
template <typename T>
cudaError_t launch_add_vu(T *out, const T *v, const T *u, double a, double b, long long N, cudaStream_t s);
// rho = re^2 + im^2
template <typename T> cudaError_t launch_abs2(T *rho, const T *re, const T *im, long long N, cudaStream_t s);
// x += f c[0]
template <typename T>
cudaError_t launch_add_scaled_scalar(T *x, const double *c, double f, long long N, cudaStream_t s);
// psi <- psi exp(i k . r), r = A^T (f - 1/2) the cell-centred position
template <typename T>
cudaError_t launch_kick(T *re, T *im, int n0, int n1, int n2, const TdCell &c, const double *k, cudaStream_t s);
// out[0..2] = sum_r r (|psi|^2 - rho0) dV (rho0 may be NULL); part holds 3 nblk partials
template <typename T>
cudaError_t launch_dipole(const T *re, const T *im, const T *rho0, int n0, int n1, int n2, const TdCell &c, double dV,
                          double *part, int nblk, double *out, cudaStream_t s);
// x += c[0] (c a device scalar)
template <typename T> cudaError_t launch_add_scalar(T *x, const double *c, long long N, cudaStream_t s);
// optimiser preconditioner on a normalised half spectrum: h(G) *= a G^2 / (G^4 + a G^2 + b), h(0) kept
template <typename C>
cudaError_t launch_precond(C *h, int n0, int n1, int n2, const double *bvec, double a, double b, cudaStream_t s);

}  // namespace ofdft
