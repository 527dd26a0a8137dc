// Smooth particle-mesh Ewald structure factor and forces (see pme.cu).
#pragma once

#include "common.cuh"

namespace ofdft {

constexpr int kPmeMaxOrder = 16;

struct PmeArgs {
    int n0, n1, n2, n2h, n_ions, p, s;   // grid, ion count, B-spline order, species filter
    double recip[9];                     // rows b_a (a_i . b_j = delta_ij), no 2 pi
    const double *pos;                   // device [n_ions][3]
    const int *species;                  // device [n_ions]
    int charge_ff = 0;                   // 1: form factor Z_s instead of v_s (Ewald sum)
};

// Q (fixed point, scale 2^40) += B-spline stencils of the ions of species a.s
cudaError_t pme_spread(const PmeArgs &a, unsigned long long *Q, cudaStream_t s);
// out = Q * 2^-40 in T; Q is zeroed for the next species
template <typename T> cudaError_t pme_fixed_to_real(unsigned long long *Q, T *out, long long N, cudaStream_t s);
// vext (+)= (1/Omega) v_s(|G|) S_s(G) from the normalised transform qhat of the charge grid;
// B = [conj b_0 (n0) | conj b_1 (n1) | conj b_2 (n2/2+1)]
template <typename C>
cudaError_t pme_vext(const PmeArgs &a, const C *qhat, const double2 *B, double Z, double rc, double count, double N,
                     double omega, C *vext, int first, cudaStream_t s);
// field = rho_hat conj(prod conj b) v_s (G != 0)
template <typename C>
cudaError_t pme_force_field(const PmeArgs &a, const C *rhohat, const double2 *B, double Z, double rc, C *field,
                            cudaStream_t s);
// F[I] = -dE/dR_I for the ions of species a.s from phi = inverse transform of the force field
template <typename T> cudaError_t pme_gather(const PmeArgs &a, const T *phi, double *F, cudaStream_t s);

}  // namespace ofdft
