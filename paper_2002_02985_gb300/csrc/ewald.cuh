// Ion-ion Ewald energy and forces (see ewald.cu).
#pragma once

#include "common.cuh"

namespace ofdft {

// Real-space part over a cell list: ions sorted by cell, each thread one ion,
// visiting the (2 kr + 1)^3 neighbouring cells with their lattice shifts.
struct EwaldReal {
    int n;                  // ions
    int nc[3], kr[3];       // cells per lattice direction, search range in cells
    double A[9];            // lattice vectors a_0, a_1, a_2 (rows, bohr)
    double eta, rc2;        // split parameter, squared cut-off radius
    const double4 *p;       // [n] sorted by cell: wrapped position (x, y, z) and charge Z
    const int *cell;        // [n] cell id of each sorted ion
    const int *cstart;      // [ncells + 1] first sorted ion of each cell
    const int *orig;        // [n] original index of each sorted ion
    double *F;              // [n][3] by original index (written)
    double *e;              // [n] by sorted index: 1/2 sum_J,L' Z_I Z_J erfc(eta r)/r (written)
};
cudaError_t ewald_real(const EwaldReal &a, cudaStream_t s);

// Reciprocal part on the grid's half spectrum: from the charge structure factor
// S_Z(G) = sum_I Z_I e^{-iG.R_I} in sz, the partials of
// sum_{G != 0} w |S_Z|^2 exp(-G^2/(4 eta^2))/G^2 (w = half-spectrum weight), and
// sz is overwritten by the force field (4 pi / Omega) exp(-G^2/(4 eta^2))/G^2 S_Z (0 at G = 0).
cudaError_t ewald_recip(int n0, int n1, int n2, const double *bvec, double eta, double omega, double2 *sz,
                        double *part, int nblk, cudaStream_t s);

// out[0] = sum of x[0..n) in a fixed order (partials: nblk doubles of scratch)
cudaError_t ewald_sum(const double *x, long long n, double *part, int nblk, double *out, cudaStream_t s);

}  // namespace ofdft
