// Ion-ion electrostatic energy and forces by Ewald summation: point charges Z_I
// in a uniform neutralising background (the electrons make the cell neutral),
// the term that turns E[rho] of Eq. efunc into a total energy for structures and
// forces.  With split parameter eta:
//   E = 1/2 sum_{I,J,L}' Z_I Z_J erfc(eta r)/r
//     + (2 pi/Omega) sum_{G != 0} |S_Z(G)|^2 exp(-G^2/(4 eta^2))/G^2
//     - eta/sqrt(pi) sum Z_I^2 - pi (sum Z_I)^2 / (2 Omega eta^2)
// The reciprocal sum runs over the FFT grid's G vectors (eta is chosen so that the
// terms beyond the grid's largest inscribed sphere are below 1e-16), the real-space
// sum over a cell list, both in FP64.
#include "ewald.cuh"

namespace ofdft {

__global__ void __launch_bounds__(128) ewald_real_kernel(EwaldReal a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const double4 pi = a.p[i];
    const int c = a.cell[i];
    const int ci[3] = {c / (a.nc[1] * a.nc[2]), (c / a.nc[2]) % a.nc[1], c % a.nc[2]};
    const double two_eta_sqrtpi = 2.0 * a.eta / sqrt(kPi);
    double e = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
    for (int d0 = -a.kr[0]; d0 <= a.kr[0]; d0++) {
        const int c0 = ci[0] + d0, s0 = (c0 >= 0) ? c0 / a.nc[0] : -((-c0 + a.nc[0] - 1) / a.nc[0]);
        const int w0 = c0 - s0 * a.nc[0];
        for (int d1 = -a.kr[1]; d1 <= a.kr[1]; d1++) {
            const int c1 = ci[1] + d1, s1 = (c1 >= 0) ? c1 / a.nc[1] : -((-c1 + a.nc[1] - 1) / a.nc[1]);
            const int w1 = c1 - s1 * a.nc[1];
            for (int d2 = -a.kr[2]; d2 <= a.kr[2]; d2++) {
                const int c2 = ci[2] + d2, s2 = (c2 >= 0) ? c2 / a.nc[2] : -((-c2 + a.nc[2] - 1) / a.nc[2]);
                const int w2 = c2 - s2 * a.nc[2];
                // lattice shift of the neighbouring cell's image
                const double Lx = s0 * a.A[0] + s1 * a.A[3] + s2 * a.A[6];
                const double Ly = s0 * a.A[1] + s1 * a.A[4] + s2 * a.A[7];
                const double Lz = s0 * a.A[2] + s1 * a.A[5] + s2 * a.A[8];
                const bool home = s0 == 0 && s1 == 0 && s2 == 0;
                const int id = (w0 * a.nc[1] + w1) * a.nc[2] + w2;
                for (int j = a.cstart[id]; j < a.cstart[id + 1]; j++) {
                    if (home && j == i) continue;
                    const double4 pj = a.p[j];
                    const double dx = pi.x - pj.x - Lx, dy = pi.y - pj.y - Ly, dz = pi.z - pj.z - Lz;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 >= a.rc2) continue;
                    const double r = sqrt(r2);
                    const double er = erfc(a.eta * r) / r;
                    const double zz = pi.w * pj.w;
                    e += 0.5 * zz * er;
                    const double fs = zz * (er + two_eta_sqrtpi * exp(-a.eta * a.eta * r2)) / r2;
                    fx += fs * dx;
                    fy += fs * dy;
                    fz += fs * dz;
                }
            }
        }
    }
    a.e[i] = e;
    const int I = a.orig[i];
    a.F[3 * (size_t)I] = fx;
    a.F[3 * (size_t)I + 1] = fy;
    a.F[3 * (size_t)I + 2] = fz;
}

cudaError_t ewald_real(const EwaldReal &a, cudaStream_t s) {
    ewald_real_kernel<<<(a.n + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) ewald_recip_kernel(int n0, int n1, int n2, double b0, double b1, double b2,
                                                          double b3, double b4, double b5, double b6, double b7,
                                                          double b8, double eta, double omega, double2 *sz,
                                                          double *part) {
    __shared__ double sd[32];
    const int n2h = n2 / 2 + 1;
    const long long NH = (long long)n0 * n1 * n2h;
    const double inv4e2 = 0.25 / (eta * eta);
    double acc = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < NH; e += (long long)gridDim.x * blockDim.x) {
        const int k2 = (int)(e % n2h);
        const long long r = e / n2h;
        const int k1 = (int)(r % n1), k0 = (int)(r / n1);
        const double m0 = (k0 <= n0 / 2) ? k0 : k0 - n0, m1 = (k1 <= n1 / 2) ? k1 : k1 - n1, m2 = k2;
        const double gx = m0 * b0 + m1 * b3 + m2 * b6, gy = m0 * b1 + m1 * b4 + m2 * b7, gz = m0 * b2 + m1 * b5 + m2 * b8;
        const double q2 = gx * gx + gy * gy + gz * gz;
        double2 out = make_double2(0.0, 0.0);
        if (q2 > 0.0) {
            const double w = (k2 == 0 || (n2 % 2 == 0 && 2 * k2 == n2)) ? 1.0 : 2.0;
            const double f = exp(-q2 * inv4e2) / q2;
            const double2 S = sz[e];
            acc += w * f * (S.x * S.x + S.y * S.y);
            const double c = 4.0 * kPi / omega * f;
            out = make_double2(c * S.x, c * S.y);
        }
        sz[e] = out;
    }
    acc = block_sum(acc, sd);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(256) sum_kernel(const double *x, long long n, double *part) {
    __shared__ double sd[32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += x[i];
    acc = block_sum(acc, sd);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

cudaError_t ewald_recip(int n0, int n1, int n2, const double *bv, double eta, double omega, double2 *sz,
                        double *part, int nblk, cudaStream_t s) {
    ewald_recip_kernel<<<nblk, 256, 0, s>>>(n0, n1, n2, bv[0], bv[1], bv[2], bv[3], bv[4], bv[5], bv[6], bv[7],
                                            bv[8], eta, omega, sz, part);
    return cudaGetLastError();
}

cudaError_t ewald_sum(const double *x, long long n, double *part, int nblk, double *out, cudaStream_t s) {
    sum_kernel<<<nblk, 256, 0, s>>>(x, n, part);
    sum_kernel<<<1, 256, 0, s>>>(part, nblk, out);
    return cudaGetLastError();
}

}  // namespace ofdft
