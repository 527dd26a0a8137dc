// Smooth particle-mesh Ewald structure factor and forces (Sec. 2.5 of the paper;
// Essmann et al. 1995), in the exp(-iG.R) convention of this library:
//
//   S(G) ~ prod_a conj(b_a(m_a)) * FFT[Q](G),  Q(k) = sum_I prod_a M_p(u_aI - k_a),
//
// u_a = n_a (R . b_a) (grid units), M_p the cardinal B-spline of even order p.
// Spreading uses 64-bit fixed-point atomics (scale 2^40), so the charge grid
// does not depend on the order in which ions are added (bit-reproducible).
#include "pme.cuh"

namespace ofdft {

// w[i] = M_p(x + i), i = 0..p-1 (x in [0,1)); d[i] = dM_p/dy at y = x + i, by the
// recursion M_k(y) = (y M_{k-1}(y) + (k - y) M_{k-1}(y - 1)) / (k - 1), M_2 = hat.
__device__ void bspline_weights(double x, int p, double *w, double *d) {
    for (int i = 0; i < p; i++) w[i] = 0.0;
    w[0] = x;
    w[1] = 1.0 - x;
    for (int k = 3; k <= p; k++) {
        if (k == p && d) {
            for (int i = 0; i < p; i++) d[i] = w[i] - (i >= 1 ? w[i - 1] : 0.0);   // M_{p-1}(y) - M_{p-1}(y-1)
        }
        for (int i = k - 1; i >= 0; i--) {
            const double a = (i >= 1) ? w[i - 1] : 0.0;
            w[i] = ((x + i) * w[i] + (k - x - i) * a) / (double)(k - 1);
        }
    }
    if (p == 2 && d) {
        d[0] = 1.0;
        d[1] = -1.0;
    }
}

__device__ __forceinline__ int wrap(int k, int n) { return ((k % n) + n) % n; }

// lanes 0..2 of the warp compute the weights of one axis each into shared memory
__device__ __forceinline__ void ion_stencil(const PmeArgs &a, int I, double (*w)[kPmeMaxOrder],
                                            double (*d)[kPmeMaxOrder], int *base, int lane) {
    if (lane < 3) {
        const double *R = a.pos + 3 * (size_t)I;
        const int n = lane == 0 ? a.n0 : (lane == 1 ? a.n1 : a.n2);
        double f = R[0] * a.recip[3 * lane] + R[1] * a.recip[3 * lane + 1] + R[2] * a.recip[3 * lane + 2];
        f -= floor(f);
        double u = f * n;
        double fl = floor(u);
        if (fl >= n) fl -= n;          // f == 1 - tiny rounding
        base[lane] = (int)fl;
        bspline_weights(u - floor(u), a.p, w[lane], d ? d[lane] : nullptr);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(256) pme_spread_kernel(PmeArgs a, unsigned long long *Q) {
    __shared__ double w[8][3][kPmeMaxOrder];
    __shared__ int base[8][3];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int I = blockIdx.x * 8 + wid;
    if (I >= a.n_ions || a.species[I] != a.s) return;      // whole warp leaves together
    ion_stencil(a, I, w[wid], nullptr, base[wid], lane);
    const int p = a.p;
    const double scale = 1099511627776.0;                   // 2^40
    for (int t = lane; t < p * p; t += 32) {
        const int j0 = t / p, j1 = t - j0 * p;
        const int k0 = wrap(base[wid][0] - j0, a.n0), k1 = wrap(base[wid][1] - j1, a.n1);
        const double w01 = w[wid][0][j0] * w[wid][1][j1];
        const size_t row = ((size_t)k0 * a.n1 + k1) * a.n2;
        for (int j2 = 0; j2 < p; j2++) {
            const int k2 = wrap(base[wid][2] - j2, a.n2);
            const double v = w01 * w[wid][2][j2];
            atomicAdd(Q + row + k2, (unsigned long long)llrint(v * scale));
        }
    }
}

template <typename T>
__global__ void pme_fixed_to_real_kernel(unsigned long long *Q, T *out, long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride) {
        out[i] = (T)((double)Q[i] * (1.0 / 1099511627776.0));
        Q[i] = 0ull;
    }
}

__device__ __forceinline__ double pme_pp_form(double q2, double Z, double rc) {
    if (q2 <= 0.0) return kPi * Z * rc * rc;
    return -4.0 * kPi * Z * exp(-q2 * rc * rc * 0.25) / q2;
}

__device__ __forceinline__ void pme_g(const PmeArgs &a, long long e, int &k0, int &k1, int &k2, double &q2) {
    k2 = (int)(e % a.n2h);
    const long long r = e / a.n2h;
    k1 = (int)(r % a.n1);
    k0 = (int)(r / a.n1);
    const double m0 = (k0 <= a.n0 / 2) ? k0 : k0 - a.n0;
    const double m1 = (k1 <= a.n1 / 2) ? k1 : k1 - a.n1;
    const double m2 = k2;
    const double tp = 2.0 * kPi;
    double g[3];
    for (int c = 0; c < 3; c++) g[c] = tp * (m0 * a.recip[c] + m1 * a.recip[3 + c] + m2 * a.recip[6 + c]);
    q2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
}

// V_ext(G) (+)= (1/Omega) v_s(|G|) S_s(G),  S_s = prod conj(b) * N * qhat;  S_s(0) = count
template <typename C>
__global__ void pme_vext_kernel(PmeArgs a, const C *qhat, const double2 *B, double Z, double rc, double count,
                                double N, double omega, C *vext, int first) {
    const long long NH = (long long)a.n0 * a.n1 * a.n2h;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= NH) return;
    int k0, k1, k2;
    double q2;
    pme_g(a, e, k0, k1, k2, q2);
    double sx, sy;
    if (q2 > 0.0) {
        const double2 b0 = B[k0], b1 = B[a.n0 + k1], b2 = B[a.n0 + a.n1 + k2];
        const double rx = b0.x * b1.x - b0.y * b1.y, ry = b0.x * b1.y + b0.y * b1.x;
        const double bx = rx * b2.x - ry * b2.y, by = rx * b2.y + ry * b2.x;
        const double qx = (double)qhat[e].x * N, qy = (double)qhat[e].y * N;
        sx = bx * qx - by * qy;
        sy = bx * qy + by * qx;
    } else {
        sx = count;
        sy = 0.0;
    }
    const double v = a.charge_ff ? Z : pme_pp_form(q2, Z, rc) / omega;
    C out;
    out.x = (decltype(out.x))(v * sx);
    out.y = (decltype(out.y))(v * sy);
    if (!first) {
        out.x += vext[e].x;
        out.y += vext[e].y;
    }
    vext[e] = out;
}

// F_s(G) = rho_hat(G) conj(prod conj b) v_s(|G|) for G != 0 (0 at G = 0), written into field
template <typename C>
__global__ void pme_force_field_kernel(PmeArgs a, const C *rhohat, const double2 *B, double Z, double rc,
                                       C *field) {
    const long long NH = (long long)a.n0 * a.n1 * a.n2h;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= NH) return;
    int k0, k1, k2;
    double q2;
    pme_g(a, e, k0, k1, k2, q2);
    C out;
    out.x = 0;
    out.y = 0;
    if (q2 > 0.0) {
        const double2 b0 = B[k0], b1 = B[a.n0 + k1], b2 = B[a.n0 + a.n1 + k2];
        const double rx = b0.x * b1.x - b0.y * b1.y, ry = b0.x * b1.y + b0.y * b1.x;
        const double bx = rx * b2.x - ry * b2.y, by = -(rx * b2.y + ry * b2.x);   // conj of the product
        const double v = a.charge_ff ? Z : pme_pp_form(q2, Z, rc);
        const double hx = rhohat[e].x, hy = rhohat[e].y;
        out.x = (decltype(out.x))(v * (hx * bx - hy * by));
        out.y = (decltype(out.y))(v * (hx * by + hy * bx));
    }
    field[e] = out;
}

// F_I = -sum_a (du_a) n_a b_a,  du_a = sum_k phi(k) dQ(k)/du_a (stencil gather, warp per ion)
template <typename T>
__global__ void __launch_bounds__(256) pme_gather_kernel(PmeArgs a, const T *phi, double *F) {
    __shared__ double w[8][3][kPmeMaxOrder];
    __shared__ double d[8][3][kPmeMaxOrder];
    __shared__ int base[8][3];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int I = blockIdx.x * 8 + wid;
    if (I >= a.n_ions || a.species[I] != a.s) return;
    ion_stencil(a, I, w[wid], d[wid], base[wid], lane);
    const int p = a.p;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int t = lane; t < p * p; t += 32) {
        const int j0 = t / p, j1 = t - j0 * p;
        const int k0 = wrap(base[wid][0] - j0, a.n0), k1 = wrap(base[wid][1] - j1, a.n1);
        const size_t row = ((size_t)k0 * a.n1 + k1) * a.n2;
        const double w0 = w[wid][0][j0], w1 = w[wid][1][j1], d0 = d[wid][0][j0], d1 = d[wid][1][j1];
        for (int j2 = 0; j2 < p; j2++) {
            const int k2 = wrap(base[wid][2] - j2, a.n2);
            const double ph = (double)phi[row + k2];
            const double w2 = w[wid][2][j2], d2 = d[wid][2][j2];
            s0 += ph * d0 * w1 * w2;
            s1 += ph * w0 * d1 * w2;
            s2 += ph * w0 * w1 * d2;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        const double du[3] = {s0 * a.n0, s1 * a.n1, s2 * a.n2};
        for (int c = 0; c < 3; c++)
            F[3 * (size_t)I + c] = -(du[0] * a.recip[c] + du[1] * a.recip[3 + c] + du[2] * a.recip[6 + c]);
    }
}

// ----------------------------------------------------------------------------- launchers
cudaError_t pme_spread(const PmeArgs &a, unsigned long long *Q, cudaStream_t s) {
    pme_spread_kernel<<<(a.n_ions + 7) / 8, 256, 0, s>>>(a, Q);
    return cudaGetLastError();
}

template <typename T> cudaError_t pme_fixed_to_real(unsigned long long *Q, T *out, long long N, cudaStream_t s) {
    pme_fixed_to_real_kernel<T><<<2048, 256, 0, s>>>(Q, out, N);
    return cudaGetLastError();
}

template <typename C>
cudaError_t pme_vext(const PmeArgs &a, const C *qhat, const double2 *B, double Z, double rc, double count, double N,
                     double omega, C *vext, int first, cudaStream_t s) {
    const long long NH = (long long)a.n0 * a.n1 * a.n2h;
    pme_vext_kernel<C><<<(unsigned)((NH + 255) / 256), 256, 0, s>>>(a, qhat, B, Z, rc, count, N, omega, vext, first);
    return cudaGetLastError();
}

template <typename C>
cudaError_t pme_force_field(const PmeArgs &a, const C *rhohat, const double2 *B, double Z, double rc, C *field,
                            cudaStream_t s) {
    const long long NH = (long long)a.n0 * a.n1 * a.n2h;
    pme_force_field_kernel<C><<<(unsigned)((NH + 255) / 256), 256, 0, s>>>(a, rhohat, B, Z, rc, field);
    return cudaGetLastError();
}

template <typename T> cudaError_t pme_gather(const PmeArgs &a, const T *phi, double *F, cudaStream_t s) {
    pme_gather_kernel<T><<<(a.n_ions + 7) / 8, 256, 0, s>>>(a, phi, F);
    return cudaGetLastError();
}

template cudaError_t pme_fixed_to_real<float>(unsigned long long *, float *, long long, cudaStream_t);
template cudaError_t pme_fixed_to_real<double>(unsigned long long *, double *, long long, cudaStream_t);
template cudaError_t pme_vext<float2>(const PmeArgs &, const float2 *, const double2 *, double, double, double,
                                      double, double, float2 *, int, cudaStream_t);
template cudaError_t pme_vext<double2>(const PmeArgs &, const double2 *, const double2 *, double, double, double,
                                       double, double, double2 *, int, cudaStream_t);
template cudaError_t pme_force_field<float2>(const PmeArgs &, const float2 *, const double2 *, double, double,
                                             float2 *, cudaStream_t);
template cudaError_t pme_force_field<double2>(const PmeArgs &, const double2 *, const double2 *, double, double,
                                              double2 *, cudaStream_t);
template cudaError_t pme_gather<float>(const PmeArgs &, const float *, double *, cudaStream_t);
template cudaError_t pme_gather<double>(const PmeArgs &, const double *, double *, cudaStream_t);

}  // namespace ofdft
