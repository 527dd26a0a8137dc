// Structure factor, forces and optimiser vector kernels (see misc.cuh).
#include "misc.cuh"

namespace ofdft {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ void gvec_of(const IonArgs &a, long long e, double &gx, double &gy, double &gz, int &k0,
                                        int &k1, int &k2) {
    k2 = (int)(e % a.n2h);
    const long long r = e / a.n2h;
    k1 = (int)(r % a.n1);
    k0 = (int)(r / a.n1);
    const double m0 = (k0 <= a.n0 / 2) ? k0 : k0 - a.n0;
    const double m1 = (k1 <= a.n1 / 2) ? k1 : k1 - a.n1;
    const double m2 = k2;
    gx = m0 * a.bvec[0] + m1 * a.bvec[3] + m2 * a.bvec[6];
    gy = m0 * a.bvec[1] + m1 * a.bvec[4] + m2 * a.bvec[7];
    gz = m0 * a.bvec[2] + m1 * a.bvec[5] + m2 * a.bvec[8];
}

// v(q) = -4 pi Z exp(-(q rc)^2/4)/q^2, v(0) = pi Z rc^2 (finite part, Coulomb tail neutralised)
__device__ __forceinline__ double pp_form(double q2, double Z, double rc) {
    if (q2 <= 0.0) return kPi * Z * rc * rc;
    return -4.0 * kPi * Z * exp(-q2 * rc * rc * 0.25) / q2;
}

__global__ void __launch_bounds__(256) vext_kernel(IonArgs a, double2 *v64, float2 *v32) {
    const long long NH = (long long)a.n0 * a.n1 * a.n2h;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= NH) return;
    double gx, gy, gz;
    int k0, k1, k2;
    gvec_of(a, e, gx, gy, gz, k0, k1, k2);
    const double q2 = gx * gx + gy * gy + gz * gz;
    double2 acc = make_double2(0.0, 0.0);
    for (int s = 0; s < a.n_species; s++) {
        double2 S = make_double2(0.0, 0.0);
        for (int I = 0; I < a.n_ions; I++) {
            if (a.species[I] != s) continue;
            const double2 p = zmul(zmul(a.ph0[(size_t)I * a.n0 + k0], a.ph1[(size_t)I * a.n1 + k1]),
                                   a.ph2[(size_t)I * a.n2h + k2]);
            S.x += p.x;
            S.y += p.y;
        }
        const double v = a.charge_ff ? a.Z[s] : pp_form(q2, a.Z[s], a.rc[s]) / a.omega;
        acc.x += v * S.x;
        acc.y += v * S.y;
    }
    if (v64) v64[e] = acc;
    if (v32) v32[e] = make_float2((float)acc.x, (float)acc.y);
}

// FP32-mixed variant: the per-ion phase products e^{-iG.R} = P0 P1 P2 are formed
// in FP32 from the FP64 tables rounded once; groups of 8 ions are summed in
// FP32 and the groups in FP64 (GB300's FP64 rate is a small fraction of FP32's).
__global__ void __launch_bounds__(256) vext_fast_kernel(IonArgs a, const float2 *ph32, float2 *v32) {
    const long long NH = (long long)a.n0 * a.n1 * a.n2h;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= NH) return;
    double gx, gy, gz;
    int k0, k1, k2;
    gvec_of(a, e, gx, gy, gz, k0, k1, k2);
    const double q2 = gx * gx + gy * gy + gz * gz;
    const float2 *P0 = ph32, *P1 = ph32 + (size_t)a.n_ions * a.n0, *P2 = P1 + (size_t)a.n_ions * a.n1;
    double ax = 0.0, ay = 0.0;
    for (int s = 0; s < a.n_species; s++) {
        double Sx = 0.0, Sy = 0.0;
        float gxs = 0.f, gys = 0.f;
        int cnt = 0;
        for (int I = 0; I < a.n_ions; I++) {
            if (a.species[I] != s) continue;
            const float2 p0 = P0[(size_t)I * a.n0 + k0], p1 = P1[(size_t)I * a.n1 + k1], p2 = P2[(size_t)I * a.n2h + k2];
            const float rx = p0.x * p1.x - p0.y * p1.y, ry = p0.x * p1.y + p0.y * p1.x;
            gxs += rx * p2.x - ry * p2.y;
            gys += rx * p2.y + ry * p2.x;
            if (++cnt == 8) {
                Sx += (double)gxs;
                Sy += (double)gys;
                gxs = gys = 0.f;
                cnt = 0;
            }
        }
        Sx += (double)gxs;
        Sy += (double)gys;
        const double v = pp_form(q2, a.Z[s], a.rc[s]) / a.omega;
        ax += v * Sx;
        ay += v * Sy;
    }
    v32[e] = make_float2((float)ax, (float)ay);
}

cudaError_t launch_vext(const IonArgs &a, double2 *vext64, float2 *vext32, cudaStream_t s, const float2 *ph32) {
    const long long NH = (long long)a.n0 * a.n1 * a.n2h;
    if (ph32 && vext32 && !vext64)
        vext_fast_kernel<<<(unsigned)((NH + 255) / 256), 256, 0, s>>>(a, ph32, vext32);
    else
        vext_kernel<<<(unsigned)((NH + 255) / 256), 256, 0, s>>>(a, vext64, vext32);
    return cudaGetLastError();
}

// FP32 copy of the FP64 phase tables
__global__ void round_phases_kernel(const double2 *in, float2 *out, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
cudaError_t launch_round_phases(const double2 *in, float2 *out, long long n, cudaStream_t s) {
    round_phases_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

// Forces, FP64 path: F_I = -sum_G w G v(|G|) Im[conj(rho_hat) e^{-iG.R_I}]; block
// (I, chunk) sums a contiguous range of the half spectrum, one partial per component.
template <typename C>
__global__ void __launch_bounds__(256) forces_kernel(IonArgs a, const C *rh, double *part, int nchunk) {
    __shared__ double sd[32];
    const int I = blockIdx.x, chunk = blockIdx.y;
    const long long NH = (long long)a.n0 * a.n1 * a.n2h;
    const long long per = (NH + nchunk - 1) / nchunk;
    const long long e0 = chunk * per, e1 = (e0 + per < NH) ? e0 + per : NH;
    const int s = a.species[I];
    const double Z = a.Z[s], rc = a.rc[s];
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        double gx, gy, gz;
        int k0, k1, k2;
        gvec_of(a, e, gx, gy, gz, k0, k1, k2);
        const double q2 = gx * gx + gy * gy + gz * gz;
        if (q2 <= 0.0) continue;
        const double w = (k2 == 0 || (a.n2 % 2 == 0 && 2 * k2 == a.n2)) ? 1.0 : 2.0;
        const double2 p = zmul(zmul(a.ph0[(size_t)I * a.n0 + k0], a.ph1[(size_t)I * a.n1 + k1]),
                               a.ph2[(size_t)I * a.n2h + k2]);
        const C r = rh[e];
        // Im[conj(r) p] = r.x p.y - r.y p.x
        const double im = (double)r.x * p.y - (double)r.y * p.x;
        const double f = -w * (a.charge_ff ? Z : pp_form(q2, Z, rc)) * im;
        fx += f * gx;
        fy += f * gy;
        fz += f * gz;
    }
    fx = block_sum(fx, sd);
    if (threadIdx.x == 0) part[((size_t)I * nchunk + chunk) * 3 + 0] = fx;
    fy = block_sum(fy, sd);
    if (threadIdx.x == 0) part[((size_t)I * nchunk + chunk) * 3 + 1] = fy;
    fz = block_sum(fz, sd);
    if (threadIdx.x == 0) part[((size_t)I * nchunk + chunk) * 3 + 2] = fz;
}

template <typename C>
cudaError_t launch_forces(const IonArgs &a, const C *rhohat, double *partials, int nchunk, cudaStream_t s) {
    dim3 g(a.n_ions, nchunk);
    forces_kernel<C><<<g, 256, 0, s>>>(a, rhohat, partials, nchunk);
    return cudaGetLastError();
}
template cudaError_t launch_forces<float2>(const IonArgs &, const float2 *, double *, int, cudaStream_t);
template cudaError_t launch_forces<double2>(const IonArgs &, const double2 *, double *, int, cudaStream_t);

// Forces, FP32-mixed path.  With G = sum_a m_a b_a (b_a: the rows of bvec, 2 pi times the
// reciprocal vectors), the force on ion I of species s is
//   F_I = sum_a b_a S_a(I),   S_a(I) = sum_G m_a Im[c(G) e^{-iG.R_I}],
//   c(G) = -w v_s(|G|) conj(rho_hat(G))   (w = 1 on the k2 = 0 and n2/2 planes, else 2).
// The phase factorises over the axes, e^{-iG.R} = P0(k0) P1(k1) P2(k2), so with the rows
// r = (k0, k1) of the half spectrum
//   U_I(r) = sum_k2 c(r, k2) P2_I(k2),   V_I(r) = sum_k2 k2 c(r, k2) P2_I(k2)
// (two complex products [rows x k2] x [k2 x ions]) and
//   S_0 += m0 Im[P01 U],  S_1 += m1 Im[P01 U],  S_2 += Im[P01 V],   P01 = P0(k0) P1(k1).
// The first step carries all the work: 16 FP32 operations per (row, k2, ion), as packed
// two-ion FP32x2 FMAs from register tiles; the second is once per (row, ion).

// the static part of c for species s, once per set of ions: gf[e] = -w v_s(|G|) (FP64, rounded once)
__global__ void __launch_bounds__(256) force_table_kernel(IonArgs a, float *gf, int s) {
    const long long NH = (long long)a.n0 * a.n1 * a.n2h;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= NH) return;
    double gx, gy, gz;
    int k0, k1, k2;
    gvec_of(a, e, gx, gy, gz, k0, k1, k2);
    const double q2 = gx * gx + gy * gy + gz * gz;
    float f = 0.f;
    if (q2 > 0.0) {
        const double w = (k2 == 0 || (a.n2 % 2 == 0 && 2 * k2 == a.n2)) ? 1.0 : 2.0;
        f = (float)(-w * pp_form(q2, a.Z[s], a.rc[s]));
    }
    gf[e] = f;
}

cudaError_t launch_force_tables(const IonArgs &a, float *gf, cudaStream_t st) {
    const long long NH = (long long)a.n0 * a.n1 * a.n2h;
    for (int s = 0; s < a.n_species; s++)
        force_table_kernel<<<(unsigned)((NH + 255) / 256), 256, 0, st>>>(a, gf + (size_t)s * NH, s);
    return cudaGetLastError();
}

// Block: kFR rows x kFI ions of one species (its ions listed in ions[0, nion)), looping over
// the row tiles blockIdx.x, blockIdx.x + gridDim.x, ...; k2 is staged kFK at a time.  Thread
// (tr, ti) = (threadIdx.x / 16, threadIdx.x % 16) owns rows 4 tr .. 4 tr + 3 and ions 4 ti ..
// 4 ti + 3 of the tile (two pairs, each pair packed (I, J) in FP32x2).  U and V are summed in
// FP32 over k2; the second step in FP32 over the thread's 4 rows, then FP64.
constexpr int kFR = 64, kFI = 64, kFK = 32;
__global__ void __launch_bounds__(256) forces_sep_kernel(IonArgs a, const float2 *ph32, const float *gf,
                                                         const float2 *rh, const int *ions, int nion, double *part) {
    __shared__ __align__(16) float2 cs[kFK][kFR + 2];          // c(r, k2), [k2][row] (padded rows)
    __shared__ __align__(16) float4 ps[kFK][kFI / 2 + 1];      // P2 of ion pairs: (re_I, re_J, im_I, im_J)
    __shared__ double red[8][kFI][3];
    const int ti = threadIdx.x & 15, tr = threadIdx.x >> 4;
    const int rows = a.n0 * a.n1, n2h = a.n2h;
    const int ion0 = blockIdx.y * kFI;
    const float2 *P0 = ph32, *P1 = ph32 + (size_t)a.n_ions * a.n0, *P2 = P1 + (size_t)a.n_ions * a.n1;
    // this thread's four ions (global indices; -1 past the species' list)
    int myI[4];
#pragma unroll
    for (int q = 0; q < 4; q++) myI[q] = (ion0 + 4 * ti + q < nion) ? ions[ion0 + 4 * ti + q] : -1;
    double S[4][3];
#pragma unroll
    for (int q = 0; q < 4; q++) S[q][0] = S[q][1] = S[q][2] = 0.0;
    const int ntile = (rows + kFR - 1) / kFR;
    for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int r0 = tile * kFR;
        float2 U[4][2][2], V[4][2][2];                         // [row][pair][re, im] (FP32x2 over the pair)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int p = 0; p < 2; p++) U[j][p][0] = U[j][p][1] = V[j][p][0] = V[j][p][1] = make_float2(0.f, 0.f);
        for (int kc = 0; kc < n2h; kc += kFK) {
            __syncthreads();                                   // the previous chunk is consumed
            for (int idx = threadIdx.x; idx < kFR * kFK; idx += 256) {
                const int i = idx / kFK, k = idx - i * kFK;
                float2 c = make_float2(0.f, 0.f);
                if (r0 + i < rows && kc + k < n2h) {
                    const long long e = (long long)(r0 + i) * n2h + kc + k;
                    const float f = gf[e];
                    const float2 r = rh[e];
                    c = make_float2(f * r.x, -f * r.y);
                }
                cs[k][i] = c;
            }
            for (int idx = threadIdx.x; idx < (kFI / 2) * kFK; idx += 256) {
                const int pp = idx / kFK, k = idx - pp * kFK;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (kc + k < n2h) {
                    const int t0 = ion0 + 2 * pp, t1 = t0 + 1;
                    const float2 u = t0 < nion ? P2[(size_t)ions[t0] * n2h + kc + k] : make_float2(0.f, 0.f);
                    const float2 w = t1 < nion ? P2[(size_t)ions[t1] * n2h + kc + k] : make_float2(0.f, 0.f);
                    v = make_float4(u.x, w.x, u.y, w.y);
                }
                ps[k][pp] = v;
            }
            __syncthreads();
            const int kn = min(kFK, n2h - kc);
#pragma unroll 2
            for (int k = 0; k < kn; k++) {
                const float4 c01 = *reinterpret_cast<const float4 *>(&cs[k][4 * tr]);
                const float4 c23 = *reinterpret_cast<const float4 *>(&cs[k][4 * tr + 2]);
                const float4 pa = ps[k][2 * ti], pb = ps[k][2 * ti + 1];
                const float kf = (float)(kc + k);
                const float cr[4] = {c01.x, c01.z, c23.x, c23.z}, ci[4] = {c01.y, c01.w, c23.y, c23.w};
                const float2 Pr[2] = {make_float2(pa.x, pa.y), make_float2(pb.x, pb.y)};
                const float2 Pi[2] = {make_float2(pa.z, pa.w), make_float2(pb.z, pb.w)};
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const float2 a_r = make_float2(cr[j], cr[j]), a_i = make_float2(ci[j], ci[j]);
                    const float2 n_i = make_float2(-ci[j], -ci[j]);
                    const float br = kf * cr[j], bi = kf * ci[j];
                    const float2 b_r = make_float2(br, br), b_i = make_float2(bi, bi), m_i = make_float2(-bi, -bi);
#pragma unroll
                    for (int p = 0; p < 2; p++) {
                        // (c P2): re = cr Pr - ci Pi, im = cr Pi + ci Pr (two ions at once)
                        U[j][p][0] = __ffma2_rn(n_i, Pi[p], __ffma2_rn(a_r, Pr[p], U[j][p][0]));
                        U[j][p][1] = __ffma2_rn(a_i, Pr[p], __ffma2_rn(a_r, Pi[p], U[j][p][1]));
                        V[j][p][0] = __ffma2_rn(m_i, Pi[p], __ffma2_rn(b_r, Pr[p], V[j][p][0]));
                        V[j][p][1] = __ffma2_rn(b_i, Pr[p], __ffma2_rn(b_r, Pi[p], V[j][p][1]));
                    }
                }
            }
        }
        // second step: the rows' P01 and the three sums of each of the thread's ions
        float s32[4][3];
#pragma unroll
        for (int q = 0; q < 4; q++) s32[q][0] = s32[q][1] = s32[q][2] = 0.f;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int r = r0 + 4 * tr + j;
            if (r >= rows) continue;
            const int k0 = r / a.n1, k1 = r - k0 * a.n1;
            const float m0 = (float)(k0 <= a.n0 / 2 ? k0 : k0 - a.n0), m1 = (float)(k1 <= a.n1 / 2 ? k1 : k1 - a.n1);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                if (myI[q] < 0) continue;
                const float2 p0 = P0[(size_t)myI[q] * a.n0 + k0], p1 = P1[(size_t)myI[q] * a.n1 + k1];
                const float pr = p0.x * p1.x - p0.y * p1.y, pi = p0.x * p1.y + p0.y * p1.x;
                const int p = q >> 1;
                const float ur = (q & 1) ? U[j][p][0].y : U[j][p][0].x, ui = (q & 1) ? U[j][p][1].y : U[j][p][1].x;
                const float vr = (q & 1) ? V[j][p][0].y : V[j][p][0].x, vi = (q & 1) ? V[j][p][1].y : V[j][p][1].x;
                const float imU = pr * ui + pi * ur, imV = pr * vi + pi * vr;
                s32[q][0] += m0 * imU;
                s32[q][1] += m1 * imU;
                s32[q][2] += imV;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int d = 0; d < 3; d++) S[q][d] += (double)s32[q][d];
    }
    // block sums: the two row groups of a warp by a shuffle, then the 8 warps in shared memory
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double v = S[q][d] + __shfl_xor_sync(0xffffffffu, S[q][d], 16);
            if (lane < 16) red[warp][4 * ti + q][d] = v;
        }
    __syncthreads();
    if (threadIdx.x < 3 * kFI) {
        const int q = threadIdx.x / 3, d = threadIdx.x - 3 * q;
        double t = 0.0;
        for (int w = 0; w < 8; w++) t += red[w][q][d];
        if (ion0 + q < nion) part[((size_t)ions[ion0 + q] * gridDim.x + blockIdx.x) * 3 + d] = t;
    }
}

// row-tile blocks of the separable force kernel: about two waves (three blocks resident per SM)
int forces_sep_blocks(const IonArgs &a, int nsm) {
    const int ntile = (a.n0 * a.n1 + kFR - 1) / kFR, target = 6 * nsm;
    return ntile < target ? ntile : target;
}

cudaError_t launch_forces_sep(const IonArgs &a, const float2 *rhohat, const float2 *ph32, const float *gf,
                              const int *sp_ions, const int *sp_off, int nrb, double *partials, cudaStream_t st) {
    const long long NH = (long long)a.n0 * a.n1 * a.n2h;
    for (int s = 0; s < a.n_species; s++) {
        const int nion = sp_off[s + 1] - sp_off[s];
        if (nion == 0) continue;
        dim3 g(nrb, (nion + kFI - 1) / kFI);
        forces_sep_kernel<<<g, 256, 0, st>>>(a, ph32, gf + (size_t)s * NH, rhohat, sp_ions + sp_off[s], nion,
                                             partials);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// F_I = sum_a b_a S_a(I), S_a(I) = the partials [n_ions][nrb][3] summed over the row tiles in order
__global__ void reduce_force_sep_kernel(IonArgs a, const double *part, int nrb, double *F) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= a.n_ions) return;
    double S[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < nrb; c++)
        for (int k = 0; k < 3; k++) S[k] += part[((size_t)I * nrb + c) * 3 + k];
    for (int d = 0; d < 3; d++) F[3 * I + d] = S[0] * a.bvec[d] + S[1] * a.bvec[3 + d] + S[2] * a.bvec[6 + d];
}
cudaError_t launch_reduce_force_sep(const IonArgs &a, const double *part, int nrb, double *F, cudaStream_t s) {
    reduce_force_sep_kernel<<<(a.n_ions + 127) / 128, 128, 0, s>>>(a, part, nrb, F);
    return cudaGetLastError();
}

// F[I][d] = sum over chunks of the partials [n_ions][nchunk][3] (fixed order)
__global__ void reduce_force_partials_kernel(const double *part, int n_ions, int nchunk, double *F) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * n_ions) return;
    const int I = t / 3, d = t - 3 * I;
    double s = 0.0;
    for (int c = 0; c < nchunk; c++) s += part[((size_t)I * nchunk + c) * 3 + d];
    F[t] = s;
}
cudaError_t launch_reduce_force_partials(const double *part, int n_ions, int nchunk, double *F, cudaStream_t s) {
    reduce_force_partials_kernel<<<(3 * n_ions + 255) / 256, 256, 0, s>>>(part, n_ions, nchunk, F);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- plain FFT along n0
template <typename T, int CAP, int DIR>
__global__ void __launch_bounds__(512) axis0_fft_kernel(typename Vec2<T>::type *data, int n0, long long P, FFTPlan p,
                                 const typename Vec2<T>::type *twg, int TW, T scale) {
    typedef typename Vec2<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = (C *)smem_raw;
    C *buf = tw + n0;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) tw[i] = twg[i];
    const long long c0 = (long long)blockIdx.x * TW;
    for (int idx = threadIdx.x; idx < n0 * TW; idx += blockDim.x) {
        const int w = idx % TW, i = idx / TW;
        buf[idx] = (c0 + w < P) ? data[(size_t)i * P + c0 + w] : cmake<C>((T)0, (T)0);
    }
    __syncthreads();
    fft_smem<DIR, CAP>(buf, TW, TW, p, tw);
    for (int idx = threadIdx.x; idx < n0 * TW; idx += blockDim.x) {
        const int w = idx % TW, i = idx / TW;
        if (c0 + w < P) data[(size_t)i * P + c0 + w] = cscale(buf[idx], scale);
    }
}

// the same with the length, the tile (TWC columns) and the radix plan fixed at compile time
template <typename T, int N, int TWC, int DIR>
__global__ void __launch_bounds__(256) axis0_fft_ct_kernel(typename Vec2<T>::type *data, long long P,
                                                           const typename Vec2<T>::type *twg, T scale) {
    typedef typename Vec2<T>::type C;
    constexpr int MAXR = sizeof(T) == 4 ? 16 : 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = (C *)smem_raw;
    C *buf = tw + N;
    for (int i = threadIdx.x; i < N; i += 256) tw[i] = twg[i];
    const long long c0 = (long long)blockIdx.x * TWC;
    for (int idx = threadIdx.x; idx < N * TWC; idx += 256) {
        const int w = idx % TWC, i = idx / TWC;
        buf[idx] = (c0 + w < P) ? data[(size_t)i * P + c0 + w] : cmake<C>((T)0, (T)0);
    }
    __syncthreads();
    ct::fft<DIR, N, TWC, TWC, 256, MAXR>(buf, tw);
    for (int idx = threadIdx.x; idx < N * TWC; idx += 256) {
        const int w = idx % TWC, i = idx / TWC;
        if (c0 + w < P) data[(size_t)i * P + c0 + w] = cscale(buf[idx], scale);
    }
}

template <typename T, int N, int TWC>
cudaError_t launch_axis0_fft_ct(typename Vec2<T>::type *data, long long P, const typename Vec2<T>::type *tw,
                                double scale, cudaStream_t s, int dir) {
    typedef typename Vec2<T>::type C;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = allow_max_dynamic_smem(axis0_fft_ct_kernel<T, N, TWC, -1>);
        if (e == cudaSuccess) e = allow_max_dynamic_smem(axis0_fft_ct_kernel<T, N, TWC, 1>);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const size_t sm = (size_t)N * sizeof(C) * (1 + TWC);
    const unsigned nb = (unsigned)((P + TWC - 1) / TWC);
    if (dir < 0) axis0_fft_ct_kernel<T, N, TWC, -1><<<nb, 256, sm, s>>>(data, P, tw, (T)scale);
    else axis0_fft_ct_kernel<T, N, TWC, 1><<<nb, 256, sm, s>>>(data, P, tw, (T)scale);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axis0_fft(typename Vec2<T>::type *data, int n0, long long P, const FFTPlan &p,
                             const typename Vec2<T>::type *tw, int TW, int thr, double scale, cudaStream_t s, int dir) {
    typedef typename Vec2<T>::type C;
    constexpr int CAP = sizeof(T) == 4 ? 16 : 8;
    // compile-time forms for the common lengths
    if (n0 == 64) return launch_axis0_fft_ct<T, 64, 32>(data, P, tw, scale, s, dir);
    if (n0 == 96) return launch_axis0_fft_ct<T, 96, 32>(data, P, tw, scale, s, dir);
    if (n0 == 128) return launch_axis0_fft_ct<T, 128, 32>(data, P, tw, scale, s, dir);
    if (n0 == 192) return launch_axis0_fft_ct<T, 192, 16>(data, P, tw, scale, s, dir);
    if (n0 == 256) return launch_axis0_fft_ct<T, 256, 16>(data, P, tw, scale, s, dir);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = allow_max_dynamic_smem(axis0_fft_kernel<T, CAP, -1>);
        if (e == cudaSuccess) e = allow_max_dynamic_smem(axis0_fft_kernel<T, CAP, 1>);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // a plain transform has one channel: wide column tiles (coalesced rows of up to 32 complex),
    // independent of the reciprocal-space kernel's tile.  Each thread stages at most CAP values
    // per pass, so a pass of radix R over TW columns needs (n0/R) TW / (CAP/R) threads: the tile
    // is narrowed until every pass fits in 512 threads and 96 KB
    (void)TW;
    (void)thr;
    auto need = [&](int cols) {
        long long nt = 32;
        for (int i = 0; i < p.npass; i++) {
            const int R = p.radix[i], mb = CAP / R;
            const long long t = ((long long)(n0 / R) * cols + mb - 1) / mb;
            nt = t > nt ? t : nt;
        }
        return (int)((nt + 31) / 32 * 32);
    };
    int tw_cols = 32;
    while (tw_cols > 1 && ((size_t)n0 * sizeof(C) * (1 + tw_cols) > 96 * 1024 || need(tw_cols) > 512)) tw_cols /= 2;
    TW = tw_cols;
    thr = need(TW) > 256 ? need(TW) : 256;
    if (thr > 512) return cudaErrorInvalidConfiguration;
    const size_t sm = (size_t)n0 * sizeof(C) * (1 + TW);
    const unsigned nb = (unsigned)((P + TW - 1) / TW);
    if (dir < 0) axis0_fft_kernel<T, CAP, -1><<<nb, thr, sm, s>>>(data, n0, P, p, tw, TW, (T)scale);
    else axis0_fft_kernel<T, CAP, 1><<<nb, thr, sm, s>>>(data, n0, P, p, tw, TW, (T)scale);
    return cudaGetLastError();
}
template cudaError_t launch_axis0_fft<float>(float2 *, int, long long, const FFTPlan &, const float2 *, int, int,
                                             double, cudaStream_t, int);
template cudaError_t launch_axis0_fft<double>(double2 *, int, long long, const FFTPlan &, const double2 *, int, int,
                                              double, cudaStream_t, int);

// ---------------------------------------------------------------- optimiser vectors
template <typename T>
__global__ void __launch_bounds__(256) dot_kernel(const T *a, const T *b, const T *c, long long N, double *part,
                                                  bool exact) {
    __shared__ double sd[32];
    double acc = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (sizeof(T) == 4 && exact) {
        for (; i < N; i += stride) acc += (double)(c ? a[i] * b[i] * c[i] : a[i] * b[i]);
    } else if (sizeof(T) == 4) {
        // FP32 products in groups of 8 grid strides, each group added in FP64 (the FP64 pipe
        // of GB300 would otherwise bound this pass)
        while (i < N) {
            T g = 0;
#pragma unroll
            for (int u = 0; u < 8; u++, i += stride)
                if (i < N) g += c ? a[i] * b[i] * c[i] : a[i] * b[i];
            acc += (double)g;
        }
    } else {
        for (; i < N; i += stride) {
            double v = (double)a[i] * (double)b[i];
            if (c) v *= (double)c[i];
            acc += v;
        }
    }
    acc = block_sum(acc, sd);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(256) sum_partials_kernel(const double *part, int n, double *out) {
    __shared__ double sd[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    acc = block_sum(acc, sd);
    if (threadIdx.x == 0) *out = acc;
}

template <typename T>
cudaError_t launch_dot(const T *a, const T *b, const T *c, long long N, double *partials, int nblk, double *out,
                       cudaStream_t s, bool exact) {
    dot_kernel<T><<<nblk, 256, 0, s>>>(a, b, c, N, partials, exact);
    sum_partials_kernel<<<1, 256, 0, s>>>(partials, nblk, out);
    return cudaGetLastError();
}

template <typename T> __global__ void axpby_kernel(T *y, const T *x, T al, T be, long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (be == (T)0) {                  // y is not read: it may hold anything, NaN included
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride) y[i] = al * x[i];
        return;
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride)
        y[i] = al * x[i] + be * y[i];
}
template <typename T>
cudaError_t launch_axpby(T *y, const T *x, double alpha, double beta, long long N, cudaStream_t s) {
    axpby_kernel<T><<<1216, 256, 0, s>>>(y, x, (T)alpha, (T)beta, N);
    return cudaGetLastError();
}

template <typename T>
__global__ void rotate_kernel(T *psl, T *rho, const T *psi, const T *p, T c, T sn, long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride) {
        const T v = psi[i] * c + p[i] * sn;
        psl[i] = v;
        rho[i] = v * v;
    }
}
template <typename T>
cudaError_t launch_rotate(T *psi_l, T *rho, const T *psi, const T *p, double c, double sn, long long N,
                          cudaStream_t s) {
    rotate_kernel<T><<<1216, 256, 0, s>>>(psi_l, rho, psi, p, (T)c, (T)sn, N);
    return cudaGetLastError();
}

template <typename T> __global__ void grad_kernel(T *g, const T *psi, const T *V, T mu, T dV2, long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride)
        g[i] = dV2 * psi[i] * (V[i] - mu);
}
template <typename T>
cudaError_t launch_grad(T *g, const T *psi, const T *V, double mu, double dV, long long N, cudaStream_t s) {
    grad_kernel<T><<<1216, 256, 0, s>>>(g, psi, V, (T)mu, (T)(2.0 * dV), N);
    return cudaGetLastError();
}

template <typename T> __global__ void square_kernel(T *rho, T *psi, T scale, long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride) {
        const T v = psi[i] * scale;
        psi[i] = v;
        rho[i] = v * v;
    }
}
template <typename T> cudaError_t launch_square(T *rho, T *psi, double scale, long long N, cudaStream_t s) {
    square_kernel<T><<<1216, 256, 0, s>>>(rho, psi, (T)scale, N);
    return cudaGetLastError();
}

template <typename T> __global__ void copy_kernel(T *d, const T *s, long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride) d[i] = s[i];
}
template <typename T> cudaError_t launch_copy(T *dst, const T *src, long long N, cudaStream_t s) {
    copy_kernel<T><<<1216, 256, 0, s>>>(dst, src, N);
    return cudaGetLastError();
}

// sources of to-index j along one full axis: up to two (index, weight)
__device__ __forceinline__ int axis_sources(int j, int nf, int nt, int *src, double *w) {
    const int m = (j <= nt / 2) ? j : j - nt;                // signed frequency on the target grid
    const int small = nf < nt ? nf : nt;
    const int am = m < 0 ? -m : m;
    if (2 * am < small) {
        src[0] = ((m % nf) + nf) % nf;
        w[0] = 1.0;
        return 1;
    }
    if (small % 2 == 0 && 2 * am == small) {
        if (nt > nf) {                                         // +-nf/2 on the target: half the Nyquist each
            src[0] = nf / 2;
            w[0] = 0.5;
            return 1;
        }
        if (nt < nf) {                                         // target Nyquist (m = +nt/2): both signs
            if (m < 0) return 0;
            src[0] = nt / 2;
            src[1] = nf - nt / 2;
            w[0] = w[1] = 1.0;
            return 2;
        }
        src[0] = j;
        w[0] = 1.0;
        return 1;
    }
    return 0;
}

template <typename C>
__global__ void spectral_map_kernel(const C *src, int f0, int f1, int f2, C *dst, int t0, int t1, int t2) {
    const int fh = f2 / 2 + 1, th = t2 / 2 + 1;
    const long long NT = (long long)t0 * t1 * th, stride = (long long)gridDim.x * blockDim.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < NT; e += stride) {
        const int j2 = (int)(e % th);
        const long long r = e / th;
        const int j1 = (int)(r % t1), j0 = (int)(r / t1);
        int s0[2], s1[2];
        double w0[2], w1[2];
        const int n0 = axis_sources(j0, f0, t0, s0, w0), n1 = axis_sources(j1, f1, t1, s1, w1);
        // last axis (half spectrum, m2 = j2 >= 0): sources (index, weight, conjugate-partner?)
        const int small2 = f2 < t2 ? f2 : t2;
        int n2 = 0, i2[2] = {0, 0}, cj[2] = {0, 0};
        double w2[2] = {0.0, 0.0};
        if (2 * j2 < small2) {
            i2[0] = j2; w2[0] = 1.0; n2 = 1;
        } else if (small2 % 2 == 0 && 2 * j2 == small2) {
            if (t2 > f2) { i2[0] = j2; w2[0] = 0.5; n2 = 1; }
            else if (t2 < f2) { i2[0] = j2; w2[0] = 1.0; i2[1] = j2; w2[1] = 1.0; cj[1] = 1; n2 = 2; }
            else { i2[0] = j2; w2[0] = 1.0; n2 = 1; }
        }
        double ax = 0.0, ay = 0.0;
        for (int a = 0; a < n0; a++)
            for (int b = 0; b < n1; b++)
                for (int c = 0; c < n2; c++) {
                    const double w = w0[a] * w1[b] * w2[c];
                    if (!cj[c]) {
                        const C v = src[((long long)s0[a] * f1 + s1[b]) * fh + i2[c]];
                        ax += w * v.x;
                        ay += w * v.y;
                    } else {                                   // coefficient at -m2: conj of (-m0, -m1, +m2)
                        const int q0 = (f0 - s0[a]) % f0, q1 = (f1 - s1[b]) % f1;
                        const C v = src[((long long)q0 * f1 + q1) * fh + i2[c]];
                        ax += w * v.x;
                        ay -= w * v.y;
                    }
                }
        C out;
        out.x = (decltype(out.x))(e == 0 ? 0.0 : ax);          // the mean is added back after the inverse
        out.y = (decltype(out.y))(e == 0 ? 0.0 : ay);
        dst[e] = out;
    }
}

template <typename C>
cudaError_t launch_spectral_map(const C *src, int f0, int f1, int f2, C *dst, int t0, int t1, int t2,
                                cudaStream_t s) {
    spectral_map_kernel<C><<<1216, 256, 0, s>>>(src, f0, f1, f2, dst, t0, t1, t2);
    return cudaGetLastError();
}
template cudaError_t launch_spectral_map<float2>(const float2 *, int, int, int, float2 *, int, int, int,
                                                 cudaStream_t);
template cudaError_t launch_spectral_map<double2>(const double2 *, int, int, int, double2 *, int, int, int,
                                                  cudaStream_t);

template <typename T> __global__ void add_scalar_kernel(T *x, const double *c, long long N) {
    const T v = (T)c[0];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride) x[i] += v;
}
template <typename T> cudaError_t launch_add_scalar(T *x, const double *c, long long N, cudaStream_t s) {
    add_scalar_kernel<T><<<1216, 256, 0, s>>>(x, c, N);
    return cudaGetLastError();
}

// G^2 of half-spectrum element e in the spectrum's own precision R (float for the FP32-mixed
// path: GB300's FP64 rate would make these elementwise passes FP64-bound)
template <typename R>
__device__ __forceinline__ R half_spectrum_g2(long long e, int n0, int n1, int n2h, const R *b) {
    const int k2 = (int)(e % n2h);
    const long long r = e / n2h;
    const int k1 = (int)(r % n1), k0 = (int)(r / n1);
    const R m0 = (R)((k0 <= n0 / 2) ? k0 : k0 - n0), m1 = (R)((k1 <= n1 / 2) ? k1 : k1 - n1), m2 = (R)k2;
    const R gx = m0 * b[0] + m1 * b[3] + m2 * b[6], gy = m0 * b[1] + m1 * b[4] + m2 * b[7],
            gz = m0 * b[2] + m1 * b[5] + m2 * b[8];
    return gx * gx + gy * gy + gz * gz;
}
struct Bvec9 {
    double v[9];
};

template <typename C>
__global__ void precond_kernel(C *h, int n0, int n1, int n2, Bvec9 bv, double pa_, double pb_) {
    typedef decltype(h[0].x) R;
    R b[9];
#pragma unroll
    for (int i = 0; i < 9; i++) b[i] = (R)bv.v[i];
    const R pa = (R)pa_, pb = (R)pb_;
    const int n2h = n2 / 2 + 1;
    const long long NH = (long long)n0 * n1 * n2h, stride = (long long)gridDim.x * blockDim.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < NH; e += stride) {
        const R q2 = half_spectrum_g2<R>(e, n0, n1, n2h, b);
        const R f = (q2 > (R)0) ? pa * q2 / (q2 * q2 + pa * q2 + pb) : (R)1;
        C v = h[e];
        v.x *= f;
        v.y *= f;
        h[e] = v;
    }
}
template <typename C>
cudaError_t launch_precond(C *h, int n0, int n1, int n2, const double *bv, double a, double b, cudaStream_t s) {
    Bvec9 b9;
    for (int i = 0; i < 9; i++) b9.v[i] = bv[i];
    precond_kernel<C><<<1216, 256, 0, s>>>(h, n0, n1, n2, b9, a, b);
    return cudaGetLastError();
}
template cudaError_t launch_precond<float2>(float2 *, int, int, int, const double *, double, double, cudaStream_t);
template cudaError_t launch_precond<double2>(double2 *, int, int, int, const double *, double, double, cudaStream_t);

// Lagrangian Hessian times q by a forward difference of the gradient 2 psi V[psi^2] dV:
// Hq = 2 dV (q Vq + psi (Vq - V) / e - mu q), Vq the potential at psi + e q.
template <typename T>
__global__ void hvp_kernel(T *Hq, const T *psi, const T *q, const T *V, const T *Vq, T inv_e, T mu, T dV2,
                           long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride) {
        const T vq = Vq[i], qi = q[i];
        Hq[i] = dV2 * (qi * (vq - mu) + psi[i] * (vq - V[i]) * inv_e);
    }
}
template <typename T>
cudaError_t launch_hvp(T *Hq, const T *psi, const T *q, const T *V, const T *Vq, double e, double mu, double dV,
                       long long N, cudaStream_t s) {
    hvp_kernel<T><<<1216, 256, 0, s>>>(Hq, psi, q, V, Vq, (T)(1.0 / e), (T)mu, (T)(2.0 * dV), N);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- real-time TD-OFDFT
// h(G) *= f(G) on a normalised half spectrum: MODE 0 the kinetic K = G^2/2 (K(0) = 0),
// MODE 1 the Crank-Nicolson normal-equation preconditioner 1 / (1 + tau^2 (G^2/2 + vbar)^2)
template <typename C, int MODE>
__global__ void spectral_factor_kernel(C *h, int n0, int n1, int n2, Bvec9 bv, double tau_, double vbar_) {
    typedef decltype(h[0].x) R;
    R b[9];
#pragma unroll
    for (int i = 0; i < 9; i++) b[i] = (R)bv.v[i];
    const R tau = (R)tau_, vbar = (R)vbar_;
    const int n2h = n2 / 2 + 1;
    const long long NH = (long long)n0 * n1 * n2h, stride = (long long)gridDim.x * blockDim.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < NH; e += stride) {
        const R kin = (R)0.5 * half_spectrum_g2<R>(e, n0, n1, n2h, b);
        R f;
        if (MODE == 0) {
            f = kin;
        } else {
            const R x = tau * (kin + vbar);
            f = (R)1 / ((R)1 + x * x);
        }
        C v = h[e];
        v.x *= f;
        v.y *= f;
        h[e] = v;
    }
}
template <typename C>
cudaError_t launch_spectral_factor(C *h, int n0, int n1, int n2, const double *bv, int mode, double tau, double vbar,
                                   cudaStream_t s) {
    Bvec9 b9;
    for (int i = 0; i < 9; i++) b9.v[i] = bv[i];
    if (mode == 0)
        spectral_factor_kernel<C, 0><<<1216, 256, 0, s>>>(h, n0, n1, n2, b9, tau, vbar);
    else
        spectral_factor_kernel<C, 1><<<1216, 256, 0, s>>>(h, n0, n1, n2, b9, tau, vbar);
    return cudaGetLastError();
}
template cudaError_t launch_spectral_factor<float2>(float2 *, int, int, int, const double *, int, double, double,
                                                    cudaStream_t);
template cudaError_t launch_spectral_factor<double2>(double2 *, int, int, int, const double *, int, double, double,
                                                     cudaStream_t);

// out = a out + b v u
template <typename T> __global__ void add_vu_kernel(T *out, const T *v, const T *u, T a, T b, long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride)
        out[i] = a * out[i] + b * v[i] * u[i];
}
template <typename T>
cudaError_t launch_add_vu(T *out, const T *v, const T *u, double a, double b, long long N, cudaStream_t s) {
    add_vu_kernel<T><<<1216, 256, 0, s>>>(out, v, u, (T)a, (T)b, N);
    return cudaGetLastError();
}

// rho = re^2 + im^2
template <typename T> __global__ void abs2_kernel(T *rho, const T *re, const T *im, long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride)
        rho[i] = re[i] * re[i] + im[i] * im[i];
}
template <typename T> cudaError_t launch_abs2(T *rho, const T *re, const T *im, long long N, cudaStream_t s) {
    abs2_kernel<T><<<1216, 256, 0, s>>>(rho, re, im, N);
    return cudaGetLastError();
}

// x += f c[0]
template <typename T> __global__ void add_scaled_scalar_kernel(T *x, const double *c, double f, long long N) {
    const T v = (T)(f * c[0]);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride) x[i] += v;
}
template <typename T>
cudaError_t launch_add_scaled_scalar(T *x, const double *c, double f, long long N, cudaStream_t s) {
    add_scaled_scalar_kernel<T><<<1216, 256, 0, s>>>(x, c, f, N);
    return cudaGetLastError();
}

// cell-centred Cartesian position of grid point i: r = A^T (f - 1/2), f = (i0/n0, i1/n1, i2/n2)
__device__ __forceinline__ void centred_position(long long i, int n0, int n1, int n2, const TdCell &c, double &x,
                                                 double &y, double &z) {
    const int i2 = (int)(i % n2);
    const long long r = i / n2;
    const int i1 = (int)(r % n1), i0 = (int)(r / n1);
    const double f0 = (double)i0 / n0 - 0.5, f1 = (double)i1 / n1 - 0.5, f2 = (double)i2 / n2 - 0.5;
    x = f0 * c.a[0] + f1 * c.a[3] + f2 * c.a[6];
    y = f0 * c.a[1] + f1 * c.a[4] + f2 * c.a[7];
    z = f0 * c.a[2] + f1 * c.a[5] + f2 * c.a[8];
}

// psi <- psi exp(i k . r)
template <typename T>
__global__ void kick_kernel(T *re, T *im, int n0, int n1, int n2, TdCell c, double kx, double ky, double kz,
                            long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride) {
        double x, y, z;
        centred_position(i, n0, n1, n2, c, x, y, z);
        double sn, cs;
        sincos(kx * x + ky * y + kz * z, &sn, &cs);
        const double a = (double)re[i], b = (double)im[i];
        re[i] = (T)(a * cs - b * sn);
        im[i] = (T)(a * sn + b * cs);
    }
}
template <typename T>
cudaError_t launch_kick(T *re, T *im, int n0, int n1, int n2, const TdCell &c, const double *k, cudaStream_t s) {
    kick_kernel<T><<<1216, 256, 0, s>>>(re, im, n0, n1, n2, c, k[0], k[1], k[2], (long long)n0 * n1 * n2);
    return cudaGetLastError();
}

// partials of sum_r r (|psi|^2 - rho0) dV: part[3 b + k], then the three sums into out[0..2].
// Positions and products in T (FP32 in the FP32-mixed path), sums in FP64.
template <typename T>
__global__ void __launch_bounds__(256) dipole_kernel(const T *re, const T *im, const T *rho0, int n0, int n1, int n2,
                                                     TdCell c, double dV, long long N, double *part) {
    __shared__ double sd[3 * 32];
    double acc[3] = {0.0, 0.0, 0.0};
    T a9[9];
#pragma unroll
    for (int k = 0; k < 9; k++) a9[k] = (T)c.a[k];
    const T r0 = (T)1 / (T)n0, r1 = (T)1 / (T)n1, r2 = (T)1 / (T)n2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride) {
        const int i2 = (int)(i % n2);
        const long long q = i / n2;
        const int i1 = (int)(q % n1), i0 = (int)(q / n1);
        const T f0 = (T)i0 * r0 - (T)0.5, f1 = (T)i1 * r1 - (T)0.5, f2 = (T)i2 * r2 - (T)0.5;
        const T a = re[i], b = im[i];
        const T d = a * a + b * b - (rho0 ? rho0[i] : (T)0);
        acc[0] += (double)((f0 * a9[0] + f1 * a9[3] + f2 * a9[6]) * d);
        acc[1] += (double)((f0 * a9[1] + f1 * a9[4] + f2 * a9[7]) * d);
        acc[2] += (double)((f0 * a9[2] + f1 * a9[5] + f2 * a9[8]) * d);
    }
    block_sum_n<3>(acc, sd);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) part[3 * blockIdx.x + k] = acc[k] * dV;
}
__global__ void __launch_bounds__(256) sum3_partials_kernel(const double *part, int n, double *out) {
    __shared__ double sd[3 * 32];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int k = 0; k < 3; k++) acc[k] += part[3 * i + k];
    block_sum_n<3>(acc, sd);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) out[k] = acc[k];
}
template <typename T>
cudaError_t launch_dipole(const T *re, const T *im, const T *rho0, int n0, int n1, int n2, const TdCell &c, double dV,
                          double *part, int nblk, double *out, cudaStream_t s) {
    dipole_kernel<T><<<nblk, 256, 0, s>>>(re, im, rho0, n0, n1, n2, c, dV, (long long)n0 * n1 * n2, part);
    sum3_partials_kernel<<<1, 256, 0, s>>>(part, nblk, out);
    return cudaGetLastError();
}

#define INST(T)                                                                                              \
    template cudaError_t launch_add_vu<T>(T *, const T *, const T *, double, double, long long, cudaStream_t); \
    template cudaError_t launch_abs2<T>(T *, const T *, const T *, long long, cudaStream_t);                 \
    template cudaError_t launch_add_scaled_scalar<T>(T *, const double *, double, long long, cudaStream_t);  \
    template cudaError_t launch_kick<T>(T *, T *, int, int, int, const TdCell &, const double *, cudaStream_t); \
    template cudaError_t launch_dipole<T>(const T *, const T *, const T *, int, int, int, const TdCell &,     \
                                          double, double *, int, double *, cudaStream_t);                    \
    template cudaError_t launch_hvp<T>(T *, const T *, const T *, const T *, const T *, double, double,      \
                                       double, long long, cudaStream_t);                                     \
    template cudaError_t launch_add_scalar<T>(T *, const double *, long long, cudaStream_t);                  \
    template cudaError_t launch_dot<T>(const T *, const T *, const T *, long long, double *, int, double *,    \
                                       cudaStream_t, bool);                                                  \
    template cudaError_t launch_axpby<T>(T *, const T *, double, double, long long, cudaStream_t);           \
    template cudaError_t launch_rotate<T>(T *, T *, const T *, const T *, double, double, long long,         \
                                          cudaStream_t);                                                     \
    template cudaError_t launch_grad<T>(T *, const T *, const T *, double, double, long long, cudaStream_t);  \
    template cudaError_t launch_square<T>(T *, T *, double, long long, cudaStream_t);                        \
    template cudaError_t launch_copy<T>(T *, const T *, long long, cudaStream_t);
INST(float)
INST(double)

}  // namespace ofdft
