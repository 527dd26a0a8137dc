// Shared-memory batched FFT engine: mixed radix 2/3/4/5/8/16 Stockham autosort.
//
// A CTA transforms B sequences of length n that live in shared memory with the
// batch index innermost: element e of sequence b sits at buf[e * ld + b].
// Consecutive threads take consecutive b, so with B >= 16 every pass reads and
// writes shared memory without bank conflicts.  Each pass stages its
// butterflies in registers (at most CAP complex values per thread) so the
// transform runs in place; the host picks the block size so that
// ceil((n/R) * B / threads) * R <= CAP for every radix R of the plan.
//
// Sign convention: DIR = -1 computes X_k = sum_j x_j e^{-2 pi i jk/n}
// (forward), DIR = +1 the unnormalised inverse.  Twiddles come from a table
// tw[k] = e^{-2 pi i k/n} built once in FP64 on the host and rounded once.
#pragma once

#include "common.cuh"

namespace ofdft {

struct FFTPlan {
    int n;
    int npass;
    int radix[OFDFT_MAX_PASS];
    int ns[OFDFT_MAX_PASS];      // product of the radices of the earlier passes
};

// ----------------------------------------------------------------- butterflies
template <int DIR, typename C> __device__ __forceinline__ void dft2(C *v) {
    C t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
}

template <int DIR, typename C> __device__ __forceinline__ void dft4x(C &a0, C &a1, C &a2, C &a3) {
    C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = cmul_si<DIR>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}
template <int DIR, typename C> __device__ __forceinline__ void dft4(C *v) { dft4x<DIR>(v[0], v[1], v[2], v[3]); }

template <int DIR, typename C> __device__ __forceinline__ void dft8(C *v) {
    typedef decltype(C::x) T;
    const T c = (T)0.7071067811865476;            // cos(pi/4)
    dft4x<DIR>(v[0], v[2], v[4], v[6]);           // E_0..E_3
    dft4x<DIR>(v[1], v[3], v[5], v[7]);           // O_0..O_3
    const T s = (T)DIR;
    // W8^1 = c (1 + s i), W8^2 = s i, W8^3 = c (-1 + s i)
    C o1 = cmake<C>(c * (v[3].x - s * v[3].y), c * (v[3].y + s * v[3].x));
    C o2 = cmul_si<DIR>(v[5]);
    C o3 = cmake<C>(-c * (v[7].x + s * v[7].y), c * (s * v[7].x - v[7].y));
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

template <int DIR, typename C> __device__ __forceinline__ void dft3(C *v) {
    typedef decltype(C::x) T;
    const T h = (T)0.8660254037844386;            // sin(2 pi/3)
    C t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    C m = cmake<C>(v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y);
    C n = cmul_si<DIR>(cscale(t2, h));
    v[0] = cadd(v[0], t1);
    v[1] = cadd(m, n);
    v[2] = csub(m, n);
}

template <int DIR, typename C> __device__ __forceinline__ void dft5(C *v) {
    typedef decltype(C::x) T;
    const T c1 = (T)0.30901699437494745, c2 = (T)-0.8090169943749473;
    const T s1 = (T)0.9510565162951535, s2 = (T)0.5877852522924732;
    C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]), t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    C m1 = cmake<C>(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
    C m2 = cmake<C>(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
    C n1 = cmul_si<DIR>(cmake<C>(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
    C n2 = cmul_si<DIR>(cmake<C>(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(m1, n1);
    v[4] = csub(m1, n1);
    v[2] = cadd(m2, n2);
    v[3] = csub(m2, n2);
}

// 16-point DFT as 4 x 4: DFT4 over n1 for each n2, twiddles W16^(n2 k1), DFT4
// over n2; X[k1 + 4 k2] = sum_n2 W4^(n2 k2) W16^(n2 k1) sum_n1 W4^(n1 k1) v[4 n1 + n2].
template <int DIR, typename C> __device__ __forceinline__ void dft16(C *v) {
    typedef decltype(C::x) T;
    const T s = (T)DIR;
    const T c8 = (T)0.9238795325112867, s8 = (T)0.3826834323650898, h = (T)0.7071067811865476;
#pragma unroll
    for (int n2 = 0; n2 < 4; n2++) dft4x<DIR>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    // v[n2 + 4 k1] holds A_n2[k1]; multiply by W16^(n2 k1), W16^e = cos(2 pi e/16) + s i sin(2 pi e/16)
    auto rot = [&](C &x, T cr, T si) {          // x *= (cr + s i si)
        const T xr = x.x, xi = x.y;
        x.x = xr * cr - s * xi * si;
        x.y = xi * cr + s * xr * si;
    };
    rot(v[5], c8, s8);          // e = 1
    rot(v[9], h, h);            // e = 2
    rot(v[13], s8, c8);         // e = 3
    rot(v[6], h, h);            // e = 2
    v[10] = cmul_si<DIR>(v[10]);// e = 4
    rot(v[14], -h, h);          // e = 6
    rot(v[7], s8, c8);          // e = 3
    rot(v[11], -h, h);          // e = 6
    rot(v[15], -c8, -s8);       // e = 9
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) dft4x<DIR>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // now v[4 k1 + k2] = X[k1 + 4 k2]: transpose the 4 x 4 index
    C t[16];
#pragma unroll
    for (int i = 0; i < 16; i++) t[i] = v[i];
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++)
#pragma unroll
        for (int k2 = 0; k2 < 4; k2++) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

template <int DIR, int R, typename C> __device__ __forceinline__ void dft(C *v) {
    if (R == 2) dft2<DIR>(v);
    else if (R == 3) dft3<DIR>(v);
    else if (R == 4) dft4<DIR>(v);
    else if (R == 5) dft5<DIR>(v);
    else if (R == 8) dft8<DIR>(v);
    else dft16<DIR>(v);
}

// ----------------------------------------------------------------- one pass
template <int DIR, int R, int CAP, typename C>
__device__ __forceinline__ void fft_pass(C *buf, int ld, int B, int n, int Ns, const C *tw) {
    constexpr int MB = CAP / R;
    const int nb = n / R;
    const int total = nb * B;
    const int stride = n / (Ns * R);
    const int nthr = blockDim.x;
    C v[MB][R];
    // CAP / R butterflies per thread, staged in registers between the read and
    // the write half so that the pass can run in place
#pragma unroll
    for (int q = 0; q < MB; q++) {
        const int idx = threadIdx.x + q * nthr;
        if (idx < total) {
            const int b = idx % B, j = idx / B, k = j % Ns;
#pragma unroll
            for (int r = 0; r < R; r++) {
                C x = buf[(j + r * nb) * ld + b];
                if (r > 0 && k > 0) {
                    C w = tw[r * k * stride];
                    if (DIR > 0) w.y = -w.y;
                    x = cmul(x, w);
                }
                v[q][r] = x;
            }
            dft<DIR, R>(v[q]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MB; q++) {
        const int idx = threadIdx.x + q * nthr;
        if (idx < total) {
            const int b = idx % B, j = idx / B, k = j % Ns;
            const int dst = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int r = 0; r < R; r++) buf[(dst + r * Ns) * ld + b] = v[q][r];
        }
    }
    __syncthreads();
}

// Full transform of B sequences (all threads of the CTA take part; the caller
// must __syncthreads() after filling buf).  On return buf holds the result.
// Kept out of line: one copy per (direction, precision) keeps the register
// allocation of the fused kernels that call it several times small.
template <int DIR, int CAP, typename C>
__device__ __noinline__ void fft_smem(C *buf, int ld, int B, const FFTPlan &p, const C *tw) {
    for (int s = 0; s < p.npass; s++) {
        const int R = p.radix[s], Ns = p.ns[s];
        if (R == 8) fft_pass<DIR, 8, CAP>(buf, ld, B, p.n, Ns, tw);
        else if (R == 4) fft_pass<DIR, 4, CAP>(buf, ld, B, p.n, Ns, tw);
        else if (R == 2) fft_pass<DIR, 2, CAP>(buf, ld, B, p.n, Ns, tw);
        else if (R == 3) fft_pass<DIR, 3, CAP>(buf, ld, B, p.n, Ns, tw);
        else fft_pass<DIR, 5, CAP>(buf, ld, B, p.n, Ns, tw);
    }
}


// ======================================================================
// Compile-time variant: length N, batch B (sequence stride 1, batch index
// innermost with element stride LD) and block size NT are template
// parameters, so every index, loop bound and twiddle stride is a constant.
// The radix sequence puts the largest power-of-two radix first (16 in FP32,
// 8 in FP64), then the remaining power of two, then 5s, then 3s.
namespace ct {

// radix sequence with power-of-two radix at most maxr (16 or 8): maxr-radix
// passes first, then one smaller power of two, then 5s, then 3s
constexpr int npass(int n, int maxr) {
    int c = 0, m = n, p2 = 0;
    while (m % 2 == 0) { m /= 2; p2++; }
    const int lr = maxr == 16 ? 4 : 3;
    c += p2 / lr + (p2 % lr ? 1 : 0);
    while (m % 5 == 0) { m /= 5; c++; }
    while (m % 3 == 0) { m /= 3; c++; }
    return c;
}

constexpr int radix(int n, int p, int maxr) {
    int m = n, p2 = 0;
    while (m % 2 == 0) { m /= 2; p2++; }
    const int lr = maxr == 16 ? 4 : 3;
    int rbig = p2 / lr, rem = p2 % lr;
    if (p < rbig) return maxr;
    p -= rbig;
    if (rem) {
        if (p == 0) return 1 << rem;
        p -= 1;
    }
    int n5 = 0;
    while (m % 5 == 0) { m /= 5; n5++; }
    if (p < n5) return 5;
    return 3;
}

constexpr int ns(int n, int p, int maxr) {
    int s = 1;
    for (int q = 0; q < p; q++) s *= radix(n, q, maxr);
    return s;
}

template <int DIR, int R, int N, int NS, int B, int LD, int NT, typename C>
__device__ __forceinline__ void pass(C *buf, const C *tw) {
    constexpr int NB = N / R, TOT = NB * B, Q = (TOT + NT - 1) / NT, STRIDE = N / (NS * R);
    C v[Q][R];
#pragma unroll
    for (int q = 0; q < Q; q++) {
        const int idx = threadIdx.x + q * NT;
        if (TOT % NT == 0 || idx < TOT) {
            const int b = idx % B, j = idx / B, k = j % NS;
#pragma unroll
            for (int r = 0; r < R; r++) {
                C x = buf[(j + r * NB) * LD + b];
                if (NS > 1 && r > 0) {
                    C w = tw[r * k * STRIDE];
                    if (DIR > 0) w.y = -w.y;
                    x = cmul(x, w);
                }
                v[q][r] = x;
            }
            dft<DIR, R>(v[q]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; q++) {
        const int idx = threadIdx.x + q * NT;
        if (TOT % NT == 0 || idx < TOT) {
            const int b = idx % B, j = idx / B, k = j % NS;
            const int dst = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; r++) buf[(dst + r * NS) * LD + b] = v[q][r];
        }
    }
    __syncthreads();
}

template <int DIR, int N, int B, int LD, int NT, int MAXR, int P, typename C>
__device__ __forceinline__ void passes(C *buf, const C *tw) {
    if constexpr (P < npass(N, MAXR)) {
        pass<DIR, radix(N, P, MAXR), N, ns(N, P, MAXR), B, LD, NT>(buf, tw);
        passes<DIR, N, B, LD, NT, MAXR, P + 1>(buf, tw);
    }
}

// B sequences of length N in buf (element e of sequence b at buf[e*LD + b]);
// the caller synchronises before the call.  MAXR caps the power-of-two radix
// (16: a 128-point transform is 16 x 8; 8: it is 8 x 8 x 2).
template <int DIR, int N, int B, int LD, int NT, int MAXR, typename C>
__device__ __forceinline__ void fft(C *buf, const C *tw) {
    passes<DIR, N, B, LD, NT, MAXR, 0>(buf, tw);
}

// Out-of-place form of the same passes: each butterfly reads its R inputs from
// `in` and writes its outputs to `out` at once, so nothing is held across a
// barrier (registers: one butterfly at a time) and a pass needs one barrier.
template <int DIR, int R, int N, int NS, int B, int LD, int NT, typename C>
__device__ __forceinline__ void pass_oop(const C *in, C *out, const C *tw) {
    constexpr int NB = N / R, TOT = NB * B, STRIDE = N / (NS * R);
#pragma unroll
    for (int idx0 = 0; idx0 < TOT; idx0 += NT) {
        const int idx = idx0 + threadIdx.x;
        if (TOT % NT == 0 || idx < TOT) {
            const int b = idx % B, j = idx / B, k = j % NS;
            C v[R];
#pragma unroll
            for (int r = 0; r < R; r++) {
                C x = in[(j + r * NB) * LD + b];
                if (NS > 1 && r > 0) {
                    C w = tw[r * k * STRIDE];
                    if (DIR > 0) w.y = -w.y;
                    x = cmul(x, w);
                }
                v[r] = x;
            }
            dft<DIR, R>(v);
            const int dst = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; r++) out[(dst + r * NS) * LD + b] = v[r];
        }
    }
    __syncthreads();
}

template <int DIR, int N, int B, int LD, int NT, int MAXR, int P, typename C>
__device__ __forceinline__ C *passes_oop(C *x, C *y, const C *tw) {
    if constexpr (P < npass(N, MAXR)) {
        pass_oop<DIR, radix(N, P, MAXR), N, ns(N, P, MAXR), B, LD, NT>(x, y, tw);
        return passes_oop<DIR, N, B, LD, NT, MAXR, P + 1>(y, x, tw);
    } else {
        return x;
    }
}

// B sequences of length N in x (layout as fft above), y a scratch buffer of the
// same size; returns the buffer that holds the transform (x or y by the parity
// of the pass count).  The caller synchronises before the call.
template <int DIR, int N, int B, int LD, int NT, int MAXR, typename C>
__device__ __forceinline__ C *fft_oop(C *x, C *y, const C *tw) {
    return passes_oop<DIR, N, B, LD, NT, MAXR, 0>(x, y, tw);
}

}  // namespace ct
}  // namespace ofdft
