// Kernel templates of one energy/potential evaluation (pipeline in eval.cuh).
//
// Every FFT-carrying kernel is written once against an FFT policy P:
//   RtPolicy<T, AX>              sizes, batch and plan read from EvalArgs (any 2^a3^b5^c)
//   CtPolicy<T, N, B, LD, NT>    size, batch, batch stride and block size fixed at
//                                compile time (specialised instantiations)
// so the physics is shared and only the transform is specialised.
#pragma once

#include "eval.cuh"
#include "gnl_fit.cuh"

#include <type_traits>

namespace ofdft {

// ======================================================================= policies
template <typename T, int AX> struct RtPolicy {
    typedef typename Vec2<T>::type C;
    static constexpr bool ct = false, oop = false;
    static constexpr int N_ = 0, B_ = 0, NT_ = 0;
    static constexpr int max_threads = kMaxThreads, min_blocks = 1, min_blocks_ax0 = 1;
    __device__ static int n(const EvalArgs<T> &a) { return AX == 0 ? a.n0 : (AX == 1 ? a.n1 : a.n2); }
    __device__ static int B(const EvalArgs<T> &a) { return AX == 0 ? a.TW0 : (AX == 1 ? a.TW1 : a.Brow); }
    __device__ static int ld(const EvalArgs<T> &a) { return AX == 2 ? a.Brow + 1 : B(a); }
    __device__ static int nt() { return blockDim.x; }
    template <int DIR> __device__ static void fft(C *buf, const EvalArgs<T> &a, const C *tw) {
        fft_smem<DIR, Cap<T>::value>(buf, ld(a), B(a), AX == 0 ? a.p0 : (AX == 1 ? a.p1 : a.p2), tw);
    }
    // transform of x with y as scratch; returns the buffer holding the result (here x)
    template <int DIR> __device__ static C *fft2(C *x, C *, const EvalArgs<T> &a, const C *tw) {
        fft<DIR>(x, a, tw);
        return x;
    }
};

template <typename T, int N, int B__, int LD_, int NT__, int MAXR = (sizeof(T) == 4 ? 16 : 8), int MINB = 0,
          bool OOP = true>
struct CtPolicy {
    typedef typename Vec2<T>::type C;
    static constexpr bool ct = true, oop = OOP;
    static constexpr int N_ = N, B_ = B__, NT_ = NT__;
    // register budget: at least 768 resident threads per SM (24 warps)
    static constexpr int max_threads = NT__;
    static constexpr int min_blocks = MINB ? MINB : ((768 / NT__) > 0 ? 768 / NT__ : 1);
    // the reciprocal-space kernel holds more live state: at least 512 threads per SM
    static constexpr int min_blocks_ax0 = MINB ? MINB : ((512 / NT__) > 0 ? 512 / NT__ : 1);
    __device__ static constexpr int n(const EvalArgs<T> &) { return N; }
    __device__ static constexpr int B(const EvalArgs<T> &) { return B__; }
    __device__ static constexpr int ld(const EvalArgs<T> &) { return LD_; }
    __device__ static constexpr int nt() { return NT__; }
    template <int DIR> __device__ static void fft(C *buf, const EvalArgs<T> &, const C *tw) {
        ct::fft<DIR, N, B__, LD_, NT__, MAXR>(buf, tw);
    }
    // x transformed with y as scratch (out of place unless OOP is false); returns the
    // buffer holding the result
    template <int DIR> __device__ static C *fft2(C *x, C *y, const EvalArgs<T> &, const C *tw) {
        if constexpr (OOP) {
            return ct::fft_oop<DIR, N, B__, LD_, NT__, MAXR>(x, y, tw);
        } else {
            ct::fft<DIR, N, B__, LD_, NT__, MAXR>(x, tw);
            return x;
        }
    }
};

// ======================================================================= G_NL
// Lindhard-derived WT kernel (Sec. 2.3, the G_NL definition below Eq. MGP):
//   G_NL(eta) = 1/F(eta) - 3 eta^2 - 1,
//   F(eta)    = 1/2 + (1 - eta^2)/(4 eta) ln|(1+eta)/(1-eta)|.
// Below eta = 1/2 and above eta = 2 the exact series of F in y = eta^2
// (resp. x = 1/eta^2) are summed, with the numerator 1 - (1 + 3 eta^2) F
// expanded term by term so that nothing cancels (a_m = 1/(4 m^2 - 1)):
//   eta < 1/2:  F = 1 - sum_m a_m y^m,   num = -(8/3) y + sum_{m>=2} (a_m + 3 a_{m-1}) y^m
//   eta > 2  :  F = sum_m a_m x^m,       num = -sum_{m>=1} (a_m + 3 a_{m+1}) x^m
// and G_NL = num / F.  The loops are unrolled, so every coefficient folds to
// a constant.  (These series serve the FP64 kernels; the FP32-mixed kernels use the
// polynomial forms of gnl_fit.cuh in the same two ranges.)
template <typename T> struct GnlTerms { static constexpr int value = 10; };
template <> struct GnlTerms<double> { static constexpr int value = 28; };

// Divisions and the logarithm of the kernel: in the FP32-mixed path the fast
// intrinsics (at most 2 ulp for these operand ranges, against the few ulp the
// FP32 sums already carry); FP64 keeps IEEE division and log.
__device__ __forceinline__ float gdiv(float a, float b) { return __fdividef(a, b); }
__host__ __device__ __forceinline__ double gdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float glog(float x) { return __logf(x); }
__host__ __device__ __forceinline__ double glog(double x) { return log(x); }
__host__ __device__ __forceinline__ double gabs(double x) { return fabs(x); }
__device__ __forceinline__ float gabs(float x) { return fabsf(x); }

// closed form between the series ranges (1/2 <= eta <= 2)
template <typename T> __host__ __device__ __forceinline__ T gnl_mid(T eta) {
    const T d = (T)1 - eta;
    if (gabs(d) < (T)1e-12) return (T)-2;
    const T F = (T)0.5 + gdiv((T)1 - eta * eta, (T)4 * eta) * glog(gabs(gdiv((T)1 + eta, d)));
    return gdiv((T)1, F) - (T)3 * eta * eta - (T)1;
}

// (host and device: the FP64 form also builds the MGP correction table).  The FP32-mixed
// kernels take G_NL below eta = 1/2 and above eta = 2 from the degree-6 polynomials of
// gnl_fit.cuh (y S(y) and L(1/eta^2), within 2e-10 of the closed form: below FP32 rounding,
// in 7 fused multiply-adds instead of two 10-term series and a division).
template <typename T> __host__ __device__ __forceinline__ T gnl(T eta) {
#ifdef __CUDA_ARCH__
    if constexpr (sizeof(T) == 4) {
        // both polynomials and the select carry no branch, so that the evaluations of a
        // thread's several G vectors interleave; only 1/2 <= eta <= 2 branches
        const float y = eta * eta;
        const float gs = y * gnl_small_s(y), gl = gnl_large_l(gdiv(1.0f, y));
        float g = eta < 0.5f ? gs : gl;
        if (eta >= 0.5f && eta <= 2.0f) g = gnl_mid(eta);
        return g;
    } else
#endif
    {
        constexpr int nt = GnlTerms<T>::value;
        // both series are sums sum_{m=1}^{nt} c_m z^m, evaluated by Horner's rule with fused
        // multiply-adds: p = c_nt, p = p z + c_m (m = nt-1..1), sum = p z
        if (eta < (T)0.5) {
            const T y = eta * eta;
            T pF = (T)(1.0 / (4.0 * nt * nt - 1.0));
            T pN = (T)(1.0 / (4.0 * nt * nt - 1.0) + 3.0 / (4.0 * (nt - 1) * (nt - 1) - 1.0));
#pragma unroll
            for (int m = nt - 1; m >= 1; m--) {
                const double am = 1.0 / (4.0 * m * m - 1.0);
                const double lo = (m >= 2) ? am + 3.0 / (4.0 * (m - 1) * (m - 1) - 1.0) : -8.0 / 3.0;
                pF = pF * y + (T)am;
                pN = pN * y + (T)lo;
            }
            return gdiv(pN * y, (T)1 - pF * y);
        } else if (eta > (T)2) {
            const T x = gdiv((T)1, eta * eta);
            T pF = (T)(1.0 / (4.0 * nt * nt - 1.0));
            T pN = (T)(1.0 / (4.0 * nt * nt - 1.0) + 3.0 / (4.0 * (nt + 1) * (nt + 1) - 1.0));
#pragma unroll
            for (int m = nt - 1; m >= 1; m--) {
                const double am = 1.0 / (4.0 * m * m - 1.0);
                const double hi = am + 3.0 / (4.0 * (m + 1) * (m + 1) - 1.0);
                pF = pF * x + (T)am;
                pN = pN * x + (T)hi;
            }
            return -gdiv(pN, pF);          // the common factor x of both sums cancels
        }
        return gnl_mid(eta);
    }
}

// MGP correction J_y(eta) by linear interpolation in u = eta / (1 + eta) of the table a.mgp_tab
// (n points, u = i/(n-1)); the kernel value of Eq. MGP is C_WT ((1 - x) G_NL + 3 x y J_y).
template <typename T> __device__ __forceinline__ T mgp_j(const T *tab, int n, T eta) {
    const T pos = gdiv(eta, (T)1 + eta) * (T)(n - 1);
    int i = (int)pos;
    i = i > n - 2 ? n - 2 : i;
    const T f = pos - (T)i, t0 = tab[i];
    return t0 + f * (tab[i + 1] - t0);
}

// The kernel of Eq. WT (C_WT G_NL) or of Eq. MGP at eta = |G| / (2k)
template <typename T, bool MGP> __device__ __forceinline__ T kernel_value(const EvalArgs<T> &a, T eta) {
    T G = gnl(eta);
    if constexpr (MGP) G = a.mgp_1mx * G + a.mgp_3xy * mgp_j(a.mgp_tab, a.mgp_n, eta);
    return (T)kCWT * G;
}

// The FP32 kernel at eta > 2, exactly as kernel_value<float, false> gives it there, for a warp
// whose every eta is known to lie above 2 (most G vectors of a bulk grid): the polynomial in
// 1/eta^2 alone, without the other range's polynomial, the select and the closed-form test.
__device__ __forceinline__ float kernel_value_large(float eta) {
    return (float)kCWT * gnl_large_l(gdiv(1.0f, eta * eta));
}
// whether the calling warp may use kernel_value_large for every element whose |G| is at least
// gmin (the caller's smallest |G|) at eta = |G| hk; always false for MGP and FP64 kernels
template <typename T, bool MGP> __device__ __forceinline__ bool warp_all_large(T gmin, T hk) {
    if constexpr (MGP || sizeof(T) != 4) return false;
    else return __all_sync(__activemask(), gmin * hk > (T)2);
}

// ======================================================================= LDA exchange-correlation
// Dirac exchange and the Perdew-Zunger (1981) fit of the Ceperley-Alder correlation,
// spin unpolarised (the xc of the paper's benchmarks, Sec. 3.1), with
// r_s = (3 / (4 pi rho))^(1/3):
//   eps_x = -(3/4) (3/pi)^(1/3) rho^(1/3),  V_x = (4/3) eps_x
//   r_s >= 1: eps_c = g / (1 + b1 sqrt(r_s) + b2 r_s),
//             V_c = eps_c (1 + (7/6) b1 sqrt(r_s) + (4/3) b2 r_s) / (1 + b1 sqrt(r_s) + b2 r_s)
//   r_s <  1: eps_c = A ln r_s + B + C r_s ln r_s + D r_s,
//             V_c = A ln r_s + (B - A/3) + (2/3) C r_s ln r_s + ((2 D - C)/3) r_s
// (V = d(rho eps)/d rho).  Returns rho eps_xc; v receives V_xc.
template <typename T> __device__ __forceinline__ T lda_xc(T rho, T &v) {
    constexpr double g = -0.1423, b1 = 1.0529, b2 = 0.3334, A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116;
    constexpr double cx = 0.7385587663820224;                 // (3/4) (3/pi)^(1/3)
    constexpr double crs = 0.6203504908994001;                // (3 / (4 pi))^(1/3)
    const T c = dcbrt(rho);
    const T ex = -(T)cx * c;
    const T rs = (T)crs / c;
    T ec, vc;
    if (rs >= (T)1) {
        const T sq = dsqrt(rs);
        const T den = (T)1 + (T)b1 * sq + (T)b2 * rs;
        ec = (T)g / den;
        vc = ec * ((T)1 + (T)(7.0 / 6.0 * b1) * sq + (T)(4.0 / 3.0 * b2) * rs) / den;
    } else {
        const T l = dlog(rs);
        ec = (T)A * l + (T)B + (T)C * rs * l + (T)D * rs;
        vc = (T)A * l + (T)(B - A / 3.0) + (T)(2.0 / 3.0 * C) * rs * l + (T)((2.0 * D - C) / 3.0) * rs;
    }
    v = (T)(4.0 / 3.0) * ex + vc;
    return rho * (ex + ec);
}

// ======================================================================= energy partials
// An FP32-mixed per-thread energy partial: terms summed in T over a short run (a tile's
// elements of one thread, a few grid points) and folded into FP64 once (the default), or,
// with the exact-sums test option, every term converted and added in FP64.  FP64 builds
// add every term in FP64 either way.
template <typename T, bool XS> struct Part {
    T f = (T)0;
    double d = 0.0;
    __device__ __forceinline__ void add(T v) {
        if constexpr (XS) d += (double)v;
        else f += v;
    }
    __device__ __forceinline__ double value() const { return XS ? d : (double)f; }
};

// ======================================================================= helpers
template <typename T> __device__ __forceinline__ int knot_interval(T kc, const T *knots, int M) {
    // largest j in [0, M-2] with knots[j] <= kc (binary search; kc already clamped)
    int lo = 0, hi = M - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (knots[mid] <= kc) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Knot interval of a clamped kF for geometric knots made from the density (s1: the end
// knots are kF of the minimum and maximum density):
// j from ln(kF / k_1) / ln(r) (ilr = 1 / ln r, r the knot ratio), then one step up and one
// down with the binary search's rule, which gives its result exactly whenever the guess is
// within one interval (ln r >= 1e-4 keeps the guess's rounding below a hundredth of an
// interval).  ilr = 0 (caller-given or arithmetic knots, near-equal knots) uses the search.
template <typename T> __device__ __forceinline__ T knot_log_scale(const EvalArgs<T> &a, const T *knots, int M) {
    if (a.frozen || a.knot_spacing != 0 || M < 3) return (T)0;
    const T lr = glog(gdiv(knots[M - 1], knots[0])) / (T)(M - 1);
    return lr > (T)1e-4 ? (T)1 / lr : (T)0;
}
template <typename T> __device__ __forceinline__ int knot_interval_fast(T kc, const T *knots, int M, T ilr) {
    if (ilr == (T)0) return knot_interval(kc, knots, M);
    int j = (int)(glog(gdiv(kc, knots[0])) * ilr);
    j = j < 0 ? 0 : (j > M - 2 ? M - 2 : j);
    if (j < M - 2 && knots[j + 1] <= kc) j++;
    if (j > 0 && knots[j] > kc) j--;
    return j;
}

// rho^alpha, rho^beta and kF = (3 pi^2 rho)^(1/3) of a floored density xf.  For the
// Lindhard-consistent exponents alpha = beta = 5/6 (the default functional) rho^(5/6) is
// formed as sqrt(rho) cbrt(rho) and kF from the same cube root: two roots per point in
// place of a general power and a second root.  Every kernel that places a point on the
// knots calls this, so the forward and the inverse rows agree on the point's interval.
template <typename T>
__device__ __forceinline__ void point_powers(const EvalArgs<T> &a, T xf, T &ra, T &rb, T &kf) {
    if (a.alpha == (T)(5.0 / 6.0) && a.beta == a.alpha) {
        const T c = dcbrt(xf);
        ra = rb = dsqrt(xf) * c;
        kf = (T)kCbrtThreePi2 * c;
    } else {
        ra = dpow(xf, a.alpha);
        rb = (a.beta == a.alpha) ? ra : dpow(xf, a.beta);
        kf = dcbrt((T)kThreePi2 * xf);
    }
}

// Whether kF(x) lies in the knot range [k_1, k_M] (the exact potential's slope term is
// applied only there).  With knots made from the density (s1) the end knots are kF of the
// floored min and max density, and kF is monotone, so the test is taken on the density
// itself: points at the minimum or maximum density (every point of a floored vacuum) are
// then inside in any precision, as they are in exact arithmetic.  Caller-given knots are
// compared in kF.
template <typename T>
__device__ __forceinline__ bool in_knot_range(const EvalArgs<T> &a, T xf, T kf, T klo, T khi, T rlo, T rhi) {
    return a.frozen ? (kf >= klo && kf <= khi) : (xf >= rlo && xf <= rhi);
}

// ======================================================================= knots (s1)
// FP64 reduction of the stats partials (read through L2: they were written by
// other blocks of the same launch), the mean density, E_TF, and the M knots
// between kF(min rho) and kF(max rho).  Called by the last stats block.
template <typename T>
__device__ __forceinline__ void knots_from_partials(const EvalArgs<T> &a, double *sd, T *st) {
    __shared__ double kn[OFDFT_MAX_KNOTS];
    __shared__ double smm[2];
    double s_rho = 0.0, s_tf = 0.0, s_xc = 0.0;
    T mn = (T)3.0e38, mx = (T)-3.0e38;
    for (int b = threadIdx.x; b < a.nb_stats; b += blockDim.x) {
        s_rho += __ldcg(a.part_stats + 3 * b);
        s_tf += __ldcg(a.part_stats + 3 * b + 1);
        s_xc += __ldcg(a.part_stats + 3 * b + 2);
        const T x = __ldcg(a.part_minmax + 2 * b), y = __ldcg(a.part_minmax + 2 * b + 1);
        mn = x < mn ? x : mn;
        mx = y > mx ? y : mx;
    }
    double r[3] = {s_rho, s_tf, s_xc};
    block_sum_n<3>(r, sd);
    s_rho = r[0];
    s_tf = r[1];
    s_xc = r[2];
    mn = block_min(mn, st);
    mx = block_max(mx, st);
    const double fl = (double)a.floor_;
    if (threadIdx.x == 0) {
        a.scal[S_SUM_RHO] = s_rho;
        a.scal[S_SUM_TF] = s_tf;
        a.scal[S_RHO_MIN] = (double)mn;
        a.scal[S_RHO_MAX] = (double)mx;
        const double mean = s_rho / (double)a.N;
        a.scal[S_RHO_MEAN] = mean;
        a.scal[S_KF_WT] = cbrt(kThreePi2 * (mean > fl ? mean : fl));
        a.energies[E_TF] = (a.terms & 1u) ? kCTF * s_tf * a.dV : 0.0;
        a.energies[E_XC] = (a.terms & 32u) ? s_xc * a.dV : 0.0;
        smm[0] = (double)mn;
        smm[1] = (double)mx;
    }
    __syncthreads();
    if (!((a.terms & 4u) && a.kernel == 0 && a.M >= 2)) return;
    // s1: one thread per knot, in FP64
    const int M = a.M, m = threadIdx.x;
    if (m < M) {
        double k;
        if (!a.frozen) {
            const double kmin = cbrt(kThreePi2 * (smm[0] > fl ? smm[0] : fl));
            const double kmax = cbrt(kThreePi2 * (smm[1] > fl ? smm[1] : fl));
            if (m == 0) k = kmin;
            else if (m == M - 1) k = kmax;
            else if (a.knot_spacing == 0) k = kmin * exp((double)m * (log(kmax / kmin) / (double)(M - 1)));
            else k = kmin + (double)m * ((kmax - kmin) / (double)(M - 1));
            a.knots_d[m] = k;
        } else {
            k = a.knots_d[m];
        }
        kn[m] = k;
        a.knots_t[m] = (T)k;
    }
    __syncthreads();
    if (m + 1 < M) {
        const double dk = kn[m + 1] - kn[m];
        a.invdk_t[m] = dk > 0.0 ? (T)(1.0 / dk) : (T)0;
    }
}

// ======================================================================= stats (s1 input)
template <typename T, bool XS>
__device__ __forceinline__ void stats_body(const EvalArgs<T> &a, const int bid, const int nblk) {
    __shared__ double sd[3 * 32];
    __shared__ T st[32];
    double s_rho = 0.0, s_tf = 0.0, s_xc = 0.0;
    T mn = (T)3.0e38, mx = (T)-3.0e38;
    int bad = 0;
    const bool xc = a.terms & 32u;
    // groups of 4 consecutive points: summed in T, then added in FP64 (keeps the FP64 pipe
    // idle); U groups a grid stride apart per iteration, all loaded before any is used
    constexpr int U = 4;
    const long long ng = (a.N + 3) / 4, stride = (long long)nblk * blockDim.x;
    const bool vec = (reinterpret_cast<uintptr_t>(a.rho) % (4 * sizeof(T)) == 0) && (a.N % 4 == 0);
    for (long long g0 = bid * (long long)blockDim.x + threadIdx.x; g0 < ng; g0 += U * stride) {
        T x[U][4];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long gi = g0 + u * stride;
            if (vec && gi < ng) {
                load4(a.rho + 4 * gi, x[u]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; q++) x[u][q] = (4 * gi + q < a.N) ? a.rho[4 * gi + q] : (T)0;
            }
        }
        // FP32-mixed: the U groups are summed in FP32 too (one FP64 add per sum per iteration);
        // with exact sums every point is added in FP64
        T r16 = 0, t16 = 0, x16 = 0;
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long gi = g0 + u * stride;
            T r4 = 0, t4 = 0, x4 = 0;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                if (4 * gi + q < a.N) {
                    const T xv = x[u][q];
                    if (!(xv >= (T)0) || !(xv < (T)3.0e38)) bad = 1;      // NaN, Inf or negative
                    const T c = dcbrt(xv);
                    T xe = 0;
                    if (xc) {
                        T vxc;
                        xe = lda_xc(xv > a.floor_ ? xv : a.floor_, vxc);   // rho eps_xc
                    }
                    if constexpr (sizeof(T) == 4 && XS) {
                        s_rho += (double)xv;
                        s_tf += (double)(xv * c * c);
                        s_xc += (double)xe;
                    } else {
                        r4 += xv;
                        t4 += xv * c * c;                                  // rho^(5/3)
                        x4 += xe;
                    }
                    mn = xv < mn ? xv : mn;
                    mx = xv > mx ? xv : mx;
                }
            }
            if (sizeof(T) == 4) {
                r16 += r4;
                t16 += t4;
                x16 += x4;
            } else {
                s_rho += (double)r4;
                s_tf += (double)t4;
                s_xc += (double)x4;
            }
        }
        if (sizeof(T) == 4) {
            s_rho += (double)r16;
            s_tf += (double)t16;
            s_xc += (double)x16;
        }
    }
    double r[3] = {s_rho, s_tf, s_xc};
    if constexpr (sizeof(T) == 4 && !XS) block_sum_n_f32warp<3>(r, sd);
    else block_sum_n<3>(r, sd);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) a.part_stats[3 * bid + k] = r[k];
    mn = block_min(mn, st);
    if (threadIdx.x == 0) a.part_minmax[2 * bid] = mn;
    mx = block_max(mx, st);
    if (threadIdx.x == 0) a.part_minmax[2 * bid + 1] = mx;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0 && bad) a.scal[S_BAD] = 1.0;
    // the last block to finish reduces every block's partials and makes the knots (thread 0
    // wrote this block's partials and flag, so only it orders them before the ticket)
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(a.ticket, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    knots_from_partials(a, sd, st);
    if (threadIdx.x == 0) *a.ticket = 0u;           // ready for the next evaluation
}

// ======================================================================= row forward (R2C along n2)
// Tile: B pairs of consecutive rows (flattened row r = i0*n1 + i1); pair p holds
// rows 2p and 2p+1, packed as z = x_2p + i x_2p+1 for one complex FFT of length n2.
// Per-point arrays use the layout o = i2 * 2B + rr (rr = row within the tile), so
// the two points of a pair are adjacent and a thread reads them as one vector.
// The density is staged through shared memory ([rr][pitch], pitch odd) so that
// both the global loads and the shared-memory transposition are conflict free.
template <typename T, class P>
__device__ __forceinline__ void row_fwd_body(const EvalArgs<T> &a, const int bid, const int nblk) {
    typedef typename Vec2<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = P::n(a), B = P::B(a), ld = P::ld(a), NT = P::nt();
    const int n2h = n / 2 + 1;
    const int PP = 2 * B * n, pitch = row_pitch(n);
    C *tw = (C *)smem_raw;
    C *buf = tw + n;
    T *stg = (T *)buf;
    T *sx = (T *)((unsigned char *)buf + row_buf_bytes<T>(n, B));
    T *sra = sx + PP;
    T *srb = sra + PP;
    T *st = srb + PP;
    unsigned char *sj = (unsigned char *)(st + PP);
    __shared__ T sk[OFDFT_MAX_KNOTS];

    const long long R = (long long)a.n0 * a.n1;
    const long long row0 = 2LL * B * bid;
    for (int i = threadIdx.x; i < n; i += NT) tw[i] = a.tw2[i];
    const bool lwt = (a.terms & 4u) && a.kernel == 0;
    const int M = a.M;
    if (lwt)
        for (int i = threadIdx.x; i < M; i += NT) sk[i] = a.knots_t[i];
    const T mean = (T)a.scal[S_RHO_MEAN];
    for (int idx = threadIdx.x; idx < PP; idx += NT) {
        const int rr = idx / n, i2 = idx - rr * n;
        const long long row = row0 + rr;
        stg[rr * pitch + i2] = (row < R) ? a.rho[row * n + i2] : (T)0;
    }
    __syncthreads();
    const T ilr = lwt ? knot_log_scale(a, sk, M) : (T)0;
    // per-point quantities (o = idx = i2 * 2B + rr)
    for (int o = threadIdx.x; o < PP; o += NT) {
        const int rr = o % (2 * B), i2 = o / (2 * B);
        const T x = stg[rr * pitch + i2];
        sx[o] = x;
        if (a.terms & 4u) {
            const T xf = x > a.floor_ ? x : a.floor_;
            T ra, rb, kf;
            point_powers(a, xf, ra, rb, kf);
            sra[o] = ra;
            srb[o] = rb;
            if (lwt) {
                kf = kf < sk[0] ? sk[0] : (kf > sk[M - 1] ? sk[M - 1] : kf);
                const int j = knot_interval_fast(kf, sk, M, ilr);
                sj[o] = (unsigned char)j;
                st[o] = (kf - sk[j]) * a.invdk_t[j];
            }
        }
    }
    __syncthreads();
    for (int ci = 0; ci < a.nfwd; ci++) {
        const int ch = a.fwd_ch[ci];
        for (int idx = threadIdx.x; idx < n * B; idx += NT) {
            const int b = idx % B, i2 = idx / B;
            const int o = 2 * idx;                      // = i2 * 2B + 2b
            T v[2];
#pragma unroll
            for (int s = 0; s < 2; s++) {
                T f;
                if (ch == CH_HPP) f = sx[o + s] - mean;
                else if (ch == CH_VW) f = dsqrt(sx[o + s] > (T)0 ? sx[o + s] : (T)0);
                else if (ch == CH_NL) f = srb[o + s];
                else if (!lwt) f = sra[o + s];                     // WT: rho^alpha field
                else {
                    const int m = ch - CH_KNOT0, j = sj[o + s];
                    const T t = st[o + s];
                    f = (j == m) ? ((T)1 - t) * sra[o + s] : ((j == m - 1) ? t * sra[o + s] : (T)0);
                }
                if (row0 + 2 * b + s >= R) f = 0;
                v[s] = f;
            }
            buf[i2 * ld + b] = cmake<C>(v[0], v[1]);
        }
        __syncthreads();
        P::template fft<-1>(buf, a, tw);
        // unpack X_2p[k] = (Z_k + conj Z_{n-k})/2, X_2p+1[k] = (Z_k - conj Z_{n-k})/(2i)
        C *out = a.chan + (size_t)ch * a.NH;
        for (int idx = threadIdx.x; idx < n2h * B; idx += NT) {
            const int b = idx / n2h, k = idx - b * n2h;
            const C A = buf[k * ld + b];
            const C Bv = buf[((n - k) % n) * ld + b];
            const long long r0 = row0 + 2 * b;
            if (r0 < R) out[r0 * n2h + k] = cmake<C>((T)0.5 * (A.x + Bv.x), (T)0.5 * (A.y - Bv.y));
            if (r0 + 1 < R) out[(r0 + 1) * n2h + k] = cmake<C>((T)0.5 * (A.y + Bv.y), (T)0.5 * (Bv.x - A.x));
        }
        __syncthreads();
    }
}

// ======================================================================= pencil (C2C along n1)

// Persistent: block b handles tiles t = b, b + gridDim.x, ... of the flattened
// (channel, column tile) range; a tile is TW consecutive columns c = k0 * n2h + k2
// (flattened over the planes, so only the last tile of a channel is ragged) times
// all n1 rows.  The next tile is prefetched with cp.async into the second of two
// buffers while the current one is transformed and stored.
template <typename T, int DIR, class P>
__device__ __forceinline__ void pencil1_body(const EvalArgs<T> &a, const int bid, const int nblk) {
    typedef typename Vec2<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = P::n(a), TW = P::B(a), n2h = a.n2h, NT = P::nt();
    C *tw = (C *)smem_raw;
    C *const b0 = tw + n, *const b1 = tw + n + n * TW;   // prefetch ping-pong (no indexed array:
    C *scr = tw + n + 2 * n * TW;                        // it would live in local memory); scratch
    for (int i = threadIdx.x; i < n; i += NT) tw[i] = a.tw1[i];
    const long long ncols = (long long)a.n0 * n2h;
    const int ntile = (int)((ncols + TW - 1) / TW);
    const int nch = DIR < 0 ? a.ncol : a.ncol_inv;
    const int total = ntile * nch;
    const long long plane = (long long)n * n2h;
    auto tile_base = [&](int t, long long &c0) -> C * {
        const int ci = t / ntile;
        c0 = (long long)(t - ci * ntile) * TW;
        const int ch = DIR < 0 ? a.col_ch[ci] : a.col_inv_ch[ci];
        return a.chan + (size_t)ch * a.NH;
    };
    // With a compile-time policy NT is a multiple of TW, so a thread keeps one column w of
    // every tile: its (k0, k2) is found once per tile with a 32-bit division (columns number
    // fewer than 2^31) and each element adds only its row offset.
    constexpr bool fixed_col = P::ct && P::B_ > 0 && (P::NT_ % (P::B_ > 0 ? P::B_ : 1) == 0);
    auto col_offset = [&](long long c0, bool &ok) -> size_t {
        const int c = (int)c0 + threadIdx.x % TW;
        ok = c < ncols;
        const int k0 = c / n2h, k2 = c - k0 * n2h;
        return ok ? (size_t)k0 * plane + k2 : 0;
    };
    auto prefetch = [&](int t, C *dst) {
        long long c0;
        const C *base = tile_base(t, c0);
        if constexpr (fixed_col) {
            bool ok;
            const C *src = base + col_offset(c0, ok);
            for (int idx = threadIdx.x; idx < n * TW; idx += NT)
                cp_async<sizeof(C)>(dst + idx, src + (ok ? (size_t)(idx / TW) * n2h : 0), ok);
        } else {
            for (int idx = threadIdx.x; idx < n * TW; idx += NT) {
                const int w = idx % TW, i = idx / TW;
                const long long c = c0 + w;
                const long long k0 = c / n2h, k2 = c - k0 * n2h;
                const bool ok = c < ncols;
                cp_async<sizeof(C)>(dst + idx, base + (ok ? k0 * plane + (long long)i * n2h + k2 : 0), ok);
            }
        }
        cp_async_commit();
    };
    int it = 0;
    if (bid < total) prefetch(bid, b0);
    for (int t = bid; t < total; t += nblk, it++) {
        C *cur = (it & 1) ? b1 : b0;
        cp_async_wait<0>();
        __syncthreads();
        if (t + (int)nblk < total) prefetch(t + nblk, (it & 1) ? b0 : b1);
        const C *res = P::template fft2<DIR>(cur, scr, a, tw);
        long long c0;
        C *base = tile_base(t, c0);
        if constexpr (fixed_col) {
            bool ok;
            C *dstc = base + col_offset(c0, ok);
            if (ok)
                for (int idx = threadIdx.x; idx < n * TW; idx += NT) dstc[(size_t)(idx / TW) * n2h] = res[idx];
        } else {
            for (int idx = threadIdx.x; idx < n * TW; idx += NT) {
                const int w = idx % TW, i = idx / TW;
                const long long c = c0 + w;
                const long long k0 = c / n2h, k2 = c - k0 * n2h;
                if (c < ncols) base[k0 * plane + (long long)i * n2h + k2] = res[idx];
            }
        }
    }
    cp_async_wait<0>();
}

// ======================================================================= axis 0 + reciprocal space
// Tile: TW consecutive columns (k1, k2) of the plane, all n0 values of k0.
// The channel tiles are read in a fixed order (Hartree+PP, vW, rho^beta, then
// the knot fields); the next one is prefetched asynchronously into the second
// of two rotating buffers while the current one is transformed.
// Partials per block: [0] sum_G w |rho_hat|^2/G^2, [1] sum_G w G^2 |psi_hat|^2,
// [2] sum_G w Re(conj(rho_hat) V_ext), [3] nonlocal energy in G space.
template <typename T, class P, bool MGP, bool XS = false>
__device__ __forceinline__ void axis0_body(const EvalArgs<T> &a, const int bid, const int nblk) {
    typedef typename Vec2<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sd[4 * 32];
    __shared__ T cvec[64][3];
    __shared__ T cw[64];
    __shared__ T sk[OFDFT_MAX_KNOTS];
    __shared__ int order[kMaxChan];
    const int n = P::n(a), TW = P::B(a), n2h = a.n2h, NT = P::nt();
    const long long PL = (long long)a.n1 * n2h;      // columns per plane
    const int NTILE = n * TW;
    C *tw = (C *)smem_raw;
    C *xa = tw + n, *xb = tw + n + NTILE;            // rotating load buffers (slots 0, 1)
    C *Rr = xb + NTILE;
    C *A = Rr + NTILE;
    C *scr = A + NTILE;                              // scratch of the out-of-place transforms
    T *gn = (T *)(scr + (P::oop ? NTILE : 0));
    const bool lwt = a.kernel == 0;
    const bool exact = a.nlpot == 0;
    // the channels this block reads, in processing order
    int nord = 0;
    if (a.terms & (8u | 16u)) nord++;
    if (a.terms & 2u) nord++;
    if (a.terms & 4u) nord += 1 + (!lwt ? 1 : (exact ? a.M : 0));
    if (threadIdx.x == 0) {
        int q = 0;
        if (a.terms & (8u | 16u)) order[q++] = CH_HPP;
        if (a.terms & 2u) order[q++] = CH_VW;
        if (a.terms & 4u) {
            order[q++] = CH_NL;
            if (!lwt) order[q++] = CH_KNOT0;
            else if (exact)
                for (int m = 0; m < a.M; m++) order[q++] = CH_KNOT0 + m;
        }
    }
    const long long c0 = (long long)bid * TW;
    auto prefetch = [&](C *dst, int ch) {
        const C *src = a.chan + (size_t)ch * a.NH;
        for (int idx = threadIdx.x; idx < NTILE; idx += NT) {
            const int w = idx % TW, i = idx / TW;
            const bool ok = c0 + w < PL;
            cp_async<sizeof(C)>(dst + idx, src + (ok ? (size_t)i * PL + c0 + w : 0), ok);
        }
        cp_async_commit();
    };
    auto store = [&](const C *srcb, int ch) {
        C *dst = a.chan + (size_t)ch * a.NH;
        for (int idx = threadIdx.x; idx < NTILE; idx += NT) {
            const int w = idx % TW, i = idx / TW;
            if (c0 + w < PL) dst[(size_t)i * PL + c0 + w] = srcb[idx];
        }
    };
    for (int i = threadIdx.x; i < n; i += NT) tw[i] = a.tw0[i];
    // per column (k1, k2): its part of the G vector and its half-spectrum weight
    for (int w = threadIdx.x; w < TW; w += NT) {
        const long long col = c0 + w;
        const int k1 = (int)(col / n2h), k2 = (int)(col % n2h);
        const double m1 = (k1 <= a.n1 / 2) ? k1 : k1 - a.n1, m2 = k2;
        for (int d = 0; d < 3; d++) cvec[w][d] = (T)(m1 * a.bvec[3 + d] + m2 * a.bvec[6 + d]);
        cw[w] = (col < PL) ? ((k2 == 0 || (a.n2 % 2 == 0 && k2 == a.n2 / 2)) ? (T)1 : (T)2) : (T)0;
    }
    if ((a.terms & 4u) && lwt)
        for (int i = threadIdx.x; i < a.M; i += NT) sk[i] = a.knots_t[i];
    __syncthreads();
    int stage = 0;
    if (nord > 0) prefetch(xa, order[0]);
    // next(): wait for the current stage's tile, start the following one; returns its slot
    auto next = [&]() -> int {
        cp_async_wait<0>();
        __syncthreads();
        const int cur = stage & 1;
        if (stage + 1 < nord) prefetch(((stage + 1) & 1) ? xb : xa, order[stage + 1]);
        stage++;
        return cur;
    };
    // transforms of the tile in buffer x, returning the buffer that holds the result; when
    // that is the scratch buffer, x becomes the scratch (callers re-point the tile's slot)
    auto fwd = [&](C *x) -> C * {
        C *r = P::template fft2<-1>(x, scr, a, tw);
        if (r != x) scr = x;
        return r;
    };
    auto inv = [&](C *x) -> C * {
        C *r = P::template fft2<+1>(x, scr, a, tw);
        if (r != x) scr = x;
        return r;
    };
    auto slot = [&](int sl) -> C * { return sl ? xb : xa; };
    auto set_slot = [&](int sl, C *p) {
        if (sl) xb = p;
        else xa = p;
    };
    const T b0x = (T)a.bvec[0], b0y = (T)a.bvec[1], b0z = (T)a.bvec[2];
    T gmin = (T)3.0e38;                       // the smallest |G| of this thread's elements
    for (int idx = threadIdx.x; idx < NTILE; idx += NT) {
        const int w = idx % TW, i = idx / TW;
        const T m0 = (T)((i <= n / 2) ? i : i - n);
        const T gx = cvec[w][0] + m0 * b0x;
        const T gy = cvec[w][1] + m0 * b0y;
        const T gz = cvec[w][2] + m0 * b0z;
        gn[idx] = dsqrt(gx * gx + gy * gy + gz * gz);
        gmin = gn[idx] < gmin ? gn[idx] : gmin;
    }
    const T invN = (T)(1.0 / (double)a.N);
    double eH = 0.0, eV = 0.0, eP = 0.0, eN = 0.0;

    // ---- Hartree + local pseudopotential
    if (a.terms & (8u | 16u)) {
        const int sl = next();
        C *S = fwd(slot(sl));
        set_slot(sl, S);
        Part<T, XS> fH, fP;     // per-thread partials, folded into FP64 once
        for (int idx = threadIdx.x; idx < NTILE; idx += NT) {
            const int w = idx % TW, i = idx / TW;
            const long long col = c0 + w;
            const C X0 = cscale(S[idx], invN);
            const T g = gn[idx];
            const T g2 = g * g;
            if (a.rhohat_out && col < PL) a.rhohat_out[(size_t)i * PL + col] = X0;
            C out = cmake<C>((T)0, (T)0);
            if (col < PL && g2 > (T)0) {
                const T wgt = cw[w];
                if (a.terms & 8u) {
                    const T f = (T)1 / g2;
                    fH.add(wgt * (X0.x * X0.x + X0.y * X0.y) * f);
                    out = cscale(X0, (T)(4.0 * kPi) * f);
                }
                if (a.terms & 16u) {
                    const C v = a.vext[(size_t)i * PL + col];
                    fP.add(wgt * (X0.x * v.x + X0.y * v.y));
                    out = cadd(out, v);
                }
            } else if (col < PL && (a.terms & 16u)) {
                out = a.vext[(size_t)i * PL + col];       // G = 0: V_ext(0) only
            }
            S[idx] = out;
        }
        eH += fH.value();
        eP += fP.value();
        __syncthreads();
        S = inv(S);
        set_slot(sl, S);
        store(S, CH_HPP);
    }
    // ---- von Weizsaecker (psi form)
    if (a.terms & 2u) {
        const int sl = next();
        C *S = fwd(slot(sl));
        set_slot(sl, S);
        Part<T, XS> fV;
        for (int idx = threadIdx.x; idx < NTILE; idx += NT) {
            const int w = idx % TW;
            const C X0 = cscale(S[idx], invN);
            const T g = gn[idx];
            const T g2 = g * g;
            fV.add(cw[w] * g2 * (X0.x * X0.x + X0.y * X0.y));
            S[idx] = cscale(X0, g2);
        }
        eV += fV.value();
        __syncthreads();
        S = inv(S);
        set_slot(sl, S);
        store(S, CH_VW);
    }
    // ---- nonlocal: s2 (kernel at each knot) and the reciprocal half of s3
    if (a.terms & 4u) {
        {
            const int sl = next();
            C *S = fwd(slot(sl));
            set_slot(sl, S);
            for (int idx = threadIdx.x; idx < NTILE; idx += NT) Rr[idx] = cscale(S[idx], invN);
        }
        if (!lwt) {
            // global-kF Wang-Teter: K * rho^beta into CH_NL, K * rho^alpha into CH_KNOT0;
            // E = Omega sum_G w Re(conj(FFT[rho^alpha]) K FFT[rho^beta])
            const T hk = (T)(0.5 / a.scal[S_KF_WT]);
            const int sl = next();
            C *S = fwd(slot(sl));
            set_slot(sl, S);
            Part<T, XS> fN;
            auto wt = [&](auto large) {
                for (int idx = threadIdx.x; idx < NTILE; idx += NT) {
                    const int w = idx % TW;
                    T K;
                    if constexpr (decltype(large)::value) K = kernel_value_large(gn[idx] * hk);
                    else K = kernel_value<T, MGP>(a, gn[idx] * hk);
                    const C Sa = cscale(S[idx], invN);
                    const C Rb = Rr[idx];
                    fN.add(cw[w] * K * (Sa.x * Rb.x + Sa.y * Rb.y));
                    Rr[idx] = cscale(Rb, K);
                    S[idx] = cscale(Sa, K);
                }
            };
            if (warp_all_large<T, MGP>(gmin, hk)) wt(std::true_type{});
            else wt(std::false_type{});
            eN += fN.value();
            __syncthreads();
            Rr = inv(Rr);
            S = inv(S);
            set_slot(sl, S);
            store(Rr, CH_NL);
            store(S, CH_KNOT0);
        } else {
            if (exact)
                for (int idx = threadIdx.x; idx < NTILE; idx += NT) A[idx] = cmake<C>((T)0, (T)0);
            for (int m = 0; m < a.M; m++) {
                const T hk = (T)0.5 / sk[m];
                int sl;
                C *S;
                if (exact) {
                    sl = next();
                    S = fwd(slot(sl));
                    set_slot(sl, S);
                } else {
                    __syncthreads();
                    sl = m & 1;
                    S = slot(sl);
                }
                Part<T, XS> fN;
                auto knot = [&](auto large) {
                    for (int idx = threadIdx.x; idx < NTILE; idx += NT) {
                        T K;
                        if constexpr (decltype(large)::value) K = kernel_value_large(gn[idx] * hk);
                        else K = kernel_value<T, MGP>(a, gn[idx] * hk);
                        if (exact) {
                            // E_NL += Omega sum_G w Re(conj(FFT[h_m rho^alpha]) K_m FFT[rho^beta])
                            const C Sm = cscale(S[idx], invN);
                            const C Rb = Rr[idx];
                            fN.add(cw[idx % TW] * K * (Sm.x * Rb.x + Sm.y * Rb.y));
                            A[idx] = cadd(A[idx], cscale(Sm, K));
                        }
                        S[idx] = cscale(Rr[idx], K);
                    }
                };
                if (warp_all_large<T, MGP>(gmin, hk)) knot(std::true_type{});
                else knot(std::false_type{});
                eN += fN.value();
                __syncthreads();
                S = inv(S);
                set_slot(sl, S);
                store(S, CH_KNOT0 + m);
            }
            if (exact) {
                __syncthreads();
                A = inv(A);
                store(A, CH_NL);
            }
        }
    }
    cp_async_wait<0>();
    double r[4] = {eH, eV, eP, eN};
    block_sum_n<4>(r, sd);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; k++) a.part_ax0[4 * bid + k] = r[k];
}

// ======================================================================= row inverse (C2R along n2) + s4 + V
template <typename T, class P, bool XS = false>
__device__ __forceinline__ void row_inv_body(const EvalArgs<T> &a, const int bid, const int nblk) {
    typedef typename Vec2<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sd[32];
    __shared__ T sk[OFDFT_MAX_KNOTS];
    __shared__ T sidk[OFDFT_MAX_KNOTS];
    const int n = P::n(a), B = P::B(a), ld = P::ld(a), NT = P::nt();
    const int n2h = n / 2 + 1;
    const int PP = 2 * B * n, pitch = row_pitch(n);
    C *tw = (C *)smem_raw;
    C *buf = tw + n;
    T *stg = (T *)buf;
    T *sv = (T *)((unsigned char *)buf + row_buf_bytes<T>(n, B));   // V accumulator
    T *sa1 = sv + PP;                      // rho^(alpha-1)
    T *sk3 = sa1 + PP;                     // exact: kF/3 inside the knot range (else 0); interp: rho^alpha
    T *svw = sk3 + PP;                     // 1 / (2 max(psi, psi_floor))
    T *sb1 = svw + PP;                     // rho^(beta-1)
    T *st = sb1 + PP;                      // spline weight t
    unsigned char *sj = (unsigned char *)(st + PP);

    const long long R = (long long)a.n0 * a.n1;
    const long long row0 = 2LL * B * bid;
    const bool lwt = (a.terms & 4u) && a.kernel == 0;
    const bool interp = a.nlpot == 1;
    const int M = a.M;
    for (int i = threadIdx.x; i < n; i += NT) tw[i] = a.tw2[i];
    if (lwt)
        for (int i = threadIdx.x; i < M; i += NT) {
            sk[i] = a.knots_t[i];
            sidk[i] = (i + 1 < M) ? a.invdk_t[i] : (T)0;
        }
    for (int idx = threadIdx.x; idx < PP; idx += NT) {
        const int rr = idx / n, i2 = idx - rr * n;
        const long long row = row0 + rr;
        stg[rr * pitch + i2] = (row < R) ? a.rho[row * n + i2] : (T)0;
    }
    __syncthreads();
    const T ilr = lwt ? knot_log_scale(a, sk, M) : (T)0;
    const T psi_floor = dsqrt(a.floor_);
    const T rlo = (T)a.scal[S_RHO_MIN] > a.floor_ ? (T)a.scal[S_RHO_MIN] : a.floor_;
    const T rhi = (T)a.scal[S_RHO_MAX] > a.floor_ ? (T)a.scal[S_RHO_MAX] : a.floor_;
    for (int o = threadIdx.x; o < PP; o += NT) {
        const int rr = o % (2 * B), i2 = o / (2 * B);
        const T x = stg[rr * pitch + i2];
        T v = 0;
        const T xp = x > (T)0 ? x : (T)0;
        if (a.terms & 1u) {
            const T c = dcbrt(xp);
            v = (T)(5.0 / 3.0 * kCTF) * c * c;          // V_TF = (5/3) C_TF rho^(2/3)
        }
        if (a.terms & 32u) {
            T vxc;
            lda_xc(x > a.floor_ ? x : a.floor_, vxc);
            v += vxc;
        }
        sv[o] = v;
        const T p = dsqrt(xp);
        svw[o] = (T)1 / ((T)2 * (p > psi_floor ? p : psi_floor));
        if (a.terms & 4u) {
            const T xf = x > a.floor_ ? x : a.floor_;
            T ra, rb, kf;
            point_powers(a, xf, ra, rb, kf);
            sa1[o] = ra / xf;
            sb1[o] = rb / xf;
            if (lwt) {
                const bool inside = in_knot_range(a, xf, kf, sk[0], sk[M - 1], rlo, rhi);
                const T kc = kf < sk[0] ? sk[0] : (kf > sk[M - 1] ? sk[M - 1] : kf);
                const int j = knot_interval_fast(kc, sk, M, ilr);
                sj[o] = (unsigned char)j;
                st[o] = (kc - sk[j]) * sidk[j];
                sk3[o] = interp ? ra : (inside ? kf * (T)(1.0 / 3.0) : (T)0);
            }
        }
    }
    __syncthreads();
    Part<T, XS> fNL;
    const T alpha_eff = interp ? (T)2 * a.alpha : a.alpha;
    // the pair of half-spectrum rows of every (pair, k) this thread packs; with a
    // compile-time policy the next channel's values are loaded into registers
    // while the current channel is transformed (latency hidden behind the FFT)
    constexpr int QP = P::ct ? (P::B_ * (P::N_ / 2 + 1) + P::NT_ - 1) / P::NT_ : 1;
    C p0[QP], p1[QP];
    auto load_pairs = [&](int ci) {
        const C *in = a.chan + (size_t)a.inv_ch[ci] * a.NH;
#pragma unroll
        for (int q = 0; q < QP; q++) {
            const int idx = threadIdx.x + q * NT;
            const C z = cmake<C>((T)0, (T)0);
            p0[q] = z;
            p1[q] = z;
            if (idx < n2h * B) {
                const int b = idx / n2h, k = idx - b * n2h;
                const long long r0 = row0 + 2 * b;
                if (r0 < R) p0[q] = in[r0 * n2h + k];
                if (r0 + 1 < R) p1[q] = in[(r0 + 1) * n2h + k];
            }
        }
    };
    auto pack = [&](int idx, C X0, C X1) {
        const int b = idx / n2h, k = idx - b * n2h;
        if (k == 0 || 2 * k == n) {
            buf[k * ld + b] = cmake<C>(X0.x, X1.x);
        } else {
            buf[k * ld + b] = cmake<C>(X0.x - X1.y, X0.y + X1.x);
            buf[(n - k) * ld + b] = cmake<C>(X0.x + X1.y, X1.x - X0.y);
        }
    };
    if constexpr (P::ct) {
        if (a.ninv > 0) load_pairs(0);
    }
    for (int ci = 0; ci < a.ninv; ci++) {
        const int kind = a.inv_kind[ci], m = a.inv_knot[ci];
        // pack the pair of half spectra into one full complex spectrum
        if constexpr (P::ct) {
#pragma unroll
            for (int q = 0; q < QP; q++) {
                const int idx = threadIdx.x + q * NT;
                if (idx < n2h * B) pack(idx, p0[q], p1[q]);
            }
            __syncthreads();
            if (ci + 1 < a.ninv) load_pairs(ci + 1);
        } else {
            const C *in = a.chan + (size_t)a.inv_ch[ci] * a.NH;
            for (int idx = threadIdx.x; idx < n2h * B; idx += NT) {
                const int b = idx / n2h, k = idx - b * n2h;
                const long long r0 = row0 + 2 * b;
                const C z = cmake<C>((T)0, (T)0);
                pack(idx, (r0 < R) ? in[r0 * n2h + k] : z, (r0 + 1 < R) ? in[(r0 + 1) * n2h + k] : z);
            }
            __syncthreads();
        }
        P::template fft<+1>(buf, a, tw);
        for (int idx = threadIdx.x; idx < n * B; idx += NT) {
            const int b = idx % B, i2 = idx / B;
            const C z = buf[i2 * ld + b];
            const int o = 2 * idx;                      // = i2 * 2B + 2b
#pragma unroll
            for (int s = 0; s < 2; s++) {
                const T y = s ? z.y : z.x;
                T acc = sv[o + s];
                if (kind == CONS_ADD) acc += y;
                else if (kind == CONS_VW) acc += y * svw[o + s];
                else if (kind == CONS_T2 || kind == CONS_WT_B) acc += a.beta * sb1[o + s] * y;
                else if (kind == CONS_WT_A) acc += a.alpha * sa1[o + s] * y;
                else {
                    const int j = sj[o + s];
                    if (j == m || j + 1 == m) {
                        const T t = st[o + s], idk = sidk[j];
                        const T h = (j == m) ? (T)1 - t : t;
                        if (interp) {
                            acc += y * alpha_eff * sa1[o + s] * h;
                            if (row0 + 2 * b + s < R) fNL.add(sk3[o + s] * h * y);
                        } else {
                            const T hp = (j == m) ? -idk : idk;
                            acc += y * sa1[o + s] * (alpha_eff * h + sk3[o + s] * hp);
                        }
                    }
                }
                sv[o + s] = acc;
            }
        }
        __syncthreads();
    }
    if (a.V) {
        for (int o = threadIdx.x; o < PP; o += NT) {
            const int rr = o % (2 * B), i2 = o / (2 * B);
            stg[rr * pitch + i2] = sv[o];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < PP; idx += NT) {
            const int rr = idx / n, i2 = idx - rr * n;
            const long long row = row0 + rr;
            if (row < R) a.V[row * n + i2] = stg[rr * pitch + i2];
        }
    }
    const double eNL = block_sum(fNL.value(), sd);
    if (threadIdx.x == 0) a.part_row[bid] = eNL;
}

// ======================================================================= rows, channel-batched form
// One pair of rows (2p, 2p+1) per block.  Instead of transforming the channels
// one after another, all channels of a group of up to G are formed and
// transformed together: the batch index of the shared-memory FFT is the channel
// slot, so every pass has work for every thread and one transform per group
// replaces one per channel.  Each thread owns fixed points of the pair (element
// e of the packed sequence = points (2p, e) and (2p+1, e)) for the whole
// kernel, so the per-point quantities (rho^alpha, knot interval, spline
// weights) live in registers and a point reads only the channels it needs: the
// semilocal ones and the two knots that bracket its kF.
template <typename T, int N, int G, int NT, int MAXR, int MINB>
struct RowPolicy2 {
    typedef typename Vec2<T>::type C;
    static constexpr int N_ = N, G_ = G, NT_ = NT, LD = (G % 2) ? G : G + 1;
    // each of the two buffers (the batch and the out-of-place transform's scratch) holds
    // N x LD elements and, when used as staging, G pairs of half-spectrum rows
    static constexpr int SCR = (N * LD > G * (N + 2)) ? N * LD : G * (N + 2);
    static constexpr int E = (N + NT - 1) / NT;      // elements (pairs of points) per thread
    static constexpr int min_blocks = MINB;
    template <int DIR> __device__ static C *fft(C *x, C *y, const C *tw) {
        return ct::fft_oop<DIR, N, G, LD, NT, MAXR>(x, y, tw);
    }
};

template <typename T, class Q>
__device__ __forceinline__ void row_fwd2_body(const EvalArgs<T> &a, const int bid, const int nblk) {
    typedef typename Vec2<T>::type C;
    constexpr int n = Q::N_, G = Q::G_, LD = Q::LD, NT = Q::NT_, E = Q::E, n2h = n / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = (C *)smem_raw;
    C *buf = tw + n;                 // the channel batch, formed here
    C *scr = buf + Q::SCR;           // scratch of the out-of-place transform
    __shared__ T sk[OFDFT_MAX_KNOTS], sdk[OFDFT_MAX_KNOTS];
    __shared__ int sch[kMaxChan], skpos;
    const long long R = (long long)a.n0 * a.n1;
    const long long row0 = 2LL * bid;
    const bool has1 = row0 + 1 < R;
    const bool nl = a.terms & 4u, lwt = nl && a.kernel == 0;
    const int M = a.M, nf = a.nfwd;
    // the block's density values are requested first, so that their latency overlaps the
    // table loads and the barrier below
    T xr[E][2];
#pragma unroll
    for (int q = 0; q < E; q++) {
        const int e = threadIdx.x + q * NT;
#pragma unroll
        for (int s = 0; s < 2; s++) xr[q][s] = (e < n && (s == 0 || has1)) ? a.rho[(row0 + s) * n + e] : (T)0;
    }
    for (int i = threadIdx.x; i < n; i += NT) tw[i] = a.tw2[i];
    if (lwt)
        for (int i = threadIdx.x; i < M; i += NT) {
            sk[i] = a.knots_t[i];
            sdk[i] = a.invdk_t[i];
        }
    for (int i = threadIdx.x; i < nf; i += NT) sch[i] = a.fwd_ch[i];
    if (threadIdx.x == 0) {
        // list position of the first knot field h_0 rho^alpha (the knots follow in order)
        int k = nf;
        if (lwt)
            for (int i = nf - 1; i >= 0; i--)
                if (a.fwd_ch[i] >= CH_KNOT0) k = i;
        skpos = k;
    }
    __syncthreads();
    const int kpos = skpos;
    const T mean = (T)a.scal[S_RHO_MEAN];
    const T ilr = lwt ? knot_log_scale(a, sk, M) : (T)0;
    // per-point channel values: vh = rho - mean, vv = psi, vb = rho^beta,
    // fa/fb = (1 - t) rho^alpha / t rho^alpha for knots j/j+1 (WT: fa = rho^alpha)
    T vh[E][2], vv[E][2], vb[E][2], fa[E][2], fb[E][2];
    int jj[E][2];
#pragma unroll
    for (int q = 0; q < E; q++) {
        const int e = threadIdx.x + q * NT;
#pragma unroll
        for (int s = 0; s < 2; s++) {
            vh[q][s] = vv[q][s] = vb[q][s] = fa[q][s] = fb[q][s] = (T)0;
            jj[q][s] = 0;
            if (e < n && (s == 0 || has1)) {
                const T x = xr[q][s];
                vh[q][s] = x - mean;
                vv[q][s] = dsqrt(x > (T)0 ? x : (T)0);
                if (nl) {
                    const T xf = x > a.floor_ ? x : a.floor_;
                    T ra, rb, kf;
                    point_powers(a, xf, ra, rb, kf);
                    vb[q][s] = rb;
                    if (lwt) {
                        kf = kf < sk[0] ? sk[0] : (kf > sk[M - 1] ? sk[M - 1] : kf);
                        const int j = knot_interval_fast(kf, sk, M, ilr);
                        const T t = (kf - sk[j]) * sdk[j];
                        jj[q][s] = j;
                        fa[q][s] = ((T)1 - t) * ra;
                        fb[q][s] = t * ra;
                    } else {
                        fa[q][s] = ra;
                    }
                }
            }
        }
    }
    for (int g0 = 0; g0 < nf; g0 += G) {
        const int gact = nf - g0 < G ? nf - g0 : G;
        // form: every slot of the element (knot slots zero), then the two knot values of each point
#pragma unroll
        for (int q = 0; q < E; q++) {
            const int e = threadIdx.x + q * NT;
            if (e < n) {
                C *row = buf + e * LD;
#pragma unroll
                for (int s = 0; s < G; s++) {
                    const int ci = g0 + s;
                    C v = cmake<C>((T)0, (T)0);
                    if (ci < kpos && ci < nf) {
                        const int ch = sch[ci];
                        if (ch == CH_HPP) v = cmake<C>(vh[q][0], vh[q][1]);
                        else if (ch == CH_VW) v = cmake<C>(vv[q][0], vv[q][1]);
                        else if (ch == CH_NL) v = cmake<C>(vb[q][0], vb[q][1]);
                        else v = cmake<C>(fa[q][0], fa[q][1]);          // WT: rho^alpha
                    }
                    row[s] = v;
                }
                if (kpos < nf) {
#pragma unroll
                    for (int s = 0; s < 2; s++) {
                        const int ca = kpos + jj[q][s] - g0;
                        if (ca >= 0 && ca < gact) ((T *)(row + ca))[s] = fa[q][s];
                        if (ca + 1 >= 0 && ca + 1 < gact) ((T *)(row + ca + 1))[s] = fb[q][s];
                    }
                }
            }
        }
        __syncthreads();
        const C *Z = Q::template fft<-1>(buf, scr, tw);
        // unpack X_2p[k] = (Z_k + conj Z_{n-k})/2, X_2p+1[k] = (Z_k - conj Z_{n-k})/(2i)
        // (plain stores: staging for bulk stores measured slower here)
        for (int idx = threadIdx.x; idx < gact * n2h; idx += NT) {
            const int s = idx / n2h, k = idx - s * n2h;
            const C A = Z[k * LD + s];
            const C Bv = Z[((n - k) % n) * LD + s];
            C *out = a.chan + (size_t)sch[g0 + s] * a.NH + row0 * n2h + k;
            out[0] = cmake<C>((T)0.5 * (A.x + Bv.x), (T)0.5 * (A.y - Bv.y));
            if (has1) out[n2h] = cmake<C>((T)0.5 * (A.y + Bv.y), (T)0.5 * (Bv.x - A.x));
        }
        __syncthreads();
    }
}

template <typename T, class Q>
__device__ __forceinline__ void row_inv2_body(const EvalArgs<T> &a, const int bid, const int nblk) {
    typedef typename Vec2<T>::type C;
    constexpr int n = Q::N_, G = Q::G_, LD = Q::LD, NT = Q::NT_, E = Q::E, n2h = n / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = (C *)smem_raw;
    C *buf = tw + n;                 // the packed channel batch
    C *scr = buf + Q::SCR;           // scratch of the out-of-place transform; stages the raw rows
    __shared__ double sd[32];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int s_ok;
    __shared__ T sk[OFDFT_MAX_KNOTS], sdk[OFDFT_MAX_KNOTS];
    __shared__ int sch[kMaxChan], skind[kMaxChan], skpos;
    const long long R = (long long)a.n0 * a.n1;
    const long long row0 = 2LL * bid;
    const bool has1 = row0 + 1 < R;
    const bool nl = a.terms & 4u, lwt = nl && a.kernel == 0, interp = a.nlpot == 1;
    const int M = a.M, ni = a.ninv;
    // bulk (TMA) loads need 16-byte aligned rows: an even channel stride, both rows present.
    // The two half-spectrum rows of each channel (contiguous in memory) are copied
    // asynchronously into the scratch buffer, one bulk copy per channel, so that all of a
    // group's loads are in flight at once; the first group's copies and the block's density
    // values are requested before anything else, so that their latency overlaps the table
    // loads, the barrier and the per-point factors below.
    const bool bulk = has1 && (a.NH % 2 == 0) && (smem_u32(scr) % 16 == 0);
    auto issue_rows = [&](int g0, int gact) {
        const unsigned bytes = (unsigned)(2 * n2h * sizeof(C));
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&mbar, bytes * (unsigned)gact);
        for (int s = 0; s < gact; s++)
            bulk_g2s(scr + 2 * s * n2h, a.chan + (size_t)a.inv_ch[g0 + s] * a.NH + row0 * n2h, bytes, &mbar);
    };
    if (bulk && threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        fence_proxy_async_smem();
        issue_rows(0, ni < G ? ni : G);
    }
    T xr[E][2];
#pragma unroll
    for (int q = 0; q < E; q++) {
        const int e = threadIdx.x + q * NT;
#pragma unroll
        for (int s = 0; s < 2; s++) xr[q][s] = (e < n && (s == 0 || has1)) ? a.rho[(row0 + s) * n + e] : (T)0;
    }
    for (int i = threadIdx.x; i < n; i += NT) tw[i] = a.tw2[i];
    if (lwt)
        for (int i = threadIdx.x; i < M; i += NT) {
            sk[i] = a.knots_t[i];
            sdk[i] = (i + 1 < M) ? a.invdk_t[i] : (T)0;
        }
    for (int i = threadIdx.x; i < ni; i += NT) {
        sch[i] = a.inv_ch[i];
        skind[i] = a.inv_kind[i];
    }
    if (threadIdx.x == 0) {
        // list position of the first knot field y_0 (the knots follow in order)
        int k = ni;
        for (int i = ni - 1; i >= 0; i--)
            if (a.inv_kind[i] == CONS_KNOT) k = i;
        skpos = k;
    }
    __syncthreads();
    const int kpos = skpos;
    unsigned phase = 0;
    const T ilr = lwt ? knot_log_scale(a, sk, M) : (T)0;
    const T psi_floor = dsqrt(a.floor_);
    const T alpha_eff = interp ? (T)2 * a.alpha : a.alpha;
    const T rlo = (T)a.scal[S_RHO_MIN] > a.floor_ ? (T)a.scal[S_RHO_MIN] : a.floor_;
    const T rhi = (T)a.scal[S_RHO_MAX] > a.floor_ ? (T)a.scal[S_RHO_MAX] : a.floor_;
    // per point: V accumulator (starts at V_TF), factors of the semilocal channels,
    // and the knot interval with the weights of its two knots in V (wa, wb) and,
    // interpolated mode, in the real-space E_NL (ea, eb)
    T acc[E][2], fvw[E][2], fa1[E][2], fb1[E][2], wa[E][2], wb[E][2], ea[E][2], eb[E][2];
    int jj[E][2];
#pragma unroll
    for (int q = 0; q < E; q++) {
        const int e = threadIdx.x + q * NT;
#pragma unroll
        for (int s = 0; s < 2; s++) {
            acc[q][s] = fvw[q][s] = fa1[q][s] = fb1[q][s] = wa[q][s] = wb[q][s] = ea[q][s] = eb[q][s] = (T)0;
            jj[q][s] = 0;
            if (e < n) {
                const bool valid = s == 0 || has1;
                const T x = xr[q][s];
                const T xp = x > (T)0 ? x : (T)0;
                if (a.terms & 1u) {
                    const T c = dcbrt(xp);
                    acc[q][s] = (T)(5.0 / 3.0 * kCTF) * c * c;        // V_TF = (5/3) C_TF rho^(2/3)
                }
                if (a.terms & 32u) {
                    T vxc;
                    lda_xc(x > a.floor_ ? x : a.floor_, vxc);
                    acc[q][s] += vxc;
                }
                const T p = dsqrt(xp);
                fvw[q][s] = (T)1 / ((T)2 * (p > psi_floor ? p : psi_floor));
                if (nl) {
                    const T xf = x > a.floor_ ? x : a.floor_;
                    T ra, rb, kf;
                    point_powers(a, xf, ra, rb, kf);
                    const T sa1 = ra / xf;
                    fa1[q][s] = a.alpha * sa1;
                    fb1[q][s] = a.beta * (rb / xf);
                    if (lwt) {
                        const bool inside = in_knot_range(a, xf, kf, sk[0], sk[M - 1], rlo, rhi);
                        const T kc = kf < sk[0] ? sk[0] : (kf > sk[M - 1] ? sk[M - 1] : kf);
                        const int j = knot_interval_fast(kc, sk, M, ilr);
                        const T t = (kc - sk[j]) * sdk[j], idk = sdk[j];
                        jj[q][s] = j;
                        if (interp) {
                            wa[q][s] = alpha_eff * sa1 * ((T)1 - t);
                            wb[q][s] = alpha_eff * sa1 * t;
                            if (valid) {
                                ea[q][s] = ra * ((T)1 - t);
                                eb[q][s] = ra * t;
                            }
                        } else {
                            const T k3 = inside ? kf * (T)(1.0 / 3.0) : (T)0;
                            wa[q][s] = sa1 * (alpha_eff * ((T)1 - t) - k3 * idk);
                            wb[q][s] = sa1 * (alpha_eff * t + k3 * idk);
                        }
                    }
                }
            }
        }
    }
    Part<T, false> fNL;
    bool alive = true;
    for (int g0 = 0; g0 < ni; g0 += G) {
        const int gact = ni - g0 < G ? ni - g0 : G;
        // the group's rows by bulk copies (the first group's are already in flight), else
        // element copies (a missing second row reads as zeros)
        if (bulk) {
            if (threadIdx.x == 0) {
                if (g0 > 0) issue_rows(g0, gact);
                s_ok = mbar_wait_bounded(&mbar, phase, a.wait_polls) ? 1 : 0;
            }
            __syncthreads();
            if (!s_ok) {
                // the copies did not arrive in time: flag it and stop working, but first let
                // them land (they target this block's shared memory, which the next block on
                // this SM may own) with a longer bounded wait; if even that expires the flag
                // says so (2: copies may still be in flight, the whole call is invalid)
                if (threadIdx.x == 0) {
                    const bool drained = mbar_wait_bounded(&mbar, phase, 1u << 26);
                    atomicAdd(a.scal + (drained ? S_TIMEOUT : S_FATAL), 1.0);
                }
                alive = false;
                break;
            }
            mbar_wait_bounded(&mbar, phase, 1u << 22);      // completed: makes the data visible here
            phase ^= 1u;
        } else {
            for (int idx = threadIdx.x; idx < gact * 2 * n2h; idx += NT) {
                const int s = idx / (2 * n2h), j = idx - s * 2 * n2h;
                const bool ok = j < n2h || has1;
                cp_async<sizeof(C)>(scr + idx, a.chan + (size_t)sch[g0 + s] * a.NH + (ok ? row0 * n2h + j : 0), ok);
            }
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
        }
        // pack each pair of half-spectrum rows into one full complex spectrum
        for (int idx = threadIdx.x; idx < gact * n2h; idx += NT) {
            const int s = idx / n2h, k = idx - s * n2h;
            const C X0 = scr[2 * s * n2h + k];
            const C X1 = scr[(2 * s + 1) * n2h + k];
            if (k == 0 || 2 * k == n) {
                buf[k * LD + s] = cmake<C>(X0.x, X1.x);
            } else {
                buf[k * LD + s] = cmake<C>(X0.x - X1.y, X0.y + X1.x);
                buf[(n - k) * LD + s] = cmake<C>(X0.x + X1.y, X1.x - X0.y);
            }
        }
        __syncthreads();
        const C *Z = Q::template fft<+1>(buf, scr, tw);
#pragma unroll
        for (int q = 0; q < E; q++) {
            const int e = threadIdx.x + q * NT;
            if (e < n) {
                const C *row = Z + e * LD;
                const int pend = kpos < g0 + gact ? kpos : g0 + gact;
                for (int ci = g0; ci < pend; ci++) {
                    const C z = row[ci - g0];
                    const int kind = skind[ci];
#pragma unroll
                    for (int s = 0; s < 2; s++) {
                        const T y = s ? z.y : z.x;
                        if (kind == CONS_ADD) acc[q][s] += y;
                        else if (kind == CONS_VW) acc[q][s] += y * fvw[q][s];
                        else if (kind == CONS_T2 || kind == CONS_WT_B) acc[q][s] += fb1[q][s] * y;
                        else if (kind == CONS_WT_A) acc[q][s] += fa1[q][s] * y;
                    }
                }
                if (kpos < ni) {
#pragma unroll
                    for (int s = 0; s < 2; s++) {
                        const int ca = kpos + jj[q][s] - g0;
                        if (ca >= 0 && ca < gact) {
                            const T y = ((const T *)(row + ca))[s];
                            acc[q][s] += y * wa[q][s];
                            fNL.add(ea[q][s] * y);
                        }
                        if (ca + 1 >= 0 && ca + 1 < gact) {
                            const T y = ((const T *)(row + ca + 1))[s];
                            acc[q][s] += y * wb[q][s];
                            fNL.add(eb[q][s] * y);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if (alive && a.V) {
#pragma unroll
        for (int q = 0; q < E; q++) {
            const int e = threadIdx.x + q * NT;
            if (e < n) {
                a.V[row0 * n + e] = acc[q][0];
                if (has1) a.V[(row0 + 1) * n + e] = acc[q][1];
            }
        }
    }
    if (lwt && interp) {                     // the only mode with a real-space E_NL
        const double eNL = block_sum(fNL.value(), sd);
        if (threadIdx.x == 0) a.part_row[bid] = eNL;
    }
}

// ======================================================================= finalize
// FP64 energies from the per-block partials of the reciprocal-space kernel (and, for
// the interpolated LWT mode, of the row kernel), summed in a fixed order.
template <typename T>
__device__ __forceinline__ void finalize_body(const EvalArgs<T> &a, const int bid, const int nblk) {
    // block k sums one kind of partial (0..3: the reciprocal-space kernel's E_H, E_vW,
    // E_PP and G-space E_NL sums; 4: the rows' real-space E_NL), so the FP64 work is
    // spread over five SMs; the last block to finish assembles the energies
    __shared__ double sd[32];
    __shared__ bool last;
    const int k = bid;
    const bool real_space = a.kernel == 0 && a.nlpot == 1;
    double acc = 0.0;
    if (k < 4) {
        for (int b = threadIdx.x; b < a.nb_ax0; b += blockDim.x) acc += a.part_ax0[4 * b + k];
    } else if ((a.terms & 4u) && real_space) {
        for (int b = threadIdx.x; b < a.nb_row; b += blockDim.x) acc += a.part_row[b];
    }
    acc = block_sum(acc, sd);
    double *sums = a.scal + S_FIN;
    if (threadIdx.x == 0) {
        sums[k] = acc;
        __threadfence();
        last = atomicAdd(a.ticket, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    const double h = __ldcg(sums), v = __ldcg(sums + 1), p = __ldcg(sums + 2), ng = __ldcg(sums + 3),
                 nl = __ldcg(sums + 4);
    double *E = a.energies;
    E[E_VW] = (a.terms & 2u) ? 0.5 * a.omega * v : 0.0;
    E[E_H] = (a.terms & 8u) ? 2.0 * kPi * a.omega * h : 0.0;
    if (a.terms & 16u) {
        const double v0 = (double)a.vext[0].x;                    // V_ext(G = 0)
        E[E_PP] = a.omega * (p + a.scal[S_RHO_MEAN] * v0);
    } else {
        E[E_PP] = 0.0;
    }
    // nonlocal: G-space sum (exact LWT, WT) or real-space sum (interpolated LWT)
    E[E_NL] = (a.terms & 4u) ? (real_space ? nl * a.dV : a.omega * ng) : 0.0;
    E[E_TOT] = E[E_TF] + E[E_VW] + E[E_NL] + E[E_H] + E[E_PP] + E[E_XC];
    *a.ticket = 0u;                                   // ready for the next evaluation
}

// ======================================================================= kernel wrappers
// Single evaluation: the arguments in the kernel's parameter space, block b = blockIdx.x.
template <typename T, bool XS = false>
__global__ void __launch_bounds__(256) stats_kernel(EvalArgs<T> a) {
    stats_body<T, XS>(a, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void __launch_bounds__(256) finalize_kernel(EvalArgs<T> a) {
    finalize_body<T>(a, blockIdx.x, gridDim.x);
}
template <typename T, class P>
__global__ void __launch_bounds__(P::max_threads, P::min_blocks) row_fwd_kernel(EvalArgs<T> a) {
    row_fwd_body<T, P>(a, blockIdx.x, gridDim.x);
}
template <typename T, int DIR, class P>
__global__ void __launch_bounds__(P::max_threads, P::min_blocks) pencil1_kernel(EvalArgs<T> a) {
    pencil1_body<T, DIR, P>(a, blockIdx.x, gridDim.x);
}
// MGP: the knots' kernels of Eq. MGP from the correction table (a separate instantiation,
// so that the Wang-Teter form carries no trace of it)
// XS: every energy term added in FP64 (the exact-sums test option; runtime-size kernels only)
template <typename T, class P, bool MGP = false, bool XS = false>
__global__ void __launch_bounds__(P::max_threads, P::min_blocks_ax0) axis0_kernel(EvalArgs<T> a) {
    axis0_body<T, P, MGP, XS>(a, blockIdx.x, gridDim.x);
}
template <typename T, class P, bool XS = false>
__global__ void __launch_bounds__(P::max_threads, P::min_blocks) row_inv_kernel(EvalArgs<T> a) {
    row_inv_body<T, P, XS>(a, blockIdx.x, gridDim.x);
}
template <typename T, class Q>
__global__ void __launch_bounds__(Q::NT_, Q::min_blocks) row_fwd2_kernel(EvalArgs<T> a) {
    row_fwd2_body<T, Q>(a, blockIdx.x, gridDim.x);
}
template <typename T, class Q>
__global__ void __launch_bounds__(Q::NT_, Q::min_blocks) row_inv2_kernel(EvalArgs<T> a) {
    row_inv2_body<T, Q>(a, blockIdx.x, gridDim.x);
}

// Grouped: one launch runs a pass of K evaluations that share one launch geometry (the
// snapshots of one grid shape in a batch).  The arguments of evaluation k sit at ga[k] in
// global memory; block b works on evaluation b / bps as that evaluation's block b mod bps,
// so every evaluation sees exactly the blocks, partial sums and reduction order of its
// single launch (bit-identical results).
#define OFDFT_GROUP_INDEX const int gk = blockIdx.x / bps, gb = blockIdx.x - gk * bps
template <typename T, bool XS = false>
__global__ void __launch_bounds__(256) stats_group(const EvalArgs<T> *__restrict__ ga, int bps) {
    OFDFT_GROUP_INDEX;
    stats_body<T, XS>(ga[gk], gb, bps);
}
template <typename T>
__global__ void __launch_bounds__(256) finalize_group(const EvalArgs<T> *__restrict__ ga, int bps) {
    OFDFT_GROUP_INDEX;
    finalize_body<T>(ga[gk], gb, bps);
}
template <typename T, class P>
__global__ void __launch_bounds__(P::max_threads, P::min_blocks) row_fwd_group(const EvalArgs<T> *__restrict__ ga,
                                                                                int bps) {
    OFDFT_GROUP_INDEX;
    row_fwd_body<T, P>(ga[gk], gb, bps);
}
template <typename T, int DIR, class P>
__global__ void __launch_bounds__(P::max_threads, P::min_blocks) pencil1_group(const EvalArgs<T> *__restrict__ ga,
                                                                                int bps) {
    OFDFT_GROUP_INDEX;
    pencil1_body<T, DIR, P>(ga[gk], gb, bps);
}
template <typename T, class P, bool MGP = false>
__global__ void __launch_bounds__(P::max_threads, P::min_blocks_ax0) axis0_group(const EvalArgs<T> *__restrict__ ga,
                                                                                  int bps) {
    OFDFT_GROUP_INDEX;
    axis0_body<T, P, MGP, false>(ga[gk], gb, bps);
}
template <typename T, class P>
__global__ void __launch_bounds__(P::max_threads, P::min_blocks) row_inv_group(const EvalArgs<T> *__restrict__ ga,
                                                                                int bps) {
    OFDFT_GROUP_INDEX;
    row_inv_body<T, P, false>(ga[gk], gb, bps);
}
template <typename T, class Q>
__global__ void __launch_bounds__(Q::NT_, Q::min_blocks) row_fwd2_group(const EvalArgs<T> *__restrict__ ga, int bps) {
    OFDFT_GROUP_INDEX;
    row_fwd2_body<T, Q>(ga[gk], gb, bps);
}
template <typename T, class Q>
__global__ void __launch_bounds__(Q::NT_, Q::min_blocks) row_inv2_group(const EvalArgs<T> *__restrict__ ga, int bps) {
    OFDFT_GROUP_INDEX;
    row_inv2_body<T, Q>(ga[gk], gb, bps);
}

}  // namespace ofdft
