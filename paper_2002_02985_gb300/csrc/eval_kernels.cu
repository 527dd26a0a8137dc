// Kernels of one energy/potential evaluation (see eval.cuh for the pipeline).
#include "eval.cuh"

namespace ofdft {

// ======================================================================= G_NL
// Lindhard-derived WT kernel (Sec. 2.3, the G_NL definition below Eq. MGP):
//   G_NL(eta) = 1/F(eta) - 3 eta^2 - 1,
//   F(eta)    = 1/2 + (1 - eta^2)/(4 eta) ln|(1+eta)/(1-eta)|.
// Below eta = 1/2 and above eta = 2 the exact series of F in y = eta^2
// (resp. x = 1/eta^2) are summed, with the numerator 1 - (1 + 3 eta^2) F
// expanded term by term so that nothing cancels:
//   eta < 1/2:  F = 1 - sum_m y^m a_m,         num = -(8/3) y + sum_{m>=2} y^m (a_m + 3 a_{m-1})
//   eta > 2  :  F = sum_m x^m a_m,             num = -sum_{m>=1} x^m (a_m + 3 a_{m+1})
// with a_m = 1/(4 m^2 - 1) and G_NL = num / F.
#define GNL_TERMS 28
__constant__ double c_gnl_a[GNL_TERMS + 2];
__constant__ double c_gnl_lo[GNL_TERMS + 2];
__constant__ double c_gnl_hi[GNL_TERMS + 2];
__constant__ float c_gnl_af[GNL_TERMS + 2];
__constant__ float c_gnl_lof[GNL_TERMS + 2];
__constant__ float c_gnl_hif[GNL_TERMS + 2];

cudaError_t upload_gnl_tables() {
    double a[GNL_TERMS + 2], lo[GNL_TERMS + 2], hi[GNL_TERMS + 2];
    float af[GNL_TERMS + 2], lof[GNL_TERMS + 2], hif[GNL_TERMS + 2];
    for (int m = 0; m < GNL_TERMS + 2; m++) {
        a[m] = m == 0 ? 0.0 : 1.0 / (4.0 * m * m - 1.0);
    }
    for (int m = 0; m < GNL_TERMS + 2; m++) {
        lo[m] = (m >= 2) ? a[m] + 3.0 * a[m - 1] : (m == 1 ? -8.0 / 3.0 : 0.0);
        hi[m] = (m >= 1 && m + 1 < GNL_TERMS + 2) ? a[m] + 3.0 * a[m + 1] : 0.0;
        af[m] = (float)a[m];
        lof[m] = (float)lo[m];
        hif[m] = (float)hi[m];
    }
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(c_gnl_a, a, sizeof(a))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_gnl_lo, lo, sizeof(lo))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_gnl_hi, hi, sizeof(hi))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_gnl_af, af, sizeof(af))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_gnl_lof, lof, sizeof(lof))) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_gnl_hif, hif, sizeof(hif));
}

template <typename T> struct GnlTab;
template <> struct GnlTab<float> {
    static constexpr int nt = 12;
    __device__ static float a(int m) { return c_gnl_af[m]; }
    __device__ static float lo(int m) { return c_gnl_lof[m]; }
    __device__ static float hi(int m) { return c_gnl_hif[m]; }
};
template <> struct GnlTab<double> {
    static constexpr int nt = GNL_TERMS;
    __device__ static double a(int m) { return c_gnl_a[m]; }
    __device__ static double lo(int m) { return c_gnl_lo[m]; }
    __device__ static double hi(int m) { return c_gnl_hi[m]; }
};

template <typename T> __device__ __forceinline__ T gnl(T eta) {
    typedef GnlTab<T> Tb;
    constexpr int nt = Tb::nt;
    if (eta < (T)0.5) {
        const T y = eta * eta;
        T sF = 0, sN = 0;
#pragma unroll
        for (int m = nt; m >= 1; m--) {
            sF = (sF + Tb::a(m)) * y;
            sN = (sN + Tb::lo(m)) * y;
        }
        return sN / ((T)1 - sF);
    } else if (eta > (T)2) {
        const T x = (T)1 / (eta * eta);
        T sF = 0, sN = 0;
#pragma unroll
        for (int m = nt; m >= 1; m--) {
            sF = (sF + Tb::a(m)) * x;
            sN = (sN + Tb::hi(m)) * x;
        }
        return -sN / sF;
    }
    const T d = (T)1 - eta;
    if (dabs(d) < (T)1e-12) return (T)-2;
    const T F = (T)0.5 + ((T)1 - eta * eta) / ((T)4 * eta) * dlog(dabs(((T)1 + eta) / d));
    return (T)1 / F - (T)3 * eta * eta - (T)1;
}

// ======================================================================= helpers
template <typename T> __device__ __forceinline__ int knot_interval(T kc, const T *knots, int M) {
    // largest j in [0, M-2] with knots[j] <= kc (binary search; kc already clamped)
    int lo = 0, hi = M - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (knots[mid] <= kc) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T> __device__ __forceinline__ T pow_guarded(T x, T e, T floor_) {
    return dpow(x > floor_ ? x : floor_, e);
}

// ======================================================================= stats (s1 input)
template <typename T>
__global__ void __launch_bounds__(256) stats_kernel(EvalArgs<T> a) {
    __shared__ double sd[32];
    __shared__ T st[32];
    double s_rho = 0.0, s_tf = 0.0;
    T mn = (T)3.0e38, mx = (T)-3.0e38;
    int bad = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.N; i += stride) {
        const T x = a.rho[i];
        if (!(x >= (T)0) || !(x < (T)3.0e38)) bad = 1;      // NaN, Inf or negative
        s_rho += (double)x;
        const T c = dcbrt(x);
        s_tf += (double)(x * c * c);                       // rho^(5/3)
        mn = x < mn ? x : mn;
        mx = x > mx ? x : mx;
    }
    s_rho = block_sum(s_rho, sd);
    if (threadIdx.x == 0) a.part_stats[2 * blockIdx.x] = s_rho;
    s_tf = block_sum(s_tf, sd);
    if (threadIdx.x == 0) a.part_stats[2 * blockIdx.x + 1] = s_tf;
    mn = block_min(mn, st);
    if (threadIdx.x == 0) a.part_minmax[2 * blockIdx.x] = mn;
    mx = block_max(mx, st);
    if (threadIdx.x == 0) a.part_minmax[2 * blockIdx.x + 1] = mx;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0 && bad) a.scal[S_BAD] = 1.0;
}

// ======================================================================= knots (s1)
template <typename T>
__global__ void __launch_bounds__(256) knots_kernel(EvalArgs<T> a) {
    __shared__ double sd[32];
    __shared__ T st[32];
    double s_rho = 0.0, s_tf = 0.0;
    T mn = (T)3.0e38, mx = (T)-3.0e38;
    for (int b = threadIdx.x; b < a.nb_stats; b += blockDim.x) {
        s_rho += a.part_stats[2 * b];
        s_tf += a.part_stats[2 * b + 1];
        const T x = a.part_minmax[2 * b], y = a.part_minmax[2 * b + 1];
        mn = x < mn ? x : mn;
        mx = y > mx ? y : mx;
    }
    s_rho = block_sum(s_rho, sd);
    s_tf = block_sum(s_tf, sd);
    mn = block_min(mn, st);
    mx = block_max(mx, st);
    if (threadIdx.x != 0) return;
    const double fl = (double)a.floor_;
    a.scal[S_SUM_RHO] = s_rho;
    a.scal[S_SUM_TF] = s_tf;
    a.scal[S_RHO_MIN] = (double)mn;
    a.scal[S_RHO_MAX] = (double)mx;
    const double mean = s_rho / (double)a.N;
    a.scal[S_RHO_MEAN] = mean;
    a.scal[S_KF_WT] = cbrt(kThreePi2 * (mean > fl ? mean : fl));
    a.energies[E_TF] = (a.terms & 1u) ? kCTF * s_tf * a.dV : 0.0;
    const int M = a.M;
    if (!(a.terms & 4u) || a.kernel != 0 || M < 2) return;
    if (!a.frozen) {
        // s1: knots between kF(min rho) and kF(max rho), FP64
        const double rmin = (double)mn > fl ? (double)mn : fl, rmax = (double)mx > fl ? (double)mx : fl;
        const double kmin = cbrt(kThreePi2 * rmin), kmax = cbrt(kThreePi2 * rmax);
        for (int m = 0; m < M; m++) {
            double k;
            if (a.knot_spacing == 0) k = kmin * exp((double)m * (log(kmax / kmin) / (double)(M - 1)));
            else k = kmin + (double)m * ((kmax - kmin) / (double)(M - 1));
            a.knots_d[m] = k;
        }
        a.knots_d[0] = kmin;
        a.knots_d[M - 1] = kmax;
    }
    for (int m = 0; m < M; m++) a.knots_t[m] = (T)a.knots_d[m];
    for (int m = 0; m + 1 < M; m++) {
        const double dk = a.knots_d[m + 1] - a.knots_d[m];
        a.invdk_t[m] = dk > 0.0 ? (T)(1.0 / dk) : (T)0;
    }
}

// ======================================================================= row forward (R2C along n2)
// Tile: Brow pairs of consecutive rows (flattened row r = i0*n1 + i1); row pair
// p holds rows 2p and 2p+1, packed as z = x_2p + i x_2p+1 for one complex FFT.
template <typename T> size_t row_fwd_smem(const EvalArgs<T> &a) {
    typedef typename Vec2<T>::type C;
    const size_t P = (size_t)2 * a.Brow * (a.n2 + 1);
    return a.n2 * sizeof(C) + (size_t)a.n2 * (a.Brow + 1) * sizeof(C) + P * (4 * sizeof(T) + 1) + 16;
}

template <typename T, int CAP>
__global__ void __launch_bounds__(kMaxThreads) row_fwd_kernel(EvalArgs<T> a) {
    typedef typename Vec2<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n2, n2h = a.n2h, B = a.Brow, ld = B + 1, pl = n + 1;
    const int P = 2 * B * pl;
    C *tw = (C *)smem_raw;
    C *buf = tw + n;
    T *sx = (T *)(buf + (size_t)n * ld);
    T *sra = sx + P;
    T *srb = sra + P;
    T *st = srb + P;
    unsigned char *sj = (unsigned char *)(st + P);
    __shared__ T sk[OFDFT_MAX_KNOTS];

    const long long R = (long long)a.n0 * a.n1;
    const long long row0 = 2LL * B * blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = a.tw2[i];
    const bool lwt = (a.terms & 4u) && a.kernel == 0;
    const int M = a.M;
    if (lwt) for (int i = threadIdx.x; i < M; i += blockDim.x) sk[i] = a.knots_t[i];
    const T mean = (T)a.scal[S_RHO_MEAN];
    __syncthreads();
    // per-point quantities, rows rr = 0..2B-1 of the tile
    for (int idx = threadIdx.x; idx < 2 * B * n; idx += blockDim.x) {
        const int rr = idx / n, i2 = idx - rr * n;
        const long long row = row0 + rr;
        const int o = rr * pl + i2;
        T x = 0;
        if (row < R) x = a.rho[row * n + i2];
        sx[o] = x;
        if (a.terms & 4u) {
            const T xf = x > a.floor_ ? x : a.floor_;
            const T ra = dpow(xf, a.alpha);
            sra[o] = ra;
            srb[o] = (a.beta == a.alpha) ? ra : dpow(xf, a.beta);
            if (lwt) {
                T kf = dcbrt((T)kThreePi2 * xf);
                kf = kf < sk[0] ? sk[0] : (kf > sk[M - 1] ? sk[M - 1] : kf);
                const int j = knot_interval(kf, sk, M);
                sj[o] = (unsigned char)j;
                st[o] = (kf - sk[j]) * a.invdk_t[j];
            }
        }
    }
    __syncthreads();
    for (int ci = 0; ci < a.nfwd; ci++) {
        const int ch = a.fwd_ch[ci];
        // channel field, packed in pairs
        for (int idx = threadIdx.x; idx < n * B; idx += blockDim.x) {
            const int b = idx % B, i2 = idx / B;
            T v[2];
#pragma unroll
            for (int s = 0; s < 2; s++) {
                const int o = (2 * b + s) * pl + i2;
                T f;
                if (ch == CH_HPP) f = sx[o] - mean;
                else if (ch == CH_VW) f = dsqrt(sx[o] > (T)0 ? sx[o] : (T)0);
                else if (ch == CH_NL) f = srb[o];
                else if (!lwt) f = sra[o];                         // WT: rho^alpha field
                else {
                    const int m = ch - CH_KNOT0, j = sj[o];
                    const T t = st[o];
                    f = (j == m) ? ((T)1 - t) * sra[o] : ((j == m - 1) ? t * sra[o] : (T)0);
                }
                if (row0 + 2 * b + s >= R) f = 0;
                v[s] = f;
            }
            buf[i2 * ld + b] = cmake<C>(v[0], v[1]);
        }
        __syncthreads();
        fft_smem<-1, CAP>(buf, ld, B, a.p2, tw);
        // unpack X_2p[k] = (Z_k + conj Z_{n-k})/2, X_2p+1[k] = (Z_k - conj Z_{n-k})/(2i)
        C *out = a.chan + (size_t)ch * a.NH;
        for (int idx = threadIdx.x; idx < n2h * B; idx += blockDim.x) {
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
template <typename T> size_t pencil_smem(int n, int TW) {
    typedef typename Vec2<T>::type C;
    return (size_t)n * sizeof(C) + (size_t)n * TW * sizeof(C);
}

// blockIdx.x: tile of TW consecutive k2, blockIdx.y: i0, blockIdx.z: channel list entry
template <typename T, int DIR, int CAP>
__global__ void __launch_bounds__(kMaxThreads) pencil1_kernel(EvalArgs<T> a) {
    typedef typename Vec2<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n1, TW = a.TW1, n2h = a.n2h;
    C *tw = (C *)smem_raw;
    C *buf = tw + n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = a.tw1[i];
    const int ch = DIR < 0 ? a.col_ch[blockIdx.z] : a.col_inv_ch[blockIdx.z];
    C *base = a.chan + (size_t)ch * a.NH + (size_t)blockIdx.y * n * n2h;
    const int c0 = blockIdx.x * TW;
    for (int idx = threadIdx.x; idx < n * TW; idx += blockDim.x) {
        const int w = idx % TW, i = idx / TW;
        buf[idx] = (c0 + w < n2h) ? base[(size_t)i * n2h + c0 + w] : cmake<C>((T)0, (T)0);
    }
    __syncthreads();
    fft_smem<DIR, CAP>(buf, TW, TW, a.p1, tw);
    for (int idx = threadIdx.x; idx < n * TW; idx += blockDim.x) {
        const int w = idx % TW, i = idx / TW;
        if (c0 + w < n2h) base[(size_t)i * n2h + c0 + w] = buf[idx];
    }
}

// ======================================================================= axis 0 + reciprocal space
template <typename T> size_t axis0_smem(int n, int TW) {
    typedef typename Vec2<T>::type C;
    return (size_t)n * sizeof(C) + 3 * (size_t)n * TW * sizeof(C) + (size_t)n * TW * sizeof(T) + 16;
}

template <typename T, int CAP>
__global__ void __launch_bounds__(kMaxThreads) axis0_kernel(EvalArgs<T> a) {
    typedef typename Vec2<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sd[32];
    __shared__ double cvec[64][3];
    __shared__ float cw[64];
    __shared__ T sk[OFDFT_MAX_KNOTS];
    const int n = a.n0, TW = a.TW0, n2h = a.n2h;
    const long long P = (long long)a.n1 * n2h;      // columns per plane
    const size_t NT = (size_t)n * TW;
    C *tw = (C *)smem_raw;
    C *S = tw + n;
    C *Rr = S + NT;
    C *A = Rr + NT;
    T *gn = (T *)(A + NT);
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = a.tw0[i];
    const long long c0 = (long long)blockIdx.x * TW;
    // per-column (k1, k2): partial G vector and half-spectrum weight
    for (int w = threadIdx.x; w < TW; w += blockDim.x) {
        const long long col = c0 + w;
        const int k1 = (int)(col / n2h), k2 = (int)(col % n2h);
        const double m1 = (k1 <= a.n1 / 2) ? k1 : k1 - a.n1, m2 = k2;
        for (int d = 0; d < 3; d++) cvec[w][d] = m1 * a.bvec[3 + d] + m2 * a.bvec[6 + d];
        cw[w] = (col < P) ? ((k2 == 0 || (a.n2 % 2 == 0 && k2 == a.n2 / 2)) ? 1.f : 2.f) : 0.f;
    }
    const bool lwt = a.kernel == 0;
    if ((a.terms & 4u) && lwt) for (int i = threadIdx.x; i < a.M; i += blockDim.x) sk[i] = a.knots_t[i];
    __syncthreads();
    for (int idx = threadIdx.x; idx < (int)NT; idx += blockDim.x) {
        const int w = idx % TW, i = idx / TW;
        const double m0 = (i <= n / 2) ? i : i - n;
        const double gx = cvec[w][0] + m0 * a.bvec[0];
        const double gy = cvec[w][1] + m0 * a.bvec[1];
        const double gz = cvec[w][2] + m0 * a.bvec[2];
        gn[idx] = (T)sqrt(gx * gx + gy * gy + gz * gz);
    }
    const T invN = (T)(1.0 / (double)a.N);
    double eH = 0.0, eV = 0.0, eP = 0.0;

    auto load = [&](C *dst, int ch) {
        const C *src = a.chan + (size_t)ch * a.NH;
        for (int idx = threadIdx.x; idx < (int)NT; idx += blockDim.x) {
            const int w = idx % TW, i = idx / TW;
            dst[idx] = (c0 + w < P) ? src[(size_t)i * P + c0 + w] : cmake<C>((T)0, (T)0);
        }
    };
    auto store = [&](const C *srcb, int ch) {
        C *dst = a.chan + (size_t)ch * a.NH;
        for (int idx = threadIdx.x; idx < (int)NT; idx += blockDim.x) {
            const int w = idx % TW, i = idx / TW;
            if (c0 + w < P) dst[(size_t)i * P + c0 + w] = srcb[idx];
        }
    };

    // ---- Hartree + local pseudopotential
    if (a.terms & (8u | 16u)) {
        load(S, CH_HPP);
        __syncthreads();
        fft_smem<-1, CAP>(S, TW, TW, a.p0, tw);
        for (int idx = threadIdx.x; idx < (int)NT; idx += blockDim.x) {
            const int w = idx % TW, i = idx / TW;
            const long long col = c0 + w;
            const C X = cscale(S[idx], invN);
            const T g = gn[idx];
            const T g2 = g * g;
            C out = cmake<C>((T)0, (T)0);
            if (col < P && g2 > (T)0) {
                const double wgt = cw[w];
                if (a.terms & 8u) {
                    const T f = (T)(4.0 * kPi) / g2;
                    eH += wgt * ((double)X.x * X.x + (double)X.y * X.y) / (double)g2;
                    out = cscale(X, f);
                }
                if (a.terms & 16u) {
                    const C v = a.vext[(size_t)i * P + col];
                    eP += wgt * ((double)X.x * v.x + (double)X.y * v.y);
                    out = cadd(out, v);
                }
            } else if (col < P && (a.terms & 16u)) {
                out = a.vext[(size_t)i * P + col];       // G = 0: V_ext(0) only
            }
            S[idx] = out;
        }
        __syncthreads();
        fft_smem<+1, CAP>(S, TW, TW, a.p0, tw);
        store(S, CH_HPP);
        __syncthreads();
    }
    // ---- von Weizsaecker (psi form)
    if (a.terms & 2u) {
        load(S, CH_VW);
        __syncthreads();
        fft_smem<-1, CAP>(S, TW, TW, a.p0, tw);
        for (int idx = threadIdx.x; idx < (int)NT; idx += blockDim.x) {
            const int w = idx % TW;
            const C X = cscale(S[idx], invN);
            const T g = gn[idx];
            const T g2 = g * g;
            eV += (double)cw[w] * (double)g2 * ((double)X.x * X.x + (double)X.y * X.y);
            S[idx] = cscale(X, g2);
        }
        __syncthreads();
        fft_smem<+1, CAP>(S, TW, TW, a.p0, tw);
        store(S, CH_VW);
        __syncthreads();
    }
    // ---- nonlocal: s2 (kernel at each knot) and the reciprocal half of s3
    if (a.terms & 4u) {
        load(Rr, CH_NL);
        __syncthreads();
        fft_smem<-1, CAP>(Rr, TW, TW, a.p0, tw);
        for (int idx = threadIdx.x; idx < (int)NT; idx += blockDim.x) Rr[idx] = cscale(Rr[idx], invN);
        __syncthreads();
        if (!lwt) {
            // global-kF Wang-Teter: K * rho^beta into CH_NL, K * rho^alpha into CH_KNOT0
            const T hk = (T)(0.5 / a.scal[S_KF_WT]);
            load(S, CH_KNOT0);
            __syncthreads();
            fft_smem<-1, CAP>(S, TW, TW, a.p0, tw);
            for (int idx = threadIdx.x; idx < (int)NT; idx += blockDim.x) {
                const T K = (T)kCWT * gnl(gn[idx] * hk);
                Rr[idx] = cscale(Rr[idx], K);
                S[idx] = cscale(S[idx], K * invN);
            }
            __syncthreads();
            fft_smem<+1, CAP>(Rr, TW, TW, a.p0, tw);
            fft_smem<+1, CAP>(S, TW, TW, a.p0, tw);
            store(Rr, CH_NL);
            store(S, CH_KNOT0);
        } else {
            const bool exact = a.nlpot == 0;
            if (exact)
                for (int idx = threadIdx.x; idx < (int)NT; idx += blockDim.x) A[idx] = cmake<C>((T)0, (T)0);
            for (int m = 0; m < a.M; m++) {
                const T hk = (T)0.5 / sk[m];
                if (exact) {
                    load(S, CH_KNOT0 + m);
                    __syncthreads();
                    fft_smem<-1, CAP>(S, TW, TW, a.p0, tw);
                }
                for (int idx = threadIdx.x; idx < (int)NT; idx += blockDim.x) {
                    const T K = (T)kCWT * gnl(gn[idx] * hk);
                    if (exact) A[idx] = cadd(A[idx], cscale(S[idx], K * invN));
                    S[idx] = cscale(Rr[idx], K);
                }
                __syncthreads();
                fft_smem<+1, CAP>(S, TW, TW, a.p0, tw);
                store(S, CH_KNOT0 + m);
                __syncthreads();
            }
            if (exact) {
                fft_smem<+1, CAP>(A, TW, TW, a.p0, tw);
                store(A, CH_NL);
            }
        }
    }
    eH = block_sum(eH, sd);
    if (threadIdx.x == 0) a.part_ax0[3 * blockIdx.x] = eH;
    eV = block_sum(eV, sd);
    if (threadIdx.x == 0) a.part_ax0[3 * blockIdx.x + 1] = eV;
    eP = block_sum(eP, sd);
    if (threadIdx.x == 0) a.part_ax0[3 * blockIdx.x + 2] = eP;
}

// ======================================================================= row inverse (C2R along n2) + s4 + V
template <typename T> size_t row_inv_smem(const EvalArgs<T> &a) {
    typedef typename Vec2<T>::type C;
    const size_t P = (size_t)2 * a.Brow * (a.n2 + 1);
    return a.n2 * sizeof(C) + (size_t)a.n2 * (a.Brow + 1) * sizeof(C) + P * (7 * sizeof(T) + 1) + 16;
}

template <typename T, int CAP>
__global__ void __launch_bounds__(kMaxThreads) row_inv_kernel(EvalArgs<T> a) {
    typedef typename Vec2<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sd[32];
    __shared__ T sk[OFDFT_MAX_KNOTS];
    __shared__ T sidk[OFDFT_MAX_KNOTS];
    const int n = a.n2, n2h = a.n2h, B = a.Brow, ld = B + 1, pl = n + 1;
    const int P = 2 * B * pl;
    C *tw = (C *)smem_raw;
    C *buf = tw + n;
    T *sv = (T *)(buf + (size_t)n * ld);   // V accumulator
    T *sx = sv + P;                        // rho
    T *sa1 = sx + P;                       // rho^(alpha-1)
    T *sb1 = sa1 + P;                      // rho^(beta-1)
    T *skf = sb1 + P;                      // kF/3 inside the knot range, else 0
    T *sea = skf + P;                      // rho^alpha
    T *st = sea + P;                       // spline weight t
    unsigned char *sj = (unsigned char *)(st + P);

    const long long R = (long long)a.n0 * a.n1;
    const long long row0 = 2LL * B * blockIdx.x;
    const bool lwt = (a.terms & 4u) && a.kernel == 0;
    const int M = a.M;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = a.tw2[i];
    if (lwt)
        for (int i = threadIdx.x; i < M; i += blockDim.x) {
            sk[i] = a.knots_t[i];
            sidk[i] = (i + 1 < M) ? a.invdk_t[i] : (T)0;
        }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 2 * B * n; idx += blockDim.x) {
        const int rr = idx / n, i2 = idx - rr * n;
        const long long row = row0 + rr;
        const int o = rr * pl + i2;
        T x = 0;
        if (row < R) x = a.rho[row * n + i2];
        sx[o] = x;
        T v = 0;
        if (a.terms & 1u) {
            const T c = dcbrt(x > (T)0 ? x : (T)0);
            v = (T)(5.0 / 3.0 * kCTF) * c * c;          // V_TF = (5/3) C_TF rho^(2/3)
        }
        sv[o] = v;
        if (a.terms & 4u) {
            const T xf = x > a.floor_ ? x : a.floor_;
            const T ra = dpow(xf, a.alpha);
            const T rb = (a.beta == a.alpha) ? ra : dpow(xf, a.beta);
            sea[o] = ra;
            sa1[o] = ra / xf;
            sb1[o] = rb / xf;
            if (lwt) {
                const T kf = dcbrt((T)kThreePi2 * xf);
                const bool inside = kf >= sk[0] && kf <= sk[M - 1];
                const T kc = kf < sk[0] ? sk[0] : (kf > sk[M - 1] ? sk[M - 1] : kf);
                const int j = knot_interval(kc, sk, M);
                sj[o] = (unsigned char)j;
                st[o] = (kc - sk[j]) * sidk[j];
                skf[o] = (inside && a.nlpot == 0) ? kf * (T)(1.0 / 3.0) : (T)0;
            }
        }
    }
    __syncthreads();
    double eNL = 0.0;
    const T psi_floor = dsqrt(a.floor_);
    const T alpha_eff = (a.nlpot == 1) ? (T)2 * a.alpha : a.alpha;
    for (int ci = 0; ci < a.ninv; ci++) {
        const int ch = a.inv_ch[ci], kind = a.inv_kind[ci], m = a.inv_knot[ci];
        const C *in = a.chan + (size_t)ch * a.NH;
        // pack the pair of half spectra into one full complex spectrum
        for (int idx = threadIdx.x; idx < n2h * B; idx += blockDim.x) {
            const int b = idx / n2h, k = idx - b * n2h;
            const long long r0 = row0 + 2 * b;
            const C z = cmake<C>((T)0, (T)0);
            const C X0 = (r0 < R) ? in[r0 * n2h + k] : z;
            const C X1 = (r0 + 1 < R) ? in[(r0 + 1) * n2h + k] : z;
            if (k == 0 || 2 * k == n) {
                buf[k * ld + b] = cmake<C>(X0.x, X1.x);
            } else {
                buf[k * ld + b] = cmake<C>(X0.x - X1.y, X0.y + X1.x);
                buf[(n - k) * ld + b] = cmake<C>(X0.x + X1.y, X1.x - X0.y);
            }
        }
        __syncthreads();
        fft_smem<+1, CAP>(buf, ld, B, a.p2, tw);
        for (int idx = threadIdx.x; idx < n * B; idx += blockDim.x) {
            const int b = idx % B, i2 = idx / B;
            const C z = buf[i2 * ld + b];
#pragma unroll
            for (int s = 0; s < 2; s++) {
                const int o = (2 * b + s) * pl + i2;
                const T y = s ? z.y : z.x;
                T acc = sv[o];
                if (kind == CONS_ADD) acc += y;
                else if (kind == CONS_VW) {
                    const T p = dsqrt(sx[o] > (T)0 ? sx[o] : (T)0);
                    acc += y / ((T)2 * (p > psi_floor ? p : psi_floor));
                } else if (kind == CONS_T2) acc += a.beta * sb1[o] * y;
                else if (kind == CONS_WT_A) {
                    acc += a.alpha * sa1[o] * y;
                    if (row0 + 2 * b + s < R) eNL += (double)sea[o] * (double)y;
                } else if (kind == CONS_WT_B) acc += a.beta * sb1[o] * y;
                else {
                    const int j = sj[o];
                    if (j == m || j + 1 == m) {
                        const T t = st[o], idk = sidk[j];
                        const T h = (j == m) ? (T)1 - t : t;
                        const T hp = (j == m) ? -idk : idk;
                        acc += y * sa1[o] * (alpha_eff * h + skf[o] * hp);
                        if (row0 + 2 * b + s < R) eNL += (double)(sea[o] * h) * (double)y;
                    }
                }
                sv[o] = acc;
            }
        }
        __syncthreads();
    }
    if (a.V) {
        for (int idx = threadIdx.x; idx < 2 * B * n; idx += blockDim.x) {
            const int rr = idx / n, i2 = idx - rr * n;
            const long long row = row0 + rr;
            if (row < R) a.V[row * n + i2] = sv[rr * pl + i2];
        }
    }
    eNL = block_sum(eNL, sd);
    if (threadIdx.x == 0) a.part_row[blockIdx.x] = eNL;
}

// ======================================================================= finalize
template <typename T>
__global__ void __launch_bounds__(256) finalize_kernel(EvalArgs<T> a) {
    __shared__ double sd[32];
    double h = 0.0, v = 0.0, p = 0.0, nl = 0.0;
    for (int b = threadIdx.x; b < a.nb_ax0; b += blockDim.x) {
        h += a.part_ax0[3 * b];
        v += a.part_ax0[3 * b + 1];
        p += a.part_ax0[3 * b + 2];
    }
    for (int b = threadIdx.x; b < a.nb_row; b += blockDim.x) nl += a.part_row[b];
    h = block_sum(h, sd);
    v = block_sum(v, sd);
    p = block_sum(p, sd);
    nl = block_sum(nl, sd);
    if (threadIdx.x != 0) return;
    double *E = a.energies;
    E[E_VW] = (a.terms & 2u) ? 0.5 * a.omega * v : 0.0;
    E[E_H] = (a.terms & 8u) ? 2.0 * kPi * a.omega * h : 0.0;
    if (a.terms & 16u) {
        const double v0 = (double)a.vext[0].x;                    // V_ext(G = 0)
        E[E_PP] = a.omega * (p + a.scal[S_RHO_MEAN] * v0);
    } else {
        E[E_PP] = 0.0;
    }
    E[E_NL] = (a.terms & 4u) ? nl * a.dV : 0.0;
    E[E_TOT] = E[E_TF] + E[E_VW] + E[E_NL] + E[E_H] + E[E_PP];
}

// ======================================================================= launcher
template <typename T, int CAP>
static cudaError_t launch_all(const EvalArgs<T> &a, cudaStream_t s, const ProfHook *ph) {
    const long long R = (long long)a.n0 * a.n1;
    const long long pairs = (R + 1) / 2;
    const int nrt = (int)((pairs + a.Brow - 1) / a.Brow);
    auto mark = [&](int id, int phase) {
        if (ph) ph->record(ph->ctx, id, phase, s);
    };
    mark(K_STATS, 0);
    stats_kernel<T><<<a.nb_stats, 256, 0, s>>>(a);
    mark(K_STATS, 1);
    mark(K_KNOTS, 0);
    knots_kernel<T><<<1, 256, 0, s>>>(a);
    mark(K_KNOTS, 1);
    if (a.nfwd > 0) {
        mark(K_ROW_FWD, 0);
        row_fwd_kernel<T, CAP><<<nrt, a.thr_rowf, row_fwd_smem(a), s>>>(a);
        mark(K_ROW_FWD, 1);
    }
    dim3 g1((a.n2h + a.TW1 - 1) / a.TW1, a.n0, a.ncol);
    if (a.ncol > 0) {
        mark(K_PENCIL_FWD, 0);
        pencil1_kernel<T, -1, CAP><<<g1, a.thr_p1, pencil_smem<T>(a.n1, a.TW1), s>>>(a);
        mark(K_PENCIL_FWD, 1);
    }
    mark(K_AXIS0, 0);
    axis0_kernel<T, CAP><<<a.nb_ax0, a.thr_ax0, axis0_smem<T>(a.n0, a.TW0), s>>>(a);
    mark(K_AXIS0, 1);
    if (a.ncol_inv > 0) {
        dim3 g2((a.n2h + a.TW1 - 1) / a.TW1, a.n0, a.ncol_inv);
        mark(K_PENCIL_INV, 0);
        pencil1_kernel<T, +1, CAP><<<g2, a.thr_p1, pencil_smem<T>(a.n1, a.TW1), s>>>(a);
        mark(K_PENCIL_INV, 1);
    }
    mark(K_ROW_INV, 0);
    row_inv_kernel<T, CAP><<<nrt, a.thr_rowi, row_inv_smem(a), s>>>(a);
    mark(K_ROW_INV, 1);
    mark(K_FINALIZE, 0);
    finalize_kernel<T><<<1, 256, 0, s>>>(a);
    mark(K_FINALIZE, 1);
    return cudaGetLastError();
}

template <typename T> static cudaError_t set_attrs() {
    constexpr int CAP = Cap<T>::value;
    cudaError_t e;
    if ((e = allow_max_dynamic_smem(row_fwd_kernel<T, CAP>))) return e;
    if ((e = allow_max_dynamic_smem(row_inv_kernel<T, CAP>))) return e;
    if ((e = allow_max_dynamic_smem(pencil1_kernel<T, -1, CAP>))) return e;
    if ((e = allow_max_dynamic_smem(pencil1_kernel<T, +1, CAP>))) return e;
    return allow_max_dynamic_smem(axis0_kernel<T, CAP>);
}

template <typename T> cudaError_t launch_eval(const EvalArgs<T> &a, cudaStream_t s, const ProfHook *prof) {
    static bool attrs = false;
    if (!attrs) {
        cudaError_t e = set_attrs<T>();
        if (e != cudaSuccess) return e;
        attrs = true;
    }
    return launch_all<T, Cap<T>::value>(a, s, prof);
}

template <typename T> cudaError_t launch_forward_rows_cols(const EvalArgs<T> &a, cudaStream_t s) {
    static bool attrs = false;
    if (!attrs) {
        cudaError_t e = set_attrs<T>();
        if (e != cudaSuccess) return e;
        attrs = true;
    }
    const long long R = (long long)a.n0 * a.n1;
    const long long pairs = (R + 1) / 2;
    const int nrt = (int)((pairs + a.Brow - 1) / a.Brow);
    stats_kernel<T><<<a.nb_stats, 256, 0, s>>>(a);
    knots_kernel<T><<<1, 256, 0, s>>>(a);
    constexpr int CAP = Cap<T>::value;
    row_fwd_kernel<T, CAP><<<nrt, a.thr_rowf, row_fwd_smem(a), s>>>(a);
    dim3 g1((a.n2h + a.TW1 - 1) / a.TW1, a.n0, a.ncol);
    pencil1_kernel<T, -1, CAP><<<g1, a.thr_p1, pencil_smem<T>(a.n1, a.TW1), s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_forward_rows_cols<float>(const EvalArgs<float> &, cudaStream_t);
template cudaError_t launch_forward_rows_cols<double>(const EvalArgs<double> &, cudaStream_t);
template cudaError_t launch_eval<float>(const EvalArgs<float> &, cudaStream_t, const ProfHook *);
template cudaError_t launch_eval<double>(const EvalArgs<double> &, cudaStream_t, const ProfHook *);
template size_t row_fwd_smem<float>(const EvalArgs<float> &);
template size_t row_fwd_smem<double>(const EvalArgs<double> &);
template size_t row_inv_smem<float>(const EvalArgs<float> &);
template size_t row_inv_smem<double>(const EvalArgs<double> &);
template size_t pencil_smem<float>(int, int);
template size_t pencil_smem<double>(int, int);
template size_t axis0_smem<float>(int, int);
template size_t axis0_smem<double>(int, int);

}  // namespace ofdft
