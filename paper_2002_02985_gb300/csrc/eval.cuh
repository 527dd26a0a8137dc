// Parameters and launch entry points of the energy/potential pipeline.
//
// One evaluation (Sec. 2.3 steps s1-s4 plus the semilocal terms) runs as:
//   stats     one pass over rho: sum rho, sum rho^(5/3), min/max rho, bad-value flag;
//             its last block reduces the partials in FP64: mean density, kF knots (s1)
//   row_fwd   per pair of rows: forms each channel field from rho and does the
//             real-to-complex FFT along n2
//   pencil    complex FFT along n1 for all channels
//   axis0     FFT along n0, the reciprocal-space products (Hartree, PP, vW,
//             per-knot kernels K_j(G), s2 and s3), FP64 energy partials, and
//             the inverse FFT along n0
//   pencil    inverse complex FFT along n1
//   row_inv   complex-to-real FFT along n2 fused with the s4 spline blend and
//             the assembly of V; FP64 partial of E_NL
//   finalize  1 block: FP64 energies in a fixed order
#pragma once

#include <vector>

#include "fft.cuh"

namespace ofdft {

// channel slots of the workspace (each one half spectrum n0*n1*(n2/2+1))
enum { CH_HPP = 0, CH_VW = 1, CH_NL = 2, CH_KNOT0 = 3 };

// row_inv consumer kinds
enum { CONS_ADD = 0, CONS_VW = 1, CONS_T2 = 2, CONS_KNOT = 3, CONS_WT_A = 4, CONS_WT_B = 5 };

// scalar slots (double) in the workspace
enum {
    S_SUM_RHO = 0, S_SUM_TF = 1, S_RHO_MIN = 2, S_RHO_MAX = 3, S_RHO_MEAN = 4, S_BAD = 5,
    S_KF_WT = 6, S_TIMEOUT = 7,   // S_TIMEOUT: bounded waits that expired (the copies then landed)
    S_FATAL = 8,                  // waits whose copies did not land within the second bound either
    S_NSCAL = 9,
    S_FIN = 16                 // [16, 21): the finalize blocks' five sums
};
// energy slots: total, TF, vW, NL, H, PP, XC
enum { E_TOT = 0, E_TF = 1, E_VW = 2, E_NL = 3, E_H = 4, E_PP = 5, E_XC = 6, E_NUM = 7 };

constexpr int kMaxChan = 3 + OFDFT_MAX_KNOTS;
constexpr int kGroupMax = 32;        // evaluations per grouped launch (tensor maps in the parameters)
constexpr int kMaxThreads = 512;     // block size bound of the FFT kernels

// complex values a thread stages per FFT pass (register budget per precision)
template <typename T> struct Cap { static constexpr int value = sizeof(T) == 4 ? 16 : 8; };

template <typename T> struct EvalArgs {
    typedef typename Vec2<T>::type C;
    int n0, n1, n2, n2h;
    long long N, NH;
    double omega, dV;
    double bvec[9];          // 2 pi b_i (rows), b = inv(cell)^T
    const T *rho;
    T *V;                    // may be null
    C *chan;                 // workspace channels, slot c at chan + c * NH
    const C *vext;           // V_ext(G) half spectrum, null if no PP
    unsigned terms;
    int kernel, nlpot, M;    // kernel: 0 LWT, 1 WT global
    const T *mgp_tab;        // MGP correction J_y on eta/(1+eta) (null: Wang-Teter kernel)
    int mgp_n;               // table points
    T mgp_1mx, mgp_3xy;      // K = C_WT ((1 - x) G_NL + 3 x y J_y)
    T alpha, beta, floor_;
    double *scal;            // S_* slots
    double *knots_d;         // [M] FP64 knots
    T *knots_t;              // [M] knots rounded to T
    T *invdk_t;              // [M-1] 1/(k_{j+1}-k_j), 0 for a zero-width interval
    int frozen;              // knots supplied by the caller
    int knot_spacing;
    double *part_stats;      // [nb_stats * 3]: sum rho, sum rho^(5/3), sum rho eps_xc
    T *part_minmax;          // [nb_stats * 2]
    double *part_ax0;        // [nb_ax0 * 3]: S_H, S_vW, S_PP
    double *part_row;        // [nb_row]: S_NL
    double *energies;        // [6] device output
    unsigned *ticket;        // completion counter of the stats blocks (zero between launches)
    int nb_stats, nb_ax0, nb_row;
    FFTPlan p0, p1, p2;
    const C *tw0, *tw1, *tw2;
    int Brow, thr_rowf, thr_rowi, TW1, thr_p1, TW0, thr_ax0;
    int grid_p1;                         // persistent grid of the n1 pencil kernels
    int row2_G;                          // channel-batched row kernels: channels per group (0: per-channel form)
    int ax0_scr;                         // the reciprocal-space kernel has a scratch tile (out-of-place transforms)
    unsigned wait_polls;                 // polls of a bounded wait for bulk copies before it gives up
    int exact_sums;                      // FP32-mixed test option: every energy term added in FP64
    C *rhohat_out;                       // if set: the normalised rho_hat (Hartree/PP channel) for the forces
    int nfwd, fwd_ch[kMaxChan];          // channels formed by row_fwd (slot ids)
    int ncol, col_ch[kMaxChan];          // channels transformed forward along n1
    int ncol_inv, col_inv_ch[kMaxChan];  // channels transformed back along n1
    int ninv, inv_ch[kMaxChan], inv_kind[kMaxChan], inv_knot[kMaxChan];
};

// Optional per-kernel timing: record(ctx, kernel_id, phase) is called with
// phase 0 just before and phase 1 just after each launch (ids: KernelId).
enum KernelId { K_STATS = 0, K_KNOTS, K_ROW_FWD, K_PENCIL_FWD, K_AXIS0, K_PENCIL_INV, K_ROW_INV, K_FINALIZE, K_NKERNEL };
struct ProfHook {
    void (*record)(void *ctx, int kernel_id, int phase, cudaStream_t s);
    void *ctx;
};

// Dynamic shared memory of the FFT-carrying kernels (tile layouts in kernels.cuh).
// row tiles: the complex FFT buffer (n x (B+1)) doubles as the density staging
// area ([2B][pitch], pitch odd), so it is sized for the larger of the two
__host__ __device__ inline int row_pitch(int n) { return n % 2 ? n + 2 : n + 1; }
template <typename T> __host__ __device__ inline size_t row_buf_bytes(int n2, int B) {
    const size_t fft = (size_t)n2 * (B + 1) * 2 * sizeof(T);
    const size_t stg = (size_t)2 * B * row_pitch(n2) * sizeof(T);
    const size_t m = fft > stg ? fft : stg;
    return (m + 15) / 16 * 16;
}
template <typename T> __host__ __device__ inline size_t row_fwd_smem_bytes(int n2, int B) {
    typedef typename Vec2<T>::type C;
    const size_t P = (size_t)2 * B * n2;
    return n2 * sizeof(C) + row_buf_bytes<T>(n2, B) + P * (4 * sizeof(T) + 1) + 16;
}
template <typename T> __host__ __device__ inline size_t pencil_smem_bytes(int n, int TW) {
    typedef typename Vec2<T>::type C;
    // twiddles + two tile buffers (prefetch ping-pong) + the transform's scratch
    return (size_t)n * sizeof(C) + 3 * (size_t)n * TW * sizeof(C);
}

// Whether the size-specialised reciprocal-space kernel for n0 = n transforms out of place
// (in place measured faster for the FP32 128-point tiles).
template <typename T> __host__ __device__ constexpr bool axis0_oop(int n) { return !(sizeof(T) == 4 && n == 128); }

template <typename T> __host__ __device__ inline size_t axis0_smem_bytes(int n, int TW, bool scratch) {
    typedef typename Vec2<T>::type C;
    // twiddles, two load buffers, rho^beta, the term-2 accumulator, the out-of-place
    // transforms' scratch (if any), |G|
    return (size_t)n * sizeof(C) + (scratch ? 5 : 4) * (size_t)n * TW * sizeof(C) + (size_t)n * TW * sizeof(T) + 16;
}

template <typename T> __host__ __device__ inline size_t row_inv_smem_bytes(int n2, int B) {
    typedef typename Vec2<T>::type C;
    const size_t P = (size_t)2 * B * n2;
    return n2 * sizeof(C) + row_buf_bytes<T>(n2, B) + P * (6 * sizeof(T) + 1) + 16;
}

// channel-batched row kernels: twiddles and two buffers, each of max(n2 x LD, G (n2 + 2))
// complex (LD = G, or G + 1 if G is even): the batch and the transform's scratch, which also
// stage G pairs of half-spectrum rows
template <typename T> __host__ __device__ inline size_t row2_smem_bytes(int n2, int G) {
    typedef typename Vec2<T>::type C;
    const int ld = (G % 2) ? G : G + 1;
    const size_t scr = ((size_t)n2 * ld > (size_t)G * (n2 + 2)) ? (size_t)n2 * ld : (size_t)G * (n2 + 2);
    return (size_t)n2 * sizeof(C) + 2 * scr * sizeof(C) + 16;
}
template <typename T> __host__ __device__ inline size_t rowf_smem(const EvalArgs<T> &a) {
    return a.row2_G ? row2_smem_bytes<T>(a.n2, a.row2_G) : row_fwd_smem_bytes<T>(a.n2, a.Brow);
}
template <typename T> __host__ __device__ inline size_t rowi_smem(const EvalArgs<T> &a) {
    return a.row2_G ? row2_smem_bytes<T>(a.n2, a.row2_G) : row_inv_smem_bytes<T>(a.n2, a.Brow);
}

// persistent pencil grid: at most grid_p1 blocks (resident capacity), never more than tiles
template <typename T> inline unsigned pencil_tiles(const EvalArgs<T> &a, int nch) {
    const long long t = (((long long)a.n0 * a.n2h + a.TW1 - 1) / a.TW1) * nch;
    return (unsigned)(t < a.grid_p1 ? t : a.grid_p1);
}

// The persistent reciprocal-space kernel (register-resident n0 transforms, tensor-map tile
// loads; recip.cuh) compiled for an n0: Wang-Teter and Eq. MGP forms, block size, dynamic
// shared memory, blocks per SM.
struct RecipLaunch {
    const void *k = nullptr, *k_mgp = nullptr;
    const void *g = nullptr, *g_mgp = nullptr;   // grouped forms (null: none compiled)
    int nt = 0, per_sm = 1;
    int tw = 32;                 // columns per tile (the tensor copies' box width)
    size_t smem = 0;
};

// The five FFT-carrying kernels of one evaluation (generic or size-specialised).
struct LaunchSet {
    const void *row_fwd = nullptr, *row_inv = nullptr;   // depend on n2
    const void *pen_fwd = nullptr, *pen_inv = nullptr;   // depend on n1
    const void *axis0 = nullptr;                         // depends on n0
    const void *axis0_mgp = nullptr;                     // the same with Eq. MGP kernels
    RecipLaunch recip;                                   // replaces axis0 when its k is set
    // grouped forms of the five (one launch over the evaluations of a batch that share a
    // launch geometry); null where none is compiled
    const void *row_fwd_g = nullptr, *row_inv_g = nullptr, *pen_fwd_g = nullptr, *pen_inv_g = nullptr;
    const void *axis0_g = nullptr, *axis0_mgp_g = nullptr;
};

// tensor maps of the persistent reciprocal-space kernel (defined in recip.cuh)
struct RecipMaps;

// role of a kernel family for the size registry
enum { ROLE_ROW = 0, ROLE_PENCIL = 1, ROLE_AXIS0 = 2, ROLE_ROW2 = 3 };

// One compiled configuration of a role: the kernel pair (rows and pencils: forward and
// inverse; the tile reciprocal-space kernel: Wang-Teter and Eq. MGP forms), its fixed batch
// (row pairs, channel group G, or column-tile width TW) and block size; for ROLE_AXIS0 the
// persistent kernel instead when recip.k is set.
struct KernelCand {
    const void *k1 = nullptr, *k2 = nullptr;
    const void *g1 = nullptr, *g2 = nullptr;   // their grouped forms
    int B = 0, nt = 0;
    bool batched = false;                 // channel-batched row kernels (B = channels per group)
    RecipLaunch recip;
    char name[48] = {0};
};

// The compiled configurations of a role for axis length n (empty: only the runtime-size
// kernels exist), the default first.  ROLE_AXIS0 lists the persistent kernels first.
template <typename T> void kernel_candidates(int role, int n, std::vector<KernelCand> &out);
// The default configuration of a role for size n; false when none is compiled.
template <typename T> bool find_specialised(int role, int n, const void **k1, const void **k2, int *B, int *nt);
// the persistent reciprocal-space kernels compiled for n0 = n (recip.cu)
template <typename T> void recip_candidates(int n, std::vector<KernelCand> &out);
// The generic (runtime-size) kernels (exact_sums: the forms that add every energy term in FP64).
template <typename T> LaunchSet generic_kernels(bool exact_sums = false);
// the grouped forms of the generic kernels (without exact sums) into ks (group_kernels.cu)
template <typename T> void generic_group_kernels(LaunchSet &ks);
// Let every kernel of the set use the device's full opt-in shared memory.
cudaError_t prepare_kernels(const LaunchSet &ks);

// maps: the tensor maps of the persistent reciprocal-space kernel (needed when ks.recip.k is set;
// a.nb_ax0 is then its grid)
template <typename T> cudaError_t launch_eval(const EvalArgs<T> &a, const LaunchSet &ks, cudaStream_t s,
                                              const ProfHook *prof = nullptr, const RecipMaps *maps = nullptr);
// Grouped launch of K <= kGroupMax evaluations sharing a's launch geometry (a: the host copy
// of any one of them; ga: all K in device memory; maps: their K tensor-map pairs when
// ks.recip.k is set).  Only when grouped_ok(ks, a): every kernel of the evaluation has a
// grouped form (FP32 kernels, without the exact-sums option).
template <typename T> bool grouped_ok(const LaunchSet &ks, const EvalArgs<T> &a);
template <typename T> cudaError_t launch_group(const EvalArgs<T> &a, const EvalArgs<T> *ga, int K, const LaunchSet &ks,
                                               cudaStream_t s, const RecipMaps *maps = nullptr);
// copies the energies and scalar slots of ga[0..n) to out (E_NUM + S_NSCAL doubles each)
template <typename T> cudaError_t launch_collect(const EvalArgs<T> *ga, int n, double *out, cudaStream_t s);
// inverse pencil along n1 + C2R rows of the channels in a.col_inv_ch / a.inv_ch (CONS_ADD), V = result
template <typename T> cudaError_t launch_inverse_cols_rows(const EvalArgs<T> &a, const LaunchSet &ks, cudaStream_t s);
// stats + knots + row_fwd + forward pencil along n1 only (the channels of a.fwd_ch / a.col_ch)
template <typename T> cudaError_t launch_forward_rows_cols(const EvalArgs<T> &a, const LaunchSet &ks, cudaStream_t s);
// Table of the MGP correction J_y(eta) = 2 int_0^1 r^(6y-1) G_NL(eta/r^2) dr at eta = u/(1-u),
// u = i/(n-1), i = 0..n-1 (FP64 Gauss-Legendre quadrature; gl = 8 nodes and 8 weights on [-1, 1])
template <typename T> cudaError_t launch_mgp_table(T *tab, int n, double y, const double *gl, cudaStream_t s);

}  // namespace ofdft
