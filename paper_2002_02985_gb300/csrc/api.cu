// C ABI of the OFDFT library: grid handle, planning, workspace, evaluation,
// forces, batched evaluation and the psi = sqrt(rho) CG optimiser.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/ofdft.h"
#include "eval.cuh"
#include "recip.cuh"
#include "ewald.cuh"
#include "misc.cuh"
#include "pme.cuh"

using namespace ofdft;

namespace {


bool factor_235(int n, std::vector<int> &radix) {
    radix.clear();
    int m = n, p2 = 0;
    while (m % 2 == 0) { m /= 2; p2++; }
    while (p2 >= 3) { radix.push_back(8); p2 -= 3; }
    if (p2 == 2) radix.push_back(4);
    if (p2 == 1) radix.push_back(2);
    while (m % 5 == 0) { m /= 5; radix.push_back(5); }
    while (m % 3 == 0) { m /= 3; radix.push_back(3); }
    return m == 1;
}

FFTPlan make_plan(int n) {
    FFTPlan p;
    std::memset(&p, 0, sizeof(p));
    std::vector<int> r;
    factor_235(n, r);
    p.n = n;
    p.npass = (int)r.size();
    int ns = 1;
    for (int i = 0; i < p.npass; i++) {
        p.radix[i] = r[i];
        p.ns[i] = ns;
        ns *= r[i];
    }
    return p;
}

// smallest multiple-of-32 thread count that keeps every pass within cap staged values
int threads_for(const FFTPlan &p, int B, int cap, int lo = 64) {
    int need = lo;
    for (int i = 0; i < p.npass; i++) {
        const int R = p.radix[i], mb = cap / R;
        const int total = (p.n / R) * B;
        const int t = (total + mb - 1) / mb;
        if (t > need) need = t;
    }
    need = (need + 31) / 32 * 32;
    return need;
}

template <typename T> struct Workspace {
    typedef typename Vec2<T>::type C;
    bool ready = false;
    int nslots = 0;
    C *chan = nullptr;
    C *tw[3] = {nullptr, nullptr, nullptr};
    C *vext = nullptr;
    double *scal = nullptr, *energies = nullptr, *knots_d = nullptr;
    T *knots_t = nullptr, *invdk_t = nullptr, *part_minmax = nullptr;
    double *part_stats = nullptr, *part_ax0 = nullptr, *part_row = nullptr, *part_misc = nullptr;
    unsigned *ticket = nullptr;       // stats completion counter
    T *opt = nullptr;                 // optimiser fields (8 * N), allocated on demand
    T *opt_ext = nullptr;             // TN / L-BFGS fields (opt_ext_fields * N), on demand
    T *td = nullptr;                  // TD-OFDFT fields (19 * N), on demand
    T *mgp_tab = nullptr;             // MGP correction table (kMgpTable points), on demand
    C *rhohat = nullptr;              // normalised rho_hat kept by an evaluation for the forces
    double mgp_y = 0.0;               // the y it was built for (0: not built)
    int opt_ext_fields = 0;
    LaunchSet ks;                     // FFT-carrying kernels (size-specialised where compiled)
    int Brow = 0, thr_rowf = 0, thr_rowi = 0, TW1 = 0, thr_p1 = 0, TW0 = 0, thr_ax0 = 0, nb_row = 0, nb_ax0 = 0;
    int grid_p1 = 0;
    int row2_G = 0;                   // channel-batched row kernels in use: channels per group
    int ax0_scr = 0;                  // the reciprocal-space kernel transforms out of place
    // plain one-channel transforms (preconditioner, interpolation, TD-OFDFT): the per-channel row
    // kernels where compiled (the channel-batched ones would leave most of each block idle)
    LaunchSet ks_plain;
    int Brow_p = 0, thr_rowf_p = 0, thr_rowi_p = 0, row2_G_p = 0;
    // persistent reciprocal-space kernel: its grid, and its tensor maps with the buffers
    // and channel count they were encoded for; the tile kernel's grid
    int recip_grid = 0, tile_nb_ax0 = 0;
    // compiled configurations per tuned role, the one in use, and the autotuner's record
    std::vector<KernelCand> cand[3];
    int pick[3] = {-1, -1, -1};
    bool tuned = false, tuning = false;
    std::string tune_report;
    RecipMaps maps;
    const void *maps_chan = nullptr, *maps_vext = nullptr;
    int maps_nslots = 0, maps_tw = 0;
};

}  // namespace

struct ofdft_grid {
    int n[3];
    int n2h;
    long long N, NH;
    double cell[9], recip[9], omega, dV;
    cudaStream_t stream;
    int device;
    int nsm;
    FFTPlan plan[3];
    Workspace<float> w32;
    Workspace<double> w64;
    // ions
    int n_ions = 0, n_species = 0;
    std::vector<double> pos, Z, rc;
    std::vector<int> species;
    bool have_ions = false;
    bool vext_fresh32 = false, vext_fresh64 = false;
    double2 *ph = nullptr;       // phase tables [n_ions][n0 + n1 + n2h]
    float2 *ph32 = nullptr;      // the same rounded to FP32 (FP32-mixed kernels)
    float *gf = nullptr;         // per-species form-factor tables of the FP32-mixed force kernel
    long long gf_len = 0;
    bool gf_fresh = false;       // the tables match the current ions (species, Z, rc)
    int *d_sp_ions = nullptr;    // the ions grouped by species (device), the groups' offsets (host)
    std::vector<int> sp_off;
    // smooth PME (ofdft_set_ions_pme): order > 0 selects it for V_ext(G) and forces
    int pme_order = 0;
    double2 *pmeB = nullptr;               // conj b_a tables [n0 | n1 | n2h]
    double *d_pos = nullptr;               // device positions
    unsigned long long *Qfix = nullptr;    // fixed-point charge grid (N)
    void *pme_real = nullptr;              // real field scratch (N, largest precision used)
    size_t pme_real_bytes = 0;
    std::vector<int> species_count;
    // asynchronous forces (batched evaluation): device partials, device F, pinned copy
    double *fpart = nullptr;
    size_t fpart_len = 0;
    double *F_dev = nullptr, *F_pinned = nullptr;
    int F_len = 0;
    unsigned long long generation = 0;     // bumped whenever device buffers are (re)allocated
    // ion-ion Ewald sum: sorted ions, cell list, results
    double4 *ew_p = nullptr;
    int *ew_cell = nullptr, *ew_orig = nullptr, *ew_cstart = nullptr;
    double *ew_F = nullptr, *ew_e = nullptr, *ew_part = nullptr;
    int ew_n = 0, ew_ncell = 0;
    int *d_species = nullptr;
    double *d_Z = nullptr, *d_rc = nullptr;
    double *h_pinned = nullptr;  // 64 doubles of pinned host memory
    std::string err;
    // ofdft_set_option
    int kernel_choice = OFDFT_KERNELS_AUTO;
    int force_pick[3] = {-1, -1, -1};    // per tuned role: a fixed candidate (-1: the autotuner's pick)
    int exact_sums = 0;                  // FP32-mixed: every energy term and dot product term in FP64
    int batch_graph = 1;
    int batch_grouped = -1;              // -1: timed both ways at a batch's first call
    std::string batch_report;            // the plan of the last batch whose first grid this was
    unsigned wait_polls = 1u << 22;
    size_t alloc_cap = 0, alloc_bytes = 0;
    // per-kernel CUDA-event timing (ofdft_profile_*)
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<cudaEvent_t> ev_pending = std::vector<cudaEvent_t>(K_NKERNEL, nullptr);
    struct Rec { int id; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    double prof_ms[K_NKERNEL] = {0};
    int prof_n[K_NKERNEL] = {0};
};

namespace {

int fail(ofdft_grid *g, int code, const char *what, cudaError_t e = cudaSuccess) {
    // a non-sticky error must not be reported again by the next call's launch check
    if (e != cudaSuccess) (void)cudaGetLastError();
    if (g) {
        char buf[512];
        if (e != cudaSuccess) std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
        else std::snprintf(buf, sizeof(buf), "%s", what);
        g->err = buf;
    }
    return code;
}

#define CK(call, what)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(g, e_ == cudaErrorMemoryAllocation ? OFDFT_ERR_OOM : OFDFT_ERR_CUDA, \
                        what, e_);                                                           \
    } while (0)

static_assert(E_NUM == OFDFT_N_ENERGIES, "energy slots");

// every device allocation of a grid goes through here: the optional cap of
// ofdft_set_option(OFDFT_OPTION_ALLOC_CAP) is checked first (out of memory past it)
template <typename P> cudaError_t gmalloc(ofdft_grid *g, P **p, size_t bytes) {
    if (g->alloc_cap && g->alloc_bytes + bytes > g->alloc_cap) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) g->alloc_bytes += bytes;
    return e;
}

template <typename T> Workspace<T> &ws(ofdft_grid *g);
template <> Workspace<float> &ws<float>(ofdft_grid *g) { return g->w32; }
template <> Workspace<double> &ws<double>(ofdft_grid *g) { return g->w64; }

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point query, so the
// library does not link libcuda); null if the driver does not provide it
PFN_cuTensorMapEncodeTiled_v12000 tensor_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return (PFN_cuTensorMapEncodeTiled_v12000)p;
    }();
    return fn;
}

// 3-D tensor map over nch half spectra of T words: [channel][k0][c], c < PL complex values,
// boxes of box_cols complex x box_rows rows x 1 channel
template <typename T>
bool encode_spectra_map(CUtensorMap *m, const void *base, long long PL, int n0, int nch, int box_rows, int box_cols) {
    const int wpc = 2;                                   // T words per complex value
    const cuuint64_t dims[3] = {(cuuint64_t)(PL * wpc), (cuuint64_t)n0, (cuuint64_t)nch};
    const cuuint64_t strides[2] = {(cuuint64_t)(PL * wpc * sizeof(T)), (cuuint64_t)(PL * n0 * wpc * sizeof(T))};
    const cuuint32_t box[3] = {(cuuint32_t)(box_cols * wpc), (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = tensor_encoder()(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                                        3, const_cast<void *>(base), dims, strides, box, estr,
                                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------- launch plan and autotuner
// Roles of the tuned kernel families: rows along n2, pencils along n1, the reciprocal-space pass.
enum { TUNE_ROWS = 0, TUNE_PENCIL = 1, TUNE_AXIS0 = 2, TUNE_NROLE = 3 };

// put a candidate of a role into the workspace's launch plan
template <typename T> int apply_cand(ofdft_grid *g, Workspace<T> &w, int role, const KernelCand &c) {
    if (role == TUNE_ROWS) {
        w.ks.row_fwd = c.k1;
        w.ks.row_inv = c.k2;
        w.ks.row_fwd_g = c.g1;
        w.ks.row_inv_g = c.g2;
        w.Brow = c.batched ? 1 : c.B;
        w.row2_G = c.batched ? c.B : 0;
        w.thr_rowf = w.thr_rowi = c.nt;
    } else if (role == TUNE_PENCIL) {
        w.ks.pen_fwd = c.k1;
        w.ks.pen_inv = c.k2;
        w.ks.pen_fwd_g = c.g1;
        w.ks.pen_inv_g = c.g2;
        // the plain one-channel transforms use the same pencils (and the same TW1, threads and grid)
        w.ks_plain.pen_fwd = c.k1;
        w.ks_plain.pen_inv = c.k2;
        w.ks_plain.pen_fwd_g = c.g1;
        w.ks_plain.pen_inv_g = c.g2;
        w.TW1 = c.B;
        w.thr_p1 = c.nt;
        // persistent pencil grid: every resident block slot of the device, once
        int per_sm = 0;
        cudaError_t e = allow_max_dynamic_smem(c.k1);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c.k1, c.nt, pencil_smem_bytes<T>(g->n[1], c.B));
        if (e != cudaSuccess) return fail(g, OFDFT_ERR_CUDA, "occupancy", e);
        w.grid_p1 = std::max(1, per_sm) * g->nsm;
    } else {
        const long long P = (long long)g->n[1] * g->n2h;
        if (c.recip.k) {
            w.ks.recip = c.recip;
            w.recip_grid = (int)std::min((P + c.recip.tw - 1) / c.recip.tw, (long long)c.recip.per_sm * g->nsm);
        } else {
            w.ks.recip = RecipLaunch();
            w.ks.axis0 = c.k1;
            w.ks.axis0_mgp = c.k2;
            w.ks.axis0_g = c.g1;
            w.ks.axis0_mgp_g = c.g2;
            w.TW0 = c.B;
            w.thr_ax0 = c.nt;
            w.ax0_scr = axis0_oop<T>(g->n[0]) ? 1 : 0;
            w.tile_nb_ax0 = (int)((P + c.B - 1) / c.B);
        }
    }
    return OFDFT_OK;
}

template <typename T> int choose_launch(ofdft_grid *g, Workspace<T> &w) {
    const size_t row_budget = 110 * 1024;
    const int cap = Cap<T>::value, tmax = kMaxThreads;
    // exact sums run the runtime-size kernels in their FP64-summing forms (the specialised ones
    // keep only the default grouping)
    const bool generic_only = g->kernel_choice == OFDFT_KERNELS_GENERIC || g->exact_sums;
    w.ks = generic_kernels<T>(g->exact_sums != 0);
    for (int r = 0; r < TUNE_NROLE; r++) {
        w.cand[r].clear();
        w.pick[r] = -1;
    }
    w.tuned = false;
    w.tune_report.clear();
    // runtime-size defaults (replaced below where compiled configurations exist)
    {
        int B = 16;
        for (; B >= 1; B /= 2)
            if (row_inv_smem_bytes<T>(g->n[2], B) <= row_budget && threads_for(g->plan[2], B, cap) <= tmax) break;
        // long FP64 rows: one row pair per block may need more than the preferred budget
        if (B < 1 && row_inv_smem_bytes<T>(g->n[2], 1) <= 200 * 1024 && threads_for(g->plan[2], 1, cap) <= tmax) B = 1;
        if (B < 1) return fail(g, OFDFT_ERR_UNSUPPORTED_SIZE, "row transform does not fit in shared memory");
        w.Brow = B;
        w.row2_G = 0;
        w.thr_rowf = w.thr_rowi = std::min(std::max(threads_for(g->plan[2], B, cap), 128), tmax);
        int TW = 16;
        while (TW > 1 && (pencil_smem_bytes<T>(g->n[1], TW) > 96 * 1024 || threads_for(g->plan[1], TW, cap) > tmax))
            TW /= 2;
        w.TW1 = TW;
        w.thr_p1 = std::min(std::max(threads_for(g->plan[1], TW, cap), 128), tmax);
        TW = 16;
        w.ax0_scr = 0;
        while (TW > 1 && (axis0_smem_bytes<T>(g->n[0], TW, false) > 200 * 1024 || threads_for(g->plan[0], TW, cap) > tmax))
            TW /= 2;
        w.TW0 = TW;
        w.thr_ax0 = std::min(std::max(threads_for(g->plan[0], TW, cap), 128), tmax);
        w.ks.recip = RecipLaunch();
    }
    const long long P = (long long)g->n[1] * g->n2h;
    if (!generic_only) {
        // rows: the channel-batched configurations (unless OFDFT_KERNELS_PER_CHANNEL_ROWS), then
        // the per-channel ones
        std::vector<KernelCand> c;
        if (g->kernel_choice != OFDFT_KERNELS_PER_CHANNEL_ROWS) {
            kernel_candidates<T>(ROLE_ROW2, g->n[2], c);
            w.cand[TUNE_ROWS] = c;
        }
        kernel_candidates<T>(ROLE_ROW, g->n[2], c);
        w.cand[TUNE_ROWS].insert(w.cand[TUNE_ROWS].end(), c.begin(), c.end());
        kernel_candidates<T>(ROLE_PENCIL, g->n[1], w.cand[TUNE_PENCIL]);
        // the reciprocal-space pass: the persistent kernels where compiled for n0 (their tensor
        // maps need rows of an even number of complex values, 16-byte strides), then the tile ones
        kernel_candidates<T>(ROLE_AXIS0, g->n[0], c);
        for (const KernelCand &k : c) {
            if (k.recip.k && (g->kernel_choice == OFDFT_KERNELS_TILE_RECIP ||
                              g->kernel_choice == OFDFT_KERNELS_PER_CHANNEL_ROWS || P % 2 != 0 || !tensor_encoder()))
                continue;
            w.cand[TUNE_AXIS0].push_back(k);
        }
    }
    // partial buffers sized for every configuration; the first of each role is the default
    w.tile_nb_ax0 = (int)((P + w.TW0 - 1) / w.TW0);
    w.nb_ax0 = w.tile_nb_ax0;
    int min_brow = w.Brow;
    for (const KernelCand &k : w.cand[TUNE_AXIS0])
        w.nb_ax0 = std::max(w.nb_ax0, k.recip.k ? (int)std::min((P + k.recip.tw - 1) / k.recip.tw,
                                                                (long long)k.recip.per_sm * g->nsm)
                                                 : (int)((P + k.B - 1) / k.B));
    for (const KernelCand &k : w.cand[TUNE_ROWS]) min_brow = std::min(min_brow, k.batched ? 1 : k.B);
    for (int r = 0; r < TUNE_NROLE; r++) {
        for (const KernelCand &k : w.cand[r]) {
            LaunchSet one;
            one.row_fwd = k.k1;
            one.row_inv = k.k2;
            one.row_fwd_g = k.g1;
            one.row_inv_g = k.g2;
            one.recip = k.recip;
            cudaError_t e = prepare_kernels(one);
            if (e != cudaSuccess) return fail(g, OFDFT_ERR_CUDA, "kernel attributes", e);
        }
        if (!w.cand[r].empty()) {
            const int fp = g->force_pick[r];
            w.pick[r] = (fp >= 0 && fp < (int)w.cand[r].size()) ? fp : 0;
            int rc = apply_cand<T>(g, w, r, w.cand[r][w.pick[r]]);
            if (rc) return rc;
        }
    }
    if (w.pick[TUNE_PENCIL] < 0) {
        int rc = apply_cand<T>(g, w, TUNE_PENCIL, KernelCand{w.ks.pen_fwd, w.ks.pen_inv, w.ks.pen_fwd_g, w.ks.pen_inv_g, w.TW1, w.thr_p1});
        if (rc) return rc;
    }
    // plain one-channel transforms: the per-channel row kernels where compiled
    w.ks_plain = w.ks;
    w.Brow_p = w.Brow;
    w.thr_rowf_p = w.thr_rowf;
    w.thr_rowi_p = w.thr_rowi;
    w.row2_G_p = w.row2_G;
    for (const KernelCand &k : w.cand[TUNE_ROWS])
        if (!k.batched) {
            w.ks_plain.row_fwd = k.k1;
            w.ks_plain.row_inv = k.k2;
            w.Brow_p = k.B;
            w.thr_rowf_p = w.thr_rowi_p = k.nt;
            w.row2_G_p = 0;
            break;
        }
    cudaError_t e = prepare_kernels(w.ks);
    if (e == cudaSuccess) e = prepare_kernels(w.ks_plain);
    if (e != cudaSuccess) return fail(g, OFDFT_ERR_CUDA, "kernel attributes", e);
    const long long R = (long long)g->n[0] * g->n[1];
    w.nb_row = (int)(((R + 1) / 2 + min_brow - 1) / min_brow);
    return OFDFT_OK;
}

template <typename T> int ensure_ws(ofdft_grid *g, int nslots) {
    typedef typename Vec2<T>::type C;
    Workspace<T> &w = ws<T>(g);
    if (!w.ready) {
        int rc = choose_launch<T>(g, w);
        if (rc) return rc;
        for (int a = 0; a < 3; a++) {
            const int n = g->n[a];
            std::vector<C> h(n);
            for (int k = 0; k < n; k++) {
                const double ang = -2.0 * kPi * (double)k / (double)n;
                h[k].x = (T)std::cos(ang);
                h[k].y = (T)std::sin(ang);
            }
            CK(gmalloc(g, &w.tw[a], n * sizeof(C)), "cudaMalloc twiddles");
            CK(cudaMemcpy(w.tw[a], h.data(), n * sizeof(C), cudaMemcpyHostToDevice), "upload twiddles");
        }
        CK(gmalloc(g, &w.scal, 64 * sizeof(double)), "cudaMalloc scalars");
        CK(cudaMemset(w.scal, 0, 64 * sizeof(double)), "memset");
        CK(gmalloc(g, &w.energies, 8 * sizeof(double)), "cudaMalloc energies");
        CK(gmalloc(g, &w.knots_d, OFDFT_MAX_KNOTS * sizeof(double)), "cudaMalloc knots");
        CK(gmalloc(g, &w.knots_t, OFDFT_MAX_KNOTS * sizeof(T)), "cudaMalloc knots");
        CK(gmalloc(g, &w.invdk_t, OFDFT_MAX_KNOTS * sizeof(T)), "cudaMalloc knots");
        const int nbs = 2 * g->nsm;
        CK(gmalloc(g, &w.part_stats, 3 * nbs * sizeof(double)), "cudaMalloc partials");
        CK(gmalloc(g, &w.part_minmax, 2 * nbs * sizeof(T)), "cudaMalloc partials");
        CK(gmalloc(g, &w.part_ax0, 4 * (size_t)w.nb_ax0 * sizeof(double)), "cudaMalloc partials");
        CK(gmalloc(g, &w.part_row, (size_t)w.nb_row * sizeof(double)), "cudaMalloc partials");
        CK(gmalloc(g, &w.part_misc, 4096 * sizeof(double)), "cudaMalloc partials");
        CK(gmalloc(g, &w.ticket, sizeof(unsigned)), "cudaMalloc ticket");
        CK(cudaMemset(w.ticket, 0, sizeof(unsigned)), "memset ticket");

        w.ready = true;
    }
    if (nslots > w.nslots) {
        if (w.chan) cudaFree(w.chan);
        w.chan = nullptr;
        w.nslots = 0;
        CK(gmalloc(g, &w.chan, (size_t)nslots * g->NH * sizeof(C)), "cudaMalloc channel workspace");
        w.nslots = nslots;
        g->generation++;
    }
    return OFDFT_OK;
}

template <typename T> void free_ws(Workspace<T> &w) {
    cudaFree(w.chan);
    for (int a = 0; a < 3; a++) cudaFree(w.tw[a]);
    cudaFree(w.vext);
    cudaFree(w.scal);
    cudaFree(w.energies);
    cudaFree(w.knots_d);
    cudaFree(w.knots_t);
    cudaFree(w.invdk_t);
    cudaFree(w.part_minmax);
    cudaFree(w.part_stats);
    cudaFree(w.part_ax0);
    cudaFree(w.part_row);
    cudaFree(w.part_misc);
    cudaFree(w.ticket);
    cudaFree(w.opt);
    cudaFree(w.opt_ext);
    cudaFree(w.td);
    cudaFree(w.mgp_tab);
    cudaFree(w.rhohat);
    w = Workspace<T>();
}

IonArgs ion_args(ofdft_grid *g) {
    IonArgs a;
    a.n0 = g->n[0];
    a.n1 = g->n[1];
    a.n2 = g->n[2];
    a.n2h = g->n2h;
    a.n_ions = g->n_ions;
    a.n_species = g->n_species;
    a.omega = g->omega;
    for (int i = 0; i < 9; i++) a.bvec[i] = 2.0 * kPi * g->recip[i];
    a.ph0 = g->ph;
    a.ph1 = g->ph + (size_t)g->n_ions * g->n[0];
    a.ph2 = a.ph1 + (size_t)g->n_ions * g->n[1];
    a.species = g->d_species;
    a.Z = g->d_Z;
    a.rc = g->d_rc;
    return a;
}

template <typename T> int build_vext_pme(ofdft_grid *g, Workspace<T> &w);

template <typename T> int ensure_vext(ofdft_grid *g) {
    typedef typename Vec2<T>::type C;
    Workspace<T> &w = ws<T>(g);
    bool &fresh = sizeof(T) == 4 ? g->vext_fresh32 : g->vext_fresh64;
    if (fresh) return OFDFT_OK;
    if (!w.vext) {
        CK(gmalloc(g, &w.vext, g->NH * sizeof(C)), "cudaMalloc V_ext(G)");
        g->generation++;
    }
    if (g->pme_order > 0) {
        int rc = build_vext_pme<T>(g, w);
        if (rc) return rc;
        fresh = true;
        return OFDFT_OK;
    }
    IonArgs a = ion_args(g);
    cudaError_t e;
    if (sizeof(T) == 4) e = launch_vext(a, nullptr, (float2 *)w.vext, g->stream, g->ph32);
    else e = launch_vext(a, (double2 *)w.vext, nullptr, g->stream);
    CK(e, "structure factor kernel");
    fresh = true;
    return OFDFT_OK;
}

int check_functional(ofdft_grid *g, const ofdft_functional *f) {
    if (!f) return fail(g, OFDFT_ERR_INVALID_ARG, "functional is NULL");
    if (f->precision != OFDFT_FP64 && f->precision != OFDFT_FP32_MIXED)
        return fail(g, OFDFT_ERR_INVALID_ARG, "unknown precision");
    if (f->terms & ~OFDFT_TERMS_VALID) return fail(g, OFDFT_ERR_INVALID_ARG, "unknown term bits");
    if (f->terms & OFDFT_TERM_NL) {
        if (f->kernel == OFDFT_KERNEL_LWT && (f->n_knots < 2 || f->n_knots > OFDFT_MAX_KNOTS))
            return fail(g, OFDFT_ERR_INVALID_ARG, "n_knots must be in [2, 64]");
        if (f->nl_potential == OFDFT_NLPOT_INTERP && f->alpha != f->beta)
            return fail(g, OFDFT_ERR_INVALID_ARG, "interpolated potential needs alpha == beta");
        if (f->kernel != OFDFT_KERNEL_LWT && f->kernel != OFDFT_KERNEL_WT_GLOBAL)
            return fail(g, OFDFT_ERR_INVALID_ARG, "unknown kernel");
        if (!std::isfinite(f->mgp_x) || std::fabs(f->mgp_x) > 10.0 ||
            (f->mgp_x != 0.0 && !(f->mgp_y > 0.0 && f->mgp_y <= 10.0)))
            return fail(g, OFDFT_ERR_INVALID_ARG, "mgp_x must be in [-10, 10], mgp_y in (0, 10]");
        if (f->knots && f->kernel == OFDFT_KERNEL_LWT)
            for (int m = 0; m + 1 < f->n_knots; m++)
                if (!(f->knots[m + 1] >= f->knots[m]) || !(f->knots[0] > 0.0))
                    return fail(g, OFDFT_ERR_INVALID_ARG, "knots must be positive and ascending");
    }
    if ((f->terms & OFDFT_TERM_PP) && !g->have_ions) return fail(g, OFDFT_ERR_NO_IONS, "PP term needs ions");
    return OFDFT_OK;
}

cudaEvent_t take_event(ofdft_grid *g) {
    if (!g->ev_pool.empty()) {
        cudaEvent_t e = g->ev_pool.back();
        g->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_record(void *ctx, int id, int phase, cudaStream_t s) {
    ofdft_grid *g = (ofdft_grid *)ctx;
    cudaEvent_t e = take_event(g);
    cudaEventRecord(e, s);
    if (phase == 0) g->ev_pending[id] = e;
    else g->recs.push_back({id, g->ev_pending[id], e});
}

void prof_collect(ofdft_grid *g) {
    cudaStreamSynchronize(g->stream);
    for (auto &r : g->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g->prof_ms[r.id] += ms;
            g->prof_n[r.id] += 1;
        }
        g->ev_pool.push_back(r.a);
        g->ev_pool.push_back(r.b);
    }
    g->recs.clear();
}

const char *kKernelNames[K_NKERNEL] = {"stats", "knots", "row_fwd", "pencil_fwd", "axis0_recip",
                                       "pencil_inv", "row_inv", "finalize"};

// ---------------------------------------------------------------- MGP kernel table
constexpr int kMgpTable = (1 << 20) + 1;

// 8-point Gauss-Legendre rule on [-1, 1]: nodes (Newton on the Legendre recurrence) then weights
void gauss_legendre8(double *out) {
    const int n = 8;
    for (int i = 0; i < n; i++) {
        double x = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        out[i] = x;
        out[n + i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

bool uses_mgp(const ofdft_functional *f) { return (f->terms & OFDFT_TERM_NL) && f->mgp_x != 0.0; }

// the correction table of the functional's y on g's stream (built once per y)
template <typename T> int ensure_mgp_table(ofdft_grid *g, const ofdft_functional *f) {
    if (!uses_mgp(f)) return OFDFT_OK;
    Workspace<T> &w = ws<T>(g);
    if (!w.mgp_tab) {
        CK(gmalloc(g, &w.mgp_tab, (size_t)kMgpTable * sizeof(T)), "cudaMalloc MGP table");
        w.mgp_y = 0.0;
    }
    if (w.mgp_y != f->mgp_y) {
        double gl[16];
        gauss_legendre8(gl);
        CK(launch_mgp_table<T>(w.mgp_tab, kMgpTable, f->mgp_y, gl, g->stream), "MGP table");
        w.mgp_y = f->mgp_y;
    }
    return OFDFT_OK;
}

template <typename T>
int enqueue_eval(ofdft_grid *g, const T *rho, const ofdft_functional *f, T *V, double *E_dev_out,
                 bool keep_rhohat = false);

// ---------------------------------------------------------------- autotuner
// Picks, per tuned role (the reciprocal-space pass, the n1 pencils, the rows), the fastest of
// the compiled configurations for the grid's sizes: at the first evaluation of a launch plan,
// each candidate of a role is timed with CUDA events over whole evaluations of the caller's
// density (the other roles at their current pick), roles in order of their share of the step.
// The picks are cached per (precision, shape, channel count) for the process, so later grids
// of the same shape skip the timing.  Evaluations are pure functions of their inputs, so the
// extra ones change nothing but the time of this first call; none runs while the stream is
// being captured (the timing is then left for a later call).
struct TuneEntry {
    int key[8];
    int pick[TUNE_NROLE];
    std::string report;
};
std::mutex &tune_mutex() {
    static std::mutex m;
    return m;
}
std::vector<TuneEntry> &tune_cache() {
    static std::vector<TuneEntry> c;
    return c;
}

// the configurations of every role with the one in use (marked *), for roles nothing timed
template <typename T> std::string plan_report(const Workspace<T> &w) {
    const char *role_name[TUNE_NROLE] = {"rows", "pencil", "recip"};
    std::string rep;
    for (int r = TUNE_NROLE - 1; r >= 0; r--) {
        if (w.cand[r].empty()) continue;
        rep += std::string(rep.empty() ? "" : "; ") + role_name[r] + ":";
        for (int c = 0; c < (int)w.cand[r].size(); c++)
            rep += std::string(" [") + w.cand[r][c].name + "]" + (c == w.pick[r] ? "*" : "");
    }
    return rep;
}

template <typename T> int autotune(ofdft_grid *g, Workspace<T> &w, const T *rho, const ofdft_functional *f) {
    bool any = false;
    for (int r = 0; r < TUNE_NROLE; r++) any = any || (w.cand[r].size() > 1 && g->force_pick[r] < 0);
    if (!any) {
        w.tuned = true;
        w.tune_report = plan_report(w) + " (nothing timed)";
        return OFDFT_OK;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(g->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        (void)cudaGetLastError();
        return OFDFT_OK;                                  // not now: timing is impossible in a capture
    }
    w.tuned = true;
    const int key[8] = {(int)sizeof(T), g->n[0], g->n[1], g->n[2], w.nslots, g->force_pick[0], g->force_pick[1],
                        g->force_pick[2]};
    {
        std::lock_guard<std::mutex> lk(tune_mutex());
        for (const TuneEntry &e : tune_cache())
            if (std::memcmp(e.key, key, sizeof(key)) == 0) {
                for (int r = 0; r < TUNE_NROLE; r++)
                    if (e.pick[r] >= 0 && e.pick[r] < (int)w.cand[r].size()) {
                        int rc = apply_cand<T>(g, w, r, w.cand[r][e.pick[r]]);
                        if (rc) return rc;
                        w.pick[r] = e.pick[r];
                    }
                w.tune_report = e.report + " (cached)";
                return OFDFT_OK;
            }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0), "event");
    cudaError_t ee = cudaEventCreate(&e1);
    if (ee != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(g, OFDFT_ERR_CUDA, "event", ee);
    }
    const int reps = g->N > (1LL << 24) ? 2 : 5;
    w.tuning = true;
    int rc = OFDFT_OK;
    std::string rep;
    const int order[TUNE_NROLE] = {TUNE_AXIS0, TUNE_PENCIL, TUNE_ROWS};
    const char *role_name[TUNE_NROLE] = {"rows", "pencil", "recip"};
    for (int oi = 0; oi < TUNE_NROLE && rc == OFDFT_OK; oi++) {
        const int r = order[oi];
        if (w.cand[r].size() < 2 || g->force_pick[r] >= 0) continue;
        int best = -1;
        float best_ms = 0.f;
        rep += std::string(rep.empty() ? "" : "; ") + role_name[r] + ":";
        for (int c = 0; c < (int)w.cand[r].size() && rc == OFDFT_OK; c++) {
            if ((rc = apply_cand<T>(g, w, r, w.cand[r][c]))) break;
            if ((rc = enqueue_eval<T>(g, rho, f, nullptr, nullptr))) break;       // warm-up
            cudaEventRecord(e0, g->stream);
            for (int i = 0; i < reps && rc == OFDFT_OK; i++) rc = enqueue_eval<T>(g, rho, f, nullptr, nullptr);
            cudaEventRecord(e1, g->stream);
            cudaError_t e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess && rc == OFDFT_OK) rc = fail(g, OFDFT_ERR_CUDA, "autotuner timing", e);
            ms /= (float)reps;
            char buf[96];
            std::snprintf(buf, sizeof(buf), " [%s] %.4f ms", w.cand[r][c].name, ms);
            rep += buf;
            if (best < 0 || ms < best_ms) {
                best = c;
                best_ms = ms;
            }
        }
        if (rc == OFDFT_OK && best >= 0) {
            rc = apply_cand<T>(g, w, r, w.cand[r][best]);
            w.pick[r] = best;
            rep += std::string(" -> ") + w.cand[r][best].name;
        }
    }
    w.tuning = false;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    w.tune_report = rep;
    std::lock_guard<std::mutex> lk(tune_mutex());
    TuneEntry te;
    std::memcpy(te.key, key, sizeof(key));
    for (int r = 0; r < TUNE_NROLE; r++) te.pick[r] = w.pick[r];
    te.report = rep;
    tune_cache().push_back(te);
    return OFDFT_OK;
}

// Fill the arguments of one evaluation (host work: the workspace, V_ext(G), the tuner's picks
// and the tensor maps are made ready first; nothing is launched).
template <typename T>
int eval_args(ofdft_grid *g, const T *rho, const ofdft_functional *f, T *V, double *E_dev_out, bool keep_rhohat,
              EvalArgs<T> &a) {
    const bool nl = f->terms & OFDFT_TERM_NL;
    const bool lwt = nl && f->kernel == OFDFT_KERNEL_LWT;
    const int M = lwt ? f->n_knots : 0;
    const int nslots = nl ? (lwt ? 3 + M : 4) : 3;
    int rc = ensure_ws<T>(g, nslots);
    if (rc) return rc;
    Workspace<T> &w = ws<T>(g);
    if (f->terms & OFDFT_TERM_PP) {
        rc = ensure_vext<T>(g);
        if (rc) return rc;
    }
    if ((rc = ensure_mgp_table<T>(g, f))) return rc;
    if (!w.tuned && !w.tuning && g->kernel_choice == OFDFT_KERNELS_AUTO && (rc = autotune<T>(g, w, rho, f)))
        return rc;
    std::memset(&a, 0, sizeof(a));
    a.n0 = g->n[0];
    a.n1 = g->n[1];
    a.n2 = g->n[2];
    a.n2h = g->n2h;
    a.N = g->N;
    a.NH = g->NH;
    a.omega = g->omega;
    a.dV = g->dV;
    for (int i = 0; i < 9; i++) a.bvec[i] = 2.0 * kPi * g->recip[i];
    a.rho = rho;
    a.V = V;
    a.chan = w.chan;
    a.vext = w.vext;
    a.terms = f->terms;
    a.kernel = f->kernel;
    if (uses_mgp(f)) {
        a.mgp_tab = w.mgp_tab;
        a.mgp_n = kMgpTable;
        a.mgp_1mx = (T)(1.0 - f->mgp_x);
        a.mgp_3xy = (T)(3.0 * f->mgp_x * f->mgp_y);
    }
    a.nlpot = f->nl_potential;
    a.M = M;
    a.alpha = (T)f->alpha;
    a.beta = (T)f->beta;
    const double fl = f->rho_floor > 0.0 ? f->rho_floor : 1e-20;
    a.floor_ = (T)(sizeof(T) == 4 && fl < 1e-30 ? 1e-30 : fl);
    a.scal = w.scal;
    a.knots_d = w.knots_d;
    a.knots_t = w.knots_t;
    a.invdk_t = w.invdk_t;
    a.frozen = (lwt && f->knots) ? 1 : 0;
    a.knot_spacing = f->knot_spacing;
    a.part_stats = w.part_stats;
    a.part_minmax = w.part_minmax;
    a.part_ax0 = w.part_ax0;
    a.part_row = w.part_row;
    a.energies = E_dev_out ? E_dev_out : w.energies;
    a.ticket = w.ticket;
    a.nb_stats = 2 * g->nsm;
    a.nb_ax0 = w.ks.recip.k ? w.recip_grid : w.tile_nb_ax0;
    a.nb_row = (int)((((long long)g->n[0] * g->n[1] + 1) / 2 + w.Brow - 1) / w.Brow);   // the row kernels' grid
    a.p0 = g->plan[0];
    a.p1 = g->plan[1];
    a.p2 = g->plan[2];
    a.tw0 = w.tw[0];
    a.tw1 = w.tw[1];
    a.tw2 = w.tw[2];
    a.Brow = w.Brow;
    a.thr_rowf = w.thr_rowf;
    a.thr_rowi = w.thr_rowi;
    a.TW1 = w.TW1;
    a.thr_p1 = w.thr_p1;
    a.TW0 = w.TW0;
    a.thr_ax0 = w.thr_ax0;
    a.grid_p1 = w.grid_p1;
    a.row2_G = w.row2_G;
    a.ax0_scr = w.ax0_scr;
    a.wait_polls = g->wait_polls;
    a.exact_sums = g->exact_sums;
    // the normalised density spectrum for the forces, written by the reciprocal-space kernel
    // (needs the Hartree/PP channel)
    if (keep_rhohat && (f->terms & (OFDFT_TERM_HARTREE | OFDFT_TERM_PP))) {
        typedef typename Vec2<T>::type C;
        if (!w.rhohat) CK(gmalloc(g, &w.rhohat, (size_t)g->NH * sizeof(C)), "cudaMalloc density spectrum");
        a.rhohat_out = w.rhohat;
    }
    // channel lists
    const bool hpp = f->terms & (OFDFT_TERM_HARTREE | OFDFT_TERM_PP);
    const bool vw = f->terms & OFDFT_TERM_VW;
    const bool exact = f->nl_potential == OFDFT_NLPOT_EXACT;
    if (hpp) { a.fwd_ch[a.nfwd++] = CH_HPP; }
    if (vw) { a.fwd_ch[a.nfwd++] = CH_VW; }
    if (nl) {
        a.fwd_ch[a.nfwd++] = CH_NL;
        if (!lwt) a.fwd_ch[a.nfwd++] = CH_KNOT0;
        else if (exact)
            for (int m = 0; m < M; m++) a.fwd_ch[a.nfwd++] = CH_KNOT0 + m;
    }
    // forward and inverse passes along n1: every channel that exists in G space
    if (hpp) a.col_ch[a.ncol++] = CH_HPP;
    if (vw) a.col_ch[a.ncol++] = CH_VW;
    if (nl) {
        a.col_ch[a.ncol++] = CH_NL;   // (interp: the forward pass needs it; the inverse is unused)
        if (!lwt) a.col_ch[a.ncol++] = CH_KNOT0;
        else
            for (int m = 0; m < M; m++) a.col_ch[a.ncol++] = CH_KNOT0 + m;
    }
    for (int i = 0; i < a.ncol; i++)
        if (!(lwt && !exact && a.col_ch[i] == CH_NL)) a.col_inv_ch[a.ncol_inv++] = a.col_ch[i];
    if (hpp) { a.inv_ch[a.ninv] = CH_HPP; a.inv_kind[a.ninv++] = CONS_ADD; }
    if (vw) { a.inv_ch[a.ninv] = CH_VW; a.inv_kind[a.ninv++] = CONS_VW; }
    if (nl) {
        if (!lwt) {
            a.inv_ch[a.ninv] = CH_NL; a.inv_kind[a.ninv++] = CONS_WT_A;
            a.inv_ch[a.ninv] = CH_KNOT0; a.inv_kind[a.ninv++] = CONS_WT_B;
        } else {
            if (exact) { a.inv_ch[a.ninv] = CH_NL; a.inv_kind[a.ninv++] = CONS_T2; }
            for (int m = 0; m < M; m++) {
                a.inv_ch[a.ninv] = CH_KNOT0 + m;
                a.inv_kind[a.ninv] = CONS_KNOT;
                a.inv_knot[a.ninv++] = m;
            }
        }
    }
    if (w.ks.recip.k && (w.maps_chan != w.chan || w.maps_vext != w.vext || w.maps_nslots != w.nslots ||
                         w.maps_tw != w.ks.recip.tw)) {
        const long long PL = (long long)g->n[1] * g->n2h;
        const int box_rows = g->n[0] > 256 ? 256 : g->n[0], tw = w.ks.recip.tw;
        if (!encode_spectra_map<T>(&w.maps.chan, w.chan, PL, g->n[0], w.nslots, box_rows, tw) ||
            !encode_spectra_map<T>(&w.maps.vext, w.vext ? (const void *)w.vext : (const void *)w.chan, PL, g->n[0],
                                   1, box_rows, tw))
            return fail(g, OFDFT_ERR_CUDA, "tensor map encoding");
        w.maps_chan = w.chan;
        w.maps_vext = w.vext;
        w.maps_nslots = w.nslots;
        w.maps_tw = tw;
    }
    return OFDFT_OK;
}

// the knots a functional supplies (frozen knots) to the evaluation's FP64 knot buffer
template <typename T> int upload_knots(ofdft_grid *g, const EvalArgs<T> &a, const ofdft_functional *f) {
    if (a.frozen)
        CK(cudaMemcpyAsync(a.knots_d, f->knots, a.M * sizeof(double), cudaMemcpyHostToDevice, g->stream),
           "upload knots");
    return OFDFT_OK;
}

// Enqueue one evaluation with filled arguments on g->stream.
template <typename T> int eval_launch(ofdft_grid *g, const EvalArgs<T> &a, const ofdft_functional *f) {
    Workspace<T> &w = ws<T>(g);
    // clears the bad-density flag, the WT kF (recomputed) and the device-wait counters
    static_assert(S_TIMEOUT == S_BAD + 2 && S_FATAL == S_BAD + 3, "flag slots");
    CK(cudaMemsetAsync(a.scal + S_BAD, 0, 4 * sizeof(double), g->stream), "memset flags");
    if (int rc = upload_knots<T>(g, a, f)) return rc;
    ProfHook hook{prof_record, g};
    CK(launch_eval<T>(a, w.ks, g->stream, g->prof_on ? &hook : nullptr, w.ks.recip.k ? &w.maps : nullptr),
       "evaluation kernels");
    return OFDFT_OK;
}

// Fill the evaluation arguments and enqueue one evaluation.
template <typename T>
int enqueue_eval(ofdft_grid *g, const T *rho, const ofdft_functional *f, T *V, double *E_dev_out, bool keep_rhohat) {
    EvalArgs<T> a;
    if (int rc = eval_args<T>(g, rho, f, V, E_dev_out, keep_rhohat, a)) return rc;
    return eval_launch<T>(g, a, f);
}

// status of the device-wait counters of an evaluation (host copies of the S_TIMEOUT and
// S_FATAL slots): bounded waits for bulk copies that expired, and those whose copies did not
// land within the second, longer bound either
int wait_status(ofdft_grid *g, const double *scal) {
    if (scal[S_FATAL] != 0.0)
        return fail(g, OFDFT_ERR_TIMEOUT, "a bounded device wait expired and bulk copies may still have been in "
                                          "flight: every result of this call is invalid");
    if (scal[S_TIMEOUT] != 0.0) return fail(g, OFDFT_ERR_TIMEOUT, "a bounded device wait expired");
    return OFDFT_OK;
}

template <typename T>
int eval_sync(ofdft_grid *g, const T *rho, const ofdft_functional *f, T *V, double *E_out) {
    int rc = enqueue_eval<T>(g, rho, f, V, nullptr);
    if (rc) return rc;
    Workspace<T> &w = ws<T>(g);
    CK(cudaMemcpyAsync(g->h_pinned, w.energies, E_NUM * sizeof(double), cudaMemcpyDeviceToHost, g->stream), "copy E");
    CK(cudaMemcpyAsync(g->h_pinned + 8, w.scal, S_NSCAL * sizeof(double), cudaMemcpyDeviceToHost, g->stream),
       "copy scalars");
    CK(cudaStreamSynchronize(g->stream), "stream synchronize");
    if ((rc = wait_status(g, g->h_pinned + 8))) return rc;
    if (g->h_pinned[8 + S_BAD] != 0.0) return fail(g, OFDFT_ERR_BAD_DENSITY, "density has NaN/Inf or negative values");
    if (E_out) std::memcpy(E_out, g->h_pinned, E_NUM * sizeof(double));
    return OFDFT_OK;
}

// ---------------------------------------------------------------- plain transforms
// EvalArgs for a plain transform of one real field through slot CH_HPP (forward:
// stats + rows + n1 pencils; the n0 pass is done by launch_axis0_fft).
template <typename T> EvalArgs<T> plain_args(ofdft_grid *g, Workspace<T> &w, const T *field) {
    EvalArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.n0 = g->n[0]; a.n1 = g->n[1]; a.n2 = g->n[2]; a.n2h = g->n2h; a.N = g->N; a.NH = g->NH;
    a.omega = g->omega; a.dV = g->dV;
    a.rho = field; a.chan = w.chan; a.terms = OFDFT_TERM_HARTREE; a.floor_ = (T)1e-30;
    a.scal = w.scal; a.knots_d = w.knots_d; a.knots_t = w.knots_t; a.invdk_t = w.invdk_t;
    a.part_stats = w.part_stats; a.part_minmax = w.part_minmax; a.energies = w.energies; a.ticket = w.ticket;
    a.part_ax0 = w.part_ax0; a.part_row = w.part_row;
    a.nb_stats = 2 * g->nsm; a.nb_ax0 = w.nb_ax0; a.nb_row = w.nb_row;
    a.p0 = g->plan[0]; a.p1 = g->plan[1]; a.p2 = g->plan[2];
    a.tw0 = w.tw[0]; a.tw1 = w.tw[1]; a.tw2 = w.tw[2];
    a.Brow = w.Brow_p; a.thr_rowf = w.thr_rowf_p; a.thr_rowi = w.thr_rowi_p;
    a.TW1 = w.TW1; a.thr_p1 = w.thr_p1; a.TW0 = w.TW0; a.thr_ax0 = w.thr_ax0; a.grid_p1 = w.grid_p1;
    a.row2_G = w.row2_G_p; a.ax0_scr = w.ax0_scr;
    a.nfwd = 1; a.fwd_ch[0] = CH_HPP; a.ncol = 1; a.col_ch[0] = CH_HPP;
    return a;
}

// normalised half spectrum (1/N) of a real field into slot CH_HPP (G = 0 is not kept)
template <typename T> int forward_plain(ofdft_grid *g, Workspace<T> &w, const T *field) {
    EvalArgs<T> a = plain_args<T>(g, w, field);
    CK(launch_forward_rows_cols<T>(a, w.ks_plain, g->stream), "forward transform");
    CK(launch_axis0_fft<T>(w.chan, g->n[0], (long long)g->n[1] * g->n2h, g->plan[0], w.tw[0], w.TW0, w.thr_ax0,
                           1.0 / (double)g->N, g->stream, -1),
       "forward transform along n0");
    return OFDFT_OK;
}

// real field out = sum_G F(G) e^{iG.r} of the half spectrum F in slot `slot` (destroys it)
template <typename T> int inverse_plain(ofdft_grid *g, Workspace<T> &w, int slot, T *out, const T *any_field) {
    typedef typename Vec2<T>::type C;
    EvalArgs<T> a = plain_args<T>(g, w, any_field);
    a.terms = 0;
    a.V = out;
    a.ncol_inv = 1;
    a.col_inv_ch[0] = slot;
    a.ninv = 1;
    a.inv_ch[0] = slot;
    a.inv_kind[0] = CONS_ADD;
    CK(launch_axis0_fft<T>((C *)w.chan + (size_t)slot * g->NH, g->n[0], (long long)g->n[1] * g->n2h, g->plan[0],
                           w.tw[0], w.TW0, w.thr_ax0, 1.0, g->stream, +1),
       "inverse transform along n0");
    CK(launch_inverse_cols_rows<T>(a, w.ks_plain, g->stream), "inverse transform");
    return OFDFT_OK;
}

template <typename T> int ensure_pme_buffers(ofdft_grid *g) {
    if (!g->Qfix) {
        CK(gmalloc(g, &g->Qfix, (size_t)g->N * sizeof(unsigned long long)), "cudaMalloc PME grid");
        g->generation++;
    }
    if (g->pme_real_bytes < (size_t)g->N * sizeof(T)) {
        cudaFree(g->pme_real);
        g->pme_real = nullptr;
        g->pme_real_bytes = 0;
        CK(gmalloc(g, &g->pme_real, (size_t)g->N * sizeof(T)), "cudaMalloc PME field");
        g->pme_real_bytes = (size_t)g->N * sizeof(T);
        g->generation++;
    }
    return OFDFT_OK;
}

PmeArgs pme_args(ofdft_grid *g, int s) {
    PmeArgs a;
    a.n0 = g->n[0];
    a.n1 = g->n[1];
    a.n2 = g->n[2];
    a.n2h = g->n2h;
    a.n_ions = g->n_ions;
    a.p = g->pme_order;
    a.s = s;
    for (int i = 0; i < 9; i++) a.recip[i] = g->recip[i];
    a.pos = g->d_pos;
    a.species = g->d_species;
    return a;
}

// V_ext(G) = (1/Omega) sum_s v_s(|G|) S_s(G) with the PME structure factor
template <typename T> int build_vext_pme(ofdft_grid *g, Workspace<T> &w) {
    typedef typename Vec2<T>::type C;
    int rc = ensure_pme_buffers<T>(g);
    if (rc) return rc;
    CK(cudaMemsetAsync(g->Qfix, 0, (size_t)g->N * sizeof(unsigned long long), g->stream), "memset");
    for (int s = 0; s < g->n_species; s++) {
        PmeArgs pa = pme_args(g, s);
        CK(pme_spread(pa, g->Qfix, g->stream), "PME spread");
        CK(pme_fixed_to_real<T>(g->Qfix, (T *)g->pme_real, g->N, g->stream), "PME grid");
        if ((rc = forward_plain<T>(g, w, (const T *)g->pme_real))) return rc;
        CK(pme_vext<C>(pa, (const C *)w.chan, g->pmeB, g->Z[s], g->rc[s], (double)g->species_count[s],
                       (double)g->N, g->omega, (C *)w.vext, s == 0, g->stream),
           "PME V_ext");
    }
    return OFDFT_OK;
}

template <typename T> int forces_pme(ofdft_grid *g, Workspace<T> &w, const T *rho, double *dF) {
    typedef typename Vec2<T>::type C;
    int rc = ensure_pme_buffers<T>(g);
    if (rc) return rc;
    if ((rc = forward_plain<T>(g, w, rho))) return rc;                  // rho_hat in slot 0
    for (int s = 0; s < g->n_species; s++) {
        PmeArgs pa = pme_args(g, s);
        C *slot1 = (C *)w.chan + g->NH;
        CK(pme_force_field<C>(pa, (const C *)w.chan, g->pmeB, g->Z[s], g->rc[s], slot1, g->stream), "PME field");
        if ((rc = inverse_plain<T>(g, w, 1, (T *)g->pme_real, rho))) return rc;
        CK(pme_gather<T>(pa, (const T *)g->pme_real, dF, g->stream), "PME gather");
    }
    return OFDFT_OK;
}

// ---------------------------------------------------------------- forces
// Force kernels in use for this grid/precision and the size of their partials.
// FP32-mixed direct forces: the separable kernel, partials [n_ions][row-tile blocks][3]; FP64 (and
// FP32 past 64 Mi half-spectrum points): one block per (ion, chunk), partials [n_ions][16][3]
template <typename T> void force_layout(ofdft_grid *g, bool &fast, int &nchunk) {
    fast = sizeof(T) == 4 && g->NH <= (64LL << 20);
    nchunk = fast ? forces_sep_blocks(ion_args(g), g->nsm) : 16;
}

// device buffers of the force computation (outside any stream capture)
template <typename T> int ensure_force_buffers(ofdft_grid *g) {
    bool fast;
    int nchunk;
    force_layout<T>(g, fast, nchunk);
    const size_t plen = (size_t)g->n_ions * nchunk * 3;
    if (g->pme_order == 0 && plen > g->fpart_len) {
        cudaFree(g->fpart);
        g->fpart = nullptr;
        g->fpart_len = 0;
        CK(gmalloc(g, &g->fpart, plen * sizeof(double)), "cudaMalloc force partials");
        g->fpart_len = plen;
        g->generation++;
    }
    if (g->pme_order == 0 && fast && g->gf_len < (long long)g->n_species * g->NH) {
        cudaFree(g->gf);
        g->gf = nullptr;
        g->gf_len = 0;
        CK(gmalloc(g, &g->gf, (size_t)g->n_species * g->NH * sizeof(float)), "cudaMalloc force tables");
        g->gf_len = (long long)g->n_species * g->NH;
        g->gf_fresh = false;
        g->generation++;
    }
    if (g->pme_order == 0 && fast && !g->gf_fresh) {
        CK(launch_force_tables(ion_args(g), g->gf, g->stream), "force tables");
        g->gf_fresh = true;
    }
    if (g->F_len < g->n_ions) {
        cudaFree(g->F_dev);
        cudaFreeHost(g->F_pinned);
        g->F_dev = g->F_pinned = nullptr;
        g->F_len = 0;
        CK(gmalloc(g, &g->F_dev, (size_t)3 * g->n_ions * sizeof(double)), "cudaMalloc forces");
        CK(cudaMallocHost(&g->F_pinned, (size_t)3 * g->n_ions * sizeof(double)), "cudaMallocHost forces");
        g->F_len = g->n_ions;
        g->generation++;
    }
    if (g->pme_order > 0) {
        int rc = ensure_pme_buffers<T>(g);
        if (rc) return rc;
    }
    return OFDFT_OK;
}

// enqueue the forces into g->F_dev (no synchronisation); rhohat: the normalised density spectrum
// an evaluation kept (null: transform rho here)
template <typename T> int forces_enqueue(ofdft_grid *g, const T *rho, const typename Vec2<T>::type *rhohat = nullptr) {
    typedef typename Vec2<T>::type C;
    int rc = ensure_ws<T>(g, 3);
    if (rc) return rc;
    if ((rc = ensure_force_buffers<T>(g))) return rc;
    Workspace<T> &w = ws<T>(g);
    if (g->pme_order > 0) return forces_pme<T>(g, w, rho, g->F_dev);
    if (!rhohat) {
        if ((rc = forward_plain<T>(g, w, rho))) return rc;      // normalised rho_hat in slot 0
        rhohat = w.chan;
    }
    bool fast;
    int nchunk;
    force_layout<T>(g, fast, nchunk);
    IonArgs ia = ion_args(g);
    if (fast) {
        CK(launch_forces_sep(ia, (const float2 *)rhohat, g->ph32, g->gf, g->d_sp_ions, g->sp_off.data(), nchunk,
                             g->fpart, g->stream),
           "forces kernel");
        CK(launch_reduce_force_sep(ia, g->fpart, nchunk, g->F_dev, g->stream), "force reduction");
    } else {
        CK(launch_forces<C>(ia, rhohat, g->fpart, nchunk, g->stream), "forces kernel");
        CK(launch_reduce_force_partials(g->fpart, g->n_ions, nchunk, g->F_dev, g->stream), "force reduction");
    }
    return OFDFT_OK;
}

template <typename T> int forces_impl(ofdft_grid *g, const T *rho, double *F) {
    int rc = forces_enqueue<T>(g, rho);
    if (rc) return rc;
    CK(cudaMemcpyAsync(F, g->F_dev, (size_t)3 * g->n_ions * sizeof(double), cudaMemcpyDeviceToHost, g->stream),
       "copy forces");
    CK(cudaStreamSynchronize(g->stream), "stream synchronize");
    return OFDFT_OK;
}

// ---------------------------------------------------------------- ion-ion Ewald sum
constexpr double kEwaldCut = 6.0;      // erfc(6) ~ 2e-17, exp(-36) ~ 2e-16
constexpr int kEwaldBlocks = 512;

int ewald_impl(ofdft_grid *g, double *E_out, double *F_out) {
    typedef double2 C;
    const int n = g->n_ions;
    // split parameter: the grid's half spectrum holds every G inside the sphere of radius
    // min_a pi n_a / |a_a|; at its surface exp(-G^2/(4 eta^2)) = exp(-36)
    const double *A = g->cell;
    double gs = 1e300;
    for (int a = 0; a < 3; a++) {
        const double len = std::sqrt(A[3 * a] * A[3 * a] + A[3 * a + 1] * A[3 * a + 1] + A[3 * a + 2] * A[3 * a + 2]);
        gs = std::min(gs, kPi * g->n[a] / len);
    }
    const double eta = gs / (2.0 * kEwaldCut), rcut = kEwaldCut / eta;
    // ---- real space: cell list over the lattice planes (host counting sort)
    EwaldReal er;
    er.n = n;
    er.eta = eta;
    er.rc2 = rcut * rcut;
    for (int i = 0; i < 9; i++) er.A[i] = A[i];
    long long ncell = 1;
    for (int a = 0; a < 3; a++) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        const double cx = A[3 * b + 1] * A[3 * c + 2] - A[3 * b + 2] * A[3 * c + 1];
        const double cy = A[3 * b + 2] * A[3 * c + 0] - A[3 * b + 0] * A[3 * c + 2];
        const double cz = A[3 * b + 0] * A[3 * c + 1] - A[3 * b + 1] * A[3 * c + 0];
        const double width = g->omega / std::sqrt(cx * cx + cy * cy + cz * cz);      // plane spacing
        er.nc[a] = (int)std::max(1.0, std::min(256.0, std::floor(width / rcut)));
        er.kr[a] = (int)std::ceil(rcut / (width / er.nc[a]));
        ncell *= er.nc[a];
    }
    std::vector<int> cell(n), cnt(ncell + 1, 0), orig(n), scell(n);
    std::vector<double4> wp(n), sp(n);
    for (int I = 0; I < n; I++) {
        const double *R = &g->pos[3 * (size_t)I];
        double f[3];
        int ci[3];
        for (int a = 0; a < 3; a++) {
            f[a] = R[0] * g->recip[3 * a] + R[1] * g->recip[3 * a + 1] + R[2] * g->recip[3 * a + 2];
            f[a] -= std::floor(f[a]);
            ci[a] = std::min(er.nc[a] - 1, (int)(f[a] * er.nc[a]));
        }
        wp[I] = make_double4(f[0] * A[0] + f[1] * A[3] + f[2] * A[6], f[0] * A[1] + f[1] * A[4] + f[2] * A[7],
                             f[0] * A[2] + f[1] * A[5] + f[2] * A[8], g->Z[g->species[I]]);
        cell[I] = (ci[0] * er.nc[1] + ci[1]) * er.nc[2] + ci[2];
        cnt[cell[I] + 1]++;
    }
    for (long long c = 0; c < ncell; c++) cnt[c + 1] += cnt[c];
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (int I = 0; I < n; I++) {
        const int k = fill[cell[I]]++;
        sp[k] = wp[I];
        orig[k] = I;
        scell[k] = cell[I];
    }
    if (n > g->ew_n || ncell > g->ew_ncell) {
        cudaFree(g->ew_p);
        cudaFree(g->ew_cell);
        cudaFree(g->ew_orig);
        cudaFree(g->ew_F);
        cudaFree(g->ew_e);
        cudaFree(g->ew_cstart);
        g->ew_p = nullptr;
        g->ew_cell = g->ew_orig = g->ew_cstart = nullptr;
        g->ew_F = g->ew_e = nullptr;
        g->ew_n = g->ew_ncell = 0;
        CK(gmalloc(g, &g->ew_p, (size_t)n * sizeof(double4)), "cudaMalloc Ewald ions");
        CK(gmalloc(g, &g->ew_cell, (size_t)n * sizeof(int)), "cudaMalloc Ewald ions");
        CK(gmalloc(g, &g->ew_orig, (size_t)n * sizeof(int)), "cudaMalloc Ewald ions");
        CK(gmalloc(g, &g->ew_F, (size_t)6 * n * sizeof(double)), "cudaMalloc Ewald forces");
        CK(gmalloc(g, &g->ew_e, (size_t)n * sizeof(double)), "cudaMalloc Ewald energies");
        CK(gmalloc(g, &g->ew_cstart, (size_t)(ncell + 1) * sizeof(int)), "cudaMalloc Ewald cells");
        g->ew_n = n;
        g->ew_ncell = (int)ncell;
    }
    if (!g->ew_part) CK(gmalloc(g, &g->ew_part, (kEwaldBlocks + 8) * sizeof(double)), "cudaMalloc Ewald partials");
    cudaStream_t st = g->stream;
    CK(cudaMemcpyAsync(g->ew_p, sp.data(), (size_t)n * sizeof(double4), cudaMemcpyHostToDevice, st), "upload");
    CK(cudaMemcpyAsync(g->ew_cell, scell.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, st), "upload");
    CK(cudaMemcpyAsync(g->ew_orig, orig.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, st), "upload");
    CK(cudaMemcpyAsync(g->ew_cstart, cnt.data(), (size_t)(ncell + 1) * sizeof(int), cudaMemcpyHostToDevice, st),
       "upload");
    er.p = g->ew_p;
    er.cell = g->ew_cell;
    er.cstart = g->ew_cstart;
    er.orig = g->ew_orig;
    er.F = g->ew_F;                                   // [n][3] real space, then [n][3] reciprocal
    er.e = g->ew_e;
    CK(ewald_real(er, st), "Ewald real space");
    double *sums = g->ew_part + kEwaldBlocks;         // [0] real-space sum, [1] reciprocal sum
    CK(ewald_sum(g->ew_e, n, g->ew_part, kEwaldBlocks, sums, st), "Ewald sum");
    // ---- reciprocal space on the grid: S_Z(G), its energy, then its forces
    int rc = ensure_ws<double>(g, 3);
    if (rc) return rc;
    Workspace<double> &w = g->w64;
    C *sz;
    if (g->pme_order > 0) {
        if ((rc = ensure_pme_buffers<double>(g))) return rc;
        sz = (C *)w.chan + 2 * g->NH;
        CK(cudaMemsetAsync(g->Qfix, 0, (size_t)g->N * sizeof(unsigned long long), st), "memset");
        for (int s = 0; s < g->n_species; s++) {
            PmeArgs pa = pme_args(g, s);
            pa.charge_ff = 1;
            CK(pme_spread(pa, g->Qfix, st), "PME spread");
            CK(pme_fixed_to_real<double>(g->Qfix, (double *)g->pme_real, g->N, st), "PME grid");
            if ((rc = forward_plain<double>(g, w, (const double *)g->pme_real))) return rc;
            CK(pme_vext<C>(pa, (const C *)w.chan, g->pmeB, g->Z[s], g->rc[s], (double)g->species_count[s],
                           (double)g->N, g->omega, sz, s == 0, st),
               "PME charge structure factor");
        }
    } else {
        sz = (C *)w.chan;
        IonArgs ia = ion_args(g);
        ia.charge_ff = 1;
        CK(launch_vext(ia, sz, nullptr, st), "charge structure factor");
    }
    double bv[9];
    for (int i = 0; i < 9; i++) bv[i] = 2.0 * kPi * g->recip[i];
    CK(ewald_recip(g->n[0], g->n[1], g->n[2], bv, eta, g->omega, sz, g->ew_part, kEwaldBlocks, st), "Ewald G sum");
    CK(ewald_sum(g->ew_part, kEwaldBlocks, g->ew_part + kEwaldBlocks + 2, 1, sums + 1, st), "Ewald sum");
    double *Frec = g->ew_F + 3 * (size_t)n;
    if (F_out) {
        if ((rc = ensure_force_buffers<double>(g))) return rc;
        if (g->pme_order > 0) {
            for (int s = 0; s < g->n_species; s++) {
                PmeArgs pa = pme_args(g, s);
                pa.charge_ff = 1;
                C *slot1 = (C *)w.chan + g->NH;
                CK(pme_force_field<C>(pa, sz, g->pmeB, g->Z[s], g->rc[s], slot1, st), "PME field");
                // (the last argument is any N-point real field the inverse rows may read; slot 0 is free)
                if ((rc = inverse_plain<double>(g, w, 1, (double *)g->pme_real, (const double *)w.chan))) return rc;
                CK(pme_gather<double>(pa, (const double *)g->pme_real, Frec, st), "PME gather");
            }
        } else {
            bool fast;
            int nchunk;
            force_layout<double>(g, fast, nchunk);
            IonArgs ia = ion_args(g);
            ia.charge_ff = 1;
            CK(launch_forces<C>(ia, sz, g->fpart, nchunk, st), "Ewald forces");
            CK(launch_reduce_force_partials(g->fpart, n, nchunk, Frec, st), "force reduction");
        }
    }
    std::vector<double> F2(F_out ? 6 * (size_t)n : 0);
    double hs[2];
    CK(cudaMemcpyAsync(hs, sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "copy energies");
    if (F_out) CK(cudaMemcpyAsync(F2.data(), g->ew_F, 6 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st),
                  "copy forces");
    CK(cudaStreamSynchronize(st), "stream synchronize");
    double zz = 0.0, zs = 0.0;
    for (int I = 0; I < n; I++) {
        const double z = g->Z[g->species[I]];
        zz += z * z;
        zs += z;
    }
    const double E = hs[0] + 2.0 * kPi / g->omega * hs[1] - eta / std::sqrt(kPi) * zz -
                     kPi * zs * zs / (2.0 * g->omega * eta * eta);
    if (E_out) *E_out = E;
    if (F_out)
        for (size_t k = 0; k < 3 * (size_t)n; k++) F_out[k] = F2[k] + F2[3 * (size_t)n + k];
    return OFDFT_OK;
}

template <typename T>
int optimize_impl(ofdft_grid *g, T *psi, const ofdft_functional *f0, double Ne, double tol, int max_iter,
                  const ofdft_opt_options &o, ofdft_opt_report *rep);
const ofdft_opt_options kOptDefaults = {OFDFT_OPT_CG, 1, 0, 0, OFDFT_UPDATE_ROTATE, OFDFT_OBJECTIVE_ENERGY};

// ---------------------------------------------------------------- Fourier interpolation between grids
bool same_cell(const ofdft_grid *a, const ofdft_grid *b) {
    for (int i = 0; i < 9; i++)
        if (std::fabs(a->cell[i] - b->cell[i]) > 1e-12 * (1.0 + std::fabs(a->cell[i]))) return false;
    return true;
}

template <typename T> int interpolate_impl(ofdft_grid *from, const T *src, ofdft_grid *to, T *dst) {
    typedef typename Vec2<T>::type C;
    ofdft_grid *g = to;                 // errors are reported on the target grid
    int rc = ensure_ws<T>(from, 3);
    if (rc) return rc;
    if ((rc = ensure_ws<T>(to, 3))) return rc;
    Workspace<T> &wf = ws<T>(from), &wt = ws<T>(to);
    if ((rc = forward_plain<T>(from, wf, src))) return rc;     // normalised spectrum, mean in the scalars
    if (from->stream != to->stream) {
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
        cudaEventRecord(ev, from->stream);
        cudaStreamWaitEvent(to->stream, ev, 0);
        cudaEventDestroy(ev);
    }
    CK(launch_spectral_map<C>((const C *)wf.chan, from->n[0], from->n[1], from->n[2], (C *)wt.chan, to->n[0],
                              to->n[1], to->n[2], to->stream),
       "spectral map");
    if ((rc = inverse_plain<T>(to, wt, 0, dst, dst))) return rc;
    CK(launch_add_scalar<T>(dst, wf.scal + S_RHO_MEAN, to->N, to->stream), "mean");
    return OFDFT_OK;
}

template <typename T>
int multistep_impl(int nlev, ofdft_grid *const *grids, T *psi, const ofdft_functional *f, double Ne, double tol,
                   int max_iter, ofdft_opt_report *rep) {
    ofdft_grid *fine = grids[nlev - 1], *g = fine;
    std::vector<T *> lev(nlev, nullptr);
    lev[nlev - 1] = psi;
    int rc = OFDFT_OK;
    for (int L = 0; L < nlev - 1 && rc == OFDFT_OK; L++) {
        cudaError_t e = gmalloc(grids[L], &lev[L], (size_t)grids[L]->N * sizeof(T));
        if (e != cudaSuccess) rc = fail(fine, OFDFT_ERR_OOM, "cudaMalloc multi-step level", e);
    }
    // the initial psi goes straight to the coarsest grid; each converged psi goes one level up
    if (rc == OFDFT_OK) rc = interpolate_impl<T>(fine, psi, grids[0], lev[0]);
    ofdft_opt_report r;
    for (int L = 0; L < nlev && rc == OFDFT_OK; L++) {
        if (L > 0) {
            if ((rc = interpolate_impl<T>(grids[L - 1], lev[L - 1], grids[L], lev[L]))) break;
            CK(cudaStreamSynchronize(grids[L - 1]->stream), "stream synchronize");
        }
        rc = optimize_impl<T>(grids[L], lev[L], f, Ne, tol, max_iter, kOptDefaults, L == nlev - 1 ? rep : &r);
        if (rc == OFDFT_ERR_NOT_CONVERGED && L < nlev - 1) rc = OFDFT_OK;   // a coarse level only seeds the next
        if (rc && L < nlev - 1 && grids[L] != fine) fine->err = grids[L]->err;
    }
    cudaStreamSynchronize(fine->stream);
    for (int L = 0; L < nlev - 1; L++) cudaFree(lev[L]);
    return rc;
}

// ---------------------------------------------------------------- optimiser
// FP64 dot products of device fields read back to the host.  The first CUDA error is kept
// in err (later products return NaN); the loops that use them check it every iteration.
template <typename T> struct Dev {
    ofdft_grid *g;
    Workspace<T> *w;
    cudaError_t err = cudaSuccess;
    double dot(const T *a, const T *b, const T *c = nullptr) {
        if (err != cudaSuccess) return std::nan("");
        cudaError_t e = launch_dot<T>(a, b, c, g->N, w->part_misc, 1024, w->part_misc + 2048, g->stream,
                                      g->exact_sums != 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->h_pinned + 40, w->part_misc + 2048, sizeof(double), cudaMemcpyDeviceToHost,
                                g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) {
            err = e;
            return std::nan("");
        }
        return g->h_pinned[40];
    }
    // OFDFT_OK, or the status of the first failed product (message kept in the handle)
    int status() const {
        return err == cudaSuccess ? OFDFT_OK : fail(g, OFDFT_ERR_CUDA, "dot product", err);
    }
};

double cubic_min(double a, double fa, double da, double b, double fb, double db, bool &ok) {
    const double d1 = da + db - 3.0 * (fa - fb) / (a - b);
    const double disc = d1 * d1 - da * db;
    ok = false;
    if (disc < 0.0) return 0.0;
    const double d2 = std::copysign(std::sqrt(disc), b - a);
    const double den = db - da + 2.0 * d2;
    if (den == 0.0) return 0.0;
    ok = true;
    return b - (b - a) * (db + d2 - d1) / den;
}

template <typename T>
int optimize_impl(ofdft_grid *g, T *psi, const ofdft_functional *f0, double Ne, double tol, int max_iter,
                  const ofdft_opt_options &o, ofdft_opt_report *rep) {
    const long long N = g->N;
    int rc = ensure_ws<T>(g, 3);
    if (rc) return rc;
    Workspace<T> &w = ws<T>(g);
    if (!w.opt) CK(gmalloc(g, &w.opt, 8 * (size_t)N * sizeof(T)), "cudaMalloc optimiser fields");
    T *rho = w.opt, *V = rho + N, *grad = V + N, *gprev = grad + N, *d = gprev + N, *p = d + N, *psil = p + N;
    T *tmp = psil + N;
    const int method = o.method;
    const int max_inner = o.max_inner > 0 ? o.max_inner : 10;
    const int lm = o.lbfgs_m > 0 ? o.lbfgs_m : 5;
    // more fields: TN's q, Hq, Vq, r; L-BFGS's m pairs (s, y)
    const int n_ext = method == OFDFT_OPT_TN ? 4 : (method == OFDFT_OPT_LBFGS ? 2 * lm : 0);
    if (n_ext > w.opt_ext_fields) {
        cudaFree(w.opt_ext);
        w.opt_ext = nullptr;
        w.opt_ext_fields = 0;
        CK(gmalloc(g, &w.opt_ext, (size_t)n_ext * (size_t)N * sizeof(T)), "cudaMalloc optimiser history");
        w.opt_ext_fields = n_ext;
    }
    T *ext = w.opt_ext;
    Dev<T> dv{g, &w};
    cudaStream_t s = g->stream;
    // Preconditioner of the gradient, P(G) = a G^2 / (G^4 + a G^2 + b), the inverse of a model
    // Hessian in psi about the mean density rho_m: G^2 from the von Weizsaecker term (it
    // grows with the grid's cut-off, so plain CG needs ever more iterations on finer grids),
    // a = (70/9) C_TF rho_m^(2/3) from the local terms, b/G^2 = 16 pi rho_m / G^2 from Hartree
    // (stiff long-wavelength charge moves; a kinetic-only preconditioner amplifies exactly
    // those and stalls).
    typedef typename Vec2<T>::type C;
    const bool precond = o.precondition != 0;
    const bool scale_upd = o.update == OFDFT_UPDATE_SCALE;
    const bool resid_obj = o.objective == OFDFT_OBJECTIVE_RESIDUAL;
    const double rho_m = Ne / g->omega;
    const double pa = 70.0 / 9.0 * kCTF * std::pow(rho_m, 2.0 / 3.0), pb = 16.0 * kPi * rho_m;
    double bv[9];
    for (int i = 0; i < 9; i++) bv[i] = 2.0 * kPi * g->recip[i];
    T *z = tmp;                        // preconditioned gradient (tmp is free until the line search)
    double zg_prev = 0.0;
    auto apply_precond = [&](const T *x, T *out) -> int {
        // the plain forward transform drops the mean (kept in the scalars); P(0) = 1 adds it back
        int r = forward_plain<T>(g, w, x);
        if (r) return r;
        CK(launch_precond<C>((C *)w.chan, g->n[0], g->n[1], g->n[2], bv, pa, pb, s), "preconditioner");
        if ((r = inverse_plain<T>(g, w, 0, out, x))) return r;
        CK(launch_add_scalar<T>(out, w.scal + S_RHO_MEAN, N, s), "preconditioner mean");
        return OFDFT_OK;
    };
    double pp = 0.0;                   // <psi, psi> of the current iterate
    auto project = [&](T *v) -> int {  // v -= (<v, psi> / <psi, psi>) psi: the tangent space
        CK(launch_axpby<T>(v, psi, -dv.dot(v, psi) / pp, 1.0, N, s), "projection");
        return OFDFT_OK;
    };
    // preconditioned steepest descent -P g (projected), or -g, into out
    auto steepest = [&](T *out) -> int {
        if (precond) {
            int r = apply_precond(grad, z);
            if (r) return r;
            CK(launch_axpby<T>(out, z, -1.0, 0.0, N, s), "axpby");
        } else {
            CK(launch_axpby<T>(out, grad, -1.0, 0.0, N, s), "axpby");
        }
        return OFDFT_OK;
    };
    const bool lwt_auto = (f0->terms & OFDFT_TERM_NL) && f0->kernel == OFDFT_KERNEL_LWT && !f0->knots;
    ofdft_functional f = *f0;
    std::vector<double> knots(OFDFT_MAX_KNOTS);
    double E[E_NUM], Enew[E_NUM];
    int evals = 0;
    // normalise psi to N_e
    const double nrm = dv.dot(psi, psi) * g->dV;
    if (!(nrm > 0.0)) return fail(g, OFDFT_ERR_BAD_DENSITY, "initial psi is zero");
    CK(launch_square<T>(rho, psi, std::sqrt(Ne / nrm), N, s), "square");
    auto refresh_knots = [&]() -> int {
        if (!lwt_auto) return OFDFT_OK;
        f.knots = nullptr;
        int r = eval_sync<T>(g, rho, &f, V, E);
        evals++;
        if (r) return r;
        cudaMemcpy(knots.data(), w.knots_d, f.n_knots * sizeof(double), cudaMemcpyDeviceToHost);
        f.knots = knots.data();
        return OFDFT_OK;
    };
    if ((rc = refresh_knots())) return rc;
    if (!lwt_auto) {
        if ((rc = eval_sync<T>(g, rho, &f, V, E))) return rc;
        evals++;
    }

    // ---- truncated Newton: inner preconditioned CG on H x = -g in the tangent space,
    // H q by a forward difference of the gradient (one evaluation per inner step)
    const double h_fd = sizeof(T) == 4 ? 1e-3 : 1e-6;   // |e q| / |psi| of the difference
    double mu = 0.0;
    auto tn_direction = [&](bool &newton) -> int {
        T *q = ext, *Hq = ext + N, *Vq = ext + 2 * N, *r = ext + 3 * N, *x = d;
        double Eq[E_NUM];
        const double gn = std::sqrt(dv.dot(grad, grad));
        // forcing term on the RMS Euler-Lagrange residual per electron, |g| / (2 sqrt(dV N_e))
        const double stop = std::min(0.5, std::sqrt(gn / (2.0 * std::sqrt(g->dV * Ne)))) * gn;
        CK(cudaMemsetAsync(x, 0, (size_t)N * sizeof(T), s), "memset");
        CK(launch_copy<T>(r, grad, N, s), "copy");
        const T *zr = r;
        int e2;
        if (precond) {
            if ((e2 = apply_precond(r, z)) || (e2 = project(z))) return e2;
            zr = z;
        }
        double rz = dv.dot(r, zr);
        CK(launch_axpby<T>(q, zr, -1.0, 0.0, N, s), "axpby");
        newton = false;
        for (int j = 0; j < max_inner; j++) {
            const double e = h_fd * std::sqrt(pp / dv.dot(q, q));
            CK(launch_rotate<T>(psil, rho, psi, q, 1.0, e, N, s), "perturb");
            if ((e2 = eval_sync<T>(g, rho, &f, Vq, Eq))) return e2;
            evals++;
            CK(launch_hvp<T>(Hq, psi, q, V, Vq, e, mu, g->dV, N, s), "Hessian product");
            if ((e2 = project(Hq))) return e2;
            const double curv = dv.dot(q, Hq);
            if (!(curv > 0.0)) break;             // non-positive curvature: keep x so far
            newton = true;
            const double a = rz / curv;
            CK(launch_axpby<T>(x, q, a, 1.0, N, s), "axpby");
            CK(launch_axpby<T>(r, Hq, a, 1.0, N, s), "axpby");
            if (j == max_inner - 1 || std::sqrt(dv.dot(r, r)) < stop) break;
            if (precond) {
                if ((e2 = apply_precond(r, z)) || (e2 = project(z))) return e2;
            }
            const double rz_new = dv.dot(r, zr);
            CK(launch_axpby<T>(q, zr, -1.0, rz_new / rz, N, s), "axpby");
            rz = rz_new;
        }
        if (!newton || !(dv.dot(x, grad) < 0.0)) {
            newton = false;
            return steepest(x);
        }
        return OFDFT_OK;
    };

    // ---- L-BFGS: two-loop recursion over a ring of m pairs (s = step of psi, y = change
    // of the projected gradient); initial inverse Hessian gamma P (or gamma I)
    std::vector<double> l_rho(lm, 0.0), l_alpha(lm, 0.0);
    int l_count = 0, l_head = 0;        // pairs stored; slot of the next pair
    bool l_pending = false;             // S(l_head) holds the last step, waiting for its y
    auto Sk = [&](int k) { return ext + (size_t)(2 * k) * (size_t)N; };
    auto Yk = [&](int k) { return ext + (size_t)(2 * k + 1) * (size_t)N; };
    auto lbfgs_direction = [&](bool &newton) -> int {
        int e2;
        if (l_pending) {
            T *y = Yk(l_head);
            CK(launch_copy<T>(y, grad, N, s), "copy");
            CK(launch_axpby<T>(y, gprev, -1.0, 1.0, N, s), "axpby");
            const double sy = dv.dot(Sk(l_head), y);
            if (sy > 0.0) {
                l_rho[l_head] = 1.0 / sy;
                l_head = (l_head + 1) % lm;
                l_count = std::min(l_count + 1, lm);
            } else {
                l_count = std::min(l_count, lm - 1);   // the slot (the oldest pair's) was overwritten
            }
            l_pending = false;
        }
        CK(launch_copy<T>(gprev, grad, N, s), "copy");
        newton = false;
        if (l_count == 0) return steepest(d);
        CK(launch_copy<T>(d, grad, N, s), "copy");
        for (int i = 0; i < l_count; i++) {             // newest to oldest
            const int k = (l_head - 1 - i + 2 * lm) % lm;
            l_alpha[k] = l_rho[k] * dv.dot(Sk(k), d);
            CK(launch_axpby<T>(d, Yk(k), -l_alpha[k], 1.0, N, s), "axpby");
        }
        const int kn = (l_head - 1 + lm) % lm;         // newest pair
        if (precond) {
            if ((e2 = apply_precond(Yk(kn), z)) || (e2 = project(z))) return e2;
            const double gamma = (1.0 / l_rho[kn]) / dv.dot(Yk(kn), z);
            if ((e2 = apply_precond(d, z)) || (e2 = project(z))) return e2;
            CK(launch_axpby<T>(d, z, gamma, 0.0, N, s), "axpby");
        } else {
            const double gamma = (1.0 / l_rho[kn]) / dv.dot(Yk(kn), Yk(kn));
            CK(launch_axpby<T>(d, d, 0.0, gamma, N, s), "axpby");
        }
        for (int i = l_count - 1; i >= 0; i--) {        // oldest to newest
            const int k = (l_head - 1 - i + 2 * lm) % lm;
            const double b = l_rho[k] * dv.dot(Yk(k), d);
            CK(launch_axpby<T>(d, Sk(k), l_alpha[k] - b, 1.0, N, s), "axpby");
        }
        CK(launch_axpby<T>(d, d, 0.0, -1.0, N, s), "axpby");
        if (dv.dot(d, grad) < 0.0) {
            newton = true;
            return OFDFT_OK;
        }
        return steepest(d);
    };
    auto forget = [&]() {               // after a failed search: no conjugacy, no history
        l_count = 0;
        l_pending = false;
    };

    double lam_prev = 0.05;
    int small = 0, it = 0, restarts = 0;
    bool have_dir = false;
    double last_dE = 0.0;
    const double c1 = 1e-4, c2 = 0.2;
    while (it < max_iter) {
        if ((rc = dv.status())) return rc;
        it++;
        // g = 2 psi (V - mu) dV, mu = int rho V / N_e
        pp = dv.dot(psi, psi);
        mu = dv.dot(psi, psi, V) * g->dV / Ne;
        CK(launch_grad<T>(grad, psi, V, mu, g->dV, N, s), "grad");
        bool newton = false;           // a TN / L-BFGS direction built from curvature
        if (method == OFDFT_OPT_TN) {
            if ((rc = tn_direction(newton))) return rc;
        } else if (method == OFDFT_OPT_LBFGS) {
            if ((rc = lbfgs_direction(newton))) return rc;
        } else {
            double beta = 0.0, zg = 0.0;
            const T *src = grad;       // the (preconditioned) steepest-descent direction
            if (precond) {
                if ((rc = apply_precond(grad, z))) return rc;
                src = z;
                zg = dv.dot(z, grad);
            }
            if (have_dir && (it % 50) != 1) {
                if (precond) {
                    // preconditioned PR+: beta = <z, g - g_prev> / <z_prev, g_prev>
                    beta = zg_prev > 0.0 ? std::max(0.0, (zg - dv.dot(z, gprev)) / zg_prev) : 0.0;
                } else {
                    const double gg = dv.dot(grad, grad), ggp = dv.dot(grad, gprev), gpgp = dv.dot(gprev, gprev);
                    beta = std::max(0.0, (gg - ggp) / gpgp);
                }
            }
            // d = -src + beta d
            if (have_dir && beta > 0.0) CK(launch_axpby<T>(d, src, -1.0, beta, N, s), "axpby");
            else CK(launch_axpby<T>(d, src, -1.0, 0.0, N, s), "axpby");
            if (dv.dot(d, grad) >= 0.0) CK(launch_axpby<T>(d, src, -1.0, 0.0, N, s), "axpby");
            CK(launch_copy<T>(gprev, grad, N, s), "copy");
            zg_prev = zg;
            have_dir = true;
        }
        // rotation: p = d - (<d,psi>/<psi,psi>) psi; scaling: p = d; then normalised to N_e
        CK(launch_copy<T>(p, d, N, s), "copy");
        if (!scale_upd) CK(launch_axpby<T>(p, psi, -dv.dot(d, psi) / pp, 1.0, N, s), "axpby");
        const double pn = dv.dot(p, p) * g->dV;
        if (!(pn > 0.0)) break;
        CK(launch_axpby<T>(p, psi, 0.0, std::sqrt(Ne / pn), N, s), "axpby");
        const double phi0 = E[0];
        // dE/dlambda at 0 = <g, p> with the projected gradient g (either update)
        const double dphi0 = dv.dot(grad, p);
        if (dphi0 >= 0.0) {
            have_dir = false;
            forget();
            if (++restarts > 3) break;
            continue;
        }
        // the trial point psi_l (and rho = psi_l^2) at step lam; c, n: the scaling's factor
        auto trial = [&](double lam, double &c, double &n) -> int {
            if (!scale_upd) {
                CK(launch_rotate<T>(psil, rho, psi, p, std::cos(lam), std::sin(lam), N, s), "rotate");
                return OFDFT_OK;
            }
            // psi_t = c (psi + t p), c = sqrt(N_e / n), n = int (psi + t p)^2
            CK(launch_rotate<T>(psil, rho, psi, p, 1.0, lam, N, s), "step");
            n = dv.dot(psil, psil) * g->dV;
            c = std::sqrt(Ne / n);
            CK(launch_square<T>(rho, psil, c, N, s), "renormalise");
            return OFDFT_OK;
        };
        auto phi = [&](double lam, double *El, double &dl) -> int {
            double c = 1.0, n = Ne;
            int r = trial(lam, c, n);
            if (r) return r;
            r = eval_sync<T>(g, rho, &f, V, El);
            evals++;
            if (r) return r;
            if (scale_upd) {
                // d psi_t/dt = c p - (int (psi + t p) p / n) psi_t, int (psi + t p) p = <psi_t, p> dV / c
                const double qp = dv.dot(psil, p) * g->dV / c;
                dl = 2.0 * g->dV * (c * dv.dot(psil, V, p) - (qp / n) * dv.dot(psil, psil, V));
                return OFDFT_OK;
            }
            // dpsi/dlambda = -psi sin + p cos into tmp (grad is free scratch here)
            CK(launch_rotate<T>(tmp, grad, psi, p, -std::sin(lam), std::cos(lam), N, s), "rotate");
            dl = 2.0 * g->dV * dv.dot(psil, V, tmp);
            return OFDFT_OK;
        };
        double lam_lo = 0.0, f_lo = phi0, d_lo = dphi0, lam_hi = -1.0, f_hi = 0.0, d_hi = 0.0;
        // a curvature-built step has a length: psi + x_perp lies on the rotation at atan(|x_perp|/|psi|)
        // (scaling: psi + d is reached at t = |d| / |psi|)
        const double step0 = scale_upd ? std::sqrt(pn / Ne) : std::atan(std::sqrt(pn / Ne));
        double lam = std::min(std::max(newton ? step0 : lam_prev, 1e-4), 0.5);
        double best_f = 1e300, best_lam = 0.0;
        bool improved = false;
        if (resid_obj) {
            // the step lowers the norm of the residual of Eq. euler2, |2 psi (V - mu) dV|:
            // backtracking from the first trial by halves until it falls by the factor 1 - c1
            const double r0 = std::sqrt(dv.dot(grad, grad));
            double best_r = r0;
            for (int ls = 0; ls < 10; ls++) {
                double cc = 1.0, nn = Ne, El[E_NUM];
                if ((rc = trial(lam, cc, nn))) return rc;
                if ((rc = eval_sync<T>(g, rho, &f, V, El))) return rc;
                evals++;
                const double mul = dv.dot(psil, psil, V) * g->dV / Ne;
                CK(launch_grad<T>(tmp, psil, V, mul, g->dV, N, s), "residual");
                const double rl = std::sqrt(dv.dot(tmp, tmp));
                if (rl < best_r) { best_r = rl; best_lam = lam; std::memcpy(Enew, El, sizeof(El)); }
                if (rl <= (1.0 - c1) * r0) break;
                lam *= 0.5;
            }
            improved = best_r < r0;
        }
        for (int ls = 0; ls < 10 && !resid_obj; ls++) {
            double El[E_NUM], dl;
            if ((rc = phi(lam, El, dl))) return rc;
            const double fl = El[0];
            if (fl < best_f) { best_f = fl; best_lam = lam; std::memcpy(Enew, El, sizeof(El)); }
            if (fl > phi0 + c1 * lam * dphi0 || (lam_hi < 0.0 && fl >= f_lo && lam_lo > 0.0)) {
                lam_hi = lam; f_hi = fl; d_hi = dl;
            } else if (std::fabs(dl) <= -c2 * dphi0) {
                break;
            } else if (dl >= 0.0) {
                lam_hi = lam_lo; f_hi = f_lo; d_hi = d_lo;
                lam_lo = lam; f_lo = fl; d_lo = dl;
            } else {
                lam_lo = lam; f_lo = fl; d_lo = dl;
                if (lam_hi < 0.0) { lam = std::min(2.0 * lam, 1.5707963267948966); continue; }
            }
            bool ok;
            double c = cubic_min(lam_lo, f_lo, d_lo, lam_hi, f_hi, d_hi, ok);
            const double lo = std::min(lam_lo, lam_hi), hi = std::max(lam_lo, lam_hi);
            if (!ok || !(c >= lo + 0.1 * (hi - lo) && c <= hi - 0.1 * (hi - lo))) c = 0.5 * (lam_lo + lam_hi);
            lam = c;
        }
        if (!resid_obj) improved = best_f < phi0;
        if (!improved) {
            have_dir = false;
            forget();
            if (++restarts > 3) break;
            // restore V at psi for the next gradient
            CK(launch_square<T>(rho, psi, 1.0, N, s), "square");
            if ((rc = eval_sync<T>(g, rho, &f, V, E))) return rc;
            evals++;
            continue;
        }
        restarts = 0;
        lam_prev = best_lam;
        // accept: psi <- the trial point at best_lam, and V at the accepted point
        {
            double c, n;
            if ((rc = trial(best_lam, c, n))) return rc;
        }
        if (method == OFDFT_OPT_LBFGS) {            // s = psi_new - psi
            CK(launch_copy<T>(Sk(l_head), psil, N, s), "copy");
            CK(launch_axpby<T>(Sk(l_head), psi, -1.0, 1.0, N, s), "axpby");
            l_pending = true;
        }
        CK(launch_copy<T>(psi, psil, N, s), "copy");
        // The rotation conserves int psi^2 exactly only in exact arithmetic; in FP32
        // the rounding drift accumulates over iterations (and lowers E with the
        // charge), so psi is renormalised to N_e with an FP64 norm.
        {
            const double nn = dv.dot(psi, psi) * g->dV;
            CK(launch_square<T>(rho, psi, std::sqrt(Ne / nn), N, s), "renormalise");
        }
        last_dE = std::fabs(Enew[0] - E[0]);
        if (lwt_auto) {
            if ((rc = refresh_knots())) return rc;
        } else {
            if ((rc = eval_sync<T>(g, rho, &f, V, E))) return rc;
            evals++;
        }
        small = (last_dE < tol * std::max(1, g->n_ions)) ? small + 1 : 0;
        if (small >= 3) break;
    }
    if (rep) {
        rep->iterations = it;
        rep->evaluations = evals;
        rep->energy = E[0];
        std::memcpy(rep->energies, E, sizeof(E));
        rep->mu = dv.dot(psi, psi, V) * g->dV / Ne;
        // residual ||(V - mu) psi|| with dV weight: sum psi^2 (V-mu)^2 dV
        CK(launch_grad<T>(grad, psi, V, rep->mu, 0.5, N, s), "grad");   // grad = psi (V - mu)
        rep->residual = std::sqrt(dv.dot(grad, grad) * g->dV);
        rep->last_dE = last_dE;
    }
    if ((rc = dv.status())) return rc;
    return small >= 3 ? OFDFT_OK : fail(g, OFDFT_ERR_NOT_CONVERGED, "the optimiser reached max_iter");
}

// ---------------------------------------------------------------- real-time TD-OFDFT
// H psi = -lap psi / 2 + v_eff psi with v_eff = d(E - T_vW)/drho; each Crank-Nicolson step
// (1 + i tau H) psi(t+dt) = (1 - i tau H) psi(t), tau = dt/2, is solved through its normal
// equations (1 + tau^2 H^2) x = (1 - i tau H)^2 psi(t): H is real, so the real and imaginary
// parts are two real symmetric positive definite systems, solved together by preconditioned
// CG with M = 1 / (1 + tau^2 (G^2/2 + vbar)^2) diagonal in G.
constexpr int kTdFields = 19;

template <typename T>
int td_impl(ofdft_grid *g, T *pre, T *pim, const T *rho0, const ofdft_functional *f0, const ofdft_td_options &o,
            double *dip, ofdft_td_report *rep) {
    typedef typename Vec2<T>::type C;
    const long long N = g->N;
    int rc = ensure_ws<T>(g, 3);
    if (rc) return rc;
    Workspace<T> &w = ws<T>(g);
    if (!w.td) CK(gmalloc(g, &w.td, (size_t)kTdFields * (size_t)N * sizeof(T)), "cudaMalloc TD fields");
    T *F[kTdFields];
    for (int k = 0; k < kTdFields; k++) F[k] = w.td + (size_t)k * (size_t)N;
    T *p0[2] = {F[0], F[1]};           // psi(t)
    T *c[2] = {F[2], F[3]};            // right-hand sides
    T *r[2] = {F[4], F[5]}, *z[2] = {F[6], F[7]}, *q[2] = {F[8], F[9]}, *Aq[2] = {F[10], F[11]};
    T *h1 = F[12], *hp[2] = {F[13], F[14]};
    T *vt = F[15], *vn = F[16], *vm = F[17], *rho = F[18];
    T *x[2] = {pre, pim};
    Dev<T> dv{g, &w};
    cudaStream_t s = g->stream;
    double bv[9];
    for (int i = 0; i < 9; i++) bv[i] = 2.0 * kPi * g->recip[i];
    TdCell cell;
    for (int i = 0; i < 9; i++) cell.a[i] = g->cell[i];
    ofdft_functional f = *f0;
    f.terms &= ~(unsigned)OFDFT_TERM_VW;
    const bool have_v = f.terms != 0;
    const double tol = o.solver_tol > 0.0 ? o.solver_tol : (sizeof(T) == 8 ? 1e-11 : 1e-5);
    const int max_it = o.max_solver_iter > 0 ? o.max_solver_iter : 200;
    const double tau = 0.5 * o.dt;
    int evals = 0, cg_total = 0;
    double max_res = 0.0;
    bool all_conv = true;
    double Ed[E_NUM];
    const int n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];

    auto veff = [&](T *v) -> int {      // v_eff at rho = |x|^2 (rho kept for vbar)
        CK(launch_abs2<T>(rho, x[0], x[1], N, s), "density");
        if (!have_v) {
            CK(cudaMemsetAsync(v, 0, (size_t)N * sizeof(T), s), "memset");
            return OFDFT_OK;
        }
        int e = eval_sync<T>(g, rho, &f, v, Ed);
        evals++;
        return e;
    };
    auto apply_h = [&](const T *u, const T *v, T *out) -> int {   // out = K u + v u
        int e = forward_plain<T>(g, w, u);
        if (e) return e;
        CK(launch_spectral_factor<C>((C *)w.chan, n0, n1, n2, bv, 0, 0.0, 0.0, s), "kinetic");
        if ((e = inverse_plain<T>(g, w, 0, out, u))) return e;
        CK(launch_add_vu<T>(out, v, u, 1.0, 1.0, N, s), "potential");
        return OFDFT_OK;
    };
    auto apply_a = [&](const T *u, const T *v, T *out) -> int {   // out = (1 + tau^2 H^2) u
        int e = apply_h(u, v, h1);
        if (e || (e = apply_h(h1, v, out))) return e;
        CK(launch_axpby<T>(out, u, 1.0, tau * tau, N, s), "axpby");
        return OFDFT_OK;
    };
    double vbar = 0.0;
    auto apply_m = [&](const T *u, T *out) -> int {              // out = M u
        int e = forward_plain<T>(g, w, u);
        if (e) return e;
        CK(launch_spectral_factor<C>((C *)w.chan, n0, n1, n2, bv, 1, tau, vbar, s), "preconditioner");
        if ((e = inverse_plain<T>(g, w, 0, out, u))) return e;
        const double a0 = tau * vbar;
        CK(launch_add_scaled_scalar<T>(out, w.scal + S_RHO_MEAN, 1.0 / (1.0 + a0 * a0), N, s), "mean");
        return OFDFT_OK;
    };
    // x <- psi(t + dt) for the Hamiltonian with potential v, x holding the initial guess
    // (x_is_psi: the guess is psi(t) itself, whose residual follows from the right-hand side)
    auto cn_solve = [&](const T *v, bool x_is_psi) -> int {
        int e;
        vbar = 0.0;
        if (have_v) {   // v weighted by the density held in rho (any vbar gives the same solution)
            const double sr = dv.dot(x[0], x[0]) + dv.dot(x[1], x[1]);
            if (sr > 0.0) vbar = dv.dot(rho, v) / sr;
        }
        // c = (1 - i tau H)^2 psi(t):  c_re = p_re + 2 tau H p_im - tau^2 H^2 p_re,
        //                               c_im = p_im - 2 tau H p_re - tau^2 H^2 p_im
        for (int j = 0; j < 2; j++)
            if ((e = apply_h(p0[j], v, hp[j]))) return e;
        for (int j = 0; j < 2; j++) {
            if ((e = apply_h(hp[j], v, c[j]))) return e;
            if (x_is_psi) {
                // r = c - (1 + tau^2 H^2) psi = -2 tau^2 H^2 p_j +- 2 tau H p_(other)
                CK(launch_copy<T>(r[j], c[j], N, s), "copy");
                CK(launch_axpby<T>(r[j], hp[1 - j], j == 0 ? 2.0 * tau : -2.0 * tau, -2.0 * tau * tau, N, s), "axpby");
            }
            CK(launch_axpby<T>(c[j], p0[j], 1.0, -tau * tau, N, s), "axpby");
            CK(launch_axpby<T>(c[j], hp[1 - j], j == 0 ? 2.0 * tau : -2.0 * tau, 1.0, N, s), "axpby");
        }
        double nc[2], rz[2];
        bool done[2];
        int its = 0;
        for (int j = 0; j < 2; j++) {
            nc[j] = std::sqrt(dv.dot(c[j], c[j]));
            done[j] = !(nc[j] > 0.0);
            if (done[j]) {
                CK(cudaMemsetAsync(x[j], 0, (size_t)N * sizeof(T), s), "memset");
                continue;
            }
            if (!x_is_psi) {
                if ((e = apply_a(x[j], v, r[j]))) return e;
                CK(launch_axpby<T>(r[j], c[j], 1.0, -1.0, N, s), "axpby");  // r = c - A x
            }
            if (std::sqrt(dv.dot(r[j], r[j])) <= tol * nc[j]) {
                done[j] = true;
                continue;
            }
            if ((e = apply_m(r[j], z[j]))) return e;
            CK(launch_copy<T>(q[j], z[j], N, s), "copy");
            rz[j] = dv.dot(r[j], z[j]);
        }
        double res = 0.0;
        while (!(done[0] && done[1]) && its < max_it) {
            its++;
            for (int j = 0; j < 2; j++) {
                if (done[j]) continue;
                if ((e = apply_a(q[j], v, Aq[j]))) return e;
                const double qAq = dv.dot(q[j], Aq[j]);
                if (!(qAq > 0.0)) {
                    done[j] = true;
                    continue;
                }
                const double a = rz[j] / qAq;
                CK(launch_axpby<T>(x[j], q[j], a, 1.0, N, s), "axpby");
                CK(launch_axpby<T>(r[j], Aq[j], -a, 1.0, N, s), "axpby");
                const double rn = std::sqrt(dv.dot(r[j], r[j])) / nc[j];
                if (rn <= tol) {
                    done[j] = true;
                    res = std::max(res, rn);
                    continue;
                }
                if ((e = apply_m(r[j], z[j]))) return e;
                const double rz_new = dv.dot(r[j], z[j]);
                CK(launch_axpby<T>(q[j], z[j], 1.0, rz_new / rz[j], N, s), "axpby");
                rz[j] = rz_new;
            }
        }
        if (!(done[0] && done[1])) {
            all_conv = false;
            for (int j = 0; j < 2; j++)
                if (!done[j]) res = std::max(res, std::sqrt(dv.dot(r[j], r[j])) / nc[j]);
        }
        cg_total += its;
        max_res = std::max(max_res, res);
        return OFDFT_OK;
    };
    auto dipole = [&](double *out) -> int {
        if (!out) return OFDFT_OK;
        CK(launch_dipole<T>(x[0], x[1], rho0, n0, n1, n2, cell, g->dV, w.part_misc + 2560, 384, w.part_misc + 3840, s),
           "dipole");
        CK(cudaMemcpyAsync(g->h_pinned + 44, w.part_misc + 3840, 3 * sizeof(double), cudaMemcpyDeviceToHost, s),
           "copy dipole");
        CK(cudaStreamSynchronize(s), "stream synchronize");
        for (int k = 0; k < 3; k++) out[k] = g->h_pinned[44 + k];
        return OFDFT_OK;
    };

    if ((rc = veff(vt))) return rc;
    if ((rc = dipole(dip))) return rc;
    int step = 0;
    for (; step < o.n_steps; step++) {
        if ((rc = dv.status())) return rc;
        for (int j = 0; j < 2; j++) CK(launch_copy<T>(p0[j], x[j], N, s), "copy");
        if ((rc = cn_solve(vt, true))) return rc;           // predictor (from psi(t))
        if ((rc = veff(vn))) return rc;
        for (int k = 0; k < o.n_corrector; k++) {           // correctors: mean of the two potentials
            CK(launch_copy<T>(vm, vt, N, s), "copy");
            CK(launch_axpby<T>(vm, vn, 0.5, 0.5, N, s), "axpby");
            if ((rc = cn_solve(vm, false))) return rc;     // from the last solution
            if ((rc = veff(vn))) return rc;
        }
        std::swap(vt, vn);
        if ((rc = dipole(dip ? dip + 3 * (size_t)(step + 1) : nullptr))) return rc;
    }
    CK(cudaStreamSynchronize(s), "stream synchronize");
    if ((rc = dv.status())) return rc;
    if (rep) {
        rep->steps = step;
        rep->evaluations = evals;
        rep->solver_iterations = cg_total;
        rep->max_residual = max_res;
    }
    return all_conv ? OFDFT_OK : fail(g, OFDFT_ERR_NOT_CONVERGED, "a Crank-Nicolson solve reached max_solver_iter");
}

// ---------------------------------------------------------------- batched evaluation
// A batch is planned once per distinct set of arguments: the snapshots are partitioned into
// groups that share one launch geometry (grid shape, compiled kernels, tiles, channel
// lists); each group of up to kGroupMax snapshots runs every pass of its evaluations as one
// grouped launch (the arguments in device memory, uploaded with the plan), single snapshots
// run the single-evaluation launches.  Groups are spread over a few internal streams forked
// from (and joined back into) the caller's stream, the heaviest first onto the least loaded
// stream; the energies and status slots of every snapshot are gathered by one kernel and
// copied to the host once.  The whole batch is captured once into a CUDA graph and replayed
// while the plan's key (the functional, the stream, every snapshot's arguments and kernels)
// is unchanged.
constexpr int kBatchStreams = 4;
constexpr int kBatchPlans = 16;

struct BatchPlan {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    void *dargs = nullptr;                 // the evaluations' arguments in plan order (device)
    double *dcol = nullptr, *hcol = nullptr;   // gathered energies and slots (device, pinned host)
    std::vector<int> order;                // plan position -> snapshot
    std::vector<int> gbeg, gstream;        // group g: positions [gbeg[g], gbeg[g + 1]), its stream
    int launches = 0;                      // kernel launches of the batch's evaluations
    std::string report;
};

std::vector<BatchPlan> &batch_plans() {
    static std::vector<BatchPlan> c;
    return c;
}

// the automatic grouping choice per batch (key without the grouping): 1 grouped, 0 not, and
// the measured times
struct BatchMode {
    std::vector<unsigned char> key;
    int grouped = 1;
    std::string note;
};
std::vector<BatchMode> &batch_modes() {
    static std::vector<BatchMode> c;
    return c;
}

void free_plan(BatchPlan &p) {
    if (p.exec) cudaGraphExecDestroy(p.exec);
    cudaFree(p.dargs);
    cudaFree(p.dcol);
    cudaFreeHost(p.hcol);
    p = BatchPlan();
}

// kBatchStreams worker streams, then the stream a batch graph is captured on (the
// caller's stream may be the legacy default stream, which cannot be captured)
cudaStream_t *batch_streams() {
    static cudaStream_t s[kBatchStreams + 1] = {nullptr};
    static int device = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (!s[0] || device != dev) {
        for (int k = 0; k <= kBatchStreams; k++) cudaStreamCreateWithFlags(&s[k], cudaStreamNonBlocking);
        device = dev;
    }
    return s;
}

template <typename T>
int prepare_batch_grid(ofdft_grid *g, const ofdft_functional *f, bool forces, const T *rho) {
    const bool nl = f->terms & OFDFT_TERM_NL;
    const bool lwt = nl && f->kernel == OFDFT_KERNEL_LWT;
    const int nslots = nl ? (lwt ? 3 + f->n_knots : 4) : 3;
    int rc = ensure_ws<T>(g, nslots);
    if (rc) return rc;
    if ((f->terms & OFDFT_TERM_PP) && (rc = ensure_vext<T>(g))) return rc;
    if (forces && (rc = ensure_force_buffers<T>(g))) return rc;
    if ((rc = ensure_mgp_table<T>(g, f))) return rc;     // before any graph capture
    Workspace<T> &w = ws<T>(g);
    if (forces && (f->terms & (OFDFT_TERM_HARTREE | OFDFT_TERM_PP)) && !w.rhohat)
        CK(gmalloc(g, &w.rhohat, (size_t)g->NH * sizeof(typename Vec2<T>::type)), "cudaMalloc density spectrum");
    if (!w.tuned && g->kernel_choice == OFDFT_KERNELS_AUTO && (rc = autotune<T>(g, w, rho, f))) return rc;
    return OFDFT_OK;
}

template <typename T> void append_bytes(std::vector<unsigned char> &key, const T &v) {
    const unsigned char *b = (const unsigned char *)&v;
    key.insert(key.end(), b, b + sizeof(T));
}

// the kernels of a launch set, field by field (no padding bytes)
void append_kernels(std::vector<unsigned char> &key, const LaunchSet &ks) {
    const void *p[] = {ks.row_fwd,   ks.row_inv,   ks.pen_fwd,     ks.pen_inv,    ks.axis0,     ks.axis0_mgp,
                       ks.recip.k,   ks.recip.k_mgp, ks.recip.g,   ks.recip.g_mgp, ks.row_fwd_g, ks.row_inv_g,
                       ks.pen_fwd_g, ks.pen_inv_g, ks.axis0_g,     ks.axis0_mgp_g};
    const long long v[] = {ks.recip.nt, ks.recip.per_sm, ks.recip.tw, (long long)ks.recip.smem};
    append_bytes(key, p);
    append_bytes(key, v);
}

// the launch geometry of an evaluation: what a grouped launch shares between its evaluations
// (the reciprocal-space pass: the persistent kernel's, or else the tile kernel's)
template <typename T> std::vector<unsigned char> launch_signature(const LaunchSet &ks_in, const EvalArgs<T> &a) {
    LaunchSet ks = ks_in;
    int tile[3] = {a.TW0, a.thr_ax0, a.ax0_scr};
    if (ks.recip.k) {
        ks.axis0 = ks.axis0_mgp = ks.axis0_g = ks.axis0_mgp_g = nullptr;
        tile[0] = tile[1] = tile[2] = 0;
    } else {
        ks.recip = RecipLaunch();
    }
    std::vector<unsigned char> k;
    append_kernels(k, ks);
    const int v[] = {a.n0,       a.n1,       a.n2,    a.nb_stats, a.nb_ax0, a.nb_row, a.Brow,     a.thr_rowf,
                     a.thr_rowi, a.TW1,      a.thr_p1, tile[0],   tile[1],  tile[2],  a.grid_p1,  a.row2_G,
                     a.nfwd,     a.ncol,     a.ncol_inv, a.exact_sums, a.mgp_tab != nullptr};
    append_bytes(k, v);
    return k;
}

// Plan a batch: groups, their streams, and the device copy of the arguments.
template <typename T>
int make_plan(ofdft_grid *g0, int n, ofdft_grid *const *grids, const std::vector<EvalArgs<T>> &args, bool grouped,
              BatchPlan &p) {
    std::vector<std::vector<unsigned char>> sig(n);
    std::vector<char> ok(n);
    for (int i = 0; i < n; i++) {
        sig[i] = launch_signature<T>(ws<T>(grids[i]).ks, args[i]);
        ok[i] = grouped && grouped_ok<T>(ws<T>(grids[i]).ks, args[i]);
    }
    // groups: snapshots of equal signature in first-seen order, cut at kGroupMax
    std::vector<char> used(n, 0);
    std::vector<long long> work;
    for (int i = 0; i < n; i++) {
        if (used[i]) continue;
        std::vector<int> mem{i};
        used[i] = 1;
        if (ok[i])
            for (int j = i + 1; j < n; j++)
                if (!used[j] && ok[j] && sig[j] == sig[i]) {
                    mem.push_back(j);
                    used[j] = 1;
                }
        for (size_t c = 0; c < mem.size(); c += kGroupMax) {
            p.gbeg.push_back((int)p.order.size());
            for (size_t m = c; m < std::min(mem.size(), c + kGroupMax); m++) p.order.push_back(mem[m]);
            work.push_back(grids[i]->N * (long long)std::min((size_t)kGroupMax, mem.size() - c));
        }
    }
    const int ng = (int)p.gbeg.size();
    p.gbeg.push_back(n);
    // what the plan launches per batch (evaluation kernels and the gather; forces excluded)
    char buf[160];
    std::snprintf(buf, sizeof(buf), "%d snapshots in %d launch groups:", n, ng);
    p.report = buf;
    p.launches = 1;
    for (int gi = 0; gi < ng; gi++) {
        const EvalArgs<T> &a = args[p.order[p.gbeg[gi]]];
        const int K = p.gbeg[gi + 1] - p.gbeg[gi];
        p.launches += (K > 1 ? 1 : 0) + 4 + (a.nfwd > 0) + (a.ncol > 0) + (a.ncol_inv > 0);
        const bool recip = ws<T>(grids[p.order[p.gbeg[gi]]]).ks.recip.k != nullptr;
        std::snprintf(buf, sizeof(buf), "%s %dx%dx%d x%d%s", gi ? "," : "", a.n0, a.n1, a.n2, K,
                      K > 1 ? (recip ? " (grouped, persistent recip)" : " (grouped)") : "");
        p.report += buf;
    }
    std::snprintf(buf, sizeof(buf), "; %d kernel launches per batch (forces excluded)", p.launches);
    p.report += buf;
    // streams: the heaviest group first onto the least loaded stream
    std::vector<int> idx(ng);
    for (int gi = 0; gi < ng; gi++) idx[gi] = gi;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return work[x] > work[y]; });
    long long load[kBatchStreams] = {0};
    p.gstream.assign(ng, 0);
    for (int gi : idx) {
        const int s = (int)(std::min_element(load, load + kBatchStreams) - load);
        p.gstream[gi] = s;
        load[s] += work[gi];
    }
    // the arguments in plan order, the gather buffers
    std::vector<EvalArgs<T>> ordered(n);
    for (int j = 0; j < n; j++) ordered[j] = args[p.order[j]];
    ofdft_grid *g = g0;
    const size_t W = E_NUM + S_NSCAL;
    CK(cudaMalloc(&p.dargs, (size_t)n * sizeof(EvalArgs<T>)), "cudaMalloc batch arguments");
    CK(cudaMalloc((void **)&p.dcol, (size_t)n * W * sizeof(double)), "cudaMalloc batch results");
    CK(cudaMallocHost((void **)&p.hcol, (size_t)n * W * sizeof(double)), "cudaMallocHost batch results");
    CK(cudaMemcpy(p.dargs, ordered.data(), (size_t)n * sizeof(EvalArgs<T>), cudaMemcpyHostToDevice),
       "upload batch arguments");
    return OFDFT_OK;
}

// forces of snapshot i on stream s and their copy to the grid's pinned buffer (if wanted)
template <typename T>
int enqueue_forces(ofdft_grid *const *grids, const void *const *rho_dev, const ofdft_functional *f,
                   double *const *F_out, int i, cudaStream_t s) {
    if (!(F_out && F_out[i])) return OFDFT_OK;
    ofdft_grid *g = grids[i];
    const cudaStream_t saved = g->stream;
    g->stream = s;
    const bool kept = f->terms & (OFDFT_TERM_HARTREE | OFDFT_TERM_PP);
    int rc = forces_enqueue<T>(g, (const T *)rho_dev[i], kept ? ws<T>(g).rhohat : nullptr);
    if (rc == OFDFT_OK) {
        cudaError_t e =
            cudaMemcpyAsync(g->F_pinned, g->F_dev, (size_t)3 * g->n_ions * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = fail(g, OFDFT_ERR_CUDA, "forces copy", e);
    }
    g->stream = saved;
    return rc;
}

// Enqueue a planned batch on the caller's stream (fork/join over the internal streams).
template <typename T>
int enqueue_batch(const BatchPlan &p, int n, ofdft_grid *const *grids, const void *const *rho_dev,
                  const ofdft_functional *f, const std::vector<EvalArgs<T>> &args, double *const *F_out,
                  cudaStream_t user) {
    cudaStream_t *st = batch_streams();
    cudaEvent_t fork, join[kBatchStreams];
    cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int k = 0; k < kBatchStreams; k++) cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming);
    int rc = OFDFT_OK;
    cudaEventRecord(fork, user);
    for (int k = 0; k < kBatchStreams; k++) cudaStreamWaitEvent(st[k], fork, 0);
    const EvalArgs<T> *dargs = (const EvalArgs<T> *)p.dargs;
    const int ng = (int)p.gstream.size();
    std::vector<cudaEvent_t> done(ng, nullptr);       // groups' evaluations complete (groups with forces)
    for (int gi = 0; gi < ng && rc == OFDFT_OK; gi++) {
        const int b = p.gbeg[gi], K = p.gbeg[gi + 1] - b;
        const cudaStream_t s = st[p.gstream[gi]];
        ofdft_grid *g = grids[p.order[b]];
        if (K == 1) {
            const cudaStream_t saved = g->stream;
            g->stream = s;
            rc = eval_launch<T>(g, args[p.order[b]], f);
            g->stream = saved;
        } else {
            RecipMaps maps[kGroupMax];
            for (int m = 0; m < K && rc == OFDFT_OK; m++) {
                ofdft_grid *gm = grids[p.order[b + m]];
                maps[m] = ws<T>(gm).maps;
                const cudaStream_t saved = gm->stream;
                gm->stream = s;
                rc = upload_knots<T>(gm, args[p.order[b + m]], f);
                gm->stream = saved;
            }
            if (rc) break;
            const Workspace<T> &w = ws<T>(g);
            cudaError_t e = launch_group<T>(args[p.order[b]], dargs + b, K, w.ks, s, w.ks.recip.k ? maps : nullptr);
            if (e != cudaSuccess) {
                rc = fail(g, OFDFT_ERR_CUDA, "grouped evaluation kernels", e);
                break;
            }
        }
        // forces (rho_hat from the evaluation): a single snapshot's right behind its evaluation;
        // a group's once all groups' evaluations are enqueued (below)
        if (K == 1) {
            rc = enqueue_forces<T>(grids, rho_dev, f, F_out, p.order[b], s);
        } else if (rc == OFDFT_OK) {
            bool any_f = false;
            for (int m = 0; m < K; m++) any_f = any_f || (F_out && F_out[p.order[b + m]]);
            if (any_f) {
                cudaError_t e = cudaEventCreateWithFlags(&done[gi], cudaEventDisableTiming);
                if (e == cudaSuccess) e = cudaEventRecord(done[gi], s);
                if (e != cudaSuccess) rc = fail(g, OFDFT_ERR_CUDA, "batch event", e);
            }
        }
    }
    // a group's forces spread over all worker streams once its evaluations are done, so that
    // they overlap one another and the other groups instead of queueing behind one stream;
    // the lightest groups (the first to finish) first
    std::vector<int> fo;
    for (int gi = 0; gi < ng; gi++)
        if (done[gi]) fo.push_back(gi);
    std::stable_sort(fo.begin(), fo.end(), [&](int x, int y) {
        return grids[p.order[p.gbeg[x]]]->N * (p.gbeg[x + 1] - p.gbeg[x]) <
               grids[p.order[p.gbeg[y]]]->N * (p.gbeg[y + 1] - p.gbeg[y]);
    });
    for (int gi : fo) {
        if (rc != OFDFT_OK) break;
        const int b = p.gbeg[gi], K = p.gbeg[gi + 1] - b;
        for (int k = 0; k < kBatchStreams; k++)
            if (k != p.gstream[gi]) cudaStreamWaitEvent(st[k], done[gi], 0);
        for (int m = 0; m < K && rc == OFDFT_OK; m++)
            rc = enqueue_forces<T>(grids, rho_dev, f, F_out, p.order[b + m], st[(p.gstream[gi] + m) % kBatchStreams]);
    }
    for (cudaEvent_t e : done)
        if (e) cudaEventDestroy(e);
    for (int k = 0; k < kBatchStreams; k++) {
        cudaEventRecord(join[k], st[k]);
        cudaStreamWaitEvent(user, join[k], 0);
    }
    cudaEventDestroy(fork);
    for (int k = 0; k < kBatchStreams; k++) cudaEventDestroy(join[k]);
    if (rc) return rc;
    ofdft_grid *g = grids[0];
    CK(launch_collect<T>(dargs, n, p.dcol, user), "gather batch results");
    CK(cudaMemcpyAsync(p.hcol, p.dcol, (size_t)n * (E_NUM + S_NSCAL) * sizeof(double), cudaMemcpyDeviceToHost,
                       user),
       "batch results copy");
    return OFDFT_OK;
}

// the key of a batch plan: the functional, the stream, the modes; per snapshot the grid, its
// buffer generation, whether forces are wanted, its kernels and its arguments (every pointer
// and size); grouped = -1 leaves the grouping out (the automatic choice's key)
template <typename T>
std::vector<unsigned char> batch_key(int n, ofdft_grid *const *grids, const ofdft_functional *f,
                                     double *const *F_out, const std::vector<EvalArgs<T>> &args, int grouped) {
    ofdft_grid *g0 = grids[0];
    bool use_graph = g0->batch_graph && !f->knots;
    for (int i = 0; i < n; i++) use_graph = use_graph && !grids[i]->prof_on;
    std::vector<unsigned char> key;
    append_bytes(key, *f);
    append_bytes(key, g0->stream);
    append_bytes(key, (int)use_graph);
    append_bytes(key, grouped);
    append_bytes(key, (int)sizeof(T));
    for (int i = 0; i < n; i++) {
        append_bytes(key, grids[i]);
        append_bytes(key, grids[i]->generation);
        append_bytes(key, (int)(F_out && F_out[i]));
        append_kernels(key, ws<T>(grids[i]).ks);
        append_bytes(key, args[i]);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    append_bytes(key, dev);
    return key;
}

// one batched call in the given mode (grouped 1 / 0); ms: if set, the device time of the
// batch's enqueued work (CUDA events on the grids' stream)
template <typename T>
int batched_run(int n, ofdft_grid *const *grids, const void *const *rho_dev, const ofdft_functional *f, double *E_out,
                void *const *V_dev, double *const *F_out, const std::vector<EvalArgs<T>> &args, int grouped,
                float *ms) {
    ofdft_grid *g0 = grids[0];
    cudaStream_t user = g0->stream;
    bool use_graph = g0->batch_graph && !f->knots;
    for (int i = 0; i < n; i++) use_graph = use_graph && !grids[i]->prof_on;
    std::vector<unsigned char> key = batch_key<T>(n, grids, f, F_out, args, grouped);
    BatchPlan *plan = nullptr;
    for (auto &bp : batch_plans())
        if (bp.key == key) plan = &bp;
    cudaError_t e;
    if (!plan) {
        if ((int)batch_plans().size() >= kBatchPlans) {
            e = cudaStreamSynchronize(user);                 // (no call leaves a batch in flight)
            if (e != cudaSuccess) return fail(g0, OFDFT_ERR_CUDA, "stream synchronize", e);
            free_plan(batch_plans().front());
            batch_plans().erase(batch_plans().begin());
        }
        BatchPlan np;
        int rc = make_plan<T>(g0, n, grids, args, grouped != 0, np);
        if (!rc && use_graph) {
            cudaGraph_t graph = nullptr;
            cudaStream_t origin = batch_streams()[kBatchStreams];
            e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) rc = fail(g0, OFDFT_ERR_CUDA, "begin capture", e);
            if (!rc) {
                rc = enqueue_batch<T>(np, n, grids, rho_dev, f, args, F_out, origin);
                e = cudaStreamEndCapture(origin, &graph);
                if (!rc && e != cudaSuccess) rc = fail(g0, OFDFT_ERR_CUDA, "end capture", e);
                if (!rc) {
                    e = cudaGraphInstantiate(&np.exec, graph, 0);
                    if (e != cudaSuccess) rc = fail(g0, OFDFT_ERR_CUDA, "graph instantiate", e);
                }
                if (graph) cudaGraphDestroy(graph);
            }
        }
        if (rc) {
            free_plan(np);
            return rc;
        }
        np.key = std::move(key);
        batch_plans().push_back(std::move(np));
        plan = &batch_plans().back();
    }
    g0->batch_report = plan->report + (plan->exec ? ", replayed as one CUDA graph" : "");
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (ms) {
        e = cudaEventCreate(&t0);
        if (e == cudaSuccess) e = cudaEventCreate(&t1);
        if (e == cudaSuccess) e = cudaEventRecord(t0, user);
        if (e != cudaSuccess) {
            if (t0) cudaEventDestroy(t0);
            if (t1) cudaEventDestroy(t1);
            return fail(g0, OFDFT_ERR_CUDA, "event", e);
        }
    }
    if (plan->exec) {
        e = cudaGraphLaunch(plan->exec, user);
        if (e != cudaSuccess) {
            if (ms) {
                cudaEventDestroy(t0);
                cudaEventDestroy(t1);
            }
            return fail(g0, OFDFT_ERR_CUDA, "graph launch", e);
        }
    } else {
        int rc = enqueue_batch<T>(*plan, n, grids, rho_dev, f, args, F_out, user);
        if (rc) {
            if (ms) {
                cudaEventDestroy(t0);
                cudaEventDestroy(t1);
            }
            return rc;
        }
    }
    if (ms) cudaEventRecord(t1, user);
    e = cudaStreamSynchronize(user);
    if (ms) {
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, t0, t1);
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
    }
    if (e != cudaSuccess) return fail(g0, OFDFT_ERR_CUDA, "stream synchronize", e);
    const int W = E_NUM + S_NSCAL;
    for (int j = 0; j < n; j++) {
        const int i = plan->order[j];
        ofdft_grid *g = grids[i];
        const double *r = plan->hcol + (size_t)j * W;
        if (int rc = wait_status(g, r + E_NUM)) return rc;
        if (r[E_NUM + S_BAD] != 0.0) return fail(g, OFDFT_ERR_BAD_DENSITY, "bad density in batch");
        std::memcpy(E_out + E_NUM * i, r, E_NUM * sizeof(double));
        if (F_out && F_out[i]) std::memcpy(F_out[i], g->F_pinned, (size_t)3 * g->n_ions * sizeof(double));
    }
    return OFDFT_OK;
}

template <typename T>
int batched_impl(int n, ofdft_grid *const *grids, const void *const *rho_dev, const ofdft_functional *f,
                 double *E_out, void *const *V_dev, double *const *F_out) {
    ofdft_grid *g0 = grids[0];
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++)
            if (grids[j] == grids[i]) return fail(g0, OFDFT_ERR_INVALID_ARG, "a grid appears twice in the batch");
    std::vector<EvalArgs<T>> args(n);
    for (int i = 0; i < n; i++) {
        const bool want_f = F_out && F_out[i];
        int rc = prepare_batch_grid<T>(grids[i], f, want_f, (const T *)rho_dev[i]);
        if (!rc) rc = eval_args<T>(grids[i], (const T *)rho_dev[i], f, V_dev ? (T *)V_dev[i] : nullptr, nullptr, want_f,
                                   args[i]);
        if (rc) return rc;
    }
    int grouped = g0->batch_grouped;
    if (grouped >= 0) return batched_run<T>(n, grids, rho_dev, f, E_out, V_dev, F_out, args, grouped, nullptr);
    // automatic: the first call of a batch runs it both ways (each once to build its plan, once
    // timed with CUDA events) and keeps the faster for the later calls with the same key
    const std::vector<unsigned char> key = batch_key<T>(n, grids, f, F_out, args, -1);
    for (const BatchMode &d : batch_modes())
        if (d.key == key) {
            int rc = batched_run<T>(n, grids, rho_dev, f, E_out, V_dev, F_out, args, d.grouped, nullptr);
            g0->batch_report += d.note;
            return rc;
        }
    float ms[2] = {0.f, 0.f};
    std::string rep[2];
    for (int m = 1; m >= 0; m--) {
        for (int r = 0; r < 2; r++)
            if (int rc = batched_run<T>(n, grids, rho_dev, f, E_out, V_dev, F_out, args, m, r ? &ms[m] : nullptr))
                return rc;
        rep[m] = g0->batch_report;
    }
    BatchMode d;
    d.key = key;
    d.grouped = ms[1] <= ms[0] ? 1 : 0;
    char buf[160];
    std::snprintf(buf, sizeof(buf), " (automatic choice: grouped %.3f ms, one launch per snapshot %.3f ms)", ms[1],
                  ms[0]);
    d.note = buf;
    g0->batch_report = rep[d.grouped] + d.note;
    if (batch_modes().size() >= 64) batch_modes().erase(batch_modes().begin());
    batch_modes().push_back(d);
    // the outputs are those of the last run: the same as the chosen mode's (E and V bit-identical)
    return OFDFT_OK;
}


}  // namespace

// ====================================================================== ABI
extern "C" {

const char *ofdft_version(void) { return "ofdft-gb300 0.1 (sm_103a)"; }

const char *ofdft_status_string(int s) {
    switch (s) {
        case OFDFT_OK: return "ok";
        case OFDFT_ERR_INVALID_ARG: return "invalid argument";
        case OFDFT_ERR_UNSUPPORTED_SIZE: return "unsupported grid size (need 2^a 3^b 5^c in [2, 1024])";
        case OFDFT_ERR_BAD_DENSITY: return "bad density (NaN, Inf or negative)";
        case OFDFT_ERR_OOM: return "out of device memory";
        case OFDFT_ERR_CUDA: return "CUDA error";
        case OFDFT_ERR_NOT_CONVERGED: return "optimiser did not converge";
        case OFDFT_ERR_NO_IONS: return "no ions set";
        case OFDFT_ERR_TIMEOUT: return "a bounded device wait expired";
        default: return "unknown status";
    }
}

const char *ofdft_last_error(const ofdft_grid *g) { return g ? g->err.c_str() : "null handle"; }

int ofdft_grid_create(const double cell[9], const int shape[3], void *cuda_stream, ofdft_grid **out) {
    if (!cell || !shape || !out) return OFDFT_ERR_INVALID_ARG;
    *out = nullptr;
    for (int a = 0; a < 3; a++) {
        std::vector<int> r;
        if (shape[a] < 2 || shape[a] > 1024 || !factor_235(shape[a], r)) return OFDFT_ERR_UNSUPPORTED_SIZE;
    }
    const double *A = cell;
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (!(std::fabs(det) > 1e-12)) return OFDFT_ERR_INVALID_ARG;
    ofdft_grid *g = new (std::nothrow) ofdft_grid();
    if (!g) return OFDFT_ERR_OOM;
    for (int a = 0; a < 3; a++) g->n[a] = shape[a];
    g->n2h = shape[2] / 2 + 1;
    g->N = (long long)shape[0] * shape[1] * shape[2];
    g->NH = (long long)shape[0] * shape[1] * g->n2h;
    std::memcpy(g->cell, cell, 9 * sizeof(double));
    // recip rows b_i = rows of inv(A)^T: b_i . a_j = delta_ij; inv(A)^T = cofactor(A) / det
    const double inv[9] = {(A[4] * A[8] - A[5] * A[7]) / det, -(A[1] * A[8] - A[2] * A[7]) / det,
                           (A[1] * A[5] - A[2] * A[4]) / det, -(A[3] * A[8] - A[5] * A[6]) / det,
                           (A[0] * A[8] - A[2] * A[6]) / det, -(A[0] * A[5] - A[2] * A[3]) / det,
                           (A[3] * A[7] - A[4] * A[6]) / det, -(A[0] * A[7] - A[1] * A[6]) / det,
                           (A[0] * A[4] - A[1] * A[3]) / det};
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) g->recip[3 * i + j] = inv[3 * j + i];
    g->omega = std::fabs(det);
    g->dV = g->omega / (double)g->N;
    g->stream = (cudaStream_t)cuda_stream;
    for (int a = 0; a < 3; a++) g->plan[a] = make_plan(shape[a]);
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess) e = cudaMallocHost(&g->h_pinned, 64 * sizeof(double));
    if (e != cudaSuccess) {
        delete g;
        return e == cudaErrorMemoryAllocation ? OFDFT_ERR_OOM : OFDFT_ERR_CUDA;
    }
    *out = g;
    return OFDFT_OK;
}

int ofdft_profile_enable(ofdft_grid *g, int enable) {
    if (!g) return OFDFT_ERR_INVALID_ARG;
    g->prof_on = enable != 0;
    return OFDFT_OK;
}

int ofdft_profile_reset(ofdft_grid *g) {
    if (!g) return OFDFT_ERR_INVALID_ARG;
    prof_collect(g);
    for (int i = 0; i < K_NKERNEL; i++) {
        g->prof_ms[i] = 0.0;
        g->prof_n[i] = 0;
    }
    return OFDFT_OK;
}

int ofdft_profile_read(ofdft_grid *g, int idx, const char **name, int *launches, double *total_ms) {
    if (!g || idx < 0 || idx >= K_NKERNEL) return OFDFT_ERR_INVALID_ARG;
    prof_collect(g);
    if (name) *name = kKernelNames[idx];
    if (launches) *launches = g->prof_n[idx];
    if (total_ms) *total_ms = g->prof_ms[idx];
    return OFDFT_OK;
}

const char *ofdft_tuning_report(const ofdft_grid *g, int precision) {
    if (!g) return "null handle";
    const std::string &r = precision == OFDFT_FP64 ? g->w64.tune_report : g->w32.tune_report;
    return r.c_str();
}

const char *ofdft_batch_report(const ofdft_grid *g) {
    if (!g) return "null handle";
    return g->batch_report.c_str();
}

int ofdft_set_option(ofdft_grid *g, int option, long long value) {
    if (!g) return OFDFT_ERR_INVALID_ARG;
    switch (option) {
        case OFDFT_OPTION_KERNELS:
            if (value != OFDFT_KERNELS_AUTO && value != OFDFT_KERNELS_GENERIC &&
                value != OFDFT_KERNELS_PER_CHANNEL_ROWS && value != OFDFT_KERNELS_TILE_RECIP)
                return fail(g, OFDFT_ERR_INVALID_ARG, "unknown kernel choice");
            if (value != g->kernel_choice) {
                // the launch plan is made with the workspaces: drop them (rebuilt on next use)
                cudaStreamSynchronize(g->stream);
                free_ws(g->w32);
                free_ws(g->w64);
                g->vext_fresh32 = g->vext_fresh64 = false;
                g->generation++;
                g->kernel_choice = (int)value;
            }
            return OFDFT_OK;
        case OFDFT_OPTION_BATCH_GRAPH:
            g->batch_graph = value != 0;
            return OFDFT_OK;
        case OFDFT_OPTION_BATCH_GROUPED:
            if (value < -1 || value > 1) return fail(g, OFDFT_ERR_INVALID_ARG, "batch grouping must be -1, 0 or 1");
            g->batch_grouped = (int)value;
            return OFDFT_OK;
        case OFDFT_OPTION_WAIT_POLLS:
            if (value < 0 || value > (1LL << 30)) return fail(g, OFDFT_ERR_INVALID_ARG, "wait polls out of range");
            g->wait_polls = (unsigned)value;
            return OFDFT_OK;
        case OFDFT_OPTION_PICK_ROWS:
        case OFDFT_OPTION_PICK_PENCIL:
        case OFDFT_OPTION_PICK_RECIP: {
            if (value < -1 || value > 255) return fail(g, OFDFT_ERR_INVALID_ARG, "candidate index out of range");
            const int r = option == OFDFT_OPTION_PICK_ROWS ? TUNE_ROWS
                        : option == OFDFT_OPTION_PICK_PENCIL ? TUNE_PENCIL : TUNE_AXIS0;
            if (g->force_pick[r] != (int)value) {
                cudaStreamSynchronize(g->stream);
                free_ws(g->w32);
                free_ws(g->w64);
                g->vext_fresh32 = g->vext_fresh64 = false;
                g->generation++;
                g->force_pick[r] = (int)value;
            }
            return OFDFT_OK;
        }
        case OFDFT_OPTION_EXACT_SUMS:
            if ((value != 0) != (g->exact_sums != 0)) {
                cudaStreamSynchronize(g->stream);
                free_ws(g->w32);
                free_ws(g->w64);
                g->vext_fresh32 = g->vext_fresh64 = false;
                g->generation++;
                g->exact_sums = value != 0;
            }
            return OFDFT_OK;
        case OFDFT_OPTION_ALLOC_CAP:
            if (value < 0) return fail(g, OFDFT_ERR_INVALID_ARG, "negative allocation cap");
            g->alloc_cap = (size_t)value;
            g->alloc_bytes = 0;
            return OFDFT_OK;
        default:
            return fail(g, OFDFT_ERR_INVALID_ARG, "unknown option");
    }
}

int ofdft_grid_destroy(ofdft_grid *g) {
    if (!g) return OFDFT_ERR_INVALID_ARG;
    cudaStreamSynchronize(g->stream);
    prof_collect(g);
    for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
    free_ws(g->w32);
    free_ws(g->w64);
    cudaFree(g->ph);
    cudaFree(g->ph32);
    cudaFree(g->gf);
    cudaFree(g->d_sp_ions);
    cudaFree(g->fpart);
    cudaFree(g->F_dev);
    cudaFreeHost(g->F_pinned);
    cudaFree(g->pmeB);
    cudaFree(g->d_pos);
    cudaFree(g->Qfix);
    cudaFree(g->pme_real);
    cudaFree(g->d_species);
    cudaFree(g->d_Z);
    cudaFree(g->d_rc);
    cudaFree(g->ew_p);
    cudaFree(g->ew_cell);
    cudaFree(g->ew_orig);
    cudaFree(g->ew_cstart);
    cudaFree(g->ew_F);
    cudaFree(g->ew_e);
    cudaFree(g->ew_part);
    cudaFreeHost(g->h_pinned);
    delete g;
    return OFDFT_OK;
}

}  // extern "C"

namespace {

// common part of both ion set-ups: validation, host copies, device species/Z/rc
int store_ions(ofdft_grid *g, const ofdft_ions *ions, const ofdft_species *sp) {
    if (!ions || !sp || ions->n < 1 || !ions->pos || !ions->species || sp->n_species < 1 || !sp->Z || !sp->rc)
        return fail(g, OFDFT_ERR_INVALID_ARG, "ions/species");
    for (int i = 0; i < ions->n; i++)
        if (ions->species[i] < 0 || ions->species[i] >= sp->n_species)
            return fail(g, OFDFT_ERR_INVALID_ARG, "species index out of range");
    CK(cudaStreamSynchronize(g->stream), "stream synchronize");
    const int n = ions->n;
    if (n != g->n_ions || sp->n_species != g->n_species) {
        cudaFree(g->ph);
        cudaFree(g->ph32);
        cudaFree(g->d_pos);
        cudaFree(g->d_species);
        cudaFree(g->d_sp_ions);
        cudaFree(g->d_Z);
        cudaFree(g->d_rc);
        g->ph = nullptr;
        g->ph32 = nullptr;
        g->d_pos = nullptr;
        g->d_species = nullptr;
        g->d_sp_ions = nullptr;
        g->d_Z = g->d_rc = nullptr;
        CK(gmalloc(g, &g->d_species, n * sizeof(int)), "cudaMalloc species");
        CK(gmalloc(g, &g->d_sp_ions, n * sizeof(int)), "cudaMalloc species lists");
        CK(gmalloc(g, &g->d_Z, sp->n_species * sizeof(double)), "cudaMalloc Z");
        CK(gmalloc(g, &g->d_rc, sp->n_species * sizeof(double)), "cudaMalloc rc");
    }
    g->n_ions = n;
    // the force tables depend on the species' Z and rc only (not on positions)
    if (g->n_species != sp->n_species || !std::equal(g->Z.begin(), g->Z.end(), sp->Z) ||
        !std::equal(g->rc.begin(), g->rc.end(), sp->rc))
        g->gf_fresh = false;
    g->n_species = sp->n_species;
    g->pos.assign(ions->pos, ions->pos + 3 * (size_t)n);
    g->species.assign(ions->species, ions->species + n);
    g->Z.assign(sp->Z, sp->Z + sp->n_species);
    g->rc.assign(sp->rc, sp->rc + sp->n_species);
    g->species_count.assign(sp->n_species, 0);
    for (int i = 0; i < n; i++) g->species_count[g->species[i]]++;
    g->sp_off.assign(sp->n_species + 1, 0);
    for (int s = 0; s < sp->n_species; s++) g->sp_off[s + 1] = g->sp_off[s] + g->species_count[s];
    std::vector<int> lists(n), fill(g->sp_off.begin(), g->sp_off.end() - 1);
    for (int i = 0; i < n; i++) lists[fill[g->species[i]]++] = i;
    CK(cudaMemcpy(g->d_species, g->species.data(), n * sizeof(int), cudaMemcpyHostToDevice), "upload species");
    CK(cudaMemcpy(g->d_sp_ions, lists.data(), n * sizeof(int), cudaMemcpyHostToDevice), "upload species lists");
    CK(cudaMemcpy(g->d_Z, g->Z.data(), g->n_species * sizeof(double), cudaMemcpyHostToDevice), "upload Z");
    CK(cudaMemcpy(g->d_rc, g->rc.data(), g->n_species * sizeof(double), cudaMemcpyHostToDevice), "upload rc");
    g->have_ions = true;
    g->vext_fresh32 = g->vext_fresh64 = false;
    return OFDFT_OK;
}

}  // namespace

extern "C" {

int ofdft_set_ions(ofdft_grid *g, const ofdft_ions *ions, const ofdft_species *sp) {
    if (!g) return OFDFT_ERR_INVALID_ARG;
    int rc = store_ions(g, ions, sp);
    if (rc) return rc;
    g->pme_order = 0;
    const int n = g->n_ions;
    if (!g->ph) {
        CK(gmalloc(g, &g->ph, (size_t)n * (g->n[0] + g->n[1] + g->n2h) * sizeof(double2)), "cudaMalloc phases");
        CK(gmalloc(g, &g->ph32, (size_t)n * (g->n[0] + g->n[1] + g->n2h) * sizeof(float2)), "cudaMalloc phases");
    }
    // per-axis phase tables e^{-2 pi i m_a f_a}, f = R . inv(cell) (fractional)
    const int na[3] = {g->n[0], g->n[1], g->n2h};
    std::vector<double2> ph((size_t)n * (na[0] + na[1] + na[2]));
    size_t off = 0;
    for (int ax = 0; ax < 3; ax++) {
        for (int I = 0; I < n; I++) {
            const double *R = &g->pos[3 * (size_t)I];
            // fractional coordinate along a_ax: R . b_ax
            const double fr = R[0] * g->recip[3 * ax] + R[1] * g->recip[3 * ax + 1] + R[2] * g->recip[3 * ax + 2];
            for (int k = 0; k < na[ax]; k++) {
                const int nn = g->n[ax];
                const double m = (ax == 2) ? k : ((k <= nn / 2) ? k : k - nn);
                double t = m * fr;
                t -= std::floor(t);
                const double ang = -2.0 * kPi * t;
                ph[off + (size_t)I * na[ax] + k] = make_double2(std::cos(ang), std::sin(ang));
            }
        }
        off += (size_t)n * na[ax];
    }
    CK(cudaMemcpy(g->ph, ph.data(), ph.size() * sizeof(double2), cudaMemcpyHostToDevice), "upload phases");
    CK(launch_round_phases(g->ph, g->ph32, (long long)ph.size(), g->stream), "round phases");
    return OFDFT_OK;
}

int ofdft_set_ions_pme(ofdft_grid *g, const ofdft_ions *ions, const ofdft_species *sp, int order) {
    if (!g) return OFDFT_ERR_INVALID_ARG;
    if (order < 4 || order > kPmeMaxOrder || order % 2) return fail(g, OFDFT_ERR_INVALID_ARG, "PME order must be even, 4..16");
    for (int a = 0; a < 3; a++)
        if (g->n[a] < order) return fail(g, OFDFT_ERR_INVALID_ARG, "grid smaller than the PME stencil");
    int rc = store_ions(g, ions, sp);
    if (rc) return rc;
    g->pme_order = order;
    if (!g->d_pos) CK(gmalloc(g, &g->d_pos, (size_t)3 * g->n_ions * sizeof(double)), "cudaMalloc positions");
    CK(cudaMemcpy(g->d_pos, g->pos.data(), (size_t)3 * g->n_ions * sizeof(double), cudaMemcpyHostToDevice),
       "upload positions");
    // conj b_a(k) = conj( e^{2 pi i (p-1) k/n} / sum_{j=0}^{p-2} M_p(j+1) e^{2 pi i k j/n} )
    std::vector<double> Mp(order + 1, 0.0);   // M_p at the integers 1..p-1
    {
        std::vector<double> w(order, 0.0);
        w[0] = 0.0;
        w[1] = 1.0;                            // order 2 at x = 0: M_2(0) = 0, M_2(1) = 1
        for (int k = 3; k <= order; k++)
            for (int i = k - 1; i >= 0; i--) {
                const double a = (i >= 1) ? w[i - 1] : 0.0;
                w[i] = ((double)i * w[i] + (double)(k - i) * a) / (double)(k - 1);
            }
        for (int i = 0; i < order; i++) Mp[i] = w[i];      // Mp[i] = M_p(i)
    }
    const int na[3] = {g->n[0], g->n[1], g->n2h};
    std::vector<double2> B((size_t)na[0] + na[1] + na[2]);
    size_t off = 0;
    for (int ax = 0; ax < 3; ax++) {
        const int n = g->n[ax];
        for (int k = 0; k < na[ax]; k++) {
            double dr = 0.0, di = 0.0;
            for (int j = 0; j <= order - 2; j++) {
                const double ang = 2.0 * kPi * (double)k * j / n;
                dr += Mp[j + 1] * std::cos(ang);
                di += Mp[j + 1] * std::sin(ang);
            }
            const double ang = 2.0 * kPi * (double)(order - 1) * k / n;
            const double nr = std::cos(ang), ni = std::sin(ang);
            const double den = dr * dr + di * di;
            const double br = (nr * dr + ni * di) / den, bi = (ni * dr - nr * di) / den;
            B[off + k] = make_double2(br, -bi);    // conjugate
        }
        off += na[ax];
    }
    if (!g->pmeB) CK(gmalloc(g, &g->pmeB, B.size() * sizeof(double2)), "cudaMalloc PME factors");
    CK(cudaMemcpy(g->pmeB, B.data(), B.size() * sizeof(double2), cudaMemcpyHostToDevice), "upload PME factors");
    return OFDFT_OK;
}

int ofdft_energy_potential(ofdft_grid *g, const void *rho_dev, const ofdft_functional *f, double *E_out,
                           void *V_dev) {
    if (!g) return OFDFT_ERR_INVALID_ARG;
    if (!rho_dev) return fail(g, OFDFT_ERR_INVALID_ARG, "rho is NULL");
    int rc = check_functional(g, f);
    if (rc) return rc;
    if (f->precision == OFDFT_FP64) return eval_sync<double>(g, (const double *)rho_dev, f, (double *)V_dev, E_out);
    return eval_sync<float>(g, (const float *)rho_dev, f, (float *)V_dev, E_out);
}

int ofdft_energy_potential_async(ofdft_grid *g, const void *rho_dev, const ofdft_functional *f, double *E_dev,
                                 void *V_dev) {
    if (!g) return OFDFT_ERR_INVALID_ARG;
    if (!rho_dev || !E_dev) return fail(g, OFDFT_ERR_INVALID_ARG, "rho or E_dev is NULL");
    int rc = check_functional(g, f);
    if (rc) return rc;
    if (f->precision == OFDFT_FP64) return enqueue_eval<double>(g, (const double *)rho_dev, f, (double *)V_dev, E_dev);
    return enqueue_eval<float>(g, (const float *)rho_dev, f, (float *)V_dev, E_dev);
}

int ofdft_forces(ofdft_grid *g, const void *rho_dev, int precision, double *F_out) {
    if (!g) return OFDFT_ERR_INVALID_ARG;
    if (!rho_dev || !F_out) return fail(g, OFDFT_ERR_INVALID_ARG, "rho or F_out is NULL");
    if (!g->have_ions) return fail(g, OFDFT_ERR_NO_IONS, "forces need ions");
    if (precision == OFDFT_FP64) return forces_impl<double>(g, (const double *)rho_dev, F_out);
    if (precision == OFDFT_FP32_MIXED) return forces_impl<float>(g, (const float *)rho_dev, F_out);
    return fail(g, OFDFT_ERR_INVALID_ARG, "unknown precision");
}

int ofdft_ewald(ofdft_grid *g, double *E_out, double *F_out) {
    if (!g) return OFDFT_ERR_INVALID_ARG;
    if (!E_out && !F_out) return fail(g, OFDFT_ERR_INVALID_ARG, "E_out and F_out are both NULL");
    if (!g->have_ions) return fail(g, OFDFT_ERR_NO_IONS, "the Ewald sum needs ions");
    return ewald_impl(g, E_out, F_out);
}

int ofdft_interpolate(ofdft_grid *from, const void *src_dev, ofdft_grid *to, void *dst_dev, int precision) {
    if (!from || !to) return OFDFT_ERR_INVALID_ARG;
    if (!src_dev || !dst_dev) return fail(to, OFDFT_ERR_INVALID_ARG, "src or dst is NULL");
    if (!same_cell(from, to)) return fail(to, OFDFT_ERR_INVALID_ARG, "the two grids must share one cell");
    int rc;
    if (precision == OFDFT_FP64) rc = interpolate_impl<double>(from, (const double *)src_dev, to, (double *)dst_dev);
    else if (precision == OFDFT_FP32_MIXED) rc = interpolate_impl<float>(from, (const float *)src_dev, to, (float *)dst_dev);
    else return fail(to, OFDFT_ERR_INVALID_ARG, "unknown precision");
    if (rc) return rc;
    ofdft_grid *g = to;
    CK(cudaStreamSynchronize(to->stream), "stream synchronize");
    return OFDFT_OK;
}

int ofdft_td_kick(ofdft_grid *g, void *psi_re, void *psi_im, const double k[3], int precision) {
    if (!g) return OFDFT_ERR_INVALID_ARG;
    if (!psi_re || !psi_im || !k) return fail(g, OFDFT_ERR_INVALID_ARG, "psi or k is NULL");
    TdCell cell;
    for (int i = 0; i < 9; i++) cell.a[i] = g->cell[i];
    if (precision == OFDFT_FP64)
        CK(launch_kick<double>((double *)psi_re, (double *)psi_im, g->n[0], g->n[1], g->n[2], cell, k, g->stream), "kick");
    else if (precision == OFDFT_FP32_MIXED)
        CK(launch_kick<float>((float *)psi_re, (float *)psi_im, g->n[0], g->n[1], g->n[2], cell, k, g->stream), "kick");
    else
        return fail(g, OFDFT_ERR_INVALID_ARG, "unknown precision");
    return OFDFT_OK;
}

int ofdft_td_propagate(ofdft_grid *g, void *psi_re, void *psi_im, const void *rho0, const ofdft_functional *f,
                       const ofdft_td_options *opt, double *dipole, ofdft_td_report *rep) {
    if (!g) return OFDFT_ERR_INVALID_ARG;
    if (!psi_re || !psi_im || !opt) return fail(g, OFDFT_ERR_INVALID_ARG, "psi or options NULL");
    if (!(std::isfinite(opt->dt) && opt->dt != 0.0) || opt->n_steps < 0 || opt->n_corrector < 0 ||
        opt->n_corrector > 16 || opt->max_solver_iter < 0 || !(opt->solver_tol >= 0.0))
        return fail(g, OFDFT_ERR_INVALID_ARG, "TD options");
    int rc = check_functional(g, f);
    if (rc) return rc;
    if (f->precision == OFDFT_FP64)
        return td_impl<double>(g, (double *)psi_re, (double *)psi_im, (const double *)rho0, f, *opt, dipole, rep);
    return td_impl<float>(g, (float *)psi_re, (float *)psi_im, (const float *)rho0, f, *opt, dipole, rep);
}

int ofdft_td_spectrum(const double *dmu, int n, double dt, double gamma, int n_omega, const double *omega,
                      double *sigma) {
    if (!dmu || !omega || !sigma || n < 1 || n_omega < 0 || !(dt != 0.0) || !(gamma >= 0.0))
        return OFDFT_ERR_INVALID_ARG;
    for (int m = 0; m < n_omega; m++) {
        // Im sum_n dmu_n e^{(i w - gamma) t_n} dt, the phase kept in [0, 2 pi) for accuracy
        double im = 0.0;
        for (int k = 0; k < n; k++) {
            const double t = k * dt;
            im += dmu[k] * std::exp(-gamma * t) * std::sin(std::fmod(omega[m] * t, 2.0 * kPi));
        }
        sigma[m] = omega[m] * im * dt;
    }
    return OFDFT_OK;
}

int ofdft_optimize_density_multistep(int n_levels, ofdft_grid *const *grids, void *psi_dev, const ofdft_functional *f,
                                     double N_e, double tol_E_per_atom, int max_iter, ofdft_opt_report *rep) {
    if (n_levels < 1 || !grids) return OFDFT_ERR_INVALID_ARG;
    ofdft_grid *fine = grids[n_levels - 1];
    for (int L = 0; L < n_levels; L++)
        if (!grids[L]) return OFDFT_ERR_INVALID_ARG;
    if (!psi_dev || !(N_e > 0.0) || max_iter < 1 || !f) return fail(fine, OFDFT_ERR_INVALID_ARG, "psi, f, N_e or max_iter");
    for (int L = 0; L < n_levels; L++) {
        if (!same_cell(grids[L], fine)) return fail(fine, OFDFT_ERR_INVALID_ARG, "all levels must share one cell");
        int rc = check_functional(grids[L], f);
        if (rc) {
            fine->err = grids[L]->err;
            return rc;
        }
    }
    if (f->precision == OFDFT_FP64)
        return multistep_impl<double>(n_levels, grids, (double *)psi_dev, f, N_e, tol_E_per_atom, max_iter, rep);
    return multistep_impl<float>(n_levels, grids, (float *)psi_dev, f, N_e, tol_E_per_atom, max_iter, rep);
}

int ofdft_optimize_density_ex(ofdft_grid *g, void *psi_dev, const ofdft_functional *f, double N_e,
                              double tol_E_per_atom, int max_iter, const ofdft_opt_options *opt,
                              ofdft_opt_report *rep) {
    if (!g) return OFDFT_ERR_INVALID_ARG;
    if (!psi_dev || !(N_e > 0.0) || max_iter < 1) return fail(g, OFDFT_ERR_INVALID_ARG, "psi, N_e or max_iter");
    const ofdft_opt_options o = opt ? *opt : kOptDefaults;
    if (o.method < OFDFT_OPT_CG || o.method > OFDFT_OPT_LBFGS || o.max_inner < 0 || o.max_inner > 100 ||
        o.lbfgs_m < 0 || o.lbfgs_m > 32 || o.update < OFDFT_UPDATE_ROTATE || o.update > OFDFT_UPDATE_SCALE ||
        o.objective < OFDFT_OBJECTIVE_ENERGY || o.objective > OFDFT_OBJECTIVE_RESIDUAL)
        return fail(g, OFDFT_ERR_INVALID_ARG, "optimiser options");
    int rc = check_functional(g, f);
    if (rc) return rc;
    if (f->precision == OFDFT_FP64)
        return optimize_impl<double>(g, (double *)psi_dev, f, N_e, tol_E_per_atom, max_iter, o, rep);
    return optimize_impl<float>(g, (float *)psi_dev, f, N_e, tol_E_per_atom, max_iter, o, rep);
}

int ofdft_optimize_density(ofdft_grid *g, void *psi_dev, const ofdft_functional *f, double N_e,
                           double tol_E_per_atom, int max_iter, ofdft_opt_report *rep) {
    return ofdft_optimize_density_ex(g, psi_dev, f, N_e, tol_E_per_atom, max_iter, nullptr, rep);
}

int ofdft_energy_potential_batched(int n, ofdft_grid *const *grids, const void *const *rho_dev,
                                   const ofdft_functional *f, double *E_out, void *const *V_dev,
                                   double *const *F_out) {
    if (n < 0 || (n > 0 && (!grids || !rho_dev || !E_out))) return OFDFT_ERR_INVALID_ARG;
    if (n == 0) return OFDFT_OK;
    for (int i = 0; i < n; i++) {
        if (!grids[i]) return OFDFT_ERR_INVALID_ARG;
        int rc = check_functional(grids[i], f);
        if (rc) return rc;
        if (grids[i]->stream != grids[0]->stream) return fail(grids[i], OFDFT_ERR_INVALID_ARG, "streams differ");
        for (int j = 0; j < i; j++)
            if (grids[j] == grids[i]) return fail(grids[i], OFDFT_ERR_INVALID_ARG, "a grid appears twice in the batch");
        if (F_out && F_out[i] && !grids[i]->have_ions) return fail(grids[i], OFDFT_ERR_NO_IONS, "forces need ions");
    }
    const bool fp64 = f->precision == OFDFT_FP64;
    return fp64 ? batched_impl<double>(n, grids, rho_dev, f, E_out, V_dev, F_out)
                : batched_impl<float>(n, grids, rho_dev, f, E_out, V_dev, F_out);
}

}  // extern "C"
