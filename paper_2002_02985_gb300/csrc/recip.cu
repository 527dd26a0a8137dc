// Instantiations of the persistent reciprocal-space kernel (recip.cuh) and its registry.
#include <cstdio>

#include "recip.cuh"

namespace ofdft {

namespace {
// TW columns per tile, MINB blocks per SM
template <typename T, int N, int E, int NSTAGE, int TW = 32, int MINB = 1> void add_recip(std::vector<KernelCand> &out) {
    typedef RecipShape<T, N, E, NSTAGE, TW> S;
    KernelCand c;
    c.recip.k = (const void *)recip_kernel<T, N, E, NSTAGE, false, TW, MINB>;
    c.recip.k_mgp = (const void *)recip_kernel<T, N, E, NSTAGE, true, TW, MINB>;
    c.recip.g = (const void *)recip_group<T, N, E, NSTAGE, false, TW, MINB>;
    c.recip.g_mgp = (const void *)recip_group<T, N, E, NSTAGE, true, TW, MINB>;
    c.recip.nt = S::NT;
    c.recip.per_sm = MINB;
    c.recip.tw = TW;
    c.recip.smem = S::smem;
    c.B = TW;
    c.nt = S::NT;
    std::snprintf(c.name, sizeof(c.name), "recip E%d s%d w%d x%d b%d", E, NSTAGE, TW, S::NT, MINB);
    out.push_back(c);
}
}  // namespace

// n0 lengths with a register-resident plan: E elements per thread (every radix divides E),
// NSTAGE channel tiles in flight; the first is the default, the autotuner times the rest
template <> void recip_candidates<float>(int n, std::vector<KernelCand> &out) {
    switch (n) {
        case 128:
            add_recip<float, 128, 8, 4, 16, 2>(out);
            add_recip<float, 128, 16, 4, 16, 2>(out);
            add_recip<float, 128, 16, 4>(out);
            add_recip<float, 128, 8, 4>(out);
            // 14 / 28 columns: the 128 x 65 columns of a 128^3 grid make 595 / 298 tiles, just under
            // two per block (16 / 32 columns: 520 / 260 tiles, so a quarter of the blocks idle
            // through the second round)
            add_recip<float, 128, 8, 4, 14, 2>(out);
            add_recip<float, 128, 8, 4, 28, 1>(out);
            add_recip<float, 128, 16, 4, 14, 2>(out);
            // 8 columns, 64 threads: a block barrier joins two warps
            add_recip<float, 128, 16, 3, 8, 4>(out);
            break;
        case 64:
            add_recip<float, 64, 8, 6>(out);
            add_recip<float, 64, 4, 4, 16, 2>(out);
            break;
        case 32: add_recip<float, 32, 4, 8>(out); break;
        case 1024:
            // 4-column tiles (32-byte rows: the tensor copies' x stays a multiple of 16 bytes), one
            // block per SM: 16 elements per thread (passes 16 16 4) or 8 (passes 8 8 8 2)
            add_recip<float, 1024, 16, 4, 4, 1>(out);
            add_recip<float, 1024, 16, 2, 4, 1>(out);
            add_recip<float, 1024, 8, 4, 4, 1>(out);
            break;
        default: break;
    }
}
template <> void recip_candidates<double>(int, std::vector<KernelCand> &) {}

}  // namespace ofdft
