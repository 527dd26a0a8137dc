// Instantiations of the persistent reciprocal-space kernel (recip.cuh) and its registry.
#include "recip.cuh"

namespace ofdft {

namespace {
template <typename T, int N, int E, int NSTAGE> void set_recip(RecipLaunch *out) {
    typedef RecipShape<T, N, E, NSTAGE> S;
    out->k = (const void *)recip_kernel<T, N, E, NSTAGE, false>;
    out->k_mgp = (const void *)recip_kernel<T, N, E, NSTAGE, true>;
    out->nt = S::NT;
    out->per_sm = 1;
    out->smem = S::smem;
}
}  // namespace

// n0 lengths with a register-resident plan: E elements per thread (every radix divides E),
// NSTAGE channel tiles in flight
template <> bool find_recip<float>(int n, RecipLaunch *out) {
    switch (n) {
        case 128: set_recip<float, 128, 16, 4>(out); return true;
        case 64: set_recip<float, 64, 8, 6>(out); return true;
        case 32: set_recip<float, 32, 4, 8>(out); return true;
        default: return false;
    }
}
template <> bool find_recip<double>(int, RecipLaunch *) { return false; }

}  // namespace ofdft
