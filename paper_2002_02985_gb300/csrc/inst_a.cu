// Specialised kernels: the 128^3 workload (FP32 and FP64) and 32.
#include <cstdlib>

#include "inst.cuh"

namespace ofdft {

template <typename T> bool find_specialised_a(int role, int n, const void **k1, const void **k2, int *B, int *nt);

// Tile-shape variants of the 128-point kernels (selected by OFDFT_VARIANT_128 for
// tuning sweeps; variant 0 is the default).
static bool variant_128(int v, int role, int n, const void **k1, const void **k2, int *B, int *nt) {
    switch (v) {
        case 1: OFDFT_SPECIALISE_X(float, 128, 8, 256, 16, 256, 8, 128, 8, 8, 0, 0) break;
        case 2: OFDFT_SPECIALISE_X(float, 128, 8, 128, 16, 256, 8, 128, 8, 16, 0, 5) break;
        case 3: OFDFT_SPECIALISE_X(float, 128, 16, 256, 16, 256, 16, 256, 8, 8, 0, 0) break;
        case 4: OFDFT_SPECIALISE_X(float, 128, 4, 128, 16, 256, 8, 256, 8, 8, 0, 0) break;
        case 5: OFDFT_SPECIALISE_ROW2(float, 128, 20, 160, 16, 4) break;
        case 6: OFDFT_SPECIALISE_X(float, 128, 8, 256, 16, 256, 8, 64, 16, 16, 0, 0) break;
        case 7: OFDFT_SPECIALISE_X(float, 128, 8, 256, 16, 256, 16, 128, 16, 16, 0, 2) break;
        case 8: OFDFT_SPECIALISE_X(float, 128, 8, 256, 16, 256, 8, 128, 16, 8, 0, 0) break;
        case 9: OFDFT_SPECIALISE_PENCIL(float, 128, 16, 256, 4) break;
        case 10: OFDFT_SPECIALISE_PENCIL(float, 128, 16, 128, 8) break;
        case 11: OFDFT_SPECIALISE_PENCIL(float, 128, 8, 128, 8) break;
        default: break;
    }
    return false;
}

template <> bool find_specialised_a<float>(int role, int n, const void **k1, const void **k2, int *B, int *nt) {
    if (n == 128) {
        const char *env = std::getenv("OFDFT_VARIANT_128");
        const int v = env ? std::atoi(env) : 0;
        if (v > 0 && variant_128(v, role, n, k1, k2, B, nt)) return true;
    }
    OFDFT_SPECIALISE_ROW2(float, 128, 20, 160, 16, 5)
    OFDFT_SPECIALISE(float, 128, 8, 256, 16, 256, 8, 128)
    OFDFT_SPECIALISE_ROW2(float, 32, 16, 64, 16, 10)
    OFDFT_SPECIALISE(float, 32, 16, 128, 16, 128, 16, 128)
    return false;
}
template <> bool find_specialised_a<double>(int role, int n, const void **k1, const void **k2, int *B, int *nt) {
    OFDFT_SPECIALISE(double, 128, 4, 256, 8, 256, 8, 256)
    return false;
}

}  // namespace ofdft
