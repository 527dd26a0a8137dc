// Specialised kernels: grid sizes 64, 80 and 96 (FP32).
#include "inst.cuh"

namespace ofdft {

template <typename T> bool find_specialised_b(int role, int n, const void **k1, const void **k2, int *B, int *nt);

template <> bool find_specialised_b<float>(int role, int n, const void **k1, const void **k2, int *B, int *nt) {
    OFDFT_SPECIALISE_ROW2(float, 64, 20, 96, 16, 6)
    OFDFT_SPECIALISE_ROW2(float, 80, 20, 128, 16, 5)
    OFDFT_SPECIALISE_ROW2(float, 96, 20, 128, 16, 5)
    OFDFT_SPECIALISE(float, 64, 16, 128, 16, 128, 16, 128)
    OFDFT_SPECIALISE(float, 80, 16, 256, 16, 256, 16, 256)
    OFDFT_SPECIALISE(float, 96, 8, 256, 16, 256, 16, 256)
    return false;
}
template <> bool find_specialised_b<double>(int, int, const void **, const void **, int *, int *) { return false; }

}  // namespace ofdft
