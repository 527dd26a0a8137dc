// Specialised kernels: grid sizes 120 and 192 (FP32).
#include "inst.cuh"

namespace ofdft {

template <typename T> bool find_specialised_c(int role, int n, const void **k1, const void **k2, int *B, int *nt);

template <> bool find_specialised_c<float>(int role, int n, const void **k1, const void **k2, int *B, int *nt) {
    OFDFT_SPECIALISE_ROW2(float, 120, 20, 160, 16, 4)
    OFDFT_SPECIALISE_ROW2(float, 192, 17, 224, 16, 3)
    OFDFT_SPECIALISE(float, 120, 8, 256, 16, 256, 16, 256)
    OFDFT_SPECIALISE(float, 192, 8, 256, 16, 512, 16, 512)
    return false;
}
template <> bool find_specialised_c<double>(int, int, const void **, const void **, int *, int *) { return false; }

}  // namespace ofdft
