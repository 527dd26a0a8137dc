// Specialised kernels: the 128^3 workload (FP32 and FP64) and 32.
#include "inst.cuh"

namespace ofdft {

template <typename T> bool find_specialised_a(int role, int n, const void **k1, const void **k2, int *B, int *nt);

template <> bool find_specialised_a<float>(int role, int n, const void **k1, const void **k2, int *B, int *nt) {
    OFDFT_SPECIALISE(float, 128, 8, 256, 16, 256, 8, 128)
    OFDFT_SPECIALISE(float, 32, 16, 128, 16, 128, 16, 128)
    return false;
}
template <> bool find_specialised_a<double>(int role, int n, const void **k1, const void **k2, int *B, int *nt) {
    OFDFT_SPECIALISE(double, 128, 4, 256, 8, 256, 8, 256)
    return false;
}

}  // namespace ofdft
