// Specialised kernels: grid size 1024 (FP32), the 1,048,576-atom configuration.
#include "inst.cuh"

namespace ofdft {

template <typename T> bool find_specialised_d(int role, int n, const void **k1, const void **k2, int *B, int *nt);

template <> bool find_specialised_d<float>(int role, int n, const void **k1, const void **k2, int *B, int *nt) {
    // rows: 8 channels per transform (two groups for 15 channels), 512 threads, one block per SM
    OFDFT_SPECIALISE_ROW2(float, 1024, 8, 512, 16, 1)
    OFDFT_SPECIALISE_PENCIL(float, 1024, 8, 512, 1)
    OFDFT_SPECIALISE_AXIS0(float, 1024, 4, 256, 16, 1)
    return false;
}
template <> bool find_specialised_d<double>(int, int, const void **, const void **, int *, int *) { return false; }

}  // namespace ofdft
