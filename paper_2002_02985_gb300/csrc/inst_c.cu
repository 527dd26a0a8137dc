// Specialised kernels: grid sizes 120 and 192 (FP32).
#include "inst.cuh"

namespace ofdft {

template <typename T> void candidates_c(int role, int n, std::vector<KernelCand> &out);

template <> void candidates_c<float>(int role, int n, std::vector<KernelCand> &out) {
    OFDFT_CAND_ROW2(float, 120, 20, 160, 16, 4)
    OFDFT_CAND_ROW2(float, 192, 17, 224, 16, 3)
    OFDFT_CAND_ALL(float, 120, 8, 256, 16, 256, 16, 256)
    OFDFT_CAND_ALL(float, 192, 8, 256, 16, 512, 16, 512)
    // alternatives for the autotuner
    OFDFT_CAND_ROW2(float, 120, 19, 152, 16, 5)
    OFDFT_CAND_ROW2(float, 120, 10, 128, 16, 8)
    OFDFT_CAND_PENCIL(float, 120, 16, 128, 16, 8)
    OFDFT_CAND_AXIS0(float, 120, 8, 128, 16, 5)
    OFDFT_CAND_AXIS0(float, 120, 16, 128, 16, 2)
    OFDFT_CAND_ROW2(float, 192, 11, 144, 16, 4)
    OFDFT_CAND_PENCIL(float, 192, 16, 256, 16, 2)
    OFDFT_CAND_AXIS0(float, 192, 8, 256, 16, 2)
    OFDFT_CAND_AXIS0(float, 192, 16, 256, 16, 1)
}
template <> void candidates_c<double>(int, int, std::vector<KernelCand> &) {}

}  // namespace ofdft
