// Specialised kernels: grid sizes 64, 80 and 96 (FP32).
#include "inst.cuh"

namespace ofdft {

template <typename T> void candidates_b(int role, int n, std::vector<KernelCand> &out);

template <> void candidates_b<float>(int role, int n, std::vector<KernelCand> &out) {
    OFDFT_CAND_ROW2(float, 64, 20, 96, 16, 6)
    OFDFT_CAND_ROW2(float, 80, 20, 128, 16, 5)
    OFDFT_CAND_ROW2(float, 96, 20, 128, 16, 5)
    OFDFT_CAND_ALL(float, 64, 16, 128, 16, 128, 16, 128)
    OFDFT_CAND_ALL(float, 80, 16, 256, 16, 256, 16, 256)
    OFDFT_CAND_ALL(float, 96, 8, 256, 16, 256, 16, 256)
    // alternatives for the autotuner
    OFDFT_CAND_PENCIL(float, 80, 16, 128, 16, 8)
    OFDFT_CAND_AXIS0(float, 80, 8, 128, 16, 5)
    OFDFT_CAND_ROW2(float, 96, 10, 128, 16, 6)
    OFDFT_CAND_PENCIL(float, 96, 16, 128, 16, 8)
    OFDFT_CAND_AXIS0(float, 96, 8, 128, 16, 5)
    OFDFT_CAND_AXIS0(float, 64, 8, 128, 16, 5)
}
template <> void candidates_b<double>(int, int, std::vector<KernelCand> &) {}

}  // namespace ofdft
