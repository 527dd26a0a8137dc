// Specialised kernels: the 128^3 workload (FP32 and FP64) and 32.
#include "inst.cuh"

namespace ofdft {

template <typename T> void candidates_a(int role, int n, std::vector<KernelCand> &out);

template <> void candidates_a<float>(int role, int n, std::vector<KernelCand> &out) {
    // 128: the bench workload's length on every axis; alternatives for the autotuner
    OFDFT_CAND_ROW2(float, 128, 20, 160, 16, 5)
    OFDFT_CAND_ROW2(float, 128, 20, 160, 16, 4)
    OFDFT_CAND_ROW2(float, 128, 19, 152, 16, 5)
    OFDFT_CAND_ROW2(float, 128, 19, 128, 16, 6)
    OFDFT_CAND_ROW2(float, 128, 10, 128, 16, 8)
    OFDFT_CAND_ALL(float, 128, 8, 256, 16, 256, 8, 128)
    OFDFT_CAND_ROW(float, 128, 8, 128, 8, 0)
    OFDFT_CAND_PENCIL(float, 128, 16, 256, 16, 4)
    OFDFT_CAND_PENCIL(float, 128, 16, 128, 16, 8)
    OFDFT_CAND_PENCIL(float, 128, 8, 128, 16, 8)
    OFDFT_CAND_AXIS0(float, 128, 16, 128, 16, 2)
    OFDFT_CAND_AXIS0(float, 128, 8, 128, 16, 5)
    OFDFT_CAND_AXIS0(float, 128, 4, 64, 16, 10)
    OFDFT_CAND_PENCIL(float, 128, 32, 256, 16, 2)
    // 32
    OFDFT_CAND_ROW2(float, 32, 16, 64, 16, 10)
    OFDFT_CAND_ALL(float, 32, 16, 128, 16, 128, 16, 128)
}
template <> void candidates_a<double>(int role, int n, std::vector<KernelCand> &out) {
    OFDFT_CAND_ALL(double, 128, 4, 256, 8, 256, 8, 256)
}

}  // namespace ofdft
