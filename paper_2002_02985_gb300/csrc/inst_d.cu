// Specialised kernels: grid size 1024 (FP32), the 1,048,576-atom configuration.
#include "inst.cuh"

namespace ofdft {

template <typename T> void candidates_d(int role, int n, std::vector<KernelCand> &out);

template <> void candidates_d<float>(int role, int n, std::vector<KernelCand> &out) {
    // rows: 8 channels per transform (two groups for 15 channels), 512 threads, one block per SM
    OFDFT_CAND_ROW2(float, 1024, 8, 512, 16, 1)
    OFDFT_CAND_PENCIL(float, 1024, 8, 512, 16, 1)
    OFDFT_CAND_AXIS0(float, 1024, 4, 256, 16, 1)
    // alternatives for the autotuner: 4-channel rows at two blocks per SM, 512 threads per
    // column tile (measured picks at 1024^3; 4-column pencils at two blocks per SM and 2-column
    // tiles were slower and are not compiled)
    OFDFT_CAND_ROW2(float, 1024, 4, 256, 16, 2)
    OFDFT_CAND_AXIS0(float, 1024, 4, 512, 16, 1)
}
template <> void candidates_d<double>(int, int, std::vector<KernelCand> &) {}

}  // namespace ofdft
