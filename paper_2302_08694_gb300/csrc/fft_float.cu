// Transform passes in FP32 (mixed precision).
#include "fft_kernels.cuh"

namespace fsib {
FSIB_FFT_INST(float)
FSIB_FFT_INST_S(float, float, float)
}  // namespace fsib
