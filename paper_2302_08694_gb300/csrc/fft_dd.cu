// Row transform passes in double-float arithmetic (FP64 mode).
#include "fft_kernels.cuh"

namespace fsib {
FSIB_FFT_INST_R(dd)
}  // namespace fsib
