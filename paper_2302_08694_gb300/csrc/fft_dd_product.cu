// Fused dealiased-product row pass in double-float arithmetic (FP64 mode).
#include "fft_kernels.cuh"

namespace fsib {
FSIB_FFT_INST_P(dd)
}  // namespace fsib
