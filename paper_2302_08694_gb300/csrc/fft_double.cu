// Transform passes in native FP64 arithmetic (the native_fp64 option).
#include "fft_kernels.cuh"

namespace fsib {
FSIB_FFT_INST(double)
FSIB_FFT_INST_S(double, double, double)
}  // namespace fsib
