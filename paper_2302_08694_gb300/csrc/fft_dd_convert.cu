// Strided transform passes in double-float arithmetic that read FP64 spectra (inverse).
#include "fft_kernels.cuh"

namespace fsib {
FSIB_FFT_INST_S(dd, double, dd)
}  // namespace fsib
