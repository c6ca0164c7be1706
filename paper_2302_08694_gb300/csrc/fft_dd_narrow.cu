// Strided transform passes in double-float arithmetic that write FP64 spectra (forward).
#include "fft_kernels.cuh"

namespace fsib {
FSIB_FFT_INST_S(dd, dd, double)
}  // namespace fsib
