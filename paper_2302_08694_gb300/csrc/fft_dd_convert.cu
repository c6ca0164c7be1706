// Strided transform passes in double-float arithmetic that read or write FP64 spectra.
#include "fft_kernels.cuh"

namespace fsib {
FSIB_FFT_INST_S(dd, double, dd)
FSIB_FFT_INST_S(dd, dd, double)
}  // namespace fsib
