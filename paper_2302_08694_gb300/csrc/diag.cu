// Arithmetic-peak microbenchmark used as the denominator of ALU rooflines:
// many independent FMA chains per thread, register resident, no memory traffic.
#include "fsib_internal.cuh"

namespace fsib {

template <typename T>
__global__ void k_fma_peak(T* out, int iters, T b, T c) {
  T a0 = T(threadIdx.x) * T(1e-3), a1 = a0 + T(1), a2 = a0 + T(2), a3 = a0 + T(3);
  T a4 = a0 + T(4), a5 = a0 + T(5), a6 = a0 + T(6), a7 = a0 + T(7);
  for (int i = 0; i < iters; ++i) {
    a0 = a0 * b + c; a1 = a1 * b + c; a2 = a2 * b + c; a3 = a3 * b + c;
    a4 = a4 * b + c; a5 = a5 * b + c; a6 = a6 * b + c; a7 = a7 * b + c;
  }
  const T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == T(-12345.678)) out[0] = s;  // keeps the chains alive
}

template <typename T>
static int measure(int iters, double* gflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FSIB_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return FSIB_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = 8 * sms, threads = 256;
  k_fma_peak<T><<<blocks, threads>>>(out, iters / 8, T(0.9999999), T(1e-7));  // warm-up
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0);
    k_fma_peak<T><<<blocks, threads>>>(out, iters, T(0.9999999), T(1e-7));
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    best = ms < best ? ms : best;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return FSIB_ECUDA;
  *gflops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e9;
  return FSIB_OK;
}

}  // namespace fsib

extern "C" int fsib_measure_peak(int kind, double* gflops) {
  if (!gflops) return FSIB_EINVAL;
  if (kind == 0) return fsib::measure<double>(4096, gflops);
  if (kind == 1) return fsib::measure<float>(65536, gflops);
  return FSIB_EINVAL;
}
