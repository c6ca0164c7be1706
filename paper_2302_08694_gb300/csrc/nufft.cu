// Point side of the NUFFTs (appendix A): bin sort, spreading onto the upsampled
// grid (Eq. type1_conv) and interpolation from it (Eq. type2_conv).
//
// Spreading kernel: "exponential of semicircle", phi(z) = exp(beta (sqrt(1 - z^2) - 1))
// for |z| <= 1, z = 2 (x - X_j)/(w h_f), w cells wide (the kernel of the NUFFT
// library the paper uses; the paper's appendix presents the Kaiser-Bessel member
// of the same family). Its Fourier transform is divided out in the transform passes.
#include "fsib_internal.cuh"

namespace fsib {

constexpr int kSpreadThreads = 256;
constexpr int kMaxW = 16;

struct PointGeom {
  int d, M, nf, w;
  double L;
  int b[3], nb[3];
};

static PointGeom geom(const Plan& p) {
  PointGeom g;
  g.d = p.d; g.M = p.M; g.nf = p.nf; g.w = p.w; g.L = p.L;
  for (int a = 0; a < 3; ++a) { g.b[a] = p.bins[a]; g.nb[a] = p.nbin[a]; }
  return g;
}

// Fine-grid coordinate t in [0, nf) of a coordinate x (periodic wrap of the unwrapped position).
__device__ __forceinline__ double grid_coord(double x, double L, int nf) {
  double xm = x - L * floor(x / L);
  double t = xm * (double)nf / L;
  if (t >= (double)nf) t -= (double)nf;
  if (t < 0.0) t = 0.0;
  return t;
}

// Window start i0 = ceil(t - w/2) of a point; its bin is B = (i0 + floor(w/2)) div b,
// clamped to the last bin. Then i0 - (B b - floor(w/2)) lies in [0, b], so the
// w-wide window of every point of bin B fits the (b + w)-wide tile at B b - floor(w/2).
__device__ __forceinline__ int window_start(double t, int w) { return (int)ceil(t - 0.5 * w); }
__device__ __forceinline__ int bin_of_start(int i0, int w, int b, int nb) {
  return min(max((i0 + w / 2) / b, 0), nb - 1);
}

__global__ void k_bin_count(PointGeom g, const double* __restrict__ X, int* __restrict__ bin_of,
                            int* __restrict__ rank, int* __restrict__ counts) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < g.M; j += gridDim.x * blockDim.x) {
    long long bin = 0, mul = 1;
    for (int a = 0; a < g.d; ++a) {
      const double t = grid_coord(X[(long long)a * g.M + j], g.L, g.nf);
      const int B = bin_of_start(window_start(t, g.w), g.w, g.b[a], g.nb[a]);
      bin += B * mul;
      mul *= g.nb[a];
    }
    bin_of[j] = (int)bin;
    rank[j] = atomicAdd(&counts[bin], 1);
  }
}

// Exclusive scan of the bin counts and list of occupied bins, in one block.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads)
k_bin_scan(const int* __restrict__ counts, long long nbins, int* __restrict__ offsets,
           int* __restrict__ occ, int* __restrict__ nocc) {
  __shared__ long long s_sum[kScanThreads];
  __shared__ int s_cnt[kScanThreads];
  const long long chunk = (nbins + kScanThreads - 1) / kScanThreads;
  const long long lo = threadIdx.x * chunk, hi = min(nbins, lo + chunk);
  long long sum = 0;
  int cnt = 0;
  for (long long i = lo; i < hi; ++i) { const int c = counts[i]; sum += c; cnt += (c > 0); }
  s_sum[threadIdx.x] = sum;
  s_cnt[threadIdx.x] = cnt;
  __syncthreads();
  // Hillis-Steele inclusive scan over the block
  for (int off = 1; off < kScanThreads; off <<= 1) {
    long long vs = 0; int vc = 0;
    if (threadIdx.x >= off) { vs = s_sum[threadIdx.x - off]; vc = s_cnt[threadIdx.x - off]; }
    __syncthreads();
    s_sum[threadIdx.x] += vs; s_cnt[threadIdx.x] += vc;
    __syncthreads();
  }
  long long run = s_sum[threadIdx.x] - sum;
  int runc = s_cnt[threadIdx.x] - cnt;
  for (long long i = lo; i < hi; ++i) {
    const int c = counts[i];
    offsets[i] = (int)run;
    if (c > 0) occ[runc++] = (int)i;
    run += c;
  }
  if (threadIdx.x == kScanThreads - 1) { offsets[nbins] = (int)s_sum[kScanThreads - 1]; *nocc = s_cnt[kScanThreads - 1]; }
}

template <typename T>
__global__ void k_bin_scatter(PointGeom g, const double* __restrict__ X, const int* __restrict__ bin_of,
                              const int* __restrict__ rank, const int* __restrict__ offsets,
                              int* __restrict__ perm, int* __restrict__ i0, T* __restrict__ delta) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < g.M; j += gridDim.x * blockDim.x) {
    const int s = offsets[bin_of[j]] + rank[j];
    perm[s] = j;
    for (int a = 0; a < g.d; ++a) {
      const double t = grid_coord(X[(long long)a * g.M + j], g.L, g.nf);
      const int c0 = window_start(t, g.w);
      i0[(long long)a * g.M + s] = c0;
      delta[(long long)a * g.M + s] = (T)((double)c0 - t);  // in [-w/2, -w/2 + 1)
    }
  }
}

void launch_bin_points(const Plan& p, Workspace& ws, const double* X, cudaStream_t st) {
  const PointGeom g = geom(p);
  cudaMemsetAsync(ws.counts, 0, sizeof(int) * (size_t)p.nbins, st);
  const int nb = (p.M + 255) / 256;
  k_bin_count<<<nb, 256, 0, st>>>(g, X, ws.bin_of, ws.rank, ws.counts);
  k_bin_scan<<<1, kScanThreads, 0, st>>>(ws.counts, p.nbins, ws.offsets, ws.occ, ws.nocc);
  if (p.prec == FSIB_FP64)
    k_bin_scatter<double><<<nb, 256, 0, st>>>(g, X, ws.bin_of, ws.rank, ws.offsets, ws.perm, ws.i0,
                                              (double*)ws.delta);
  else
    k_bin_scatter<float><<<nb, 256, 0, st>>>(g, X, ws.bin_of, ws.rank, ws.offsets, ws.perm, ws.i0,
                                             (float*)ws.delta);
}

// ---------------------------------------------------------------------------
// Kernel weights of one point along one axis, computed by lanes 0..w-1 of a warp.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T es_kernel(T z, T beta) {
  const T s = T(1) - z * z;
  return s > T(0) ? exp(beta * (sqrt(s) - T(1))) : T(0);
}

template <typename T, int D>
__device__ __forceinline__ void point_weights(T* wts /*[D][kMaxW]*/, const T* __restrict__ delta,
                                              long long s, int M, int w, T beta, int lane) {
  if (lane < w) {
    const T two_w = T(2) / T(w);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const T z = two_w * (T(lane) + delta[(long long)a * M + s]);
      wts[a * kMaxW + lane] = es_kernel<T>(z, beta);
    }
  }
  __syncwarp();
}

// Compensated atomic accumulation: the hardware sum s = old + v is rounded, and the
// exact rounding error (Knuth's TwoSum of old and v) goes to a second accumulator.
__device__ __forceinline__ void atomic_add_comp(float* hi, float* lo, float v) {
  const float old = atomicAdd(hi, v);
  const float s = __fadd_rn(old, v);
  const float bb = __fsub_rn(s, old);
  const float e = __fadd_rn(__fsub_rn(old, __fsub_rn(s, bb)), __fsub_rn(v, bb));
  if (e != 0.0f) atomicAdd(lo, e);
}

// ---------------------------------------------------------------------------
// Spread: one block per occupied bin (grid-stride), tile of (b+w)^D cells in
// shared memory, one warp per point, flush with global atomics.
// ---------------------------------------------------------------------------
template <typename T, int D, bool COMP>
__global__ void __launch_bounds__(kSpreadThreads)
k_spread(PointGeom g, T beta, const double* __restrict__ cw, const double* __restrict__ omega,
         const int* __restrict__ perm, const int* __restrict__ offsets, const int* __restrict__ occ,
         const int* __restrict__ nocc, const int* __restrict__ i0s, const T* __restrict__ delta,
         T* __restrict__ grid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = g.w, nf = g.nf, M = g.M;
  const int Tx = g.b[0] + w, Ty = g.b[1] + w, Tz = (D == 3) ? g.b[2] + w : 1;
  const int tcells = Tx * Ty * Tz;
  const int nwarp = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  T* wts_all = reinterpret_cast<T*>(smem_raw);               // [nwarp][D][kMaxW]
  T* tile = wts_all + nwarp * D * kMaxW;                     // [D][tcells]
  float* lo = reinterpret_cast<float*>(tile + D * tcells);   // [D][tcells] when COMP
  T* wts = wts_all + warp * D * kMaxW;
  const long long gcells = (long long)nf * nf * (D == 3 ? nf : 1);
  const int nb_occ = *nocc;
  for (int k = blockIdx.x; k < nb_occ; k += gridDim.x) {
    const int bin = occ[k];
    const int Bx = bin % g.nb[0];
    const int By = (bin / g.nb[0]) % g.nb[1];
    const int Bz = (D == 3) ? bin / (g.nb[0] * g.nb[1]) : 0;
    const int half = w / 2;
    const int ox = Bx * g.b[0] - half, oy = By * g.b[1] - half, oz = (D == 3) ? Bz * g.b[2] - half : 0;
    for (int i = threadIdx.x; i < D * tcells; i += blockDim.x) {
      tile[i] = T(0);
      if (COMP) lo[i] = 0.0f;
    }
    __syncthreads();
    const int s0 = offsets[bin], s1 = offsets[bin + 1];
    for (int s = s0 + warp; s < s1; s += nwarp) {
      const int j = perm[s];
      point_weights<T, D>(wts, delta, s, M, w, beta, lane);
      const double om = omega ? omega[j] : 1.0;
      T cv[D];
#pragma unroll
      for (int a = 0; a < D; ++a) cv[a] = (T)(om * cw[(long long)a * M + j]);
      const int bx = i0s[s] - ox, by = i0s[(long long)M + s] - oy;
      const int bz = (D == 3) ? i0s[2LL * M + s] - oz : 0;
      const int wd = (D == 3) ? w * w * w : w * w;
      for (int idx = lane; idx < wd; idx += 32) {
        const int qx = idx % w, qy = (idx / w) % w, qz = (D == 3) ? idx / (w * w) : 0;
        T wt = wts[qx] * wts[kMaxW + qy];
        if (D == 3) wt *= wts[2 * kMaxW + qz];
        const int cell = ((bz + qz) * Ty + (by + qy)) * Tx + (bx + qx);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          if (COMP) atomic_add_comp((float*)&tile[a * tcells + cell], &lo[a * tcells + cell], (float)(cv[a] * wt));
          else atomicAdd(&tile[a * tcells + cell], cv[a] * wt);
        }
      }
      __syncwarp();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < tcells; i += blockDim.x) {
      const int cx = i % Tx, cy = (i / Tx) % Ty, cz = i / (Tx * Ty);
      int gx = ox + cx, gy = oy + cy, gz = oz + cz;
      gx += (gx < 0) ? nf : 0; gx -= (gx >= nf) ? nf : 0;
      gy += (gy < 0) ? nf : 0; gy -= (gy >= nf) ? nf : 0;
      if (D == 3) { gz += (gz < 0) ? nf : 0; gz -= (gz >= nf) ? nf : 0; }
      const long long gi = ((long long)gz * nf + gy) * nf + gx;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        T v = tile[a * tcells + i];
        if (COMP) v = (T)((float)v + lo[a * tcells + i]);
        if (v != T(0)) atomicAdd(&grid[a * gcells + gi], v);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Interp: one warp per (sorted) point, gather of the w^D window, warp reduction.
// ---------------------------------------------------------------------------
template <typename T, int D>
__global__ void __launch_bounds__(kSpreadThreads)
k_interp(PointGeom g, T beta, const int* __restrict__ perm, const int* __restrict__ i0s,
         const T* __restrict__ delta, const T* __restrict__ grid, double* __restrict__ U) {
  __shared__ T wts_all[(kSpreadThreads / 32) * 3 * kMaxW];
  const int w = g.w, nf = g.nf, M = g.M;
  const int nwarp = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  T* wts = wts_all + warp * D * kMaxW;
  const long long gcells = (long long)nf * nf * (D == 3 ? nf : 1);
  const int wd = (D == 3) ? w * w * w : w * w;
  for (long long s = (long long)blockIdx.x * nwarp + warp; s < M; s += (long long)gridDim.x * nwarp) {
    point_weights<T, D>(wts, delta, s, M, w, beta, lane);
    const int bx = i0s[s], by = i0s[(long long)M + s], bz = (D == 3) ? i0s[2LL * M + s] : 0;
    T acc[D];
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] = T(0);
    for (int idx = lane; idx < wd; idx += 32) {
      const int qx = idx % w, qy = (idx / w) % w, qz = (D == 3) ? idx / (w * w) : 0;
      T wt = wts[qx] * wts[kMaxW + qy];
      if (D == 3) wt *= wts[2 * kMaxW + qz];
      int gx = bx + qx, gy = by + qy, gz = bz + qz;
      gx += (gx < 0) ? nf : 0; gx -= (gx >= nf) ? nf : 0;
      gy += (gy < 0) ? nf : 0; gy -= (gy >= nf) ? nf : 0;
      if (D == 3) { gz += (gz < 0) ? nf : 0; gz -= (gz >= nf) ? nf : 0; }
      const long long gi = ((long long)gz * nf + gy) * nf + gx;
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] += wt * __ldg(&grid[a * gcells + gi]);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      T v = acc[a];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      acc[a] = v;
    }
    if (lane == 0) {
      const int j = perm[s];
#pragma unroll
      for (int a = 0; a < D; ++a) U[(long long)a * M + j] = (double)acc[a];
    }
    __syncwarp();
  }
}

static int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <typename T>
void launch_spread(const Plan& p, Workspace& ws, const double* cw, const double* omega, T* grid,
                   cudaStream_t st) {
  const PointGeom g = geom(p);
  const int D = p.d;
  const int tcells = (g.b[0] + g.w) * (g.b[1] + g.w) * (D == 3 ? g.b[2] + g.w : 1);
  const bool comp = (sizeof(T) == 4);
  const size_t smem = sizeof(T) * (size_t)((kSpreadThreads / 32) * D * kMaxW + D * tcells) +
                      (comp ? sizeof(float) * (size_t)D * tcells : 0);
  const int blocks = 4 * num_sms();
  const T beta = (T)p.beta;
  if (D == 3) {
    auto kern = comp ? k_spread<T, 3, true> : k_spread<T, 3, false>;
    raise_smem_limit(reinterpret_cast<const void*>(kern));
    kern<<<blocks, kSpreadThreads, smem, st>>>(g, beta, cw, omega, ws.perm, ws.offsets, ws.occ, ws.nocc,
                                               ws.i0, (const T*)ws.delta, grid);
  } else {
    auto kern = comp ? k_spread<T, 2, true> : k_spread<T, 2, false>;
    raise_smem_limit(reinterpret_cast<const void*>(kern));
    kern<<<blocks, kSpreadThreads, smem, st>>>(g, beta, cw, omega, ws.perm, ws.offsets, ws.occ, ws.nocc,
                                               ws.i0, (const T*)ws.delta, grid);
  }
}

template <typename T>
void launch_interp(const Plan& p, Workspace& ws, const T* grid, double* U, cudaStream_t st) {
  const PointGeom g = geom(p);
  const int nwarp = kSpreadThreads / 32;
  long long blocks = (p.M + nwarp - 1) / nwarp;
  if (blocks > 16LL * num_sms()) blocks = 16LL * num_sms();
  const T beta = (T)p.beta;
  if (p.d == 3)
    k_interp<T, 3><<<(unsigned)blocks, kSpreadThreads, 0, st>>>(g, beta, ws.perm, ws.i0, (const T*)ws.delta, grid, U);
  else
    k_interp<T, 2><<<(unsigned)blocks, kSpreadThreads, 0, st>>>(g, beta, ws.perm, ws.i0, (const T*)ws.delta, grid, U);
}

template void launch_spread<float>(const Plan&, Workspace&, const double*, const double*, float*, cudaStream_t);
template void launch_spread<double>(const Plan&, Workspace&, const double*, const double*, double*, cudaStream_t);
template void launch_interp<float>(const Plan&, Workspace&, const float*, double*, cudaStream_t);
template void launch_interp<double>(const Plan&, Workspace&, const double*, double*, cudaStream_t);

}  // namespace fsib
