// Point side of the NUFFTs (appendix A): bin sort, spreading onto the upsampled
// grid (Eq. type1_conv) and interpolation from it (Eq. type2_conv).
//
// Spreading kernel: "exponential of semicircle", phi(z) = exp(beta (sqrt(1 - z^2) - 1))
// for |z| <= 1, z = 2 (x - X_j)/(w h_f), w cells wide (the kernel of the NUFFT
// library the paper uses; the paper's appendix presents the Kaiser-Bessel member
// of the same family). Its Fourier transform is divided out in the transform passes.
#include <algorithm>
#include <type_traits>

#include "fsib_internal.cuh"

namespace fsib {

constexpr int kSpreadThreads = 256;
constexpr int kMaxW = 16;

struct PointGeom {
  int d, M, nf, w;
  double L, invL, scale;  // scale = nf / L (reciprocals: FP64 division is slow on this GPU)
  int b[3], nb[3];
  int slice;  // candidates per slice of a 3D gather box
  const unsigned char* band;  // row bands reached by a window (RowBands), or nullptr
};

static PointGeom geom(const Plan& p) {
  PointGeom g;
  g.d = p.d; g.M = p.M; g.nf = p.nf; g.w = p.w; g.L = p.L;
  g.invL = 1.0 / p.L; g.scale = (double)p.nf / p.L;
  for (int a = 0; a < 3; ++a) { g.b[a] = p.bins[a]; g.nb[a] = p.nbin[a]; }
  g.slice = p.slice;
  g.band = nullptr;
  return g;
}

// Fine-grid coordinate t in [0, nf) of a coordinate x (periodic wrap of the unwrapped position).
__device__ __forceinline__ double grid_coord(double x, const PointGeom& g) {
  const double xm = fma(-g.L, floor(x * g.invL), x);
  double t = xm * g.scale;
  if (t >= (double)g.nf) t -= (double)g.nf;
  if (!(t >= 0.0 && t < (double)g.nf)) t = 0.0;  // rounding just below 0, or a non-finite position
  return t;
}

// Window start i0 = ceil(t - w/2) of a point (i0 >= -w/2, so it may be negative); its bin
// is B = (i0 mod nf) div b. Then (i0 - B b) mod nf lies in [0, b), so the w-wide window of
// every point of bin B fits the (b + w - 1)-wide tile at B b, and the windows that meet the
// box [B b, B b + b) start in bins B - ceil((w - 1)/b) .. B: two bins per axis when w <= b + 1.
__device__ __forceinline__ int window_start(double t, int w) { return (int)ceil(t - 0.5 * w); }
__device__ __forceinline__ int bin_of_start(int i0, int nf, int b, int nb) {
  const int r = (i0 < 0) ? i0 + nf : (i0 >= nf ? i0 - nf : i0);
  return min(r / b, nb - 1);
}

// Bin of every point and its rank within the bin. Lanes of a warp that fall in the same
// bin (neighbouring points usually do) share one atomic increment.
struct KBinCount {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(PointGeom g, const double* __restrict__ X, int* __restrict__ bin_of,
                            int* __restrict__ rank, int* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  for (long long j0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; j0 < g.M;
       j0 += (long long)gridDim.x * blockDim.x) {
    const long long j = j0 + lane;
    const bool ok = j < g.M;
    int bin = -1;
    if (ok) {
      long long b = 0, mul = 1;
      for (int a = 0; a < g.d; ++a) {
        const double t = grid_coord(X[(long long)a * g.M + j], g);
        const int B = bin_of_start(window_start(t, g.w), g.nf, g.b[a], g.nb[a]);
        b += B * mul;
        mul *= g.nb[a];
      }
      bin = (int)b;
    }
    const unsigned same = __match_any_sync(0xffffffffu, bin);
    const int leader = __ffs(same) - 1;
    int base = 0;
    if (ok && lane == leader) base = atomicAdd(&counts[bin], __popc(same));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (ok) {
      bin_of[j] = bin;
      rank[j] = base + __popc(same & ((1u << lane) - 1u));
    }
  }
}
};

// Single-block exclusive scans. A tile is kScanThreads x kScanPer consecutive entries;
// each thread owns kScanPer of them (eight 16-byte loads when the tile is full), scans
// them in registers, and the block combines the thread totals with warp shuffles and one
// pair of barriers per tile; a running carry links the tiles.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 32;

template <int PER>
__device__ __forceinline__ void scan_load(const int* __restrict__ p, long long i0, long long n, int (&c)[PER]) {
  if (i0 + PER <= n) {
    const int4* q = reinterpret_cast<const int4*>(p + i0);
#pragma unroll
    for (int k = 0; k < PER / 4; ++k) {
      const int4 v = q[k];
      c[4 * k] = v.x; c[4 * k + 1] = v.y; c[4 * k + 2] = v.z; c[4 * k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < PER; ++k) c[k] = (i0 + k < n) ? p[i0 + k] : 0;
  }
}

template <int PER>
__device__ __forceinline__ void scan_store(int* __restrict__ p, long long i0, long long n, const int (&c)[PER]) {
  if (i0 + PER <= n) {
    int4* q = reinterpret_cast<int4*>(p + i0);
#pragma unroll
    for (int k = 0; k < PER / 4; ++k) q[k] = make_int4(c[4 * k], c[4 * k + 1], c[4 * k + 2], c[4 * k + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < PER; ++k)
      if (i0 + k < n) p[i0 + k] = c[k];
  }
}

// Block-wide exclusive prefix of NV per-thread totals (in place); tot receives the block totals.
template <int NV>
__device__ __forceinline__ void block_prefix(int (&v)[NV], int (&tot)[NV], int (*wsum)[32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    incl[q] = v[q];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl[q], off);
      if (lane >= off) incl[q] += t;
    }
    if (lane == 31) wsum[q][warp] = incl[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      int x = wsum[q][lane];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += t;
      }
      wsum[q][lane] = x;  // inclusive over warps
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    v[q] = (warp ? wsum[q][warp - 1] : 0) + incl[q] - v[q];
    tot[q] = wsum[q][31];
  }
  __syncthreads();  // wsum is reused by the next tile
}

// Bin offsets (exclusive scan of the counts, total at [nbins]) and the list of occupied bins.
// OCC: also list the occupied bins (the scatter spread walks them; the gather does not).
// It also clears the row-band flags (nband bytes) that the scatter then marks, and, without
// them, leaves the counts at zero for the next binning (no memset node in the step graph).
template <bool OCC>
struct KBinScan {
  static constexpr int kThreads = kScanThreads, kMinBlocks = 0;
  static constexpr bool kAnyGrid = false;
  __device__ static void run(int* __restrict__ counts, long long nbins, int* __restrict__ offsets,
           int* __restrict__ occ, int* __restrict__ nocc, unsigned char* __restrict__ band,
           unsigned char* __restrict__ band_dil, int nband) {
  constexpr int NV = OCC ? 2 : 1;
  __shared__ int wsum[NV][32];
  int carry = 0, carry_o = 0;
  if (band)
    for (int i = threadIdx.x; i < nband; i += blockDim.x) band[i] = 0;
  if (band_dil)
    for (int i = threadIdx.x; i < nband; i += blockDim.x) band_dil[i] = 0;
  for (long long base = 0; base < nbins; base += (long long)kScanThreads * kScanPer) {
    const long long i0 = base + (long long)threadIdx.x * kScanPer;
    int c[kScanPer];
    scan_load(counts, i0, nbins, c);
    if (!band) {  // with row bands, the scatter clears the counts of the occupied bins
      int z[kScanPer];
#pragma unroll
      for (int k = 0; k < kScanPer; ++k) z[k] = 0;
      scan_store(counts, i0, nbins, z);
    }
    int v[NV], tot[NV];
    v[0] = 0;
    if constexpr (OCC) v[1] = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      v[0] += c[k];
      if constexpr (OCC) v[1] += (c[k] > 0);
    }
    block_prefix<NV>(v, tot, wsum);
    int run = carry + v[0], runo = 0;
    if constexpr (OCC) runo = carry_o + v[1];
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      if constexpr (OCC) { if (c[k] > 0) occ[runo++] = (int)(i0 + k); }
      const int t = c[k];
      c[k] = run;
      run += t;
    }
    scan_store(offsets, i0, nbins, c);
    carry += tot[0];
    if constexpr (OCC) carry_o += tot[1];
  }
  if (threadIdx.x == 0) { offsets[nbins] = carry; if (OCC) *nocc = carry_o; }
}
};

// Exclusive scans of two int arrays of length n, one per block (blockIdx.x = 0: a, 1: b);
// out arrays hold n + 1 entries.
struct KScan2 {
  static constexpr int kThreads = kScanThreads, kMinBlocks = 0;
  static constexpr bool kAnyGrid = false;
  __device__ static void run(const int* __restrict__ a, const int* __restrict__ b, int n, int* __restrict__ oa, int* __restrict__ ob) {
  __shared__ int wsum[1][32];
  const int* in = blockIdx.x ? b : a;
  int* out = blockIdx.x ? ob : oa;
  int carry = 0;
  for (long long base = 0; base < n; base += (long long)kScanThreads * kScanPer) {
    const long long i0 = base + (long long)threadIdx.x * kScanPer;
    int x[kScanPer];
    scan_load(in, i0, n, x);
    int v[1] = {0}, tot[1];
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) v[0] += x[k];
    block_prefix<1>(v, tot, wsum);
    int r = carry + v[0];
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      const int t = x[k];
      x[k] = r;
      r += t;
    }
    scan_store(out, i0, n, x);
    carry += tot[0];
  }
  if (threadIdx.x == 0) out[n] = carry;
}
};

// Row bands (boxes along y and z) that the windows of an occupied bin reach: windows starting in
// bin B cover cells [B b, B b + b + w - 1), boxes B .. B + reach per axis; band_dil one box more
// each way (the bands still hold the windows after a move of under a box). The scan has cleared
// the flags; the stores are unconditional (one lane of a warp marks its bin: a read before each
// store would wait on memory 34 times in a row).
__device__ __forceinline__ void band_mark(const PointGeom& g, int bin, unsigned char* __restrict__ band,
                                          unsigned char* __restrict__ band_dil, int reach) {
  const int nby = g.nb[1], nbz = (g.d == 3) ? g.nb[2] : 1;
  const int rz = (g.d == 3) ? reach : 0, z0 = (g.d == 3) ? -1 : 0;
  const int by = (bin / g.nb[0]) % nby, bz = bin / (g.nb[0] * nby);
  for (int dz = 0; dz <= rz; ++dz)
    for (int dy = 0; dy <= reach; ++dy) {
      band[((bz + dz) % nbz) * nby + (by + dy) % nby] = 1;
    }
  if (band_dil)
    for (int dz = z0; dz <= rz - z0; ++dz)
      for (int dy = -1; dy <= reach + 1; ++dy) {
        band_dil[((bz + dz + nbz) % nbz) * nby + (by + dy + nby) % nby] = 1;
      }
}

template <typename T>
struct KBinScatter {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  // With row bands (band != nullptr): the first point of each occupied bin (rank 0) also marks
  // the bands its bin's windows reach (band_mark) and returns the bin's count to zero for the
  // next binning (empty bins were never counted).
  __device__ static void run(PointGeom g, const double* __restrict__ X, const int* __restrict__ bin_of,
                              const int* __restrict__ rank, const int* __restrict__ offsets,
                              int* __restrict__ perm, int* __restrict__ i0, T* __restrict__ delta,
                              int* __restrict__ counts, unsigned char* __restrict__ band,
                              unsigned char* __restrict__ band_dil, int reach) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < g.M; j += gridDim.x * blockDim.x) {
    const int bin = bin_of[j], rk = rank[j];
    const int s = offsets[bin] + rk;
    perm[s] = j;
    if (band && rk == 0) {
      counts[bin] = 0;
      band_mark(g, bin, band, band_dil, reach);
    }
    for (int a = 0; a < g.d; ++a) {
      const double t = grid_coord(X[(long long)a * g.M + j], g);
      const int c0 = window_start(t, g.w);
      i0[(long long)a * g.M + s] = c0;
      delta[(long long)a * g.M + s] = (T)((double)c0 - t);  // in [-w/2, -w/2 + 1)
    }
  }
}
};

static int num_sms();

// The whole binning of a small problem in one block (one launch instead of four): bins and
// ranks with shared-memory atomics, the exclusive scan of the bin counts in shared memory, the
// row bands and the scatter. Used when the points are few (the positions' FP64 grid
// coordinates, computed twice per point, run on one SM) and the bins fit in shared memory.
constexpr int kSmallBins = 8192;
constexpr int kSmallM = 2048;

template <typename T>
struct KBinSmall {
  static constexpr int kThreads = 1024, kMinBlocks = 0;
  static constexpr bool kAnyGrid = false;
  __device__ static void run(PointGeom g, const double* __restrict__ X, int* __restrict__ bin_of, int* __restrict__ rank,
            int* __restrict__ offsets, int* __restrict__ perm, int* __restrict__ i0, T* __restrict__ delta,
            unsigned char* __restrict__ band, unsigned char* __restrict__ band_dil, int nband, int reach) {
  __shared__ int sc[kSmallBins];
  __shared__ int wsum[1][32];
  const int nbins = g.nb[0] * g.nb[1] * (g.d == 3 ? g.nb[2] : 1);
  const int M = g.M;
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) sc[i] = 0;
  for (int i = threadIdx.x; band && i < nband; i += blockDim.x) band[i] = 0;
  for (int i = threadIdx.x; band_dil && i < nband; i += blockDim.x) band_dil[i] = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    int b = 0, mul = 1;
    for (int a = 0; a < g.d; ++a) {
      const double t = grid_coord(X[(long long)a * M + j], g);
      b += bin_of_start(window_start(t, g.w), g.nf, g.b[a], g.nb[a]) * mul;
      mul *= g.nb[a];
    }
    bin_of[j] = b;
    rank[j] = atomicAdd(&sc[b], 1);
  }
  __syncthreads();
  // exclusive scan: thread t owns the bins [t per, (t + 1) per)
  const int per = (nbins + (int)blockDim.x - 1) / (int)blockDim.x;
  const int b0 = threadIdx.x * per;
  int loc = 0;
  for (int k = 0; k < per; ++k)
    if (b0 + k < nbins) loc += sc[b0 + k];
  int v[1] = {loc}, tot[1];
  block_prefix<1>(v, tot, wsum);
  int run = v[0];
  const int nby = g.nb[1], nbz = (g.d == 3) ? g.nb[2] : 1;
  const int rz = (g.d == 3) ? reach : 0, z0 = (g.d == 3) ? -1 : 0;
  for (int k = 0; k < per; ++k) {
    const int bin = b0 + k;
    if (bin >= nbins) break;
    const int c = sc[bin];
    sc[bin] = run;
    offsets[bin] = run;
    run += c;
    if (c > 0 && band) {  // row bands of this bin's windows (see band_mark)
      const int by = (bin / g.nb[0]) % nby, bz = bin / (g.nb[0] * nby);
      for (int dz = 0; dz <= rz; ++dz)
        for (int dy = 0; dy <= reach; ++dy) band[((bz + dz) % nbz) * nby + (by + dy) % nby] = 1;
      if (band_dil)
        for (int dz = z0; dz <= rz - z0; ++dz)
          for (int dy = -1; dy <= reach + 1; ++dy) band_dil[((bz + dz + nbz) % nbz) * nby + (by + dy + nby) % nby] = 1;
    }
  }
  if (threadIdx.x == 0) offsets[nbins] = tot[0];
  __syncthreads();
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const int s = sc[bin_of[j]] + rank[j];
    perm[s] = j;
    for (int a = 0; a < g.d; ++a) {
      const double t = grid_coord(X[(long long)a * M + j], g);
      const int c0 = window_start(t, g.w);
      i0[(long long)a * M + s] = c0;
      delta[(long long)a * M + s] = (T)((double)c0 - t);
    }
  }
}
};

void launch_bin_points(const Plan& p, Workspace& ws, const double* X, cudaStream_t st, bool occupied,
                       bool dilate) {
  const PointGeom g = geom(p);
  // counts are zero here: the workspace starts zeroed and every scan clears them after use
  const int nb = (p.M + 255) / 256;
  unsigned char* band = occupied ? nullptr : ws.band;  // row bands for the gather path
  unsigned char* band_dil = (occupied || !dilate) ? nullptr : ws.band_dil;
  const int nband = p.nbin[1] * (p.d == 3 ? p.nbin[2] : 1);
  const int reach = (p.bins[1] + p.w - 2) / p.bins[1];
  if (!occupied && p.M <= kSmallM && p.nbins <= kSmallBins) {  // gather path, small problem
    if (p.prec == FSIB_FP64)
      launch<KBinSmall<double>>(1, 1024, 0, st, g, X, ws.bin_of, ws.rank, ws.offsets, ws.perm, ws.i0,
                                             (double*)ws.delta, band, band_dil, nband, reach);
    else
      launch<KBinSmall<float>>(1, 1024, 0, st, g, X, ws.bin_of, ws.rank, ws.offsets, ws.perm, ws.i0,
                                            (float*)ws.delta, band, band_dil, nband, reach);
    return;
  }
  launch<KBinCount>(nb, 256, 0, st, g, X, ws.bin_of, ws.rank, ws.counts);
  if (occupied) launch<KBinScan<true>>(1, kScanThreads, 0, st, ws.counts, p.nbins, ws.offsets, ws.occ, ws.nocc, band, band_dil, nband);
  else launch<KBinScan<false>>(1, kScanThreads, 0, st, ws.counts, p.nbins, ws.offsets, ws.occ, ws.nocc, band, band_dil, nband);
  if (p.prec == FSIB_FP64)
    launch<KBinScatter<double>>(nb, 256, 0, st, g, X, ws.bin_of, ws.rank, ws.offsets, ws.perm, ws.i0,
                                (double*)ws.delta, ws.counts, band, band_dil, reach);
  else
    launch<KBinScatter<float>>(nb, 256, 0, st, g, X, ws.bin_of, ws.rank, ws.offsets, ws.perm, ws.i0,
                               (float*)ws.delta, ws.counts, band, band_dil, reach);
}

// ---------------------------------------------------------------------------
// Kernel weights of one point along one axis, computed by lanes 0..w-1 of a warp.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T es_kernel(T z, T beta) {
  const T s = T(1) - z * z;
  return s > T(0) ? exp(beta * (sqrt(s) - T(1))) : T(0);
}

__device__ __forceinline__ float warp_sum(float v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ dd warp_sum(dd v) {
  for (int off = 16; off > 0; off >>= 1)
    v = v + dd(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
  return v;
}
__device__ __forceinline__ double to_double_val(float v) { return (double)v; }
__device__ __forceinline__ double to_double_val(dd v) { return dd_to_double(v); }

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
struct KSpreadScatter {
  static constexpr int kThreads = kSpreadThreads, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(PointGeom g, T beta, const double* __restrict__ cw, const double* __restrict__ omega,
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
    const int ox = Bx * g.b[0], oy = By * g.b[1], oz = (D == 3) ? Bz * g.b[2] : 0;
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
      int bx = i0s[s] - ox, by = i0s[(long long)M + s] - oy;  // in [0, b) after the periodic wrap
      int bz = (D == 3) ? i0s[2LL * M + s] - oz : 0;
      bx += (bx < 0) ? nf : 0; by += (by < 0) ? nf : 0; bz += (bz < 0) ? nf : 0;
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
};

// ---------------------------------------------------------------------------
// Interp: one warp per (sorted) point, gather of the w^D window, warp reduction.
// ---------------------------------------------------------------------------
template <typename T, int D>
struct KInterp {
  static constexpr int kThreads = kSpreadThreads, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(PointGeom g, T beta, const int* __restrict__ perm, const int* __restrict__ i0s,
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
};

// ---------------------------------------------------------------------------
// Kernel weights in the transform arithmetic: float evaluates phi in FP32, dd
// evaluates it in FP64 and splits the value into a double-float pair.
// ---------------------------------------------------------------------------
template <typename T> struct DeltaT;
template <> struct DeltaT<float> { using type = float; };
template <> struct DeltaT<dd> { using type = double; };

__device__ __forceinline__ float es_weight(float z, double beta) { return es_kernel<float>(z, (float)beta); }

// s2w = 2/w and bdd = beta as double-float constants (used by the double-float version).
template <typename T>
__device__ __forceinline__ T weight_of(typename DeltaT<T>::type delta, int q, int w, double beta, dd s2w, dd bdd);
template <>
__device__ __forceinline__ float weight_of<float>(float delta, int q, int w, double beta, dd, dd) {
  const float z = (2.0f / (float)w) * ((float)q + delta);
  return es_kernel<float>(z, (float)beta);
}
template <>
__device__ __forceinline__ dd weight_of<dd>(double delta, int q, int, double, dd s2w, dd bdd) {
  // phi(z) = exp(beta (sqrt(1 - z^2) - 1)), z = (2/w)(q + delta), in double-float on the FP32
  // pipes (the FP64 pipe of this GPU is the slow one): delta split into a pair, q added to it.
  const dd z = (dd((float)q) + dd_from_double(delta)) * s2w;
  const dd s = dd(1.0f) - z * z;
  if (!(s.hi > 0.0f)) return dd(0.0f);
  return dd_exp_nonpos((dd_sqrt(s) - dd(1.0f)) * bdd);
}


// ---------------------------------------------------------------------------
// Transform modes float / dd, gather formulation.
//
// k_point_prep: for every sorted point s, the kernel weights W[s][a][q] =
//   phi(2 (i0_a + q - t_a)/w) (in double-float on the FP32 pipes for dd, in float for float) and, for
//   a spread, the weighted force C[s][a] = omega_j c_a,j.
// k_spread_gather: one block per output box of bx * by (* bz) grid cells. Every point
//   whose window meets the box lies in one of the neighbouring bins, so the block
//   walks those bins' point ranges, stages the candidates in shared memory, and each
//   thread adds the contributions to its own run of 8 cells of one component in
//   registers. Each grid cell is written once, by plain stores (no atomics, no
//   separate zero fill); boxes with no candidate write zeros.
// k_interp_warp: one warp per point; the warp first tabulates the window's rows (their
//   grid offsets and weight products w_y w_z) in shared memory, then lane = qx + w k reads
//   row segments of the window (coalesced along x), four rows at a time, accumulates
//   g * (w_y w_z), and finally multiplies by w_x.
// ---------------------------------------------------------------------------
constexpr int kSeg = 8;  // cells per thread run along x in the gather

template <typename T, int D>
struct KPointPrep {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(PointGeom g, double beta, const typename DeltaT<T>::type* __restrict__ delta,
                             const int* __restrict__ perm, const double* __restrict__ cw,
                             const double* __restrict__ omega, T* __restrict__ W, T* __restrict__ Cw, dd s2w, dd bdd) {
  const int w = g.w, M = g.M;
  const long long nw = (long long)M * D * w;
  auto entry = [&](long long s, int r) {
    const int a = r / w, q = r - a * w;
    W[s * D * w + r] = weight_of<T>(delta[(long long)a * M + s], q, w, beta, s2w, bdd);
    if (Cw && q == 0) {
      const int j = perm[s];
      const double om = omega ? omega[j] : 1.0;
      const double c = om * cw[(long long)a * M + j];
      if constexpr (std::is_same<T, dd>::value) Cw[s * D + a] = dd_from_double(c);
      else Cw[s * D + a] = T(c);
    }
  };
  if (nw < (1LL << 31)) {  // 32-bit index arithmetic (the usual case)
    const unsigned per = (unsigned)(D * w);
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < (unsigned)nw; t += gridDim.x * blockDim.x) {
      const unsigned s = t / per;
      entry((long long)s, (int)(t - s * per));
    }
  } else {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nw; t += (long long)gridDim.x * blockDim.x) {
      const long long s = t / (D * w);
      entry(s, (int)(t - s * (D * w)));
    }
  }
}
};

__device__ __forceinline__ void fma_acc(float& acc, float a, float b) { acc = __fmaf_rn(a, b, acc); }
__device__ __forceinline__ void fma_acc(dd& acc, dd a, dd b) { dd_fma_acc(acc, a, b); }
__device__ __forceinline__ float acc_norm(float a) { return a; }
__device__ __forceinline__ dd acc_norm(dd a) { return dd_norm(a); }

// Compensated FP32 sum (Kahan's compensation in Neumaier's form, with Knuth's TwoSum so that no
// ordering of magnitudes is assumed): s is the rounded running sum, c the sum of the exact
// rounding errors of the additions; the sum is s + c. The error of a compensated sum of n terms is
// about 2u sum|x_i| + O(n u^2) sum|x_i| instead of the (n - 1) u sum|x_i| of recursive summation.
struct cf {
  float s, c;
  __host__ __device__ constexpr cf(float v = 0.0f) : s(v), c(0.0f) {}
};
__device__ __forceinline__ void add_comp(cf& a, float x) {
  float s, e;
  two_sum(a.s, x, s, e);
  a.s = s;
  a.c = __fadd_rn(a.c, e);
}
__device__ __forceinline__ void fma_acc(cf& acc, float a, float b) { add_comp(acc, __fmul_rn(a, b)); }
__device__ __forceinline__ float acc_norm(cf a) { return __fadd_rn(a.s, a.c); }

// Summation of the FP32 gather spreads (option "spread_sum"): kSumPlain adds every term with an
// FMA; kSumTerm adds every term into a compensated sum; kSumChunk adds the terms of one staged
// chunk of candidates with FMAs and the chunk's partial sum into a compensated sum. Double-float
// accumulators are compensated by construction and ignore the option.
constexpr int kSumPlain = 0, kSumTerm = 1, kSumChunk = 2;
template <typename T, int COMP> struct SumAcc { using type = T; };
template <> struct SumAcc<float, kSumTerm> { using type = cf; };

constexpr int kGatherChunk = 128;  // candidates staged per round (2D gather)
constexpr int kGatherSliceMin = 256;  // fewest candidates a block takes when blocks share a 2D box

// Loads that bypass L1 (other blocks wrote the data during this kernel).
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ dd ld_cg(const dd* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return dd(v.x, v.y);
}


// Neighbouring bins whose window starts can reach box (Bx, By, Bz) (defined below).
__device__ __forceinline__ int nb_list(const PointGeom& g, int dlo, int dhi, int Bx, int By, int Bz, int lane,
                                       int* bin);

template <typename T, int D, int COMP>
struct KSpreadGather {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = false;
  __device__ static void run(PointGeom g, int dlo, int dhi, const int* __restrict__ offsets, const int* __restrict__ i0s,
                             const T* __restrict__ W, const T* __restrict__ Cw, T* __restrict__ grid, int KS,
                             T* __restrict__ partials, int* __restrict__ done) {
  // KS > 1: blocks ks = 0 .. KS - 1 of each box (block index box + ks * nbox) share its candidates
  // when there are enough of them (kGatherSliceMin a block), store partial boxes, and the block
  // that finishes the box's last slice adds them in slice order (done: a counter per box, back
  // to zero when the box is stored).
  __shared__ __align__(16) T sW[kGatherChunk * D * kMaxW];
  __shared__ T sC[kGatherChunk * D];
  __shared__ int sI[kGatherChunk * 3];
  const int w = g.w, nf = g.nf, M = g.M;
  const int bxs = g.b[0], bys = g.b[1], bzs = (D == 3) ? g.b[2] : 1;
  const int nseg = bxs / kSeg;
  const int nbox = g.nb[0] * g.nb[1] * (D == 3 ? g.nb[2] : 1);
  const int box = blockIdx.x % nbox, ks = blockIdx.x / nbox;
  const int Bx = box % g.nb[0], By = (box / g.nb[0]) % g.nb[1], Bz = (D == 3) ? box / (g.nb[0] * g.nb[1]) : 0;
  if (g.band && !g.band[Bz * g.nb[1] + By]) return;  // a row band that no window reaches: never read
  const int ox = Bx * bxs, oy = By * bys, oz = Bz * bzs;
  // task: (component, z, y, segment) -> a run of kSeg cells along x. The block holds G = blockDim
  // / ntask groups of ntask threads; group q takes candidates q, q + G, ... of every staged chunk,
  // and the groups' partial sums are added at the end (dense boxes hold thousands of candidates).
  const int ntask = D * bzs * bys * nseg;
  const int G = blockDim.x / ntask;
  const int task = threadIdx.x % ntask, group = threadIdx.x / ntask;
  const int seg = task % nseg, ty = (task / nseg) % bys, tz = (task / (nseg * bys)) % bzs;
  const int comp = task / (nseg * bys * bzs);
  const int cx0 = ox + seg * kSeg, cy = oy + ty, cz = oz + tz;
  using A = typename SumAcc<T, COMP>::type;
  A acc[kSeg];
  cf tot[kSeg];  // kSumChunk: compensated sums of the chunks' partial sums
#pragma unroll
  for (int i = 0; i < kSeg; ++i) { acc[i] = A(0); tot[i] = cf(0.0f); }
  const long long gcells = (long long)nf * nf * (D == 3 ? nf : 1);
  // candidates: the points of the neighbouring bins (B + dlo .. B + dhi per axis, mod nb), as
  // one list of ranges (first point, prefix of lengths) built by warp 0, staged kGatherChunk at a time
  __shared__ int sStart[32], sPre[33], sSp[kGatherChunk];
  __shared__ int sNr;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int bin = 0;
    const int nnb = nb_list(g, dlo, dhi, Bx, By, Bz, lane, &bin);
    int p0 = 0, len = 0;
    if (lane < nnb) { p0 = offsets[bin]; len = offsets[bin + 1] - p0; }
    int incl = len;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += t;
    }
    const unsigned nonempty = __ballot_sync(0xffffffffu, len > 0);
    if (len > 0) {
      const int slot = __popc(nonempty & ((1u << lane) - 1u));
      sStart[slot] = p0;
      sPre[slot] = incl - len;
    }
    if (lane == 31) { sNr = __popc(nonempty); sPre[__popc(nonempty)] = incl; }
  }
  __syncthreads();
  const int nr = sNr, total = sPre[nr];
  const int slices = (KS > 1) ? min(KS, max(1, (total + kGatherSliceMin - 1) / kGatherSliceMin)) : 1;
  if (ks >= slices) return;  // uniform across the block
  const int fb = (int)((long long)total * ks / slices), fe = (int)((long long)total * (ks + 1) / slices);
  for (int c0 = fb; c0 < fe; c0 += kGatherChunk) {
    const int nc = min(kGatherChunk, fe - c0);
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const int f = c0 + c;
      int lo = 0, hi = nr - 1;  // last range with sPre <= f
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sPre[mid] <= f) lo = mid; else hi = mid - 1;
      }
      const int sp = sStart[lo] + (f - sPre[lo]);
      sSp[c] = sp;
      for (int a = 0; a < D; ++a) {
        sI[c * 3 + a] = i0s[(long long)a * M + sp];
        sC[c * D + a] = Cw[(long long)sp * D + a];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nc * D * w; i += blockDim.x) {
      const int c = i / (D * w), r = i % (D * w);
      sW[c * D * kMaxW + r] = W[(long long)sSp[c] * D * w + r];
    }
    __syncthreads();
    for (int c = group; c < nc; c += G) {
      // window index of this thread's cells: (cell - i0) mod nf must lie in [0, w). With
      // cell in [0, nf) and i0 in [-w/2, nf - w/2] one wrap suffices; since w + b <= nf a
      // window meets the box through one periodic image only.
      int qy = cy - sI[c * 3 + 1];
      qy += (qy < 0) ? nf : 0; qy -= (qy >= nf) ? nf : 0;
      if (qy >= w) continue;
      int qz = 0;
      if (D == 3) {
        qz = cz - sI[c * 3 + 2];
        qz += (qz < 0) ? nf : 0; qz -= (qz >= nf) ? nf : 0;
        if (qz >= w) continue;
      }
      int qx0 = cx0 - sI[c * 3 + 0];
      qx0 += (qx0 < 0) ? nf : 0; qx0 -= (qx0 >= nf) ? nf : 0;
      if (qx0 > nf - kSeg) qx0 -= nf;  // run starts just before the window start
      if (qx0 >= w) continue;
      const T* wc = sW + c * D * kMaxW;  // axis a at offset a * w (layout of W)
      T t = sC[c * D + comp] * wc[w + qy];
      if (D == 3) t = t * wc[2 * w + qz];
#pragma unroll
      for (int i = 0; i < kSeg; ++i) {
        const int qx = qx0 + i;
        if (qx >= 0 && qx < w) {
          if constexpr (COMP == kSumTerm && std::is_same<T, float>::value) fma_acc(acc[i], t, wc[qx]);
          else acc[i] = acc[i] + t * wc[qx];
        }
      }
    }
    if constexpr (COMP == kSumChunk && std::is_same<T, float>::value) {
#pragma unroll
      for (int i = 0; i < kSeg; ++i) { add_comp(tot[i], acc[i]); acc[i] = A(0); }
    }
  }
  // partial sums of the groups: groups 1.. store theirs (in the weight buffer, free now), group 0
  // adds them (compensated in FP32) and writes the cells
  T part[kSeg];
#pragma unroll
  for (int i = 0; i < kSeg; ++i) {
    if constexpr (COMP == kSumChunk && std::is_same<T, float>::value) part[i] = acc_norm(tot[i]);
    else part[i] = acc_norm(acc[i]);
  }
  if (G > 1) {
    T* red = sW;  // [G - 1][ntask][kSeg] <= blockDim.x * kSeg values
    __syncthreads();
    if (group > 0) {
#pragma unroll
      for (int i = 0; i < kSeg; ++i) red[((group - 1) * ntask + task) * kSeg + i] = part[i];
    }
    __syncthreads();
    if (group == 0) {
      if constexpr (std::is_same<T, float>::value) {
#pragma unroll
        for (int i = 0; i < kSeg; ++i) {
          cf s(part[i]);
          for (int q = 1; q < G; ++q) add_comp(s, red[((q - 1) * ntask + task) * kSeg + i]);
          part[i] = acc_norm(s);
        }
      } else {
#pragma unroll
        for (int i = 0; i < kSeg; ++i)
          for (int q = 1; q < G; ++q) part[i] = part[i] + red[((q - 1) * ntask + task) * kSeg + i];
      }
    }
  }
  T* out = grid + comp * gcells + ((long long)cz * nf + cy) * nf + cx0;
  if (slices == 1) {
    if (group == 0) {
#pragma unroll
      for (int i = 0; i < kSeg; ++i) out[i] = part[i];
    }
    return;
  }
  // a slice of a shared box: its partial box, then the last block adds the slices in order
  T* pp = partials + (((long long)box * KS + ks) * ntask + task) * kSeg;
  if (group == 0) {
#pragma unroll
    for (int i = 0; i < kSeg; ++i) pp[i] = part[i];
  }
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(&done[box], 1) == slices - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (group == 0) {
    const T* p0 = partials + ((long long)box * KS * ntask + task) * kSeg;
#pragma unroll
    for (int i = 0; i < kSeg; ++i) {
      if constexpr (std::is_same<T, float>::value) {
        cf s(0.0f);
        for (int k = 0; k < slices; ++k) add_comp(s, ld_cg(p0 + (long long)k * ntask * kSeg + i));
        out[i] = acc_norm(s);
      } else {
        T v = T(0);
        for (int k = 0; k < slices; ++k) v = v + ld_cg(p0 + (long long)k * ntask * kSeg + i);
        out[i] = v;
      }
    }
  }
  if (threadIdx.x == 0) done[box] = 0;
  }
};


// Work list of the 3D gather: box b is split into K_b = ceil(cand_b / slice_size) slices
// (cand_b = points in its neighbouring bins; K_b = 0 for a box that no window reaches).

__device__ __forceinline__ int nb_list(const PointGeom& g, int dlo, int dhi, int Bx, int By, int Bz, int lane,
                                       int* bin) {
  const int span = dhi - dlo + 1;
  const int sx = min(span, g.nb[0]), sy = min(span, g.nb[1]), sz = min(span, g.nb[2]);
  const int bx0 = (span >= g.nb[0]) ? 0 : Bx + dlo, by0 = (span >= g.nb[1]) ? 0 : By + dlo;
  const int bz0 = (span >= g.nb[2]) ? 0 : Bz + dlo;
  const int nnb = sx * sy * sz;
  if (lane < nnb) {
    int nbx = bx0 + lane % sx, nby = by0 + (lane / sx) % sy, nbz = bz0 + lane / (sx * sy);
    nbx = (nbx % g.nb[0] + g.nb[0]) % g.nb[0];
    nby = (nby % g.nb[1] + g.nb[1]) % g.nb[1];
    nbz = (nbz % g.nb[2] + g.nb[2]) % g.nb[2];
    *bin = (nbz * g.nb[1] + nby) * g.nb[0] + nbx;
  }
  return nnb;
}

// Candidates per slice of a box with c candidates: the plan's slice size, or more when that
// would cut the box into more than kMaxSlices slices (dense point sets), so that the
// partial boxes never exceed kMaxSlices per box.
constexpr int kMaxSlices = 16;
__device__ __forceinline__ int slice_size(const PointGeom& g, int c) {
  return max(g.slice, (c + kMaxSlices - 1) / kMaxSlices);
}

// One warp per box: number of slices of the box.
struct KBoxSlices {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = false;
  __device__ static void run(PointGeom g, int dlo, int dhi, const int* __restrict__ offsets,
                             int* __restrict__ nslice, int* __restrict__ npart, int* __restrict__ done) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  const int nbox = g.nb[0] * g.nb[1] * g.nb[2];
  if (warp >= nbox) return;
  const int Bx = warp % g.nb[0], By = (warp / g.nb[0]) % g.nb[1], Bz = warp / (g.nb[0] * g.nb[1]);
  int bin = 0;
  const int nnb = nb_list(g, dlo, dhi, Bx, By, Bz, lane, &bin);
  int c = (lane < nnb) ? offsets[bin + 1] - offsets[bin] : 0;
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if (lane == 0) {
    const int sz = slice_size(g, c);
    const int K = (c + sz - 1) / sz;  // 0 for a box that no window reaches; at most kMaxSlices
    nslice[warp] = K;
    npart[warp] = (K > 1) ? K : 0;
    done[warp] = 0;
  }
}
};

// Box of every slice: box_item[slice_off[b] + k] = b for k < K_b; and the order in which
// the gather takes them: the slices of split boxes (K_b > 1, the densest, whose slices
// are the longest) first, then the single-slice boxes, so that the work left at the end of
// the launch is short. part_off (prefix of K_b over split boxes) numbers the first group;
// slice_off[b] - part_off[b] counts the single-slice boxes before b.
// Also resets the gather's work counters for the launch that follows.
struct KSliceBoxes {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(int nbox, const int* __restrict__ slice_off, const int* __restrict__ part_off,
                              int* __restrict__ box_item, int* __restrict__ sched, int* __restrict__ work) {
  if (blockIdx.x == 0 && threadIdx.x < 2) work[threadIdx.x] = 0;
  const int nsplit = part_off[nbox];
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) {
    const int s0 = slice_off[b], K = slice_off[b + 1] - s0;
    for (int k = 0; k < K; ++k) {
      box_item[s0 + k] = b;
      sched[(K > 1) ? part_off[b] + k : nsplit + (s0 - part_off[b])] = s0 + k;
    }
  }
}
};

// Next work of the calling block (dynamic scheduling, so that heavy and light slices spread
// evenly over the SMs): a slice (work[0]) and, with it, a run of boxes to zero (work[1]), so
// that the zero stores overlap the gathers. All threads of the block call it; it ends with
// a barrier.
__device__ __forceinline__ int next_slice(int* __restrict__ work, int* s_item, int* run) {
  __syncthreads();  // every thread has read the previous item
  if (threadIdx.x == 0) { s_item[0] = atomicAdd(&work[0], 1); s_item[1] = atomicAdd(&work[1], 1); }
  __syncthreads();
  *run = s_item[1];
  return s_item[0];
}

// Zeroing of the boxes that no window reaches but whose row band another box's windows reach
// (the forward row pass reads those rows whole), in runs of 32 boxes claimed from a counter
// (work[1]): 16-byte stores along x.
template <typename T>
__device__ __forceinline__ void zero_box(const PointGeom& g, int box, T* __restrict__ grid, int lane) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "grid element");
  constexpr int v_per_row = 8 * (int)sizeof(T) / 16;  // 16-byte vectors per 8-cell box row
  const int nf = g.nf;
  const long long gcells = (long long)nf * nf * nf;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const int Bx = box % g.nb[0], By = (box / g.nb[0]) % g.nb[1], Bz = box / (g.nb[0] * g.nb[1]);
  for (int i = lane; i < 3 * 64 * v_per_row; i += 32) {
    const int v = i % v_per_row, row = i / v_per_row;  // row = (a * 8 + z) * 8 + y
    const int y = row & 7, z = (row >> 3) & 7, a = row >> 6;
    T* r = grid + a * gcells + ((long long)(Bz * 8 + z) * nf + (By * 8 + y)) * nf + Bx * 8;
    reinterpret_cast<float4*>(r)[v] = z4;
  }
}

// A box that no window reaches is zeroed when its row band is read by the forward row pass.
__device__ __forceinline__ bool box_empty(const PointGeom& g, const int* __restrict__ slice_off, int nbox, int box) {
  if (box >= nbox || slice_off[box + 1] != slice_off[box]) return false;
  if (!g.band) return true;
  const int by = (box / g.nb[0]) % g.nb[1], bz = box / (g.nb[0] * g.nb[1]);
  return g.band[bz * g.nb[1] + by] != 0;
}

// One run by the whole block: warp w takes boxes 4w .. 4w + 3 of the run.
template <typename T>
__device__ __forceinline__ void zero_run_block(const PointGeom& g, const int* __restrict__ slice_off, int nbox,
                                               T* __restrict__ grid, int run) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
  for (int k = 0; k < 4; ++k) {
    const int box = run * 32 + warp * 4 + k;
    if (box_empty(g, slice_off, nbox, box)) zero_box<T>(g, box, grid, lane);  // uniform across the warp
  }
}

// The runs left when the slices are done, claimed warp by warp.
template <typename T>
__device__ __forceinline__ void zero_empty_boxes(const PointGeom& g, const int* __restrict__ slice_off, int nbox,
                                                 T* __restrict__ grid, int* __restrict__ work) {
  const int lane = threadIdx.x & 31;
  const int nruns = (nbox + 31) / 32;
  for (;;) {
    int run = 0;
    if (lane == 0) run = atomicAdd(&work[1], 1);
    run = __shfl_sync(0xffffffffu, run, 0);
    if (run >= nruns) break;
    const int b0 = run * 32;
    unsigned m = __ballot_sync(0xffffffffu, box_empty(g, slice_off, nbox, b0 + lane));
    while (m) {
      const int box = b0 + __ffs(m) - 1;
      m &= m - 1;
      zero_box<T>(g, box, grid, lane);
    }
  }
}

// After a block has stored the partial box of slice ks of a split box (K > 1 slices): the
// block that finishes last adds the K partials in slice order and stores the box (the
// fences make every partial visible before the count that reports it).
template <typename T>
__device__ __forceinline__ void finish_split_box(const PointGeom& g, int box, int K, const int* __restrict__ part_off,
                                                 const T* part, T* __restrict__ grid, int* __restrict__ done,
                                                 int* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_flag = (atomicAdd(&done[box], 1) == K - 1);
  __syncthreads();
  if (!*s_flag) return;
  __threadfence();
  const int nf = g.nf;
  const int Bx = box % g.nb[0], By = (box / g.nb[0]) % g.nb[1], Bz = box / (g.nb[0] * g.nb[1]);
  const long long gcells = (long long)nf * nf * nf;
  for (int i = threadIdx.x; i < 3 * 512; i += blockDim.x) {
    const int a = i / 512, c = i % 512;
    T v = T(0);
    for (int k = 0; k < K; ++k) v = v + ld_cg(part + ((long long)(part_off[box] + k) * 3 + a) * 512 + c);
    const int x = c % 8, y = (c / 8) % 8, z = c / 64;
    grid[a * gcells + ((long long)(Bz * 8 + z) * nf + (By * 8 + y)) * nf + (Bx * 8 + x)] = v;
  }
}

// 3D gather with an 8^3 box: warp z owns the box plane oz + z, lane l owns the cells
// (x, y) = (l % 8, l / 8) and (l % 8, l / 8 + 4) of that plane for all three
// components, in registers. The candidates (points of the neighbouring bins, taken in
// bin order) are staged in shared memory, a chunk at a time and double buffered, as
// box-relative weights: for axis a and box offset l, the kernel weight of the cell
// o_a + l, or zero where the point's window misses it. A lane then needs no index
// arithmetic (a zero weight adds nothing), and a candidate whose window misses a
// warp's plane is skipped by the whole warp.
constexpr int kBoxChunk = 64;
__device__ __forceinline__ bool is_zero(float v) { return v == 0.0f; }
__device__ __forceinline__ bool is_zero(double v) { return v == 0.0; }
__device__ __forceinline__ bool is_zero(dd v) { return v.hi == 0.0f; }

template <typename T, int COMP>
struct KSpreadBox3 {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(PointGeom g, int dlo, int dhi, const int* __restrict__ offsets, const int* __restrict__ i0s,
              const T* __restrict__ W, const T* __restrict__ Cw, const int* __restrict__ slice_off,
              const int* __restrict__ box_item, const int* __restrict__ sched, const int* __restrict__ part_off,
              T* __restrict__ part,
              T* __restrict__ grid, int* __restrict__ work, int* __restrict__ done) {
  __shared__ __align__(16) T sB[2][kBoxChunk * 24];  // [c][axis][8] box-relative weights
  __shared__ T sC[2][kBoxChunk * 3];
  __shared__ int sStart[32], sPre[33];  // non-empty neighbour ranges: first point, prefix of lengths
  __shared__ int sNr;
  const int w = g.w, nf = g.nf, M = g.M;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int lx = lane & 7, ly = lane >> 3;
  const int nbox = g.nb[0] * g.nb[1] * g.nb[2];
  const int nslices = slice_off[nbox];
  __shared__ int s_item[2], s_flag;
  for (;;) {
    int run;
    const int it = next_slice(work, s_item, &run);
    if (run < (nbox + 31) / 32) zero_run_block(g, slice_off, nbox, grid, run);
    if (it >= nslices) break;
    const int sl = sched[it];
    const int box = box_item[sl], ks = sl - slice_off[box], K = slice_off[box + 1] - slice_off[box];
    const int Bx = box % g.nb[0], By = (box / g.nb[0]) % g.nb[1], Bz = box / (g.nb[0] * g.nb[1]);
    const int o[3] = {Bx * 8, By * 8, Bz * 8};
    __syncthreads();
    if (warp == 0) {  // candidate ranges of the neighbouring bins, in one round trip
      int bin = 0;
      const int nnb = nb_list(g, dlo, dhi, Bx, By, Bz, lane, &bin);
      int p0 = 0, len = 0;
      if (lane < nnb) { p0 = offsets[bin]; len = offsets[bin + 1] - p0; }
      int incl = len;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
      }
      const unsigned nonempty = __ballot_sync(0xffffffffu, len > 0);
      if (len > 0) {
        const int slot = __popc(nonempty & ((1u << lane) - 1u));
        sStart[slot] = p0;
        sPre[slot] = incl - len;
      }
      if (lane == 31) { sNr = __popc(nonempty); sPre[__popc(nonempty)] = incl; }
    }
    __syncthreads();
    const int nr = sNr;
    // this slice takes candidates [ks * slice, (ks + 1) * slice) of the concatenated ranges
    const int sz = slice_size(g, sPre[nr]);
    const int f0 = ks * sz, f1 = min(sPre[nr], f0 + sz);
    // stage candidates [fa, fb) into buffer bb: one thread per (candidate, axis)
    auto stage = [&](int fa, int fb, int bb) {
      for (int i = threadIdx.x; i < (fb - fa) * 3; i += blockDim.x) {
        const int c = i / 3, a = i - 3 * c, f = fa + c;
        int lo = 0, hi = nr - 1;  // last range with sPre <= f
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (sPre[mid] <= f) lo = mid; else hi = mid - 1;
        }
        const long long sp = sStart[lo] + (f - sPre[lo]);
        int q0 = o[a] - i0s[(long long)a * M + sp];  // (o_a - i0) mod nf
        q0 += (q0 < 0) ? nf : 0; q0 -= (q0 >= nf) ? nf : 0;
        const T* wsrc = W + sp * 3 * w + a * w;
        T* dst = &sB[bb][(c * 3 + a) * 8];
        T wv[8];
#pragma unroll
        for (int l = 0; l < 8; ++l) {
          int q = q0 + l;
          q -= (q >= nf) ? nf : 0;
          wv[l] = (q < w) ? wsrc[q] : T(0);
        }
        if constexpr (sizeof(T) == 4) {  // two 16-byte stores: the threads' rows are 32 bytes apart
          reinterpret_cast<float4*>(dst)[0] = make_float4(wv[0], wv[1], wv[2], wv[3]);
          reinterpret_cast<float4*>(dst)[1] = make_float4(wv[4], wv[5], wv[6], wv[7]);
        } else {
#pragma unroll
          for (int l = 0; l < 8; ++l) dst[l] = wv[l];
        }
        sC[bb][c * 3 + a] = Cw[sp * 3 + a];
      }
    };
    using A = typename SumAcc<T, COMP>::type;
    A acc[2][3];
    cf tot[2][3];  // kSumChunk: compensated sums of the chunks' partial sums
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int a = 0; a < 3; ++a) { acc[k][a] = A(0); tot[k][a] = cf(0.0f); }
    int bb = 0;
    stage(f0, min(f1, f0 + kBoxChunk), 0);
    __syncthreads();
    for (int c0 = f0; c0 < f1; c0 += kBoxChunk) {
      const int nc = min(kBoxChunk, f1 - c0);
      if (c0 + kBoxChunk < f1) stage(c0 + kBoxChunk, min(f1, c0 + 2 * kBoxChunk), bb ^ 1);
      const T* B = sB[bb];
      const T* Cc = sC[bb];
      for (int c = 0; c < nc; ++c) {
        const T wz = B[c * 24 + 16 + warp];
        if (is_zero(wz)) continue;  // uniform across the warp
        const T wxz = B[c * 24 + lx] * wz;
        const T t0 = wxz * B[c * 24 + 8 + ly], t1 = wxz * B[c * 24 + 12 + ly];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const T cv = Cc[c * 3 + a];
          fma_acc(acc[0][a], cv, t0);
          fma_acc(acc[1][a], cv, t1);
        }
      }
      if constexpr (COMP == kSumChunk && std::is_same<T, float>::value) {
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int a = 0; a < 3; ++a) { add_comp(tot[k][a], acc[k][a]); acc[k][a] = A(0); }
      }
      __syncthreads();
      bb ^= 1;
    }
    const long long gcells = (long long)nf * nf * nf;
    const int cx = o[0] + lx, cz = o[2] + warp;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int yk = ly + 4 * k;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        T v;
        if constexpr (COMP == kSumChunk && std::is_same<T, float>::value) v = acc_norm(tot[k][a]);
        else v = acc_norm(acc[k][a]);
        if (K == 1) {
          grid[a * gcells + ((long long)cz * nf + (o[1] + yk)) * nf + cx] = v;
        } else {
          // partial box, layout [slot][a][z][y][x]
          part[((long long)(part_off[box] + ks) * 3 + a) * 512 + (warp * 8 + yk) * 8 + lx] = v;
        }
      }
    }
    if (K > 1) finish_split_box<T>(g, box, K, part_off, part, grid, done, &s_flag);  // uniform across the block
  }
  zero_empty_boxes<T>(g, slice_off, nbox, grid, work);
}
};

// Double-float variant of the 3D gather. The per-lane work is six double-float
// multiply-adds per candidate and plane, so the weight products are formed once per block
// while staging: a group of eight threads per candidate evaluates the box-relative weights
// of offset t on each axis, shares them by shuffles, and writes the candidate's 8 x 8 table
// of w_x w_y products and its d x 8 values C_a w_z (plus w_z for the plane test).
constexpr int kBoxChunkDD = 32;   // candidates per chunk (eight threads each; one per lane of a warp)
static_assert(kBoxChunkDD == 32, "the double-float gather keeps a chunk's candidate lists in one ballot word");
constexpr int kXYStride = 72;     // per-candidate stride of the x-y table (64 + 8: staging stores hit all banks)
struct KSpreadBox3DD {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(PointGeom g, int dlo, int dhi, const int* __restrict__ offsets, const int* __restrict__ i0s,
                 const dd* __restrict__ W, const dd* __restrict__ Cw, const int* __restrict__ slice_off,
                 const int* __restrict__ box_item, const int* __restrict__ sched, const int* __restrict__ part_off,
                 dd* __restrict__ part,
                 dd* __restrict__ grid, int* __restrict__ work, int* __restrict__ done) {
  // dynamic shared memory (above the 48 KB static limit): two buffers of
  //   [c][y][x] w_x w_y (stride kXYStride), [c][a][z] C_a w_z, [c] mask: bits 0-7 the z planes
  //   the candidate reaches, bits 8 and 9 the lower and upper y halves (0 when its window misses
  //   the box along x)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd (*sXY)[kBoxChunkDD * kXYStride] = reinterpret_cast<dd (*)[kBoxChunkDD * kXYStride]>(smem_raw);
  dd (*sCz)[kBoxChunkDD * 24] = reinterpret_cast<dd (*)[kBoxChunkDD * 24]>(sXY + 2);
  unsigned (*sMask)[kBoxChunkDD] = reinterpret_cast<unsigned (*)[kBoxChunkDD]>(sCz + 2);
  __shared__ int sStart[32], sPre[33];
  __shared__ int sNr;
  const int w = g.w, nf = g.nf, M = g.M;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int lx = lane & 7, ly = lane >> 3;
  const int nbox = g.nb[0] * g.nb[1] * g.nb[2];
  const int nslices = slice_off[nbox];
  __shared__ int s_item[2], s_flag;
  for (;;) {
    int run;
    const int it = next_slice(work, s_item, &run);
    if (run < (nbox + 31) / 32) zero_run_block(g, slice_off, nbox, grid, run);
    if (it >= nslices) break;
    const int sl = sched[it];
    const int box = box_item[sl], ks = sl - slice_off[box], K = slice_off[box + 1] - slice_off[box];
    const int Bx = box % g.nb[0], By = (box / g.nb[0]) % g.nb[1], Bz = box / (g.nb[0] * g.nb[1]);
    const int o[3] = {Bx * 8, By * 8, Bz * 8};
    __syncthreads();
    if (warp == 0) {  // candidate ranges of the neighbouring bins, in one round trip
      int bin = 0;
      const int nnb = nb_list(g, dlo, dhi, Bx, By, Bz, lane, &bin);
      int p0 = 0, len = 0;
      if (lane < nnb) { p0 = offsets[bin]; len = offsets[bin + 1] - p0; }
      int incl = len;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
      }
      const unsigned nonempty = __ballot_sync(0xffffffffu, len > 0);
      if (len > 0) {
        const int slot = __popc(nonempty & ((1u << lane) - 1u));
        sStart[slot] = p0;
        sPre[slot] = incl - len;
      }
      if (lane == 31) { sNr = __popc(nonempty); sPre[__popc(nonempty)] = incl; }
    }
    __syncthreads();
    const int nr = sNr;
    const int sz = slice_size(g, sPre[nr]);
    const int f0 = ks * sz, f1 = min(sPre[nr], f0 + sz);
    // stage candidates [fa, fb) into buffer bb: eight threads per candidate, t = offset
    auto stage = [&](int fa, int fb, int bb) {
      const int c = threadIdx.x >> 3, t = threadIdx.x & 7;
      const bool on = c < fb - fa;
      dd wa[3] = {dd(0.0f), dd(0.0f), dd(0.0f)};
      dd cv = dd(0.0f);
      if (on) {
        const int f = fa + c;
        int lo = 0, hi = nr - 1;  // last range with sPre <= f
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (sPre[mid] <= f) lo = mid; else hi = mid - 1;
        }
        const long long sp = sStart[lo] + (f - sPre[lo]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          int q = o[a] + t - i0s[(long long)a * M + sp];  // (o_a + t - i0) mod nf
          q += (q < 0) ? nf : 0; q -= (q >= nf) ? nf : 0; q -= (q >= nf) ? nf : 0;
          wa[a] = (q < w) ? W[sp * 3 * w + a * w + q] : dd(0.0f);
        }
        if (t < 3) cv = Cw[sp * 3 + t];
      }
      // products: thread t owns column x = t of the x-y table and plane z = t of C w_z
      dd* xy = &sXY[bb][c * kXYStride + t];
#pragma unroll
      for (int y = 0; y < 8; ++y) {
        const float yh = __shfl_sync(0xffffffffu, wa[1].hi, (lane & ~7) | y);
        const float yl = __shfl_sync(0xffffffffu, wa[1].lo, (lane & ~7) | y);
        if (on) xy[y * 8] = wa[0] * dd(yh, yl);
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float ch = __shfl_sync(0xffffffffu, cv.hi, (lane & ~7) | a);
        const float cl = __shfl_sync(0xffffffffu, cv.lo, (lane & ~7) | a);
        if (on) sCz[bb][c * 24 + a * 8 + t] = dd(ch, cl) * wa[2];
      }
      // which offsets carry weight, per axis, for the eight lanes of this candidate
      const int gs = lane & ~7;
      const unsigned bx = (__ballot_sync(0xffffffffu, on && wa[0].hi != 0.0f) >> gs) & 0xffu;
      const unsigned by = (__ballot_sync(0xffffffffu, on && wa[1].hi != 0.0f) >> gs) & 0xffu;
      const unsigned bz = (__ballot_sync(0xffffffffu, on && wa[2].hi != 0.0f) >> gs) & 0xffu;
      if (on && t == 0)
        sMask[bb][c] = bx ? (bz | ((by & 0x0Fu) ? 0x100u : 0u) | ((by & 0xF0u) ? 0x200u : 0u)) : 0u;
    };
    // Lane (lx, ly) of warp v owns two cells: (lx, ly, v) in the lower y half and (lx, ly + 4,
    // 7 - v) in the upper y half. A candidate's work on a half is skipped when its window misses
    // the plane or the half (both tests uniform across the warp), and pairing plane v with 7 - v
    // evens out the work of the warps: the windows of a box's candidates cover its middle planes
    // more often than its outer ones.
    const int zA = warp, zB = 7 - warp;
    dd acc[2][3];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int a = 0; a < 3; ++a) acc[k][a] = dd(0.0f);
    int bb = 0;
    stage(f0, min(f1, f0 + kBoxChunkDD), 0);
    __syncthreads();
    for (int c0 = f0; c0 < f1; c0 += kBoxChunkDD) {
      const int nc = min(kBoxChunkDD, f1 - c0);
      if (c0 + kBoxChunkDD < f1) stage(c0 + kBoxChunkDD, min(f1, c0 + 2 * kBoxChunkDD), bb ^ 1);
      const dd* XY = sXY[bb];
      const dd* CZ = sCz[bb];
      const unsigned* MK = sMask[bb];
      // the chunk's candidates that reach each of this warp's two cell groups, as bit lists
      // (kBoxChunkDD == 32: one candidate per lane), then only those candidates are visited
      const unsigned m = lane < nc ? MK[lane] : 0u;
      unsigned la = __ballot_sync(0xffffffffu, (m >> zA) & (m >> 8) & 1u);
      unsigned lb = __ballot_sync(0xffffffffu, (m >> zB) & (m >> 9) & 1u);
      while (la) {
        const int c = __ffs(la) - 1;
        la &= la - 1;
        const dd t0 = XY[c * kXYStride + ly * 8 + lx];
#pragma unroll
        for (int a = 0; a < 3; ++a) dd_fma_acc(acc[0][a], CZ[c * 24 + a * 8 + zA], t0);
      }
      while (lb) {
        const int c = __ffs(lb) - 1;
        lb &= lb - 1;
        const dd t1 = XY[c * kXYStride + (ly + 4) * 8 + lx];
#pragma unroll
        for (int a = 0; a < 3; ++a) dd_fma_acc(acc[1][a], CZ[c * 24 + a * 8 + zB], t1);
      }
      __syncthreads();
      bb ^= 1;
    }
    const long long gcells = (long long)nf * nf * nf;
    const int cx = o[0] + lx;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int yk = ly + 4 * k, zk = k ? zB : zA;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const dd v = dd_norm(acc[k][a]);
        if (K == 1) {
          grid[a * gcells + ((long long)(o[2] + zk) * nf + (o[1] + yk)) * nf + cx] = v;
        } else {
          part[((long long)(part_off[box] + ks) * 3 + a) * 512 + (zk * 8 + yk) * 8 + lx] = v;
        }
      }
    }
    if (K > 1) finish_split_box<dd>(g, box, K, part_off, part, grid, done, &s_flag);  // uniform across the block
  }
  zero_empty_boxes<dd>(g, slice_off, nbox, grid, work);
}
};


template <typename T, int D>
struct KInterpWarp {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(PointGeom g, const int* __restrict__ perm, const int* __restrict__ i0s, const T* __restrict__ W,
              const T* __restrict__ grid, double* __restrict__ U, const unsigned char* __restrict__ guard,
              unsigned int* miss_flag) {
  // per warp: the window's rows (y, z) as grid offsets and their weight products w_y w_z
  constexpr int kRows = (D == 3) ? kMaxW * kMaxW : kMaxW;
  __shared__ int sOff[8][kRows];
  __shared__ T sWyz[8][kRows];
  const int w = g.w, nf = g.nf, M = g.M;
  const int nwarp = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int K = 32 / w;                 // lane groups
  const int qx = lane % w, kg = lane / w;
  const bool on = kg < K;
  const long long gcells = (long long)nf * nf * (D == 3 ? nf : 1);
  const int nrow = (D == 3) ? w * w : w;
  int* off = sOff[warp];
  T* wyz = sWyz[warp];
  for (long long s = (long long)blockIdx.x * nwarp + warp; s < M; s += (long long)gridDim.x * nwarp) {
    const T* ws = W + s * D * w;
    const int bx = i0s[s], by = i0s[(long long)M + s], bz = (D == 3) ? i0s[2LL * M + s] : 0;
    __syncwarp();
    bool miss = false;  // a window row outside the bands the grid holds
    for (int r = lane; r < nrow; r += 32) {
      const int qz = (D == 3) ? r / w : 0, qy = r - qz * w;
      int gy = by + qy, gz = bz + qz;
      gy += (gy < 0) ? nf : 0; gy -= (gy >= nf) ? nf : 0;
      if (D == 3) { gz += (gz < 0) ? nf : 0; gz -= (gz >= nf) ? nf : 0; }
      if (guard && !guard[(D == 3 ? gz / g.b[2] : 0) * g.nb[1] + gy / g.b[1]]) miss = true;
      off[r] = (D == 3) ? (gz * nf + gy) * nf : gy * nf;
      T v = ws[w + qy];
      if (D == 3) v = v * ws[2 * w + qz];
      wyz[r] = v;
    }
    __syncwarp();
    int gx = bx + qx;
    gx += (gx < 0) ? nf : 0; gx -= (gx >= nf) ? nf : 0;
    const T* gp = grid + gx;
    T acc[D];
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] = T(0);
    if (on) {
      // four rows per iteration: all loads are issued before the arithmetic
      int r = kg;
      for (; r + 3 * K < nrow; r += 4 * K) {
        T gv[4][D], wv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int o = off[r + u * K];
#pragma unroll
          for (int a = 0; a < D; ++a) gv[u][a] = gp[a * gcells + o];
          wv[u] = wyz[r + u * K];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int a = 0; a < D; ++a) fma_acc(acc[a], gv[u][a], wv[u]);
      }
      for (; r < nrow; r += K) {
        const int o = off[r];
        const T wv = wyz[r];
#pragma unroll
        for (int a = 0; a < D; ++a) fma_acc(acc[a], gp[a * gcells + o], wv);
      }
      const T wxq = ws[qx];
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] = acc_norm(acc[a]) * wxq;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] = warp_sum(acc[a]);
    const bool bad = __any_sync(0xffffffffu, miss);
    if (lane == 0) {
      const int j = perm[s];
#pragma unroll
      for (int a = 0; a < D; ++a) U[(long long)a * M + j] = bad ? __longlong_as_double(0x7ff8000000000000LL)
                                                                 : to_double_val(acc[a]);
      if (bad && miss_flag) *(volatile unsigned int*)miss_flag = 1u;
    }
  }
}
};

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
    auto run = [&](auto k) {
      using K = typename decltype(k)::type;
      raise_smem_limit(kernel_ptr<K>());
      launch<K>(blocks, kSpreadThreads, smem, st, g, beta, cw, omega, ws.perm, ws.offsets, ws.occ, ws.nocc, ws.i0,
                (const T*)ws.delta, grid);
    };
    if (comp) run(type_tag<KSpreadScatter<T, 3, true>>());
    else run(type_tag<KSpreadScatter<T, 3, false>>());
  } else {
    auto run = [&](auto k) {
      using K = typename decltype(k)::type;
      raise_smem_limit(kernel_ptr<K>());
      launch<K>(blocks, kSpreadThreads, smem, st, g, beta, cw, omega, ws.perm, ws.offsets, ws.occ, ws.nocc, ws.i0,
                (const T*)ws.delta, grid);
    };
    if (comp) run(type_tag<KSpreadScatter<T, 2, true>>());
    else run(type_tag<KSpreadScatter<T, 2, false>>());
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
    launch<KInterp<T, 3>>((unsigned)blocks, kSpreadThreads, 0, st, g, beta, ws.perm, ws.i0, (const T*)ws.delta, grid, U);
  else
    launch<KInterp<T, 2>>((unsigned)blocks, kSpreadThreads, 0, st, g, beta, ws.perm, ws.i0, (const T*)ws.delta, grid, U);
}

template <typename T>
void launch_point_prep(const Plan& p, Workspace& ws, const double* cw, const double* omega, cudaStream_t st) {
  const PointGeom g = geom(p);
  using Td = typename DeltaT<T>::type;
  const long long nw = (long long)p.M * p.d * p.w;
  long long blocks = (nw + 255) / 256;
  if (blocks > 64LL * num_sms()) blocks = 64LL * num_sms();
  T* Cw = cw ? (T*)ws.cwp : nullptr;
  if (p.d == 3)
    launch<KPointPrep<T, 3>>((unsigned)blocks, 256, 0, st, g, p.beta, (const Td*)ws.delta, ws.perm, cw, omega, (T*)ws.wts, Cw,
                                                      dd(2.0 / p.w), dd(p.beta));
  else
    launch<KPointPrep<T, 2>>((unsigned)blocks, 256, 0, st, g, p.beta, (const Td*)ws.delta, ws.perm, cw, omega, (T*)ws.wts, Cw,
                                                      dd(2.0 / p.w), dd(p.beta));
}

// Blocks per box of the 2D gather: with dense points (16 or more per box on average; a curve
// puts thousands in the boxes it crosses) enough to give about four blocks per SM, at most 16;
// one block per box otherwise. A block takes at least kGatherSliceMin of its box's candidates.
int gather2d_slices(const Plan& p) {
  const long long nbox = p.nbins;
  if (p.d != 2 || (long long)p.M < 16 * nbox) return 1;
  const long long ks = (4LL * num_sms() + nbox - 1) / nbox;
  return (int)std::max(1LL, std::min(16LL, ks));
}
// Bytes of the partial boxes of the 2D gather (8-byte elements cover both precisions).
size_t gather2d_part_bytes(const Plan& p) {
  return sizeof(double) * (size_t)p.nbins * (size_t)gather2d_slices(p) * 2 * (size_t)p.bins[0] * p.bins[1];
}

template <typename T>
void launch_spread_gather(const Plan& p, Workspace& ws, T* grid, cudaStream_t st) {
  PointGeom g = geom(p);
  g.band = ws.band;  // boxes in bands that no window reaches are neither gathered nor zeroed
  const int b = p.bins[0];
  // neighbour bins holding window starts that reach the box: floor((-w + 1)/b) .. 0
  const int dlo = -((p.w - 1 + b - 1) / b), dhi = 0;
  const int nbox = (int)p.nbins;
  if (p.d == 3) {
    // slices per box, their prefix sums, then the sliced gather and the partial reduction
    launch<KBoxSlices>((nbox * 32 + 255) / 256, 256, 0, st, g, dlo, dhi, ws.offsets, ws.box_ns, ws.box_np,
                                                           ws.box_done);
    launch<KScan2>(2, 1024, 0, st, ws.box_ns, ws.box_np, nbox, ws.box_so, ws.box_po);
    launch<KSliceBoxes>((nbox + 255) / 256, 256, 0, st, nbox, ws.box_so, ws.box_po, ws.box_item, ws.box_sched,
                                                       ws.box_work);
    if constexpr (std::is_same<T, dd>::value) {
      constexpr size_t smem = 2 * sizeof(dd) * kBoxChunkDD * (kXYStride + 24) + 2 * sizeof(unsigned) * kBoxChunkDD;
      static const int per_sm = [] {
        raise_smem_limit(kernel_ptr<KSpreadBox3DD>());
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel_ptr<KSpreadBox3DD>(), 256, smem) != cudaSuccess ||
            n < 1)
          n = 4;
        return n;
      }();
      launch<KSpreadBox3DD>(per_sm * num_sms(), 256, smem, st, g, dlo, dhi, ws.offsets, ws.i0, (const dd*)ws.wts,
                            (const dd*)ws.cwp, ws.box_so, ws.box_item, ws.box_sched, ws.box_po, (dd*)ws.part, grid,
                            ws.box_work, ws.box_done);
    } else {
      auto run = [&](auto k) {
        using K = typename decltype(k)::type;
        static int per_sm = 0;
        if (!per_sm) {
          if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_ptr<K>(), 256, 0) != cudaSuccess ||
              per_sm < 1)
            per_sm = 4;
        }
        launch<K>(per_sm * num_sms(), 256, 0, st, g, dlo, dhi, ws.offsets, ws.i0, (const T*)ws.wts, (const T*)ws.cwp,
                  ws.box_so, ws.box_item, ws.box_sched, ws.box_po, (T*)ws.part, grid, ws.box_work, ws.box_done);
      };
      if (p.spread_sum == kSumTerm) run(type_tag<KSpreadBox3<T, kSumTerm>>());
      else if (p.spread_sum == kSumChunk) run(type_tag<KSpreadBox3<T, kSumChunk>>());
      else run(type_tag<KSpreadBox3<T, kSumPlain>>());
    }
  } else {
    // one thread per (component, row, run of kSeg cells) of the box, times the candidate groups
    // (up to 256 threads; every box side is a multiple of 8, so ntask = b^2/4 divides 256 or is 256)
    const int ntask = 2 * p.bins[1] * (p.bins[0] / kSeg);
    const int groups = std::max(1, std::min(16, 256 / ntask));
    const int threads = ntask * groups;
    const int mode = std::is_same<T, float>::value ? p.spread_sum : kSumPlain;
    const int KS = gather2d_slices(p);
    auto run = [&](auto k) {
      using K = typename decltype(k)::type;
      launch<K>(nbox * KS, threads, 0, st, g, dlo, dhi, ws.offsets, ws.i0, (const T*)ws.wts, (const T*)ws.cwp, grid,
                KS, (T*)ws.part, ws.box_done);
    };
    if (mode == kSumTerm) run(type_tag<KSpreadGather<T, 2, kSumTerm>>());
    else if (mode == kSumChunk) run(type_tag<KSpreadGather<T, 2, kSumChunk>>());
    else run(type_tag<KSpreadGather<T, 2, kSumPlain>>());
  }
}

template <typename T>
void launch_interp_warp(const Plan& p, Workspace& ws, const T* grid, double* U, cudaStream_t st,
                        const unsigned char* guard, unsigned int* miss) {
  const PointGeom g = geom(p);
  long long blocks = (p.M + 7) / 8;
  if (blocks > 32LL * num_sms()) blocks = 32LL * num_sms();
  if (p.d == 3)
    launch<KInterpWarp<T, 3>>((unsigned)blocks, 256, 0, st, g, ws.perm, ws.i0, (const T*)ws.wts, grid, U, guard, miss);
  else
    launch<KInterpWarp<T, 2>>((unsigned)blocks, 256, 0, st, g, ws.perm, ws.i0, (const T*)ws.wts, grid, U, guard, miss);
}

template void launch_point_prep<float>(const Plan&, Workspace&, const double*, const double*, cudaStream_t);
template void launch_point_prep<dd>(const Plan&, Workspace&, const double*, const double*, cudaStream_t);
template void launch_spread_gather<float>(const Plan&, Workspace&, float*, cudaStream_t);
template void launch_spread_gather<dd>(const Plan&, Workspace&, dd*, cudaStream_t);
template void launch_interp_warp<float>(const Plan&, Workspace&, const float*, double*, cudaStream_t,
                                        const unsigned char*, unsigned int*);
template void launch_interp_warp<dd>(const Plan&, Workspace&, const dd*, double*, cudaStream_t, const unsigned char*,
                                     unsigned int*);


template void launch_spread<float>(const Plan&, Workspace&, const double*, const double*, float*, cudaStream_t);
template void launch_spread<double>(const Plan&, Workspace&, const double*, const double*, double*, cudaStream_t);
template void launch_interp<float>(const Plan&, Workspace&, const float*, double*, cudaStream_t);
template void launch_interp<double>(const Plan&, Workspace&, const double*, double*, cudaStream_t);

}  // namespace fsib
