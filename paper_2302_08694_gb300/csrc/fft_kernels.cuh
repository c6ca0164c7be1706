// Transform passes between real grids and half spectra.
//
// A d-dimensional real transform is split into passes, one per axis:
//  * rows (x axis, contiguous): real rows of length n <-> the N/2 kept modes
//    m_x = 0..N/2-1. Two real rows are packed into one complex line.
//  * strided (y or z axis): complex lines along an axis of stride `inner`,
//    processed P adjacent lines at a time so that every global access is a run
//    of P consecutive complex values.
// Forward passes keep the modes of K_N (pruned output, the unpaired mode -N/2
// written as zero); inverse passes read K_N and zero-pad to n. The deconvolution
// of appendix A (division by the kernel's Fourier transform) or a plain scale is
// applied where all mode indices are known: on the output of the last forward
// pass and on the input of the first inverse pass.
// Kernel and launcher templates; fft_float.cu, fft_dd.cu and fft_double.cu instantiate
// them per arithmetic type so that the three compile in parallel.
#pragma once
#include <algorithm>
#include <type_traits>
#include "wfft.cuh"

namespace fsib {

// Launch shapes (tunable per plan): fl.tile_p adjacent lines per strided tile,
// fl.rows_q row pairs per CTA in the row passes.
constexpr int kThreads = 256;

// Run the line transforms with the compile-time plan when NC > 0.
template <typename T, bool INV, int NC>
__device__ __forceinline__ C<T>* fft_lines(C<T>* a, C<T>* b, int nl, int ls, int es, bool lines_fast,
                                           const FftLen& fl, const C<T>* __restrict__ tw) {
  if constexpr (NC > 0) {
    return smem_fft_ct<T, INV, NC>(a, b, nl, lines_fast ? __ffs(nl) - 1 : 0, ls, es, lines_fast, tw);
  } else {
    return smem_fft<T, INV>(a, b, nl, ls, es, lines_fast, fl, tw);
  }
}

// ---------------------------------------------------------------------------
// Strided pass
// ---------------------------------------------------------------------------
template <typename T, bool INV, typename Tin, typename Tout, int NC>
struct KFftStrided {
  static constexpr int kThreads = fsib::kThreads, kMinBlocks = 0;
  static constexpr bool kAnyGrid = false;
  static constexpr bool kMerge = std::is_same<T, float>::value;  // batches merge FP32 transforms only
  __device__ static void run(const C<Tin>* __restrict__ in, C<Tout>* __restrict__ out, int inner, int Nk,
              FftLen fl, Mult<T> mult, const C<T>* __restrict__ twg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = NC ? NC : fl.n, kP = fl.tile_p, lgP = __ffs(kP) - 1;
  C<T>* tw = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* a = tw + n;
  C<T>* b = a + n * kP;
  const int ntile = (inner + kP - 1) / kP;
  const long long co = blockIdx.x / ntile;       // component * outer + outer index
  const int q0 = (blockIdx.x % ntile) * kP;
  const int Lin = INV ? Nk : n, Lout = INV ? n : Nk;
  const int h = Nk / 2;
  const C<Tin>* src = in + co * (long long)Lin * inner;
  C<Tout>* dst = out + co * (long long)Lout * inner;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[fl.tw_off + i];
  for (int t = threadIdx.x; t < n * kP; t += blockDim.x) {
    const int p = t & (kP - 1), i = t >> lgP, q = q0 + p;
    C<T> v = mk<T>(T(0), T(0));
    if (q < inner) {
      if (!INV) {
        v = ccvt<T, Tin>(src[(long long)i * inner + q]);
      } else {
        // FFT position i holds mode i (i < N/2) or i - n (i > n - N/2); the rest is padding
        const int si = (i < h) ? i : ((i > n - h) ? i - (n - Nk) : -1);
        if (si >= 0) {
          v = ccvt<T, Tin>(src[(long long)si * inner + q]);
          T s = mult.scale;
          if (mult.dline) s *= mult.dline[si];
          if (mult.dplane) s *= mult.dplane[q];
          v = cscale<T>(v, s);
        }
      }
    }
    a[i * kP + p] = v;
  }
  __syncthreads();
  C<T>* r = fft_lines<T, INV, NC>(a, b, kP, 1, kP, true, fl, tw);
  if (!INV) {
    for (int t = threadIdx.x; t < Nk * kP; t += blockDim.x) {
      const int p = t & (kP - 1), io = t >> lgP, q = q0 + p;
      if (q >= inner) continue;
      C<T> v = mk<T>(T(0), T(0));
      if (io != h) {
        const int fi = (io < h) ? io : io + (n - Nk);
        v = r[fi * kP + p];
        T s = mult.scale;
        if (mult.dline) s *= mult.dline[io];
        if (mult.dplane) s *= mult.dplane[q];
        v = cscale<T>(v, s);
      }
      dst[(long long)io * inner + q] = ccvt<Tout, T>(v);
    }
  } else {
    for (int t = threadIdx.x; t < n * kP; t += blockDim.x) {
      const int p = t & (kP - 1), i = t >> lgP, q = q0 + p;
      if (q < inner) dst[(long long)i * inner + q] = ccvt<Tout, T>(r[i * kP + p]);
    }
  }
}
};

// ---------------------------------------------------------------------------
// Row passes: real rows (length n) <-> half spectra (N/2 modes)
// ---------------------------------------------------------------------------
template <typename T, int NC>
struct KRowsR2C {
  static constexpr int kThreads = fsib::kThreads, kMinBlocks = 0;
  static constexpr bool kAnyGrid = false;
  static constexpr bool kMerge = std::is_same<T, float>::value;  // batches merge FP32 transforms only
  __device__ static void run(const T* __restrict__ in, C<T>* __restrict__ out, long long npairs, int Nk, FftLen fl,
           const C<T>* __restrict__ twg, RowBands rb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = NC ? NC : fl.n, ls = n + 1, h = Nk / 2, kQrows = fl.rows_q;
  C<T>* tw = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* a = tw + n;
  C<T>* b = a + kQrows * ls;
  const long long pr0 = (long long)blockIdx.x * kQrows;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[fl.tw_off + i];
  for (int t = threadIdx.x; t < kQrows * n; t += blockDim.x) {
    const int p = t / n, x = t % n;
    const long long pr = pr0 + p;
    C<T> v = mk<T>(T(0), T(0));
    if (pr < npairs && rb.on(2 * pr)) v = mk<T>(in[(2 * pr) * n + x], in[(2 * pr + 1) * n + x]);
    a[p * ls + x] = v;
  }
  __syncthreads();
  C<T>* r = fft_lines<T, false, NC>(a, b, kQrows, ls, 1, false, fl, tw);
  for (int t = threadIdx.x; t < kQrows * h; t += blockDim.x) {
    const int p = t / h, k = t % h;
    const long long pr = pr0 + p;
    if (pr >= npairs) continue;
    const C<T> Z = r[p * ls + k];
    const C<T> Zc = cconj<T>(r[p * ls + (k == 0 ? 0 : n - k)]);
    const CPair<T> ab = untangle_pair<T>(Z, Zc);
    out[(2 * pr) * h + k] = ab.a;
    out[(2 * pr + 1) * h + k] = ab.b;
  }
}
};

// Build the packed complex spectrum Z = A + iB of two real rows from their half spectra.
template <typename T>
__device__ __forceinline__ C<T> pack_rows(const C<T>* __restrict__ A, const C<T>* __restrict__ B,
                                          int k, int n, int h) {
  if (k == 0) return mk<T>(A[0].x, B[0].x);  // Hermitian part of the m_x = 0 column
  if (k < h) {
    const C<T> a = A[k], bb = B[k];
    return mk<T>(ssub<T>(a.x, bb.y), sadd<T>(a.y, bb.x));
  }
  if (k > n - h) {
    const C<T> a = A[n - k], bb = B[n - k];  // conj(A) + i conj(B)
    return mk<T>(sadd<T>(a.x, bb.y), sadd<T>(-a.y, bb.x));
  }
  return mk<T>(T(0), T(0));
}

template <typename T, int NC>
struct KRowsC2R {
  static constexpr int kThreads = fsib::kThreads, kMinBlocks = 0;
  static constexpr bool kAnyGrid = false;
  static constexpr bool kMerge = std::is_same<T, float>::value;  // batches merge FP32 transforms only
  __device__ static void run(const C<T>* __restrict__ in, T* __restrict__ out, long long npairs, int Nk,
           FftLen fl, const C<T>* __restrict__ twg, RowBands rb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = NC ? NC : fl.n, ls = n + 1, h = Nk / 2, kQrows = fl.rows_q;
  C<T>* tw = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* a = tw + n;
  C<T>* b = a + kQrows * ls;
  const long long pr0 = (long long)blockIdx.x * kQrows;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[fl.tw_off + i];
  for (int t = threadIdx.x; t < kQrows * n; t += blockDim.x) {
    const int p = t / n, k = t % n;
    const long long pr = pr0 + p;
    C<T> v = mk<T>(T(0), T(0));
    if (pr < npairs) v = pack_rows<T>(in + (2 * pr) * h, in + (2 * pr + 1) * h, k, n, h);
    a[p * ls + k] = v;
  }
  __syncthreads();
  C<T>* r = fft_lines<T, true, NC>(a, b, kQrows, ls, 1, false, fl, tw);
  for (int t = threadIdx.x; t < kQrows * n; t += blockDim.x) {
    const int p = t / n, x = t % n;
    const long long pr = pr0 + p;
    if (pr >= npairs || !rb.on(2 * pr)) continue;
    const C<T> z = r[p * ls + x];
    out[(2 * pr) * n + x] = z.x;
    out[(2 * pr + 1) * n + x] = z.y;
  }
}
};

// ---------------------------------------------------------------------------
// Products of the velocity components on the dealiasing grid (three-halves rule):
// half spectra of u_a along x -> real rows u_a(x) -> u_a u_b -> half spectra of
// the d(d+1)/2 products. Input [d][nrows][N/2], output [d(d+1)/2][nrows][N/2],
// products ordered (xx, xy, xz, yy, yz, zz) in 3D and (xx, xy, yy) in 2D.
// ---------------------------------------------------------------------------
template <typename T, int NC>
struct KRowsProduct {
  static constexpr int kThreads = fsib::kThreads, kMinBlocks = 0;
  static constexpr bool kAnyGrid = false;
  static constexpr bool kMerge = std::is_same<T, float>::value;  // batches merge FP32 transforms only
  __device__ static void run(const C<T>* __restrict__ in, C<T>* __restrict__ out, int d, long long nrows,
               int Nk, FftLen fl, const C<T>* __restrict__ twg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = NC ? NC : fl.n, ls = n + 1, h = Nk / 2, kQrows = fl.rows_q;
  const int np = d * (d + 1) / 2;
  const long long npairs = nrows / 2;
  C<T>* tw = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* a = tw + n;
  C<T>* b = a + kQrows * np * ls;  // np >= d lines per row pair in each buffer
  const long long pr0 = (long long)blockIdx.x * kQrows;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[fl.tw_off + i];
  for (int t = threadIdx.x; t < kQrows * d * n; t += blockDim.x) {
    const int k = t % n, line = t / n, p = line / d, c = line % d;
    const long long pr = pr0 + p;
    C<T> v = mk<T>(T(0), T(0));
    if (pr < npairs) {
      const C<T>* base = in + ((long long)c * nrows + 2 * pr) * h;
      v = pack_rows<T>(base, base + h, k, n, h);
    }
    a[line * ls + k] = v;
  }
  __syncthreads();
  C<T>* r = fft_lines<T, true, NC>(a, b, kQrows * d, ls, 1, false, fl, tw);
  C<T>* o = (r == a) ? b : a;
  // products: re holds row 2p, im holds row 2p+1
  for (int t = threadIdx.x; t < kQrows * np * n; t += blockDim.x) {
    const int x = t % n, line = t / n, p = line / np, ab = line % np;
    int ca = 0, cb = ab;
    if (d == 3) {
      const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
      ca = ia[ab]; cb = ib[ab];
    } else {
      const int ia[3] = {0, 0, 1}, ib[3] = {0, 1, 1};
      ca = ia[ab]; cb = ib[ab];
    }
    const C<T> ua = r[(p * d + ca) * ls + x], ub = r[(p * d + cb) * ls + x];
    o[line * ls + x] = mk<T>(ua.x * ub.x, ua.y * ub.y);
  }
  __syncthreads();
  C<T>* f = fft_lines<T, false, NC>(o, r, kQrows * np, ls, 1, false, fl, tw);
  for (int t = threadIdx.x; t < kQrows * np * h; t += blockDim.x) {
    const int k = t % h, line = t / h, p = line / np, ab = line % np;
    const long long pr = pr0 + p;
    if (pr >= npairs) continue;
    const C<T> Z = f[line * ls + k];
    const C<T> Zc = cconj<T>(f[line * ls + (k == 0 ? 0 : n - k)]);
    C<T>* ob = out + ((long long)ab * nrows + 2 * pr) * h;
    const CPair<T> u = untangle_pair<T>(Z, Zc);
    ob[k] = u.a;
    ob[h + k] = u.b;
  }
}
};

// ---------------------------------------------------------------------------
// Row passes with the warp-level transform (lengths with a warp plan, wfft.cuh).
// Persistent blocks; each warp takes 32/L row pairs at a time, one per L lanes.
// Shared memory: the lane-ordered twiddle table, then per line its exchange buffer
// (and, in the product pass, the d inverse-transformed components).
// ---------------------------------------------------------------------------
// Packed line Z = A + iB of two half spectra in the warp transform's input order
// (element l + L i). In FP32 every load is issued before any element is assembled; the
// double-float version assembles element by element (its registers are the tighter limit).
template <typename T, int N>
__device__ __forceinline__ void wfft_load_packed(C<T> (&v)[wfft_M(N)], const C<T>* __restrict__ A,
                                                 const C<T>* __restrict__ B, int l, int h, bool valid) {
  constexpr int M = wfft_M(N), L = wfft_L(N), NN = wfft_n(N);
  if constexpr (sizeof(C<T>) != 8) {
#pragma unroll
    for (int i = 0; i < M; ++i) v[i] = valid ? pack_rows<T>(A, B, l + L * i, NN, h) : mk<T>(T(0), T(0));
  } else {
  C<T> a[M], b[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int k = l + L * i;
    const bool lo = k < h, hi = k > NN - h;
    const int kk = lo ? k : NN - k;
    const bool ok = valid && (lo || hi);
    a[i] = ok ? A[kk] : mk<T>(T(0), T(0));
    b[i] = ok ? B[kk] : mk<T>(T(0), T(0));
  }
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int k = l + L * i;
    if (k == 0) v[i] = mk<T>(a[i].x, b[i].x);                       // Hermitian part of m_x = 0
    else if (k < h) v[i] = mk<T>(a[i].x - b[i].y, a[i].y + b[i].x);   // A + iB
    else v[i] = mk<T>(a[i].x + b[i].y, b[i].x - a[i].y);              // conj(A) + i conj(B), or 0
  }
  }
}

template <typename T, int N>
__device__ __forceinline__ void wrows_c2r_body(const C<T>* __restrict__ in, T* __restrict__ out, long long npairs,
                                               int Nk, const C<T>* __restrict__ twg, RowBands rb) {
  constexpr int M = wfft_M(N), L = wfft_L(N), LPW = 32 / L, SL = wfft_stride(N, (int)sizeof(C<T>));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* tw = reinterpret_cast<C<T>*>(smem_raw);  // lane-ordered twiddles (wfft_tw_size(N))
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int l = lane % L, sub = lane / L;
  C<T>* buf = tw + wfft_tw_size(N) + (warp * LPW + sub) * SL;
  wfft_build_twiddles<T, N>(tw, twg);
  __syncthreads();
  const int h = Nk / 2;
  for (long long g = (long long)blockIdx.x * nwarp + warp; g * LPW < npairs; g += (long long)gridDim.x * nwarp) {
    const long long pr = g * LPW + sub;
    const bool valid = pr < npairs && rb.on(2 * pr);  // rows that no window reads are not written
    if (!__any_sync(0xffffffffu, valid)) continue;
    C<T> v[M];
    wfft_load_packed<T, N>(v, in + (2 * pr) * h, in + (2 * pr + 1) * h, l, h, valid);
    wfft<T, true, N>(v, buf, l, tw);
    if (valid) {
#pragma unroll
      for (int i = 0; i < M; ++i) {
        const int x = wfft_out_index<N>(l, i);
        out[(2 * pr) * N + x] = v[i].x;
        out[(2 * pr + 1) * N + x] = v[i].y;
      }
    }
  }
}

// FP32 lines ask for three resident blocks per SM (the pass is bound by the transforms' latency
// once the row bands cut its traffic); double-float lines keep the compiler's register choice
// (a minimum-blocks hint of one raises it).
template <typename T, int N>
struct KWRowsC2R {
  static constexpr int kThreads = 256, kMinBlocks = 3;
  static constexpr bool kAnyGrid = true;
  static constexpr bool kMerge = std::is_same<T, float>::value;  // batches merge FP32 transforms only
  __device__ static void run(const C<T>* __restrict__ in, T* __restrict__ out, long long npairs, int Nk,
            const C<T>* __restrict__ twg, RowBands rb) {
  wrows_c2r_body<T, N>(in, out, npairs, Nk, twg, rb);
}
};
template <typename T, int N>
struct KWRowsC2RDD {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  static constexpr bool kMerge = false;  // batches merge FP32 transforms only
  __device__ static void run(const C<T>* __restrict__ in, T* __restrict__ out, long long npairs, int Nk,
               const C<T>* __restrict__ twg, RowBands rb) {
  wrows_c2r_body<T, N>(in, out, npairs, Nk, twg, rb);
}
};
template <typename T, int N>
using WRowsC2R = std::conditional_t<sizeof(C<T>) == 8, KWRowsC2R<T, N>, KWRowsC2RDD<T, N>>;

// Untangle the spectra of two real rows packed as Z = A + iB: A[k] = (Z[k] + conj Z[N-k]) / 2,
// B[k] = (Z[k] - conj Z[N-k]) / 2i, for the kept modes k < h. v holds Z in output order.
template <typename T, int N>
__device__ __forceinline__ void wfft_untangle(const C<T> (&v)[wfft_M(N)], C<T>* buf, int l, bool valid, int h,
                                              C<T>* __restrict__ outA, C<T>* __restrict__ outB) {
  constexpr int M = wfft_M(N), L = wfft_L(N), NN = wfft_n(N);
#pragma unroll
  for (int i = 0; i < M; ++i) buf[wfft_out_index<N>(l, i)] = v[i];
  __syncwarp();
  if (valid) {
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const int k = l + L * i;
      if (k < h) {
        const C<T> Z = buf[k];
        const C<T> Zc = cconj<T>(buf[k == 0 ? 0 : NN - k]);
        const CPair<T> u = untangle_pair<T>(Z, Zc);
        outA[k] = u.a;
        outB[k] = u.b;
      }
    }
  }
  __syncwarp();
}

// The same for Z in strided order (lane l holds Z[l + L i] in v[i], as wfft_fwd_transposed leaves
// it): only the partners Z[N - k] of the kept modes, Z[j] for j >= N - h, go through buf.
template <typename T, int PC>
__device__ __forceinline__ void wfft_untangle_strided(const C<T> (&v)[wfft_M(PC)], C<T>* buf, int l, bool valid,
                                                      int h, C<T>* __restrict__ outA, C<T>* __restrict__ outB) {
  constexpr int M = wfft_M(PC), L = wfft_L(PC), NN = wfft_n(PC);
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int j = l + L * i;
    if (j >= NN - h) buf[j - (NN - h)] = v[i];
  }
  __syncwarp();
  if (valid) {
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const int k = l + L * i;
      if (k < h) {
        const C<T> Z = v[i];
        const C<T> Zc = cconj<T>(k == 0 ? Z : buf[h - k]);
        const CPair<T> u = untangle_pair<T>(Z, Zc);
        outA[k] = u.a;
        outB[k] = u.b;
      }
    }
  }
  __syncwarp();
}

template <typename T, int N>
__device__ __forceinline__ void wrows_r2c_body(const T* __restrict__ in, C<T>* __restrict__ out, long long npairs,
                                               int Nk, const C<T>* __restrict__ twg, RowBands rb) {
  constexpr int M = wfft_M(N), L = wfft_L(N), LPW = 32 / L, SL = wfft_stride(N, (int)sizeof(C<T>));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* tw = reinterpret_cast<C<T>*>(smem_raw);  // lane-ordered twiddles (wfft_tw_size(N))
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int l = lane % L, sub = lane / L;
  C<T>* buf = tw + wfft_tw_size(N) + (warp * LPW + sub) * SL;
  wfft_build_twiddles<T, N>(tw, twg);
  __syncthreads();
  const int h = Nk / 2;
  for (long long g = (long long)blockIdx.x * nwarp + warp; g * LPW < npairs; g += (long long)gridDim.x * nwarp) {
    const long long pr = g * LPW + sub;
    const bool valid = pr < npairs;
    const bool on = valid && rb.on(2 * pr);  // both rows of a pair lie in one band
    if (!__any_sync(0xffffffffu, on)) {      // every row of this warp is zero: so is its spectrum
      if (valid) {
#pragma unroll
        for (int i = 0; i < M; ++i) {
          const int k = l + L * i;
          if (k < h) { out[(2 * pr) * h + k] = mk<T>(T(0), T(0)); out[(2 * pr + 1) * h + k] = mk<T>(T(0), T(0)); }
        }
      }
      continue;
    }
    C<T> v[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const int x = l + L * i;
      v[i] = on ? mk<T>(in[(2 * pr) * N + x], in[(2 * pr + 1) * N + x]) : mk<T>(T(0), T(0));
    }
    wfft<T, false, N>(v, buf, l, tw);
    wfft_untangle<T, N>(v, buf, l, valid, h, out + (2 * pr) * h, out + (2 * pr + 1) * h);
  }
}

// FP32 lines: three resident blocks per SM, as for the c2r pass; double-float lines keep the
// compiler's register choice.
template <typename T, int N>
struct KWRowsR2C {
  static constexpr int kThreads = 256, kMinBlocks = 3;
  static constexpr bool kAnyGrid = true;
  static constexpr bool kMerge = std::is_same<T, float>::value;  // batches merge FP32 transforms only
  __device__ static void run(const T* __restrict__ in, C<T>* __restrict__ out, long long npairs, int Nk,
            const C<T>* __restrict__ twg, RowBands rb) {
  wrows_r2c_body<T, N>(in, out, npairs, Nk, twg, rb);
}
};
template <typename T, int N>
struct KWRowsR2CDD {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  static constexpr bool kMerge = false;  // batches merge FP32 transforms only
  __device__ static void run(const T* __restrict__ in, C<T>* __restrict__ out, long long npairs, int Nk,
               const C<T>* __restrict__ twg, RowBands rb) {
  wrows_r2c_body<T, N>(in, out, npairs, Nk, twg, rb);
}
};
template <typename T, int N>
using WRowsR2C = std::conditional_t<sizeof(C<T>) == 8, KWRowsR2C<T, N>, KWRowsR2CDD<T, N>>;

// Schedule of the product pass (see k_wrows_product): kind 0 = inverse transform of
// component a into slot b; kind 1 = product ab of slots a and b; x = slot used for the
// transform's exchanges (encoded kind | a << 4 | b << 8 | x << 12 | ab << 16).
static __constant__ int kProdSched3[9] = {0 | 0 << 4 | 0 << 8 | 2 << 12,            1 << 4 | 1 << 8 | 2 << 12,
                                    1 | 0 << 4 | 0 << 8 | 2 << 12 | 0 << 16,  1 | 0 << 4 | 1 << 8 | 2 << 12 | 1 << 16,
                                    1 | 1 << 4 | 1 << 8 | 2 << 12 | 3 << 16,  0 | 2 << 4 | 2 << 8 | 2 << 12,
                                    1 | 0 << 4 | 2 << 8 | 0 << 12 | 2 << 16,  1 | 1 << 4 | 2 << 8 | 1 << 12 | 4 << 16,
                                    1 | 2 << 4 | 2 << 8 | 2 << 12 | 5 << 16};
static __constant__ int kProdSched2[5] = {0 | 0 << 4 | 0 << 8 | 2 << 12,            1 << 4 | 1 << 8 | 2 << 12,
                                    1 | 0 << 4 | 0 << 8 | 2 << 12 | 0 << 16,  1 | 0 << 4 | 1 << 8 | 2 << 12 | 1 << 16,
                                    1 | 1 << 4 | 1 << 8 | 2 << 12 | 2 << 16};

// Schedule of the product pass for one-exchange plans (see k_wrows_product): kind 0 = inverse
// transform of component a into the registers u, stored to slot stash - 1 as well when stash > 0;
// kind 1 = product of u with slot src - 1 (with u itself when src = 0) into output ab
// (encoded kind | a << 4 | stash << 8 | src << 12 | ab << 16).
static __constant__ int kProdSchedT3[9] = {0 | 0 << 4 | 1 << 8, 1 | 0 << 12 | 0 << 16, 0 | 1 << 4 | 2 << 8,
                                           1 | 1 << 12 | 1 << 16, 1 | 0 << 12 | 3 << 16, 0 | 2 << 4,
                                           1 | 1 << 12 | 2 << 16, 1 | 2 << 12 | 4 << 16, 1 | 0 << 12 | 5 << 16};
static __constant__ int kProdSchedT2[5] = {0 | 0 << 4 | 1 << 8, 1 | 0 << 12 | 0 << 16, 0 | 1 << 4,
                                           1 | 1 << 12 | 1 << 16, 1 | 0 << 12 | 2 << 16};

// Products of the velocity components (three-halves rule), one row pair per L lanes, in
// three line buffers S0..S2 of shared memory: u_x and u_y are transformed into S0 and S1
// (exchanging through S2) and give xx, xy, yy (exchanging through S2); u_z then goes to S2,
// and xz, yz, zz each exchange through the buffer of a component they no longer need (S0,
// S1, S2), which takes three line buffers per row pair instead of four. Blocks of 128 threads.
// Warp plan of the product pass: FP32 lines of 96 and 192 points take the one-exchange plans
// (the pass is bound by its shared-memory exchanges), double-float lines the default ones.
template <typename T, int N>
constexpr int prod_plan() {
  return (std::is_same<T, float>::value && wfft_has(N | kOneExchange)) ? (N | kOneExchange) : N;
}

template <typename T, int N>
struct KWRowsProduct {
  static constexpr int kThreads = 128, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  static constexpr bool kMerge = std::is_same<T, float>::value;  // batches merge FP32 transforms only
  __device__ static void run(const C<T>* __restrict__ in, C<T>* __restrict__ out, int d, long long nrows, int Nk,
                const C<T>* __restrict__ twg) {
  constexpr int PC = prod_plan<T, N>();
  constexpr int M = wfft_M(PC), L = wfft_L(PC), LPW = 32 / L, SL = wfft_stride(PC, (int)sizeof(C<T>));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* tw = reinterpret_cast<C<T>*>(smem_raw);  // lane-ordered twiddles (wfft_tw_size(PC))
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int l = lane % L, sub = lane / L;
  if constexpr (wfft_one(PC)) {
    // One-exchange plans: the inverse transforms leave u_a in registers in the plan's output
    // order; the products are formed there and go forward through wfft_fwd_transposed, which
    // reads that order, then through the untangle of the strided order. Shared memory carries
    // the transforms' exchanges (S2) and u_x, u_y for the products that pair them with a later
    // component (S0, S1), not both factors of every product.
    C<T>* twt = tw + wfft_tw_size(PC);  // w^{n1 k2} of the transposed transform
    C<T>* S = twt + wfft_twt_size<PC>() + (warp * LPW + sub) * 3 * SL;
    C<T>* X = S + 2 * SL;
    wfft_build_twiddles<T, PC>(tw, twg);
    wfft_build_twiddles_t<T, PC>(twt, twg);
    __syncthreads();
    const int h = Nk / 2;
    const long long npairs = nrows / 2;
    for (long long g = (long long)blockIdx.x * nwarp + warp; g * LPW < npairs; g += (long long)gridDim.x * nwarp) {
      const long long pr = g * LPW + sub;
      const bool valid = pr < npairs;
      // u_a of rows 2p (real part) and 2p + 1 (imaginary part), inverse = conj F conj
      auto inverse = [&](int a, C<T> (&u)[M]) {
        const C<T>* base = in + ((long long)a * nrows + 2 * pr) * h;
        wfft_load_packed<T, PC>(u, base, base + h, l, h, valid);
#pragma unroll
        for (int i = 0; i < M; ++i) u[i] = cconj<T>(u[i]);
        wfft<T, false, PC>(u, X, l, tw);
#pragma unroll
        for (int i = 0; i < M; ++i) u[i] = cconj<T>(u[i]);
      };
      auto forward = [&](C<T> (&v)[M], int ab) {
        wfft_fwd_transposed<T, PC>(v, X, l, twt);
        C<T>* ob = out + ((long long)ab * nrows + 2 * pr) * h;
        wfft_untangle_strided<T, PC>(v, X, l, valid, h, ob, ob + h);
      };
      // one component in registers at a time (u); u_x and u_y also go to this lane's slots of S0
      // and S1, from which the products that pair them with a later component read them. A loop
      // over the schedule holds one copy of each transform's code (the pass is short enough that
      // unrolled copies overflow the instruction cache).
      C<T> u[M], v[M];
      const int nst = (d == 3) ? 9 : 5;
#pragma unroll 1
      for (int q = 0; q < nst; ++q) {
        const int e = (d == 3) ? kProdSchedT3[q] : kProdSchedT2[q];
        const int kind = e & 15, a = (e >> 4) & 15, stash = ((e >> 8) & 15) - 1, src = ((e >> 12) & 15) - 1;
        if (kind == 0) {
          inverse(a, u);
          if (stash >= 0) {
#pragma unroll
            for (int i = 0; i < M; ++i) S[stash * SL + i * L + l] = u[i];
          }
        } else {
#pragma unroll
          for (int i = 0; i < M; ++i) {
            const C<T> f = src < 0 ? u[i] : S[src * SL + i * L + l];
            v[i] = mk<T>(f.x * u[i].x, f.y * u[i].y);
          }
          forward(v, e >> 16);
        }
      }
    }
    return;
  }
  C<T>* S = tw + wfft_tw_size(PC) + (warp * LPW + sub) * 3 * SL;  // S0, S1, S2
  wfft_build_twiddles<T, PC>(tw, twg);
  __syncthreads();
  const int h = Nk / 2;
  const long long npairs = nrows / 2;
  const int nst = (d == 3) ? 9 : 5;
  for (long long g = (long long)blockIdx.x * nwarp + warp; g * LPW < npairs; g += (long long)gridDim.x * nwarp) {
    const long long pr = g * LPW + sub;
    const bool valid = pr < npairs;
#pragma unroll 1
    for (int q = 0; q < nst; ++q) {
      const int e = (d == 3) ? kProdSched3[q] : kProdSched2[q];
      const int kind = e & 15, sa = (e >> 4) & 15, sb = (e >> 8) & 15, x = (e >> 12) & 15, ab = e >> 16;
      C<T>* X = S + x * SL;
      C<T> v[M];
      // One forward transform serves both directions (the inverse is conj(F(conj(x)))), so
      // the loop holds a single copy of the transform code.
      if (kind == 0) {
        const C<T>* base = in + ((long long)sa * nrows + 2 * pr) * h;
        wfft_load_packed<T, PC>(v, base, base + h, l, h, valid);
#pragma unroll
        for (int i = 0; i < M; ++i) v[i] = cconj<T>(v[i]);
      } else {
        // the real part holds row 2p, the imaginary part row 2p+1
#pragma unroll
        for (int i = 0; i < M; ++i) {
          const C<T> ua = S[sa * SL + l + L * i], ub = S[sb * SL + l + L * i];
          v[i] = mk<T>(ua.x * ub.x, ua.y * ub.y);
        }
        __syncwarp();  // the exchange slot may hold a factor
      }
      wfft<T, false, PC>(v, X, l, tw);
      if (kind == 0) {
#pragma unroll
        for (int i = 0; i < M; ++i) S[sb * SL + wfft_out_index<PC>(l, i)] = cconj<T>(v[i]);
        __syncwarp();
      } else {
        C<T>* ob = out + ((long long)ab * nrows + 2 * pr) * h;
        wfft_untangle<T, PC>(v, X, l, valid, h, ob, ob + h);
      }
    }
  }
}
};

// ---------------------------------------------------------------------------
// Strided pass in two register stages, N = R1 x R2 (radices up to 16; the lengths below).
// A block holds a tile of S2P adjacent lines (16 x S2P threads); line p of the tile is
// column p of a [N][S2P] shared array, so the threads of a warp (consecutive lines, then
// consecutive butterflies) touch consecutive addresses. Stage 1 (radix R1, no twiddles)
// reads x[j + r N/R1] and writes y[j R1 + r] after a barrier (in place); stage 2 (radix R2)
// reads y[j + r R1], multiplies by w^{j r} and writes back to the same places, which leaves
// the transform in natural order. Loads, pruning, padding and multipliers as in k_fft_strided.
// ---------------------------------------------------------------------------
constexpr bool s2_has(int n) {
  return n == 48 || n == 64 || n == 72 || n == 96 || n == 128 || n == 144 || n == 192 || n == 256;
}
constexpr int s2_R1(int n) {
  return n == 48 ? 12 : n == 64 ? 8 : n == 72 ? 8 : n == 96 ? 12 : n == 128 ? 16 : n == 144 ? 12 : 16;
}
constexpr int s2_P(int E) { return E == 8 ? 16 : 8; }  // lines per tile: 128-byte rows

template <typename T, bool INV, typename Tin, typename Tout, int N>
__device__ __forceinline__ void fft_s2_body(const C<Tin>* __restrict__ in, C<Tout>* __restrict__ out, int inner,
                                            int Nk, int ntile, Mult<T> mult, const C<T>* __restrict__ twg,
                                            ZSkip zs) {
  constexpr int P = s2_P((int)sizeof(C<T>)), R1 = s2_R1(N), R2 = N / R1, NT = 16 * P;
  constexpr int RM = R1 > R2 ? R1 : R2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* tw = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* tile = tw + N;  // [N][P]
  const long long co = blockIdx.x / ntile;
  const int q0 = (blockIdx.x % ntile) * P;
  const int Lin = INV ? Nk : N, Lout = INV ? N : Nk;
  const int h = Nk / 2;
  const C<Tin>* src = in + co * (long long)Lin * inner;
  C<Tout>* dst = out + co * (long long)Lout * inner;
  if (zs.flag) {  // a z-slab that no window reaches (uniform across the block)
    const int bz = (int)(co % zs.outer) / zs.b;
    bool any = false;
    for (int by = 0; by < zs.nby; ++by) any |= zs.flag[bz * zs.nby + by] != 0;
    if (!any) {
      if (zs.zero)
        for (int t = threadIdx.x; t < Lout * P; t += NT) {
          const int i = t / P, q = q0 + t % P;
          if (q < inner) dst[(long long)i * inner + q] = C<Tout>{};
        }
      return;
    }
  }
  for (int i = threadIdx.x; i < N; i += NT) tw[i] = twg[i];
  {
    // every load of this thread is issued before the first shared-memory store
    constexpr int NL = (N * P + NT - 1) / NT;  // N P need not be a multiple of the block size
    const int p = threadIdx.x % P, q = q0 + p;
    const bool qok = q < inner;
    C<Tin> raw[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int i = (threadIdx.x + k * NT) / P;
      const int si = (i >= N) ? -1 : INV ? ((i < h) ? i : ((i > N - h) ? i - (N - Nk) : -1)) : i;
      raw[k] = (qok && si >= 0) ? src[(long long)si * inner + q] : C<Tin>{};
    }
#pragma unroll
    constexpr bool kHoist = std::is_same<T, float>::value;  // FP32 lines: the plane factor once a thread
    const T dpq = (kHoist && INV && qok && mult.dplane) ? mult.dplane[q] : T(1);
    for (int k = 0; k < NL; ++k) {
      const int t = threadIdx.x + k * NT, i = t / P;
      if (t >= N * P) break;
      C<T> v = ccvt<T, Tin>(raw[k]);
      if (INV) {
        const int si = (i < h) ? i : ((i > N - h) ? i - (N - Nk) : -1);
        if (qok && si >= 0) {
          T sc = mult.dline ? mult.scale * mult.dline[si] : mult.scale;
          if (mult.dplane) sc = sc * (kHoist ? dpq : mult.dplane[q]);
          v = cscale<T>(v, sc);
        } else {
          v = mk<T>(T(0), T(0));
        }
      }
      tile[t] = v;  // t = i * P + p
    }
  }
  __syncthreads();
  const int p = threadIdx.x % P, j = threadIdx.x / P;  // j < 16
  C<T> v[RM];
  if (j < N / R1) {
#pragma unroll
    for (int r = 0; r < R1; ++r) v[r] = tile[(j + r * (N / R1)) * P + p];
    dft_r<T, INV, R1>(v);
  }
  __syncthreads();
  if (j < N / R1) {
#pragma unroll
    for (int r = 0; r < R1; ++r) tile[(j * R1 + r) * P + p] = v[r];
  }
  __syncthreads();
  if (j < R1) {
#pragma unroll
    for (int r = 0; r < R2; ++r) v[r] = tile[(j + r * R1) * P + p];
#pragma unroll
    for (int r = 1; r < R2; ++r) {
      C<T> w = tw[j * r];
      if (INV) w = cconj<T>(w);
      v[r] = cmul<T>(v[r], w);
    }
    dft_r<T, INV, R2>(v);
#pragma unroll
    for (int r = 0; r < R2; ++r) tile[(j + r * R1) * P + p] = v[r];
  }
  __syncthreads();
  if constexpr (std::is_same<T, float>::value) {
    // a thread keeps its line (t mod P is fixed, NT being a multiple of P) and steps 16 rows
    {
      const int pp = threadIdx.x % P, q = q0 + pp;
      if (q < inner) {
        C<Tout>* dq = dst + q;
        if (!INV) {
          const T dpq = mult.dplane ? mult.dplane[q] : T(1);  // (scale dline) dplane, as in the inverse
          for (int io = threadIdx.x / P; io < Nk; io += NT / P) {
            C<T> v = mk<T>(T(0), T(0));
            if (io != h) {
              const int fi = (io < h) ? io : io + (N - Nk);
              T sc = mult.dline ? mult.scale * mult.dline[io] : mult.scale;
              if (mult.dplane) sc = sc * dpq;
              v = cscale<T>(tile[fi * P + pp], sc);
            }
            dq[(long long)io * inner] = ccvt<Tout, T>(v);
          }
        } else {
          for (int i = threadIdx.x / P; i < N; i += NT / P) dq[(long long)i * inner] = ccvt<Tout, T>(tile[i * P + pp]);
        }
      }
    }
  } else {  // double-float and double lines measured faster with the per-element form
    if (!INV) {
      for (int t = threadIdx.x; t < Nk * P; t += NT) {
        const int pp = t % P, io = t / P, q = q0 + pp;
        if (q >= inner) continue;
        C<T> v = mk<T>(T(0), T(0));
        if (io != h) {
          const int fi = (io < h) ? io : io + (N - Nk);
          T sc = mult.scale;
          if (mult.dline) sc *= mult.dline[io];
          if (mult.dplane) sc *= mult.dplane[q];
          v = cscale<T>(tile[fi * P + pp], sc);
        }
        dst[(long long)io * inner + q] = ccvt<Tout, T>(v);
      }
    } else {
      for (int t = threadIdx.x; t < N * P; t += NT) {
        const int pp = t % P, i = t / P, q = q0 + pp;
        if (q < inner) dst[(long long)i * inner + q] = ccvt<Tout, T>(tile[t]);
      }
    }
  }
}

// FP32 tiles ask for three resident blocks per SM (at most 80 registers a thread): the
// strided passes wait on memory, and the third block hides more of it. Double-float tiles
// keep the compiler's own register choice (a minimum-blocks hint of one raises it).
template <typename T, bool INV, typename Tin, typename Tout, int N>
struct KFftS2 {
  static constexpr int kThreads = 16 * s2_P(8), kMinBlocks = 3;
  static constexpr bool kAnyGrid = false;
  static constexpr bool kMerge = std::is_same<T, float>::value;  // batches merge FP32 transforms only
  __device__ static void run(const C<Tin>* __restrict__ in, C<Tout>* __restrict__ out, int inner, int Nk, int ntile,
         Mult<T> mult, const C<T>* __restrict__ twg, ZSkip zs) {
  fft_s2_body<T, INV, Tin, Tout, N>(in, out, inner, Nk, ntile, mult, twg, zs);
}
};
template <typename T, bool INV, typename Tin, typename Tout, int N>
struct KFftS2DD {
  static constexpr int kThreads = 16 * s2_P(16), kMinBlocks = 0;
  static constexpr bool kAnyGrid = false;
  static constexpr bool kMerge = false;  // batches merge FP32 transforms only
  __device__ static void run(const C<Tin>* __restrict__ in, C<Tout>* __restrict__ out, int inner, int Nk, int ntile,
            Mult<T> mult, const C<T>* __restrict__ twg, ZSkip zs) {
  fft_s2_body<T, INV, Tin, Tout, N>(in, out, inner, Nk, ntile, mult, twg, zs);
}
};
template <typename T, bool INV, typename Tin, typename Tout, int N>
using FftS2 = std::conditional_t<sizeof(C<T>) == 8, KFftS2<T, INV, Tin, Tout, N>, KFftS2DD<T, INV, Tin, Tout, N>>;

// Persistent grid of a warp-transform kernel: resident blocks per SM times the SMs,
// or fewer when there is less work.
static unsigned wrows_grid(const void* kern, int threads, size_t smem, long long groups) {
  int dev = 0, sms = 1, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess || per < 1) per = 1;
  const long long need = (groups + threads / 32 - 1) / (threads / 32);
  return (unsigned)std::max<long long>(1, std::min<long long>(need, (long long)per * sms));
}

// A warp-level row pass runs one chain of transforms per warp. With fewer warps than this
// (small 2D grids) most of the GPU idles on that chain, and the block-level kernels, which
// spread each row pair over a whole block, finish first; they then take one row pair per
// block when the pairs do not fill the SMs twice.
constexpr long long kWarpRowsMin = 128;
static FftLen small_rows(const FftLen& fl, long long npairs) {
  static const int sms = [] {
    int dev = 0, n = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
  }();
  FftLen f = fl;
  if (npairs < 2LL * sms * f.rows_q) f.rows_q = 1;
  return f;
}

// ---------------------------------------------------------------------------
// Launchers: each dispatches on the FFT length (a compile-time kernel for the
// lengths in FSIB_FFT_SIZES, the runtime-length kernel otherwise).
// ---------------------------------------------------------------------------
// Calls f(std::integral_constant<int, NC>) with NC = n for a specialised length, else NC = 0.
template <typename F>
static void with_fft_len(int n, F&& f) {
  switch (n) {
#define FSIB_CASE(K) case K: f(std::integral_constant<int, K>()); return;
    FSIB_FFT_SIZES(FSIB_CASE)
#undef FSIB_CASE
    default: f(std::integral_constant<int, 0>()); return;
  }
}

// Shared memory of the block-level kernels: the twiddles (n) and two buffers of `lines` lines
// of `ls` elements. Long lines take fewer lines per block, down to the fewest that fit the
// opt-in limit (a power of two for the strided tiles); every length up to the largest
// transform of a plan fits with one line pair per block.
template <typename T>
static int fit_lines(int want, int n, int lines_per_unit, int ls, bool pow2) {
  int q = std::max(1, want);
  while (q > 1 && sizeof(C<T>) * ((size_t)n + 2 * (size_t)q * lines_per_unit * ls) > smem_optin())
    q = pow2 ? q / 2 : q - 1;
  return q;
}

template <typename T, typename Tin, typename Tout>
void launch_fft_strided(const C<Tin>* in, C<Tout>* out, int ncomp, int outer, int inner, int Nk,
                        const FftLen& flr, bool inverse, Mult<T> mult, const C<T>* tw,
                        cudaStream_t st, ZSkip zs) {
  FftLen fl = flr;
  fl.tile_p = fit_lines<T>(fl.tile_p, fl.n, 1, fl.n, true);
  const int kP = fl.tile_p;
  const int ntile = (inner + kP - 1) / kP;
  const long long blocks = (long long)ncomp * outer * ntile;
  const size_t smem = sizeof(C<T>) * (size_t)(fl.n + 2 * fl.n * kP);
  // A pass that converts between types runs in one direction only: a forward pass
  // may narrow its output (Tout != T), an inverse pass may widen its input (Tin != T).
  // The unused direction keeps the runtime-length kernel.
  constexpr bool fwd_only = !std::is_same<Tout, T>::value, inv_only = !std::is_same<Tin, T>::value;
  with_fft_len(fl.n, [&](auto nc) {
    constexpr int NC = decltype(nc)::value;
    constexpr int NCI = fwd_only ? 0 : NC, NCF = inv_only ? 0 : NC;
    if constexpr (s2_has(NC)) {
      constexpr int P2 = s2_P((int)sizeof(C<T>));
      const int nt2 = (inner + P2 - 1) / P2;
      const long long blocks2 = (long long)ncomp * outer * nt2;
      const size_t smem2 = sizeof(C<T>) * (size_t)(NC + NC * P2);
      if (inverse && !fwd_only) {
        using K = FftS2<T, true, Tin, Tout, NC>;
        raise_smem_limit(kernel_ptr<K>());
        launch<K>((unsigned)blocks2, 16 * P2, smem2, st, in, out, inner, Nk, nt2, mult, tw + fl.tw_off, zs);
        return;
      }
      if (!inverse && !inv_only) {
        using K = FftS2<T, false, Tin, Tout, NC>;
        raise_smem_limit(kernel_ptr<K>());
        launch<K>((unsigned)blocks2, 16 * P2, smem2, st, in, out, inner, Nk, nt2, mult, tw + fl.tw_off, zs);
        return;
      }
    }
    if (inverse) {
      using K = KFftStrided<T, true, Tin, Tout, NCI>;
      raise_smem_limit(kernel_ptr<K>());
      launch<K>((unsigned)blocks, kThreads, smem, st, in, out, inner, Nk, fl, mult, tw);
    } else {
      using K = KFftStrided<T, false, Tin, Tout, NCF>;
      raise_smem_limit(kernel_ptr<K>());
      launch<K>((unsigned)blocks, kThreads, smem, st, in, out, inner, Nk, fl, mult, tw);
    }
  });
}

template <typename T>
void launch_fft_rows_r2c(const T* in, C<T>* out, long long nrows, int Nk, const FftLen& fl,
                         const C<T>* tw, cudaStream_t st, RowBands rb) {
  const long long npairs = nrows / 2;
  FftLen fs = small_rows(fl, npairs);
  fs.rows_q = fit_lines<T>(fs.rows_q, fl.n, 1, fl.n + 1, false);
  const int kQrows = fs.rows_q;
  const long long blocks = (npairs + kQrows - 1) / kQrows;
  const size_t smem = sizeof(C<T>) * (size_t)(fl.n + 2 * kQrows * (fl.n + 1));
  with_fft_len(fl.n, [&](auto nc) {
    constexpr int NC = decltype(nc)::value;
    constexpr int LPW = wfft_has(NC) ? 32 / wfft_L(NC) : 1;
    if constexpr (wfft_has(NC)) if ((npairs + LPW - 1) / LPW >= kWarpRowsMin) {
      const size_t ws = sizeof(C<T>) * (size_t)(wfft_tw_size(NC) + 8 * LPW * wfft_stride(NC, (int)sizeof(C<T>)));
      using K = WRowsR2C<T, NC>;
      raise_smem_limit(kernel_ptr<K>());
      launch<K>(wrows_grid(kernel_ptr<K>(), 256, ws, (npairs + LPW - 1) / LPW), 256, ws, st, in, out, npairs, Nk,
                tw + fl.tw_off, rb);
      return;
    }
    using K = KRowsR2C<T, decltype(nc)::value>;
    raise_smem_limit(kernel_ptr<K>());
    launch<K>((unsigned)blocks, kThreads, smem, st, in, out, npairs, Nk, fs, tw, rb);
  });
}

template <typename T>
void launch_fft_rows_c2r(const C<T>* in, T* out, long long nrows, int Nk, const FftLen& fl,
                         const C<T>* tw, cudaStream_t st, RowBands rb) {
  const long long npairs = nrows / 2;
  FftLen fs = small_rows(fl, npairs);
  fs.rows_q = fit_lines<T>(fs.rows_q, fl.n, 1, fl.n + 1, false);
  const int kQrows = fs.rows_q;
  const long long blocks = (npairs + kQrows - 1) / kQrows;
  const size_t smem = sizeof(C<T>) * (size_t)(fl.n + 2 * kQrows * (fl.n + 1));
  with_fft_len(fl.n, [&](auto nc) {
    constexpr int NC = decltype(nc)::value;
    constexpr int LPW = wfft_has(NC) ? 32 / wfft_L(NC) : 1;
    if constexpr (wfft_has(NC)) if ((npairs + LPW - 1) / LPW >= kWarpRowsMin) {
      const size_t ws = sizeof(C<T>) * (size_t)(wfft_tw_size(NC) + 8 * LPW * wfft_stride(NC, (int)sizeof(C<T>)));
      using K = WRowsC2R<T, NC>;
      raise_smem_limit(kernel_ptr<K>());
      launch<K>(wrows_grid(kernel_ptr<K>(), 256, ws, (npairs + LPW - 1) / LPW), 256, ws, st, in, out, npairs, Nk,
                tw + fl.tw_off, rb);
      return;
    }
    using K = KRowsC2R<T, decltype(nc)::value>;
    raise_smem_limit(kernel_ptr<K>());
    launch<K>((unsigned)blocks, kThreads, smem, st, in, out, npairs, Nk, fs, tw, rb);
  });
}

template <typename T>
void launch_rows_product(const C<T>* in, C<T>* out, int d, long long nrows, int Nk,
                         const FftLen& fl, const C<T>* tw, cudaStream_t st) {
  const long long npairs = nrows / 2;
  const int lp = (d == 3) ? 6 : 3;  // lines per row pair: max(d, d(d+1)/2)
  FftLen fs = small_rows(fl, npairs);
  fs.rows_q = fit_lines<T>(fs.rows_q, fl.n, lp, fl.n + 1, false);
  const int kQrows = fs.rows_q;
  const long long blocks = (npairs + kQrows - 1) / kQrows;
  const size_t smem = sizeof(C<T>) * (size_t)(fl.n + 2 * kQrows * lp * (fl.n + 1));
  with_fft_len(fl.n, [&](auto nc) {
    constexpr int NC = decltype(nc)::value;
    constexpr int PC = wfft_has(NC) ? prod_plan<T, NC>() : NC;
    constexpr int LPW = wfft_has(NC) ? 32 / wfft_L(PC) : 1;
    if constexpr (wfft_has(NC)) if ((npairs + LPW - 1) / LPW >= kWarpRowsMin) {
      // Blocks of two warps measured no faster: double-float length 96 (five resident blocks instead
      // of two) 127.0 against 127.4 us a step, FP32 one-exchange length 192 80.6 against 74.6 us.
      // Blocks of three warps for the one-exchange plans (three resident blocks, nine warps an SM
      // instead of eight) measured slower too: 191.8 against 143.3 us a step at length 192.
      constexpr int PT = 128;
      const size_t ws = sizeof(C<T>) * (size_t)(wfft_tw_size(PC) + wfft_twt_size<PC>() +
                                                (PT / 32) * LPW * 3 * wfft_stride(PC, (int)sizeof(C<T>)));
      using K = KWRowsProduct<T, NC>;
      raise_smem_limit(kernel_ptr<K>());
      launch<K>(wrows_grid(kernel_ptr<K>(), PT, ws, (npairs + LPW - 1) / LPW), PT, ws, st, in, out, d, nrows, Nk,
                tw + fl.tw_off);
      return;
    }
    using K = KRowsProduct<T, decltype(nc)::value>;
    raise_smem_limit(kernel_ptr<K>());
    launch<K>((unsigned)blocks, kThreads, smem, st, in, out, d, nrows, Nk, fs, tw);
  });
}

#define FSIB_FFT_INST_R(T)                                                                       \
  template void launch_fft_rows_r2c<T>(const T*, C<T>*, long long, int, const FftLen&,           \
                                       const C<T>*, cudaStream_t, RowBands);                     \
  template void launch_fft_rows_c2r<T>(const C<T>*, T*, long long, int, const FftLen&,           \
                                       const C<T>*, cudaStream_t, RowBands);
#define FSIB_FFT_INST_P(T)                                                                       \
  template void launch_rows_product<T>(const C<T>*, C<T>*, int, long long, int, const FftLen&,   \
                                       const C<T>*, cudaStream_t);
#define FSIB_FFT_INST(T) FSIB_FFT_INST_R(T) FSIB_FFT_INST_P(T)
#define FSIB_FFT_INST_S(T, Ti, To)                                                               \
  template void launch_fft_strided<T, Ti, To>(const C<Ti>*, C<To>*, int, int, int, int,          \
                                              const FftLen&, bool, Mult<T>, const C<T>*,         \
                                              cudaStream_t, ZSkip);

}  // namespace fsib
