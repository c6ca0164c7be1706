// Shared-memory mixed-radix FFT used by every transform pass.
//
// Self-sorting (Stockham) formulation: stage s with radix R reads element
// j + r*n/R (r = 0..R-1) of each line, multiplies by twiddles
// w^{(j mod Ns) r n/(Ns R)}, does an R-point DFT and writes to
// (j div Ns) Ns R + (j mod Ns) + r Ns, where Ns is the product of the radices
// of the earlier stages. The output is in natural order after the last stage.
// Lines live in shared memory; element i of line l is at base[l*ls + i*es].
// Two buffers alternate between stages.
#pragma once
#include <type_traits>
#include "fsib_internal.cuh"

namespace fsib {

// Butterfly sums: double-float sums inside a DFT skip their renormalisation (dd_add_nr); the
// twiddle and constant products between the DFTs renormalise. Other types: plain sums.
template <typename T> __device__ __forceinline__ T sadd(T a, T b) {
  if constexpr (std::is_same<T, dd>::value) return dd_add_nr(a, b);
  else return a + b;
}
template <typename T> __device__ __forceinline__ T ssub(T a, T b) {
  if constexpr (std::is_same<T, dd>::value) return dd_add_nr(a, -b);
  else return a - b;
}
template <typename T> __device__ __forceinline__ C<T> badd(C<T> a, C<T> b) {
  return mk<T>(sadd<T>(a.x, b.x), sadd<T>(a.y, b.y));
}
template <typename T> __device__ __forceinline__ C<T> bsub(C<T> a, C<T> b) {
  return mk<T>(ssub<T>(a.x, b.x), ssub<T>(a.y, b.y));
}

// Spectra A, B of the two real rows packed as z = a + i b, from Z[k] and Zc = conj Z[N - k]:
// A[k] = (Z[k] + Zc) / 2, B[k] = (Z[k] - Zc) / 2i. Double-float: non-renormalising sums and
// exact halving; other types: the plain expressions.
template <typename T> struct CPair { C<T> a, b; };
template <typename T> __device__ __forceinline__ CPair<T> untangle_pair(C<T> Z, C<T> Zc) {
  if constexpr (std::is_same<T, dd>::value) {
    const C<T> s = badd<T>(Z, Zc), df = bsub<T>(Z, Zc);
    return {mk<T>(dd_half(s.x), dd_half(s.y)), mk<T>(dd_half(df.y), -dd_half(df.x))};
  } else {
    const C<T> s = cadd<T>(Z, Zc), df = csub<T>(Z, Zc);
    return {mk<T>(T(0.5) * s.x, T(0.5) * s.y), mk<T>(T(0.5) * df.y, T(-0.5) * df.x)};
  }
}

// sqrt(3)/2 in each arithmetic type
template <typename T> __device__ __forceinline__ T sqrt3_2();
template <> __device__ __forceinline__ float sqrt3_2<float>() { return 0.866025403784438646763723170752936183f; }
template <> __device__ __forceinline__ double sqrt3_2<double>() { return 0.866025403784438646763723170752936183; }
template <> __device__ __forceinline__ dd sqrt3_2<dd>() {
  constexpr dd v(0.866025403784438646763723170752936183);
  return v;
}

// 1/sqrt(2) in each arithmetic type
template <typename T> __device__ __forceinline__ T rsqrt2();
template <> __device__ __forceinline__ float rsqrt2<float>() { return 0.707106781186547524400844362104849039f; }
template <> __device__ __forceinline__ double rsqrt2<double>() { return 0.707106781186547524400844362104849039; }
template <> __device__ __forceinline__ dd rsqrt2<dd>() {
  constexpr dd v(0.707106781186547524400844362104849039);
  return v;
}

template <typename T, bool INV>
__device__ __forceinline__ void dft2(C<T>* v) {
  C<T> a = v[0], b = v[1];
  v[0] = badd<T>(a, b);
  v[1] = bsub<T>(a, b);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft3(C<T>* v) {
  // forward: y1 = v0 - (v1+v2)/2 - i s3 (v1 - v2), y2 = v0 - (v1+v2)/2 + i s3 (v1 - v2)
  C<T> s = badd<T>(v[1], v[2]);
  C<T> d = bsub<T>(v[1], v[2]);
  C<T> m;
  if constexpr (std::is_same<T, dd>::value) m = bsub<T>(v[0], mk<T>(dd_half(s.x), dd_half(s.y)));
  else m = mk<T>(v[0].x - T(0.5) * s.x, v[0].y - T(0.5) * s.y);
  C<T> t = cscale<T>(d, sqrt3_2<T>());
  C<T> it = INV ? cmul_i<T>(t) : cmul_mi<T>(t);
  v[0] = badd<T>(v[0], s);
  v[1] = badd<T>(m, it);
  v[2] = bsub<T>(m, it);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(C<T>* v) {
  C<T> s02 = badd<T>(v[0], v[2]), d02 = bsub<T>(v[0], v[2]);
  C<T> s13 = badd<T>(v[1], v[3]), d13 = bsub<T>(v[1], v[3]);
  C<T> id = INV ? cmul_i<T>(d13) : cmul_mi<T>(d13);
  v[0] = badd<T>(s02, s13);
  v[2] = bsub<T>(s02, s13);
  v[1] = badd<T>(d02, id);
  v[3] = bsub<T>(d02, id);
}

template <typename T, bool INV, int R>
__device__ __forceinline__ void stage_item(const C<T>* __restrict__ src, C<T>* __restrict__ dst,
                                           int l, int j, int n, int Ns, int ls, int es,
                                           const C<T>* __restrict__ tw) {
  const int nb = n / R;
  C<T> v[R];
  const C<T>* s = src + l * ls;
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = s[(j + r * nb) * es];
  const int k = j % Ns;
  if (Ns > 1) {
    const int step = n / (Ns * R);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      C<T> w = tw[k * r * step];  // k r step < n since k < Ns, r < R
      if (INV) w = cconj<T>(w);
      v[r] = cmul<T>(v[r], w);
    }
  }
  if (R == 2) dft2<T, INV>(v);
  if (R == 3) dft3<T, INV>(v);
  if (R == 4) dft4<T, INV>(v);
  C<T>* d = dst + l * ls;
  const int o = (j / Ns) * Ns * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) d[(o + r * Ns) * es] = v[r];
}

// Transform nl lines; returns the buffer that holds the result (a or b).
// lines_fast: consecutive threads take consecutive lines (strided layouts) rather
// than consecutive butterflies of one line (contiguous rows).
// Must be called by all threads of the block; ends with a barrier.
template <typename T, bool INV>
__device__ C<T>* smem_fft(C<T>* a, C<T>* b, int nl, int ls, int es, bool lines_fast,
                          const FftLen& fl, const C<T>* __restrict__ tw) {
  const int n = fl.n;
  int Ns = 1;
  for (int s = 0; s < fl.nstages; ++s) {
    const int R = fl.radix[s];
    const int nb = n / R;
    const int total = nl * nb;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      int l, j;
      if (lines_fast) { l = t % nl; j = t / nl; } else { j = t % nb; l = t / nb; }
      if (R == 4) stage_item<T, INV, 4>(a, b, l, j, n, Ns, ls, es, tw);
      else if (R == 2) stage_item<T, INV, 2>(a, b, l, j, n, Ns, ls, es, tw);
      else stage_item<T, INV, 3>(a, b, l, j, n, Ns, ls, es, tw);
    }
    __syncthreads();
    C<T>* t = a; a = b; b = t;
    Ns *= R;
  }
  return a;
}

// ---------------------------------------------------------------------------
// The same transform with the length N known at compile time: the radix plan,
// the butterfly index arithmetic and the twiddle strides fold to constants.
// lines_fast requires nl to be a power of two (lgnl = log2 nl).
// ---------------------------------------------------------------------------
constexpr int ct_radix(int n, int s) {
  int m = n, st = 0;
  while (m % 4 == 0) { if (st == s) return 4; m /= 4; ++st; }
  while (m % 2 == 0) { if (st == s) return 2; m /= 2; ++st; }
  while (m % 3 == 0) { if (st == s) return 3; m /= 3; ++st; }
  return 0;
}
constexpr int ct_nstages(int n) {
  int s = 0;
  while (ct_radix(n, s)) ++s;
  return s;
}

template <typename T, bool INV, int R, int N, int NS>
__device__ __forceinline__ void stage_item_ct(const C<T>* __restrict__ src, C<T>* __restrict__ dst, int l, int j,
                                              int ls, int es, const C<T>* __restrict__ tw) {
  constexpr int nb = N / R;
  C<T> v[R];
  const C<T>* s = src + l * ls;
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = s[(j + r * nb) * es];
  const int k = j % NS;
  if (NS > 1) {
    constexpr int step = N / (NS * R);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      C<T> w = tw[k * r * step];
      if (INV) w = cconj<T>(w);
      v[r] = cmul<T>(v[r], w);
    }
  }
  if (R == 2) dft2<T, INV>(v);
  if (R == 3) dft3<T, INV>(v);
  if (R == 4) dft4<T, INV>(v);
  C<T>* d = dst + l * ls;
  const int o = (j / NS) * NS * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) d[(o + r * NS) * es] = v[r];
}

template <typename T, bool INV, int N, int S = 0, int NS = 1>
__device__ __forceinline__ C<T>* smem_fft_ct(C<T>* a, C<T>* b, int nl, int lgnl, int ls, int es, bool lines_fast,
                                             const C<T>* __restrict__ tw) {
  if constexpr (S == ct_nstages(N)) {
    return a;
  } else {
    constexpr int R = ct_radix(N, S);
    constexpr int nb = N / R;
    const int total = nl * nb;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      int l, j;
      if (lines_fast) { l = t & (nl - 1); j = t >> lgnl; } else { j = t % nb; l = t / nb; }
      stage_item_ct<T, INV, R, N, NS>(a, b, l, j, ls, es, tw);
    }
    __syncthreads();
    return smem_fft_ct<T, INV, N, S + 1, NS * R>(b, a, nl, lgnl, ls, es, lines_fast, tw);
  }
}

// Dispatch on the FFT lengths used by the workloads; other lengths take the runtime plan (0).
#define FSIB_FFT_SIZES(X) X(32) X(48) X(64) X(72) X(96) X(128) X(144) X(192) X(256)

}  // namespace fsib
