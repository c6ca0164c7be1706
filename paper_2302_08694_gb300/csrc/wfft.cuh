// Warp-level FFT of one line held in registers (row passes of the lengths below). The N of the
// templates below is a plan code (see wfft_n): the line length for the default plans.
//
// A line of length N is owned by L lanes of a warp (32/L lines per warp); lane l holds
// M = N/L elements. The transform is the self-sorting (Stockham) factorisation of
// fft_device.cuh with the radix sequence R_0 = M, R_1, ... chosen so that every radix
// divides M: in stage s each lane computes M/R_s butterflies j = l + L b entirely in
// registers. Stage 0 reads x[l + L i] (i < M), which is the order in which the lane
// loads its line from global memory. Between stages the lanes exchange values through a
// per-line shared-memory buffer, synchronised with __syncwarp only; each exchange uses an
// XOR swizzle of the element index (e ^ ((e >> sh) & mk)) chosen so that the stores and
// the loads of a warp hit distinct banks. After the last stage lane l holds
// X[l + L b + (N/R_last) r] in v[b R_last + r].
#pragma once
#include "fft_device.cuh"

namespace fsib {

// A warp plan is named by a code: the line length n, plus kOneExchange for the plans with 24
// elements per lane (lengths 96 and 192, FP32 lines), whose radix-24 first stage leaves a single
// exchange (24 x 4 and 24 x 8) instead of two; they double a lane's registers, so the
// double-float passes keep the default plans.
constexpr int kOneExchange = 1 << 16;
constexpr int wfft_n(int c) { return c & 0xFFFF; }
constexpr bool wfft_one(int c) { return (c & kOneExchange) != 0; }
// Lengths with a warp plan: 64, 128, 256 (M = 8), 48, 96, 192 (M = 12), 72 and 144 (M = 18: 4 and 8
// lanes a line, radices 18 x 2 x 2 and 18 x 2 x 2 x 2); one-exchange plans of 96 and 192 (M = 24).
constexpr bool wfft_has(int c) {
  return wfft_one(c) ? (wfft_n(c) == 96 || wfft_n(c) == 192)
                     : (c == 64 || c == 128 || c == 256 || c == 48 || c == 96 || c == 192 || c == 144 ||
                        c == 72);
}
constexpr int wfft_M(int c) {
  return wfft_one(c) ? 24 : (c == 48 || c == 96 || c == 192) ? 12 : (c == 144 || c == 72) ? 18 : 8;
}
constexpr int wfft_L(int c) { return wfft_n(c) / wfft_M(c); }
constexpr int wfft_radix(int c, int s) {
  return c == 64    ? (s == 0 ? 8 : s == 1 ? 8 : 0)
         : c == 128 ? (s == 0 ? 8 : s == 1 ? 4 : s == 2 ? 4 : 0)
         : c == 256 ? (s == 0 ? 8 : s == 1 ? 8 : s == 2 ? 4 : 0)
         : c == 48  ? (s == 0 ? 12 : s == 1 ? 4 : 0)
         : c == 96  ? (s == 0 ? 12 : s == 1 ? 4 : s == 2 ? 2 : 0)
         : c == 192 ? (s == 0 ? 12 : s == 1 ? 4 : s == 2 ? 4 : 0)
         : c == 144 ? (s == 0 ? 18 : s <= 3 ? 2 : 0)
         : c == 72  ? (s == 0 ? 18 : s <= 2 ? 2 : 0)
         : c == (96 | kOneExchange)  ? (s == 0 ? 24 : s == 1 ? 4 : 0)
         : c == (192 | kOneExchange) ? (s == 0 ? 24 : s == 1 ? 8 : 0)
                    : 0;
}
constexpr int wfft_nstages(int c) {
  int s = 0;
  while (wfft_radix(c, s)) ++s;
  return s;
}
// Swizzle of the exchange after stage ex for elements of E bytes: shift (hi 8 bits) and mask.
// One-exchange plans (FP32 only): chosen with the same bank model, the 16 addresses of each
// half-warp access (8-byte elements) in distinct bank pairs for the stores after the radix-24
// stage and the loads before the last one.
constexpr int wfft_swz(int c, int E, int ex) {
  return wfft_one(c) ? (E == 8 && ex == 0 ? (wfft_n(c) == 192 ? (3 << 8 | 7) : (3 << 8 | 3)) : 0)
         : E == 8 ? (c == 64    ? (ex == 0 ? (3 << 8 | 7) : 0)
                   : c == 128 ? (ex == 0 ? (3 << 8 | 15) : ex == 1 ? (2 << 8 | 15) : 0)
                   : c == 256 ? (ex == 0 ? (3 << 8 | 15) : ex == 1 ? (3 << 8 | 15) : 0)
                   : c == 48  ? (ex == 0 ? (2 << 8 | 3) : 0)
                   : c == 96  ? (ex == 0 ? (2 << 8 | 7) : ex == 1 ? (3 << 8 | 7) : 0)
                   : c == 192 ? (ex == 0 ? (2 << 8 | 15) : ex == 1 ? (2 << 8 | 7) : 0)
                   : c == 144 ? (ex == 0 ? (3 << 8 | 1) : 0)
                   : c == 72  ? (ex == 0 ? (2 << 8 | 1) : 0)
                              : 0)
                : (c == 64    ? (ex == 0 ? (3 << 8 | 7) : 0)
                   : c == 128 ? (ex == 0 ? (3 << 8 | 7) : 0)
                   : c == 256 ? (ex == 0 ? (3 << 8 | 7) : 0)
                   : c == 48  ? (ex == 0 ? (2 << 8 | 3) : 0)
                   : c == 96  ? (ex == 0 ? (2 << 8 | 7) : ex == 1 ? (3 << 8 | 7) : 0)
                   : c == 192 ? (ex == 0 ? (2 << 8 | 7) : ex == 1 ? (3 << 8 | 7) : 0)
                   : c == 144 ? (ex == 0 ? (3 << 8 | 1) : 0)
                   : c == 72  ? (ex == 0 ? (2 << 8 | 1) : 0)
                              : 0);
}
// Elements per line buffer (n plus bank padding; the one-exchange plans' line strides are 8 and
// 4 mod 16 elements, so the lines of a half-warp also fall in distinct bank pairs).
constexpr int wfft_stride(int c, int E) {
  return wfft_one(c) ? wfft_n(c) + (wfft_n(c) == 192 ? 8 : 4)
                     : c + (E == 8 ? (c == 64 ? 8 : c == 48 ? 4 : c == 96 ? 8 : c == 144 ? 8 : c == 72 ? 4 : 0)
                                   : (c == 48 ? 4 : c == 72 ? 4 : 0));
}
template <int SW>
__device__ __forceinline__ int wswz(int e) {
  return (SW & 255) ? (e ^ ((e >> (SW >> 8)) & (SW & 255))) : e;
}

// 8-point DFT: radix-2 split into two 4-point DFTs.
template <typename T, bool INV>
__device__ __forceinline__ void dft8(C<T>* v) {
  C<T> e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
  dft4<T, INV>(e);
  dft4<T, INV>(o);
  const T h = rsqrt2<T>();
  // w^k o[k], w = exp(-+ 2 pi i / 8)
  const C<T> o1 = INV ? mk<T>(ssub<T>(o[1].x, o[1].y) * h, sadd<T>(o[1].x, o[1].y) * h)
                      : mk<T>(sadd<T>(o[1].x, o[1].y) * h, ssub<T>(o[1].y, o[1].x) * h);
  const C<T> o2 = INV ? cmul_i<T>(o[2]) : cmul_mi<T>(o[2]);
  const C<T> o3 = INV ? mk<T>(-sadd<T>(o[3].x, o[3].y) * h, ssub<T>(o[3].x, o[3].y) * h)
                      : mk<T>(ssub<T>(o[3].y, o[3].x) * h, -sadd<T>(o[3].x, o[3].y) * h);
  v[0] = badd<T>(e[0], o[0]); v[4] = bsub<T>(e[0], o[0]);
  v[1] = badd<T>(e[1], o1);   v[5] = bsub<T>(e[1], o1);
  v[2] = badd<T>(e[2], o2);   v[6] = bsub<T>(e[2], o2);
  v[3] = badd<T>(e[3], o3);   v[7] = bsub<T>(e[3], o3);
}

// 12-point DFT by the prime-factor mapping 12 = 3 x 4 (no twiddles): input index
// (4 n1 + 3 n2) mod 12, output index (4 k1 + 9 k2) mod 12.
template <typename T, bool INV>
__device__ __forceinline__ void dft12(C<T>* v) {
  C<T> a[4][3];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < 3; ++n1) a[n2][n1] = v[(4 * n1 + 3 * n2) % 12];
    dft3<T, INV>(a[n2]);
  }
#pragma unroll
  for (int k1 = 0; k1 < 3; ++k1) {
    C<T> b[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    dft4<T, INV>(b);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[(4 * k1 + 9 * k2) % 12] = b[k2];
  }
}

// 18-point DFT by the prime-factor mapping 18 = 2 x 9 (no twiddles): input index
// (9 n1 + 2 n2) mod 18, output index (9 k1 + 10 k2) mod 18.
template <typename T, bool INV>
__device__ __forceinline__ void dft18(C<T>* v);

// 24-point DFT by the prime-factor mapping 24 = 3 x 8 (no twiddles): input index
// (8 n1 + 3 n2) mod 24, output index (16 k1 + 9 k2) mod 24.
template <typename T, bool INV>
__device__ __forceinline__ void dft24(C<T>* v) {
  C<T> a[8][3];
#pragma unroll
  for (int n2 = 0; n2 < 8; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < 3; ++n1) a[n2][n1] = v[(8 * n1 + 3 * n2) % 24];
    dft3<T, INV>(a[n2]);
  }
#pragma unroll
  for (int k1 = 0; k1 < 3; ++k1) {
    C<T> b[8] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1], a[4][k1], a[5][k1], a[6][k1], a[7][k1]};
    dft8<T, INV>(b);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) v[(16 * k1 + 9 * k2) % 24] = b[k2];
  }
}

// Constants in each arithmetic type (the double-float values are split at compile time).
#define FSIB_TRIG_CONST(name, val)                                                        \
  template <typename T> __device__ __forceinline__ T name();                              \
  template <> __device__ __forceinline__ float name<float>() { return (float)(val); }    \
  template <> __device__ __forceinline__ double name<double>() { return (val); }         \
  template <> __device__ __forceinline__ dd name<dd>() {                                  \
    constexpr dd v(val);                                                                  \
    return v;                                                                             \
  }
FSIB_TRIG_CONST(cos_pi8, 0.92387953251128675612818318939678829)
FSIB_TRIG_CONST(sin_pi8, 0.38268343236508977172845998403039887)
FSIB_TRIG_CONST(cos_2pi9, 0.76604444311897803520239265055541667)
FSIB_TRIG_CONST(sin_2pi9, 0.64278760968653932632264340990727188)
FSIB_TRIG_CONST(cos_4pi9, 0.17364817766693034885171662676931466)
FSIB_TRIG_CONST(sin_4pi9, 0.98480775301220805936674302458952301)
FSIB_TRIG_CONST(cos_8pi9, -0.93969262078590838405410927732473147)
FSIB_TRIG_CONST(sin_8pi9, 0.34202014332566873304409961468225958)
#undef FSIB_TRIG_CONST

// v * (cr - i si) forward, v * (cr + i si) inverse: multiplication by w^m, w = exp(-+ 2 pi i / R).
template <typename T, bool INV>
__device__ __forceinline__ C<T> crot(C<T> v, T cr, T si) {
  const T ci = INV ? si : -si;
  if constexpr (std::is_same<T, dd>::value) return mk<T>(dd_dot2(v.x, cr, -v.y, ci), dd_dot2(v.x, ci, v.y, cr));
  else return mk<T>(v.x * cr - v.y * ci, v.x * ci + v.y * cr);
}

// 16-point DFT: 4 x 4 Cooley-Tukey (inner twiddles w^{n2 k1}, w = exp(-+ 2 pi i / 16)).
template <typename T, bool INV>
__device__ __forceinline__ void dft16(C<T>* v) {
  C<T> a[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    a[n2][0] = v[n2]; a[n2][1] = v[4 + n2]; a[n2][2] = v[8 + n2]; a[n2][3] = v[12 + n2];
    dft4<T, INV>(a[n2]);
  }
  const T c1 = cos_pi8<T>(), s1 = sin_pi8<T>(), h = rsqrt2<T>();
  a[1][1] = crot<T, INV>(a[1][1], c1, s1);   // w^1
  a[1][2] = crot<T, INV>(a[1][2], h, h);     // w^2
  a[1][3] = crot<T, INV>(a[1][3], s1, c1);   // w^3
  a[2][1] = crot<T, INV>(a[2][1], h, h);     // w^2
  a[2][2] = INV ? cmul_i<T>(a[2][2]) : cmul_mi<T>(a[2][2]);  // w^4
  a[2][3] = crot<T, INV>(a[2][3], -h, h);    // w^6
  a[3][1] = crot<T, INV>(a[3][1], s1, c1);   // w^3
  a[3][2] = crot<T, INV>(a[3][2], -h, h);    // w^6
  a[3][3] = crot<T, INV>(a[3][3], -c1, -s1); // w^9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C<T> b[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    dft4<T, INV>(b);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
  }
}

// 9-point DFT: 3 x 3 Cooley-Tukey (inner twiddles w^{n2 k1}, w = exp(-+ 2 pi i / 9)).
template <typename T, bool INV>
__device__ __forceinline__ void dft9(C<T>* v) {
  C<T> a[3][3];
#pragma unroll
  for (int n2 = 0; n2 < 3; ++n2) {
    a[n2][0] = v[n2]; a[n2][1] = v[3 + n2]; a[n2][2] = v[6 + n2];
    dft3<T, INV>(a[n2]);
  }
  a[1][1] = crot<T, INV>(a[1][1], cos_2pi9<T>(), sin_2pi9<T>());  // w^1
  a[1][2] = crot<T, INV>(a[1][2], cos_4pi9<T>(), sin_4pi9<T>());  // w^2
  a[2][1] = crot<T, INV>(a[2][1], cos_4pi9<T>(), sin_4pi9<T>());  // w^2
  a[2][2] = crot<T, INV>(a[2][2], cos_8pi9<T>(), sin_8pi9<T>());  // w^4
#pragma unroll
  for (int k1 = 0; k1 < 3; ++k1) {
    C<T> b[3] = {a[0][k1], a[1][k1], a[2][k1]};
    dft3<T, INV>(b);
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2) v[k1 + 3 * k2] = b[k2];
  }
}

template <typename T, bool INV>
__device__ __forceinline__ void dft18(C<T>* v) {
  C<T> a[9][2];
#pragma unroll
  for (int n2 = 0; n2 < 9; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < 2; ++n1) a[n2][n1] = v[(9 * n1 + 2 * n2) % 18];
    dft2<T, INV>(a[n2]);
  }
#pragma unroll
  for (int k1 = 0; k1 < 2; ++k1) {
    C<T> b[9] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1], a[4][k1], a[5][k1], a[6][k1], a[7][k1], a[8][k1]};
    dft9<T, INV>(b);
#pragma unroll
    for (int k2 = 0; k2 < 9; ++k2) v[(9 * k1 + 10 * k2) % 18] = b[k2];
  }
}

template <typename T, bool INV, int R>
__device__ __forceinline__ void dft_r(C<T>* v) {
  if constexpr (R == 2) dft2<T, INV>(v);
  else if constexpr (R == 3) dft3<T, INV>(v);
  else if constexpr (R == 4) dft4<T, INV>(v);
  else if constexpr (R == 8) dft8<T, INV>(v);
  else if constexpr (R == 9) dft9<T, INV>(v);
  else if constexpr (R == 12) dft12<T, INV>(v);
  else if constexpr (R == 16) dft16<T, INV>(v);
  else if constexpr (R == 18) dft18<T, INV>(v);
  else if constexpr (R == 24) dft24<T, INV>(v);
}

// Twiddles in lane order: for stage s >= 1, butterfly slot b, r = 1..R-1 and lane l, entry
// wfft_tw_off(N, s) + (b (R-1) + r - 1) L + l holds w^{(j mod NS) r N/(NS R)}, j = l + L b,
// w = exp(-2 pi i / N), so that the lanes of a warp read consecutive entries.
constexpr int wfft_tw_off(int c, int s) {
  int off = 0;
  for (int t = 1; t < s; ++t) off += (wfft_n(c) / wfft_radix(c, t)) * (wfft_radix(c, t) - 1);
  return off;
}
constexpr int wfft_tw_size(int c) { return wfft_tw_off(c, wfft_nstages(c)); }

// Build the lane-ordered table from the natural table tw[k] = exp(-2 pi i k / N) (global).
template <typename T, int N>
__device__ __forceinline__ void wfft_build_twiddles(C<T>* twl, const C<T>* __restrict__ tw) {
  constexpr int L = wfft_L(N), NN = wfft_n(N);
  for (int e = threadIdx.x; e < wfft_tw_size(N); e += blockDim.x) {
    int s = 1, NS = wfft_radix(N, 0);
    while (e >= wfft_tw_off(N, s + 1)) { NS *= wfft_radix(N, s); ++s; }
    const int R = wfft_radix(N, s), q = e - wfft_tw_off(N, s);
    const int l = q % L, br = q / L, b = br / (R - 1), r = br % (R - 1) + 1;
    const int j = l + L * b;
    twl[e] = tw[(j % NS) * r * (NN / (NS * R))];
  }
}

// Stage S of the warp transform (NS = product of the earlier radices). buf: this line's
// exchange buffer; twl: the lane-ordered twiddle table in shared memory.
template <typename T, bool INV, int N, int S = 0, int NS = 1>
__device__ __forceinline__ void wfft(C<T> (&v)[wfft_M(N)], C<T>* buf, int l, const C<T>* __restrict__ twl) {
  constexpr int M = wfft_M(N), L = wfft_L(N), R = wfft_radix(N, S), NB = M / R, NN = wfft_n(N);
  constexpr int E = (int)sizeof(C<T>);
  if constexpr (S > 0) {
    // gather this stage's inputs x[j + r N/R], j = l + L b, from the previous stage's outputs
    constexpr int SW = wfft_swz(N, E, S - 1);
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int r = 0; r < R; ++r) v[b * R + r] = buf[wswz<SW>(l + L * b + r * (NN / R))];
    __syncwarp();
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C<T> w = twl[wfft_tw_off(N, S) + (b * (R - 1) + r - 1) * L + l];
        if (INV) w = cconj<T>(w);
        v[b * R + r] = cmul<T>(v[b * R + r], w);
      }
    }
    dft_r<T, INV, R>(&v[b * R]);
  }
  if constexpr (S + 1 < wfft_nstages(N)) {
    constexpr int SW = wfft_swz(N, E, S);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = l + L * b;
      const int o = (j / NS) * NS * R + j % NS;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[wswz<SW>(o + r * NS)] = v[b * R + r];
    }
    __syncwarp();
    wfft<T, INV, N, S + 1, NS * R>(v, buf, l, twl);
  }
}

// Natural index of register slot i after the last stage.
template <int N>
__device__ __forceinline__ int wfft_out_index(int l, int i) {
  constexpr int RL = wfft_radix(N, wfft_nstages(N) - 1);
  return l + wfft_L(N) * (i / RL) + (wfft_n(N) / RL) * (i % RL);
}

// Forward transform of a one-exchange plan (N = 24 L) that takes its input in the order the
// plan leaves its output: lane l holds x[n1 + 24 n2] in v[b L + n2], n1 = l + L b (b < 24/L,
// n2 < L), and leaves X[l + L k1] in v[k1] (k1 < 24), the order in which the plan's own
// transform reads its input. It is the plan's factorisation taken the other way round:
// with n = n1 + 24 n2 and k = k2 + L k1,
//   X[k2 + L k1] = sum_n1 w24^{n1 k1} w^{n1 k2} sum_n2 wL^{n2 k2} x[n1 + 24 n2],
// so every lane first runs its 24/L DFTs of length L (over n2, in registers), multiplies by
// w^{n1 k2}, and after one exchange (lane k2 gathers all n1 of column k2) runs a DFT of length
// 24. twt: the lane-ordered table of w^{n1 k2} (wfft_twt_size entries, see
// wfft_build_twiddles_t); buf: the line's exchange buffer (L rows of 25 elements: the rows of
// a half-warp's lines fall in distinct bank pairs).
constexpr int kTRow = 25;
template <int PC>
constexpr int wfft_twt_size() {
  return wfft_one(PC) ? (24 / wfft_L(PC)) * (wfft_L(PC) - 1) * wfft_L(PC) : 0;
}
template <typename T, int PC>
__device__ __forceinline__ void wfft_build_twiddles_t(C<T>* twt, const C<T>* __restrict__ tw) {
  constexpr int L = wfft_L(PC), NN = wfft_n(PC);
  for (int e = threadIdx.x; e < wfft_twt_size<PC>(); e += blockDim.x) {
    const int l = e % L, q = e / L, b = q / (L - 1), k2 = q % (L - 1) + 1;
    twt[e] = tw[((l + L * b) * k2) % NN];
  }
}
template <typename T, int PC>
__device__ __forceinline__ void wfft_fwd_transposed(C<T> (&v)[24], C<T>* buf, int l, const C<T>* __restrict__ twt) {
  static_assert(wfft_one(PC) && wfft_M(PC) == 24, "one-exchange plans only");
  constexpr int L = wfft_L(PC), NB = 24 / L;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    dft_r<T, false, L>(&v[b * L]);
#pragma unroll
    for (int k2 = 1; k2 < L; ++k2) v[b * L + k2] = cmul<T>(v[b * L + k2], twt[(b * (L - 1) + k2 - 1) * L + l]);
  }
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int k2 = 0; k2 < L; ++k2) buf[k2 * kTRow + l + L * b] = v[b * L + k2];
  __syncwarp();
#pragma unroll
  for (int n1 = 0; n1 < 24; ++n1) v[n1] = buf[l * kTRow + n1];
  __syncwarp();
  dft24<T, false>(v);
}

}  // namespace fsib
