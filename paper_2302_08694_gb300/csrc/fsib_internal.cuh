// Internal declarations of the FSIB library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/fsib.h"
#include "dd.cuh"
#include "launch.cuh"

namespace fsib {

// ---------------------------------------------------------------------------
// Complex numbers: plain two-component structs so that loads are 8/16-byte vectors.
// Element types: float (mixed mode), double (API arrays in FP64 mode, native
// FP64 kernels) and dd (double-float, the FP64-mode transform arithmetic).
// ---------------------------------------------------------------------------
template <typename T> struct cplx_t;
template <> struct cplx_t<float>  { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<dd>     { using type = dd2; };
template <typename T> using C = typename cplx_t<T>::type;

template <typename T> __device__ __forceinline__ C<T> mk(T x, T y) { C<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ C<T> cadd(C<T> a, C<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C<T> csub(C<T> a, C<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C<T> cmul(C<T> a, C<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// double-float: each component as one two-term dot product (one renormalisation instead of three)
template <> __device__ __forceinline__ C<dd> cmul<dd>(C<dd> a, C<dd> b) {
  return mk<dd>(dd_dot2(a.x, b.x, -a.y, b.y), dd_dot2(a.x, b.y, a.y, b.x));
}
template <typename T> __device__ __forceinline__ C<T> cconj(C<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ C<T> cscale(C<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// multiply by +i (or -i)
template <typename T> __device__ __forceinline__ C<T> cmul_i(C<T> a) { return mk<T>(-a.y, a.x); }
template <typename T> __device__ __forceinline__ C<T> cmul_mi(C<T> a) { return mk<T>(a.y, -a.x); }

// Element conversions at the boundary between API arrays and the transform type.
__device__ __forceinline__ void cvt(float& o, float i) { o = i; }
__device__ __forceinline__ void cvt(double& o, double i) { o = i; }
__device__ __forceinline__ void cvt(dd& o, dd i) { o = i; }
__device__ __forceinline__ void cvt(dd& o, double i) { o = dd_from_double(i); }
__device__ __forceinline__ void cvt(double& o, dd i) { o = dd_to_double(i); }
template <typename To, typename From>
__device__ __forceinline__ C<To> ccvt(const C<From>& i) {
  C<To> o;
  cvt(o.x, i.x);
  cvt(o.y, i.y);
  return o;
}

// ---------------------------------------------------------------------------
// 1-D FFT plan of one length n = 2^a 3^b (radix stages of 4, 2 and 3).
// ---------------------------------------------------------------------------
constexpr int kMaxStages = 12;
// Longest transform per axis: 2048 in 2D (N up to 1024 at sigma = 2); 512 in 3D, where a
// fine grid of 512^3 cells per component keeps every element index within 32 bits.
constexpr int kMaxFFT2 = 2048;
constexpr int kMaxFFT3 = 512;

struct FftLen {
  int n = 0;
  int nstages = 0;
  int radix[kMaxStages] = {0};
  int tw_off = 0;  // offset of exp(-2 pi i j/n), j = 0..n-1, in the twiddle table
  int tile_p = 8;  // strided passes: adjacent lines per CTA
  int rows_q = 4;  // row passes: row pairs per CTA
};

// Multiplier applied at the mode end of a strided pass:
//   value *= scale * dline[m_line] * (dplane ? dplane[q] : 1)
// where m_line indexes the pass axis (length-N FFT order) and q the inner index.
template <typename T> struct Mult {
  T scale = T(1);
  const T* dline = nullptr;
  const T* dplane = nullptr;
};

// ---------------------------------------------------------------------------
// Plan and workspaces of one problem (owned by fsib_plan).
// ---------------------------------------------------------------------------
struct Plan {
  int d = 3, N = 0, M = 0;
  double L = 1.0, mu = 1.0, rho = 1.0, dt = 1e-3, tol = 1e-12;
  bool stokes = false;
  int prec = FSIB_FP64;
  double sigma = 2.0;
  int width_opt = 0, bin_opt = 0;
  int use_graph = 1, check_finite = 0;
  int native_fp64 = 0;  // FP64 mode: 0 = double-float transforms, 1 = native FP64 arithmetic
  double fbody[3] = {0.0, 0.0, 0.0};  // uniform body force density, added to f-hat(0) (Navier-Stokes)
  // launch-shape tunables (chosen by fsib_autotune)
  int fft_p = 8, fft_q = 4, slice = 256;
  // summation in the FP32 gather spreads: 0 plain FMAs, 1 compensated per term, 2 compensated
  // per staged chunk of candidates (see kSumPlain, kSumTerm, kSumChunk)
  int spread_sum = 2;

  // derived
  int nf = 0;        // fine grid per axis
  int w = 0;         // kernel width (cells)
  double beta = 0;   // ES shape
  int Nt = 0;        // dealias grid per axis
  int bins[3] = {1, 1, 1}, nbin[3] = {1, 1, 1};
  long long nbins = 1;
  FftLen fl_nf, fl_nt;
};

struct Workspace {
  // twiddles (double and float copies), deconvolution tables
  void* tw = nullptr;        // C<T> table, T per precision
  void* dline = nullptr;     // T[N]
  void* dplane = nullptr;    // T[N*N/2] (3D) or T[N/2] (2D)
  // fine grid (real, d components) and two complex scratch buffers
  void* grid = nullptr;  size_t grid_bytes = 0;
  void* s1 = nullptr;    size_t s1_bytes = 0;
  void* s2 = nullptr;    size_t s2_bytes = 0;
  void* s3 = nullptr;    // second scratch pair (s1_bytes each, Navier-Stokes only): the
  void* s4 = nullptr;    // nonlinear term of u^m, computed beside the point side of the step
  void* grid2 = nullptr;  // second fine grid (Navier-Stokes only): type-2 prep of u^{m+1} beside the U^{m+1/2} interp
  void* fhat = nullptr;  size_t spec_bytes = 0;  // d * N^{d-1} * N/2 complex
  void* uhalf = nullptr;
  // sort
  int* bin_of = nullptr;      // [M]
  int* rank = nullptr;        // [M]
  int* counts = nullptr;      // [nbins]
  int* offsets = nullptr;     // [nbins + 1]
  int* occ = nullptr;         // [nbins] occupied bins; occ count at offsets[nbins]? (see nocc)
  int* nocc = nullptr;        // [1]
  int* perm = nullptr;        // [M] sorted -> original
  int* i0 = nullptr;          // [d][M] window start per axis (sorted order)
  void* delta = nullptr;      // T[d][M] i0 - t (sorted order)
  // Lagrangian scratch (double)
  double* Xh = nullptr;       // [d][M]
  double* cw = nullptr;       // [d][M] omega * F
  double* Uh = nullptr;       // [d][M]
  double* omega_ones = nullptr;
  // force models
  int force_kind = 0;         // 0 none, 1 curve, 2 mesh, 3 target points, 4 surface tension
  double curve_K = 0.0;
  double* target = nullptr;   // [d][M] target points (force kind 3)
  double target_wK = 0.0;     // omega K of the target springs
  double stiffness = 1.0;     // K (curve) or sigma (mesh): the force is linear in it
  int* csr_ptr = nullptr; int* csr_col = nullptr; double* csr_k = nullptr; int nnz = 0;
  int* tri = nullptr; int ntri = 0;
  int2* inc_jk = nullptr;     // surface tension: (j, k) of each triangle at a node, CSR rows csr_ptr
  // reductions
  double* red = nullptr;      // partial sums
  int red_blocks = 0;
  int* flag = nullptr;
  void* wts = nullptr;               // T[M][d][w] kernel weights per sorted point
  void* cwp = nullptr;               // T[M][d] weighted forces per sorted point
  void* ktab = nullptr;              // T[N] wave numbers (2 pi / L) m(i), m(i) = i or i - N, in the
                                     // spectral precision (float for FSIB_MIXED, double otherwise)
  int* box_ns = nullptr;             // [nbins] slices per gather box (3D)
  int* box_np = nullptr;             // [nbins] partial slots per box
  int* box_so = nullptr;             // [nbins + 1] slice offsets
  int* box_po = nullptr;             // [nbins + 1] partial-slot offsets
  int* box_item = nullptr;           // [slices] box of each slice (non-empty boxes only)
  int* box_sched = nullptr;          // [slices] order in which the gather takes the slices
  int* box_work = nullptr;           // [2] gather work counters: next slice, next run of empty boxes
  int* box_done = nullptr;           // [nbins] slices of a split box finished (the last one adds the partials)
  unsigned char* band = nullptr;     // [nb_z][nb_y] row bands reached by a window (gather path; see RowBands)
  unsigned char* band_dil = nullptr; // the same, widened by one box each way (kept from the X^{m+1/2} binning)
  // Set to 1 by an interpolation from a grid that holds only the widened bands when a window
  // leaves them (the point gets NaN); page-locked host memory mapped into the device, so the
  // host reads it at the next call without a synchronisation (miss_host) and clears it.
  unsigned int* miss_host = nullptr;
  unsigned int* miss_dev = nullptr;
  void* part = nullptr;              // T[slots][3][512] partial boxes
  size_t part_slots = 0;
  // reverse mode (allocated on first use)
  void* adj_spec = nullptr;          // 3 spectra: u-hat, w-hat, i k_b * spectrum
  double* adj_pts = nullptr;         // point buffers: Gu, Gw (d*d*M each), w, fw, c, a, lam, tmp (d*M each)
  double* adj_ckpt = nullptr;        // checkpoints and segment positions
  size_t adj_ckpt_bytes = 0;
  double* adj_part = nullptr;        // sigma partial sums
  double* adj_sig = nullptr;         // sigma gradient accumulator
  // staging for host pointers
  void* stage[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t stage_bytes[4] = {0, 0, 0, 0};
};

// ---------------------------------------------------------------------------
// Launchers (implemented in the .cu files). All enqueue on `st`.
// ---------------------------------------------------------------------------
// Strided passes along y of a 3D grid [comp][z][y][x] (outer = z): the z-slabs of boxes whose
// row bands are all off (RowBands flags) are skipped; zero: write zeros there instead (their
// input column is zero). The two-stage kernels honour it; other lengths compute every line.
struct ZSkip {
  const unsigned char* flag = nullptr;  // [nb_z][nb_y]
  int outer = 1, b = 1, nby = 1, zero = 0;
};
template <typename T, typename Tin = T, typename Tout = T>
void launch_fft_strided(const C<Tin>* in, C<Tout>* out, int ncomp, int outer, int inner,
                        int Nk, const FftLen& fl, bool inverse, Mult<T> mult,
                        const C<T>* tw, cudaStream_t st, ZSkip zs = ZSkip());
// Rows of the fine grid (along x) that no window of the current point binning reaches, by
// band of boxes (y div b, z div b): the gather spread leaves them unwritten, the first forward
// row pass takes them as zeros, and the last inverse row pass skips them (no interpolation
// window reads them). flag == nullptr: every row is on.
struct RowBands {
  const unsigned char* flag = nullptr;  // [nb_z][nb_y]
  int n = 1, b = 1, nby = 1, d3 = 0;    // row length (fine grid), box side, boxes along y, d == 3
  __device__ __forceinline__ bool on(long long row) const {
    if (!flag) return true;
    const int y = (int)(row % n);
    const int z = d3 ? (int)((row / n) % n) : 0;
    return flag[(z / b) * nby + y / b] != 0;
  }
};

template <typename T>
void launch_fft_rows_r2c(const T* in, C<T>* out, long long nrows, int Nk, const FftLen& fl,
                         const C<T>* tw, cudaStream_t st, RowBands rb = RowBands());
template <typename T>
void launch_fft_rows_c2r(const C<T>* in, T* out, long long nrows, int Nk, const FftLen& fl,
                         const C<T>* tw, cudaStream_t st, RowBands rb = RowBands());
template <typename T>
void launch_rows_product(const C<T>* in, C<T>* out, int d, long long nrows, int Nk,
                         const FftLen& fl, const C<T>* tw, cudaStream_t st);

// occupied: also list the occupied bins (needed by the scatter spread, launch_spread). Otherwise
// the row bands are marked; dilate: also the widened bands (ws.band_dil).
void launch_bin_points(const Plan& p, Workspace& ws, const double* X, cudaStream_t st, bool occupied = true,
                       bool dilate = false);
template <typename T>
void launch_spread(const Plan& p, Workspace& ws, const double* cw, const double* omega,
                   T* grid, cudaStream_t st);
template <typename T>
void launch_interp(const Plan& p, Workspace& ws, const T* grid, double* U, cudaStream_t st);

template <typename T>
void launch_point_prep(const Plan& p, Workspace& ws, const double* cw, const double* omega, cudaStream_t st);
template <typename T>
void launch_spread_gather(const Plan& p, Workspace& ws, T* grid, cudaStream_t st);
// guard: row bands the grid holds (RowBands flags); a point whose window leaves them gets NaN
// and sets *miss (when miss is not null).
template <typename T>
void launch_interp_warp(const Plan& p, Workspace& ws, const T* grid, double* U, cudaStream_t st,
                        const unsigned char* guard = nullptr, unsigned int* miss = nullptr);

template <typename T>
void launch_stokeslet(const Plan& p, const C<T>* fhat, C<T>* uhat, cudaStream_t st);
template <typename T>
void launch_pressure(const Plan& p, const C<T>* prod, const C<T>* fhat, C<T>* phat, cudaStream_t st);
// prod: the product coefficients, C<T> values, or double-float pairs (dd2) when prod_pairs (FP64
// mode with double-float transforms only).
template <typename T>
void launch_ns_update(const Plan& p, const void* ktab, const void* prod, bool prod_pairs, const C<T>* fhat,
                      const C<T>* ubase, C<T>* out, bool half, cudaStream_t st);

void launch_axpy(double* y, const double* x, const double* v, double a, long long n, cudaStream_t st);
void launch_force(const Plan& p, const Workspace& ws, const double* X, double* c, cudaStream_t st);
void launch_mesh_stiffness(const double* Xref, const int* tri, int ntri, int M, double sigma,
                           int* csr_ptr, int* csr_col, double* csr_k, int nnz, cudaStream_t st);
template <typename T>
int run_invariants(const Plan& p, Workspace& ws, const double* X, const C<T>* uhat,
                   double* out, cudaStream_t st);
template <typename T>
int run_band_flux(const Plan& p, Workspace& ws, const C<T>* uhat, int comp, int axis, double y0, double y1,
                  double* flux, cudaStream_t st);

template <typename T>
void launch_mul_ik(const Plan& p, int b, const C<T>* in, C<T>* out, cudaStream_t st);
void launch_vjp_combine(int d, int M, double s, double sigma, const double* Gu, const double* Gw,
                        const double* lam, const double* c, const double* fw, const double* w, double* gX,
                        double* part, int nblk, double* gsig, cudaStream_t st);

int check_last(const char* where);
void raise_smem_limit(const void* kernel);
// Blocks per box of the 2D gather and the bytes of its partial boxes.
int gather2d_slices(const Plan& p);
size_t gather2d_part_bytes(const Plan& p);
// Dynamic shared memory a block of a kernel without static shared memory may request
// (the device's opt-in limit per block).
size_t smem_optin();

}  // namespace fsib
