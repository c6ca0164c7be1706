// Lagrangian side in double precision: position updates (Eqs. spatial_1, spatial_4),
// force laws (Eq. elstic_force_2d; cot-weight springs of Sec. 6.2.3; target-point
// springs of the Poiseuille channel, Sec. 5.2.2), the invariants of Sec. 4 (enclosed
// area/volume, energies, zero mode, divergence) and the channel flux of Eq. poiseuille_flux.
#include <cmath>

#include "fsib_internal.cuh"

namespace fsib {

static unsigned blocks_for(long long n, int bs = 256) {
  long long b = (n + bs - 1) / bs;
  if (b > 65535LL * 8) b = 65535LL * 8;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// y = x + a v
struct KAxpy {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ v,
                             double a, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
      y[i] = x[i] + a * v[i];
  }
};

void launch_axpy(double* y, const double* x, const double* v, double a, long long n, cudaStream_t st) {
  launch<KAxpy>(blocks_for(n), 256, 0, st, y, x, v, a, n);
}

// Closed curve: c_j = omega F_j = K (X_{j+1} + X_{j-1} - 2 X_j)/dtheta, dtheta = 2 pi/M.
struct KForceCurve {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(const double* __restrict__ X, double* __restrict__ c, int M, double K_over_dth) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
      const int jp = (j + 1 == M) ? 0 : j + 1, jm = (j == 0) ? M - 1 : j - 1;
      for (int a = 0; a < 2; ++a) {
        const double* x = X + (long long)a * M;
        c[(long long)a * M + j] = K_over_dth * ((x[jp] - x[j]) + (x[jm] - x[j]));
      }
    }
  }
};

// Springs: c_i = sum_j K_ij (X_j - X_i), CSR adjacency (omega = 1).
// Eight lanes per vertex: the lanes take the vertex's CSR entries in strides of eight
// and reduce with shuffles, so that a vertex of high degree (a pole of a latitude-
// longitude mesh joins every point of the first ring) costs few rounds.
struct KForceMesh {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(const double* __restrict__ X, double* __restrict__ c, int M,
                             const int* __restrict__ ptr, const int* __restrict__ col,
                             const double* __restrict__ kv) {
  const int sl = threadIdx.x & 7, sub = (threadIdx.x >> 3) & 3, lane = threadIdx.x & 31;
  // warp-uniform loop over groups of four vertices (the shuffles need the whole warp)
  for (long long w0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4; w0 < M;
       w0 += (((long long)gridDim.x * blockDim.x) >> 5) * 4) {
    const int i = (int)(w0 + sub);
    const bool ok = i < M;
    // A vertex of high degree (a pole of a lat-long mesh joins a whole ring) would keep its
    // eight lanes for degree/8 rounds: such a warp takes its four vertices one at a time, all
    // 32 lanes on each.
    const int deg = ok ? ptr[i + 1] - ptr[i] : 0;
    if (__reduce_max_sync(0xffffffffu, (unsigned)deg) > 32u) {
      for (int q = 0; q < 4; ++q) {
        const int iq = (int)(w0 + q);
        if (iq >= M) break;  // uniform across the warp
        const double x0 = X[iq], x1 = X[M + iq], x2 = X[2LL * M + iq];
        double g0 = 0, g1 = 0, g2 = 0;
        for (int e = ptr[iq] + lane; e < ptr[iq + 1]; e += 32) {
          const int j = col[e];
          const double k = kv[e];
          g0 += k * (X[j] - x0);
          g1 += k * (X[M + j] - x1);
          g2 += k * (X[2LL * M + j] - x2);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          g0 += __shfl_xor_sync(0xffffffffu, g0, off);
          g1 += __shfl_xor_sync(0xffffffffu, g1, off);
          g2 += __shfl_xor_sync(0xffffffffu, g2, off);
        }
        if (lane == 0) { c[iq] = g0; c[M + iq] = g1; c[2LL * M + iq] = g2; }
      }
      continue;
    }
    double f0 = 0, f1 = 0, f2 = 0;
    if (ok) {
      const double x0 = X[i], x1 = X[M + i], x2 = X[2LL * M + i];
      for (int e = ptr[i] + sl; e < ptr[i + 1]; e += 8) {
        const int j = col[e];
        const double k = kv[e];
        f0 += k * (X[j] - x0);
        f1 += k * (X[M + j] - x1);
        f2 += k * (X[2LL * M + j] - x2);
      }
    }
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) {
      f0 += __shfl_xor_sync(0xffffffffu, f0, off, 8);
      f1 += __shfl_xor_sync(0xffffffffu, f1, off, 8);
      f2 += __shfl_xor_sync(0xffffffffu, f2, off, 8);
    }
    if (ok && sl == 0) { c[i] = f0; c[M + i] = f1; c[2LL * M + i] = f2; }
  }
  }
};

// Target points: c = omega K (X~ - X) over all d*M entries (Sec. 5.2.2).
struct KForceTarget {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(const double* __restrict__ X, const double* __restrict__ Xt,
                             double* __restrict__ c, long long n, double wK) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
      c[i] = wK * (Xt[i] - X[i]);
  }
};

// Surface tension E = gamma S (Sec. 6.2.4): F_i = -(gamma/2) sum over the triangles (i, j, k)
// at node i of (X_j - X_k) x n_ijk, n_ijk the unit normal of (X_i, X_j, X_k) (omega = 1).
// inc[e] = (j, k) lists each triangle at node i in its counter-clockwise order from i
// (CSR rows ptr). Eight lanes per vertex as in k_force_mesh.
struct KForceTension {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(const double* __restrict__ X, double* __restrict__ c, int M,
                             const int* __restrict__ ptr, const int2* __restrict__ inc, double half_gamma) {
  const int sl = threadIdx.x & 7, sub = (threadIdx.x >> 3) & 3;
  for (long long w0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4; w0 < M;
       w0 += (((long long)gridDim.x * blockDim.x) >> 5) * 4) {
    const int i = (int)(w0 + sub);
    const bool ok = i < M;
    double f0 = 0, f1 = 0, f2 = 0;
    if (ok) {
      const double x0 = X[i], x1 = X[M + i], x2 = X[2LL * M + i];
      for (int e = ptr[i] + sl; e < ptr[i + 1]; e += 8) {
        const int2 jk = inc[e];
        const double a0 = X[jk.x] - x0, a1 = X[M + jk.x] - x1, a2 = X[2LL * M + jk.x] - x2;
        const double b0 = X[jk.y] - x0, b1 = X[M + jk.y] - x1, b2 = X[2LL * M + jk.y] - x2;
        double n0 = a1 * b2 - a2 * b1, n1 = a2 * b0 - a0 * b2, n2 = a0 * b1 - a1 * b0;
        const double inv = 1.0 / sqrt(n0 * n0 + n1 * n1 + n2 * n2);
        n0 *= inv; n1 *= inv; n2 *= inv;
        const double e0 = a0 - b0, e1 = a1 - b1, e2 = a2 - b2;  // X_j - X_k
        f0 -= half_gamma * (e1 * n2 - e2 * n1);
        f1 -= half_gamma * (e2 * n0 - e0 * n2);
        f2 -= half_gamma * (e0 * n1 - e1 * n0);
      }
    }
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) {
      f0 += __shfl_xor_sync(0xffffffffu, f0, off, 8);
      f1 += __shfl_xor_sync(0xffffffffu, f1, off, 8);
      f2 += __shfl_xor_sync(0xffffffffu, f2, off, 8);
    }
    if (ok && sl == 0) { c[i] = f0; c[M + i] = f1; c[2LL * M + i] = f2; }
  }
  }
};

void launch_force(const Plan& p, const Workspace& ws, const double* X, double* c, cudaStream_t st) {
  if (ws.force_kind == 1) {
    const double dth = 2.0 * 3.14159265358979323846 / p.M;
    launch<KForceCurve>(blocks_for(p.M), 256, 0, st, X, c, p.M, ws.curve_K / dth);
  } else if (ws.force_kind == 3) {
    const long long n = (long long)p.d * p.M;
    launch<KForceTarget>(blocks_for(n), 256, 0, st, X, ws.target, c, n, ws.target_wK);
  } else if (ws.force_kind == 4) {
    launch<KForceTension>(blocks_for(8LL * p.M), 256, 0, st, X, c, p.M, ws.csr_ptr, ws.inc_jk, 0.5 * ws.stiffness);
  } else {
    launch<KForceMesh>(blocks_for(8LL * p.M), 256, 0, st, X, c, p.M, ws.csr_ptr, ws.csr_col, ws.csr_k);
  }
}

// K_AB = sum over the triangles of edge AB of (sigma/8)(a0^2 + b0^2 - c0^2)/S0 (Sec. 6.2.3),
// added to both CSR slots of the edge. Each slot receives at most two terms, so
// the result does not depend on the order of the atomic additions.
__device__ __forceinline__ int find_slot(const int* __restrict__ ptr, const int* __restrict__ col, int i, int j) {
  int lo = ptr[i], hi = ptr[i + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int v = col[mid];
    if (v == j) return mid;
    if (v < j) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

__global__ void k_mesh_stiffness(const double* __restrict__ Xr, const int* __restrict__ tri, int ntri, int M,
                                 double sigma, const int* __restrict__ ptr, const int* __restrict__ col,
                                 double* __restrict__ kv) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += gridDim.x * blockDim.x) {
    int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
    double P[3][3];
    for (int q = 0; q < 3; ++q)
      for (int a = 0; a < 3; ++a) P[q][a] = Xr[(long long)a * M + v[q]];
    double e2[3];  // e2[q] = squared length of the edge opposite vertex q
    for (int q = 0; q < 3; ++q) {
      const int u = (q + 1) % 3, w = (q + 2) % 3;
      double s = 0;
      for (int a = 0; a < 3; ++a) { const double dd = P[u][a] - P[w][a]; s += dd * dd; }
      e2[q] = s;
    }
    double ab[3], ac[3];
    for (int a = 0; a < 3; ++a) { ab[a] = P[1][a] - P[0][a]; ac[a] = P[2][a] - P[0][a]; }
    const double cx = ab[1] * ac[2] - ab[2] * ac[1], cy = ab[2] * ac[0] - ab[0] * ac[2],
                 cz = ab[0] * ac[1] - ab[1] * ac[0];
    const double S0 = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
    for (int q = 0; q < 3; ++q) {  // edge opposite vertex q joins the other two
      const int u = v[(q + 1) % 3], w = v[(q + 2) % 3];
      const double kval = sigma / 8.0 * (e2[(q + 1) % 3] + e2[(q + 2) % 3] - e2[q]) / S0;
      const int s1 = find_slot(ptr, col, u, w), s2 = find_slot(ptr, col, w, u);
      if (s1 >= 0) atomicAdd(&kv[s1], kval);
      if (s2 >= 0) atomicAdd(&kv[s2], kval);
    }
  }
}

void launch_mesh_stiffness(const double* Xref, const int* tri, int ntri, int M, double sigma,
                           int* csr_ptr, int* csr_col, double* csr_k, int nnz, cudaStream_t st) {
  cudaMemsetAsync(csr_k, 0, sizeof(double) * (size_t)nnz, st);
  k_mesh_stiffness<<<blocks_for(ntri), 256, 0, st>>>(Xref, tri, ntri, M, sigma, csr_ptr, csr_col, csr_k);
}

// ---------------------------------------------------------------------------
// Reverse mode of one velocity evaluation (quasi-static Stokes):
//   gX_b += s (sum_a Gu[b][a] lam_a + sum_a Gw[b][a] c_a + fw_b),  gsig += s sum_a w_a c_a / sigma
// with Gu = grad u, Gw = grad w at the points ([d][d][M]), fw = spring law applied to w.
// The sigma term goes to per-block partial sums, added in block order by k_vjp_sigma.
// ---------------------------------------------------------------------------
constexpr int kVjpThreads = 256;
__global__ void __launch_bounds__(kVjpThreads)
k_vjp_combine(int d, int M, double s, double inv_sigma, const double* __restrict__ Gu, const double* __restrict__ Gw,
              const double* __restrict__ lam, const double* __restrict__ c, const double* __restrict__ fw,
              const double* __restrict__ w, double* __restrict__ gX, double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
    for (int b = 0; b < d; ++b) {
      double v = fw[(long long)b * M + j];
      for (int a = 0; a < d; ++a) {
        const long long gi = ((long long)b * d + a) * M + j;
        v += Gu[gi] * lam[(long long)a * M + j] + Gw[gi] * c[(long long)a * M + j];
      }
      gX[(long long)b * M + j] += s * v;
    }
    for (int a = 0; a < d; ++a) acc += w[(long long)a * M + j] * c[(long long)a * M + j];
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += sh[i];
    part[blockIdx.x] = s * inv_sigma * t;
  }
}

__global__ void k_vjp_sigma(const double* __restrict__ part, int nblk, double* __restrict__ gsig) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < nblk; ++i) t += part[i];
  *gsig += t;
}

void launch_vjp_combine(int d, int M, double s, double sigma, const double* Gu, const double* Gw,
                        const double* lam, const double* c, const double* fw, const double* w, double* gX,
                        double* part, int nblk, double* gsig, cudaStream_t st) {
  k_vjp_combine<<<nblk, kVjpThreads, 0, st>>>(d, M, s, 1.0 / sigma, Gu, Gw, lam, c, fw, w, gX, part);
  k_vjp_sigma<<<1, 32, 0, st>>>(part, nblk, gsig);
}

// ---------------------------------------------------------------------------
// Invariants: per-block partial sums, then one block adds the partials in a fixed
// order (deterministic).
// Slots: 0 volume/area, 1 E_p, 2 sum |u|^2 (full spectrum), 3..5 u(0) components (real parts),
//        6 max |k.u|/|k|, 7 max |u|, 8 sum |k|^2 |u|^2, 9 non-finite count
// ---------------------------------------------------------------------------
constexpr int kRedSlots = 10;
constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0;
  if (threadIdx.x == 0) for (int i = 0; i < (int)(blockDim.x / 32); ++i) r += sh[i];
  return r;
}
__device__ __forceinline__ double block_max(double v, double* sh) {
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0;
  if (threadIdx.x == 0) for (int i = 0; i < (int)(blockDim.x / 32); ++i) r = fmax(r, sh[i]);
  return r;
}

struct InvGeom {
  int d, M, force_kind, ntri, N, h;
  long long nspec;
  double kunit, curve_K, target_wK, gamma;
};

__global__ void __launch_bounds__(kRedThreads)
k_inv_points(InvGeom g, const double* __restrict__ X, const int* __restrict__ tri,
             const int* __restrict__ ptr, const int* __restrict__ col, const double* __restrict__ kv,
             const double* __restrict__ Xt, double* __restrict__ part) {
  __shared__ double sh[32];
  double vol = 0, ep = 0, bad = 0;
  const int M = g.M;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g.d == 2) {
    const double dth = 2.0 * 3.14159265358979323846 / M;
    for (long long i = t0; i < M; i += stride) {
      const long long ip = (i + 1 == M) ? 0 : i + 1;
      const double x = X[i], y = X[M + i], xp = X[ip], yp = X[M + ip];
      if (g.force_kind != 3) vol += 0.5 * (x * yp - xp * y);  // open walls enclose no area
      if (g.force_kind == 1) ep += 0.5 * g.curve_K / dth * ((xp - x) * (xp - x) + (yp - y) * (yp - y));
      if (!isfinite(x) || !isfinite(y)) bad += 1;
    }
  } else {
    for (long long t = t0; t < g.ntri; t += stride) {
      const int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
      const double ax = X[a], ay = X[M + a], az = X[2LL * M + a];
      const double bx = X[b], by = X[M + b], bz = X[2LL * M + b];
      const double cx = X[c], cy = X[M + c], cz = X[2LL * M + c];
      vol += (ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx)) / 6.0;
      if (g.force_kind == 4) {  // E_p = gamma S
        const double u0 = bx - ax, u1 = by - ay, u2 = bz - az, v0 = cx - ax, v1 = cy - ay, v2 = cz - az;
        const double n0 = u1 * v2 - u2 * v1, n1 = u2 * v0 - u0 * v2, n2 = u0 * v1 - u1 * v0;
        ep += 0.5 * g.gamma * sqrt(n0 * n0 + n1 * n1 + n2 * n2);
      }
    }
    for (long long i = t0; i < M; i += stride) {
      const double x0 = X[i], x1 = X[M + i], x2 = X[2LL * M + i];
      if (!isfinite(x0) || !isfinite(x1) || !isfinite(x2)) bad += 1;
      if (g.force_kind == 2) {
        for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
          const int j = col[e];
          const double d0 = X[j] - x0, d1 = X[M + j] - x1, d2 = X[2LL * M + j] - x2;
          ep += 0.25 * kv[e] * (d0 * d0 + d1 * d1 + d2 * d2);  // each edge seen twice
        }
      }
    }
  }
  if (g.force_kind == 3) {  // E_p = (omega K / 2) sum |X~ - X|^2
    for (long long i = t0; i < (long long)g.d * M; i += stride) {
      const double e = Xt[i] - X[i];
      ep += 0.5 * g.target_wK * e * e;
    }
  }
  const double r0 = block_sum(vol, sh);
  const double r1 = block_sum(ep, sh);
  const double r9 = block_sum(bad, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x * kRedSlots + 0] = r0;
    part[blockIdx.x * kRedSlots + 1] = r1;
    part[blockIdx.x * kRedSlots + 9] = r9;
  }
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads)
k_inv_spectrum(InvGeom g, const C<T>* __restrict__ u, double* __restrict__ part) {
  __shared__ double sh[32];
  double e = 0, dk = 0, mdiv = 0, mu = 0, bad = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int N = g.N, h = g.h;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nspec; idx += stride) {
    const int ix = (int)(idx % h);
    const long long r = idx / h;
    const int iy = (int)(r % N), iz = (g.d == 3) ? (int)(r / N) : 0;
    if (iy == N / 2 || (g.d == 3 && iz == N / 2)) continue;
    const int my = iy < N / 2 ? iy : iy - N, mz = iz < N / 2 ? iz : iz - N;
    const double k[3] = {g.kunit * ix, g.kunit * my, g.kunit * mz};
    const double k2 = k[0] * k[0] + k[1] * k[1] + (g.d == 3 ? k[2] * k[2] : 0.0);
    // represented value: H(m) for m_x > 0, Hermitian part (H(m) + conj H(-m))/2 on m_x = 0
    long long mirror = idx;
    if (ix == 0) {
      const int jy = (N - iy) % N, jz = (N - iz) % N;
      mirror = ((long long)jz * N + jy) * h;
    }
    const double wgt = (ix == 0) ? 1.0 : 2.0;  // m_x > 0 stands for m and -m
    double kr = 0, ki = 0, n2 = 0;
    for (int a = 0; a < g.d; ++a) {
      C<T> v = u[a * g.nspec + idx];
      double vr = (double)v.x, vi = (double)v.y;
      if (ix == 0) {
        const C<T> m = u[a * g.nspec + mirror];
        vr = 0.5 * (vr + (double)m.x);
        vi = 0.5 * (vi - (double)m.y);
      }
      if (!isfinite(vr) || !isfinite(vi)) bad += 1;
      n2 += vr * vr + vi * vi;
      kr += k[a] * vr; ki += k[a] * vi;
      if (idx == 0) part[3 + a] = vr;  // k = 0; idx 0 is handled by thread 0 of block 0
    }
    e += wgt * n2;
    dk += wgt * k2 * n2;
    mu = fmax(mu, sqrt(n2));
    if (k2 > 0) mdiv = fmax(mdiv, sqrt((kr * kr + ki * ki) / k2));
  }
  const double r2 = block_sum(e, sh);
  const double r8 = block_sum(dk, sh);
  const double r9 = block_sum(bad, sh);
  const double r6 = block_max(mdiv, sh);
  const double r7 = block_max(mu, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x * kRedSlots + 2] = r2;
    part[blockIdx.x * kRedSlots + 6] = r6;
    part[blockIdx.x * kRedSlots + 7] = r7;
    part[blockIdx.x * kRedSlots + 8] = r8;
    part[blockIdx.x * kRedSlots + 9] += r9;
  }
}

__global__ void k_inv_final(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[kRedSlots] = {0};
  for (int b = 0; b < nblk; ++b) {
    const int sum_slots[5] = {0, 1, 2, 8, 9};
    for (int qi = 0; qi < 5; ++qi) s[sum_slots[qi]] += part[b * kRedSlots + sum_slots[qi]];
    s[6] = fmax(s[6], part[b * kRedSlots + 6]);
    s[7] = fmax(s[7], part[b * kRedSlots + 7]);
  }
  s[3] = part[3]; s[4] = part[4]; s[5] = part[5];
  for (int q = 0; q < kRedSlots; ++q) out[q] = s[q];
}

template <typename T>
int run_invariants(const Plan& p, Workspace& ws, const double* X, const C<T>* uhat, double* out,
                   cudaStream_t st) {
  InvGeom g;
  g.d = p.d; g.M = p.M; g.force_kind = ws.force_kind; g.ntri = ws.ntri; g.N = p.N; g.h = p.N / 2;
  g.nspec = (long long)g.h * p.N * (p.d == 3 ? p.N : 1);
  g.kunit = 2.0 * 3.14159265358979323846 / p.L;
  g.curve_K = ws.curve_K;
  g.target_wK = ws.target_wK;
  g.gamma = ws.stiffness;
  const int nblk = ws.red_blocks;
  double* part = ws.red;
  double* res = ws.red + (size_t)nblk * kRedSlots;
  cudaMemsetAsync(part, 0, sizeof(double) * ((size_t)nblk * kRedSlots + kRedSlots), st);
  k_inv_points<<<nblk, kRedThreads, 0, st>>>(g, X, ws.tri, ws.csr_ptr, ws.csr_col, ws.csr_k, ws.target, part);
  if (uhat) k_inv_spectrum<T><<<nblk, kRedThreads, 0, st>>>(g, uhat, part);
  k_inv_final<<<1, 32, 0, st>>>(part, nblk, res);
  double h[kRedSlots];
  if (cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return FSIB_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FSIB_ECUDA;
  const double rho = p.stokes ? 1.0 : p.rho;
  const double Ld = (p.d == 3) ? p.L * p.L * p.L : p.L * p.L;
  out[0] = h[0];
  out[1] = h[1];
  out[2] = uhat ? 0.5 * rho * Ld * h[2] : 0.0;
  out[3] = uhat ? sqrt(h[3] * h[3] + h[4] * h[4] + (p.d == 3 ? h[5] * h[5] : 0.0)) : 0.0;
  out[4] = (uhat && h[7] > 0) ? h[6] / h[7] : 0.0;
  out[5] = uhat ? p.mu * Ld * h[8] : 0.0;
  return h[9] > 0 ? FSIB_ENONFINITE : FSIB_OK;
}

// Channel flux (Eq. poiseuille_flux): Phi = int_{y0}^{y1} ubar(y) dy with ubar the average of
// u_comp over the axes other than `axis`. Only the modes m e_axis survive the average, so
// Phi = Re sum_m u-hat(m e_axis) I(m) with I(0) = y1 - y0 and
// I(m) = (e^{i k y1} - e^{i k y0}) / (i k), k = 2 pi m / L. Along x the half spectrum
// holds m >= 0 and each m > 0 stands for m and -m (twice the real part). One block.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
k_band_flux(const C<T>* __restrict__ u, int N, long long nspec, int comp, int axis, double kunit,
            double y0, double y1, double* __restrict__ out) {
  __shared__ double sh[32];
  const int h = N / 2;
  const int nm = (axis == 0) ? h : N;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nm; i += blockDim.x) {
    if (axis != 0 && i == h) continue;  // unpaired mode -N/2 (zero)
    const int m = (axis == 0 || i < h) ? i : i - N;
    const long long idx = (axis == 0) ? i : (axis == 1 ? (long long)i * h : (long long)i * N * h);
    double Ir = y1 - y0, Ii = 0.0;
    if (m != 0) {
      const double k = kunit * m;
      double s1, c1, s0, c0;
      sincos(k * y1, &s1, &c1);
      sincos(k * y0, &s0, &c0);
      Ir = (s1 - s0) / k;
      Ii = (c0 - c1) / k;
    }
    const C<T> v = u[comp * nspec + idx];
    const double re = (double)v.x * Ir - (double)v.y * Ii;
    acc += (axis == 0 && m > 0) ? 2.0 * re : re;
  }
  const double r = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = r;
}

template <typename T>
int run_band_flux(const Plan& p, Workspace& ws, const C<T>* uhat, int comp, int axis, double y0, double y1,
                  double* flux, cudaStream_t st) {
  const long long nspec = (long long)(p.N / 2) * p.N * (p.d == 3 ? p.N : 1);
  k_band_flux<T><<<1, kRedThreads, 0, st>>>(uhat, p.N, nspec, comp, axis, 2.0 * 3.14159265358979323846 / p.L,
                                            y0, y1, ws.red);
  if (cudaMemcpyAsync(flux, ws.red, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return FSIB_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FSIB_ECUDA;
  return std::isfinite(*flux) ? FSIB_OK : FSIB_ENONFINITE;
}

template int run_band_flux<float>(const Plan&, Workspace&, const C<float>*, int, int, double, double, double*, cudaStream_t);
template int run_band_flux<double>(const Plan&, Workspace&, const C<double>*, int, int, double, double, double*, cudaStream_t);

template int run_invariants<float>(const Plan&, Workspace&, const double*, const C<float>*, double*, cudaStream_t);
template int run_invariants<double>(const Plan&, Workspace&, const double*, const C<double>*, double*, cudaStream_t);

}  // namespace fsib
