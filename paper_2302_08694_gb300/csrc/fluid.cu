// Fourier-space fluid solves on the half spectrum (Secs. 3.1-3.3, 6.1).
#include <cstdio>
#include <cstdlib>
#include <type_traits>

#include "fsib_internal.cuh"

namespace fsib {

struct SpecGeom {
  int d, N, h;          // h = N/2 modes along x
  long long nspec;      // modes per component
  double kunit;         // 2 pi / L
};

static SpecGeom sgeom(const Plan& p) {
  SpecGeom g;
  g.d = p.d; g.N = p.N; g.h = p.N / 2;
  g.nspec = (long long)g.h * p.N * (p.d == 3 ? p.N : 1);
  g.kunit = 2.0 * 3.14159265358979323846 / p.L;
  return g;
}

// Decode a half-spectrum index into wavevector components; false on a Nyquist mode.
template <typename T>
__device__ __forceinline__ bool decode_mode(const SpecGeom& g, long long idx, T* k) {
  // 32-bit arithmetic: fewer than 2^31 modes at every supported size
  const unsigned u = (unsigned)idx, r = u / (unsigned)g.h;
  const int ix = (int)(u - r * (unsigned)g.h);
  const int iy = (int)(r % (unsigned)g.N);
  const int iz = (g.d == 3) ? (int)(r / (unsigned)g.N) : 0;
  if (iy == g.N / 2 || (g.d == 3 && iz == g.N / 2)) return false;
  const int my = iy < g.N / 2 ? iy : iy - g.N;
  const int mz = iz < g.N / 2 ? iz : iz - g.N;
  k[0] = (T)(g.kunit * ix);
  k[1] = (T)(g.kunit * my);
  k[2] = (T)(g.kunit * mz);
  return true;
}

// u = mu^-1 (I/|k|^2 - k k^T/|k|^4) f, u(0) = 0 (Eq. stokeslet)
template <typename T>
struct KStokeslet {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  __device__ static void run(SpecGeom g, T inv_mu, const C<T>* __restrict__ f, C<T>* __restrict__ u) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nspec;
       idx += (long long)gridDim.x * blockDim.x) {
    T k[3];
    const bool ok = decode_mode<T>(g, idx, k);
    const T k2 = k[0] * k[0] + k[1] * k[1] + (g.d == 3 ? k[2] * k[2] : T(0));
    C<T> fa[3];
    C<T> kf = mk<T>(T(0), T(0));
    for (int a = 0; a < g.d; ++a) {
      fa[a] = f[a * g.nspec + idx];
      kf = cadd<T>(kf, cscale<T>(fa[a], k[a]));
    }
    for (int a = 0; a < g.d; ++a) {
      C<T> v = mk<T>(T(0), T(0));
      if (ok && k2 > T(0)) {
        const T ik2 = T(1) / k2;
        v = cscale<T>(csub<T>(fa[a], cscale<T>(kf, k[a] * ik2)), inv_mu * ik2);
      }
      u[a * g.nspec + idx] = v;
    }
  }
  }
};

// NS substep (Eqs. spatial_2, spatial_3 with V of Algorithm 2):
//   s_a = sum_b i k_b p_ab (divergence form of the dealiased nonlinear term),
//   P = f/rho - s, Q = P - k (k.P)/|k|^2 (|k|^2 := 1 at k = 0), lam = mu dt |k|^2 / rho,
//   half: out = (dt/2 Q + base)/(1 + lam/2); full: out = (dt Q + (1 - lam/2) base)/(1 + lam/2).
// A uniform body force density fb (Sec. 5.2.2) is the coefficient at k = 0 and is added there.
struct Body { double f[3]; };

template <typename T, int D>
struct KNsUpdate {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  // ktab: (T)(kunit m(i)) for i < N (the same value decode_mode forms); mode indices are 32-bit
  // (fewer than 2^31 modes at every supported size)
  __device__ static void run(SpecGeom g, const T* __restrict__ ktab, T inv_rho, T mu_dt_over_rho, T dt, bool half,
                             Body fb, const C<T>* __restrict__ prod, const C<T>* __restrict__ f,
                             const C<T>* __restrict__ base, C<T>* __restrict__ out) {
  const unsigned nspec = (unsigned)g.nspec, h = (unsigned)g.h, N = (unsigned)g.N;
  for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nspec; idx += gridDim.x * blockDim.x) {
    const unsigned ix = idx % h, r = idx / h;
    const unsigned iy = (D == 3) ? r % N : r, iz = (D == 3) ? r / N : 0u;
    const bool ok = iy != N / 2 && (D != 3 || iz != N / 2);  // not a Nyquist mode
    const T k[3] = {ktab[ix], ktab[iy], (D == 3) ? ktab[iz] : T(0)};
    const T k2 = k[0] * k[0] + k[1] * k[1] + (D == 3 ? k[2] * k[2] : T(0));
    C<T> P[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      C<T> s = mk<T>(T(0), T(0));
#pragma unroll
      for (int b = 0; b < D; ++b) {
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        const int ab = (D == 3) ? (lo == 0 ? hi : (lo == 1 ? 2 + hi : 5)) : (lo + hi);
        s = cadd<T>(s, cscale<T>(prod[ab * g.nspec + idx], k[b]));
      }
      s = cmul_i<T>(s);
      C<T> fa = f[a * g.nspec + idx];
      if (idx == 0) fa.x += (T)fb.f[a];
      P[a] = csub<T>(cscale<T>(fa, inv_rho), s);
    }
    C<T> kP = mk<T>(T(0), T(0));
#pragma unroll
    for (int a = 0; a < D; ++a) kP = cadd<T>(kP, cscale<T>(P[a], k[a]));
    const T ik2 = (k2 > T(0)) ? T(1) / k2 : T(1);
    const T lam = mu_dt_over_rho * k2;
    const T den = T(1) / (T(1) + T(0.5) * lam);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      C<T> v = mk<T>(T(0), T(0));
      if (ok) {
        const C<T> Q = csub<T>(P[a], cscale<T>(kP, k[a] * ik2));
        const C<T> b = base[a * g.nspec + idx];
        if (half) v = cscale<T>(cadd<T>(cscale<T>(Q, T(0.5) * dt), b), den);
        else v = cscale<T>(cadd<T>(cscale<T>(Q, dt), cscale<T>(b, T(1) - T(0.5) * lam)), den);
      }
      out[a * g.nspec + idx] = v;
    }
  }
  }
};

// Pressure (Eq. pressure_poisson_k): p = -i k.(f - rho s)/|k|^2 with p(0) = 0 (mean-free).
// With the divergence form s_a = i sum_b k_b P_ab of the dealiased products P_ab = (u_a u_b)^,
// k.s = i sum_ab k_a k_b P_ab, so p = (-i k.f - rho sum_ab k_a k_b P_ab)/|k|^2.
// prod == nullptr drops the nonlinear term (Stokes). One output component.
template <typename T>
__global__ void k_pressure(SpecGeom g, T rho, const C<T>* __restrict__ prod, const C<T>* __restrict__ f,
                           C<T>* __restrict__ out) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nspec;
       idx += (long long)gridDim.x * blockDim.x) {
    T k[3];
    const bool ok = decode_mode<T>(g, idx, k);
    const int d = g.d;
    const T k2 = k[0] * k[0] + k[1] * k[1] + (d == 3 ? k[2] * k[2] : T(0));
    C<T> v = mk<T>(T(0), T(0));
    if (ok && k2 > T(0)) {
      C<T> kf = mk<T>(T(0), T(0));
      for (int a = 0; a < d; ++a) kf = cadd<T>(kf, cscale<T>(f[a * g.nspec + idx], k[a]));
      v = mk<T>(kf.y, -kf.x);  // -i k.f
      if (prod) {
        C<T> kk = mk<T>(T(0), T(0));
        for (int a = 0; a < d; ++a)
          for (int b = a; b < d; ++b) {
            const int ab = (d == 3) ? (a == 0 ? b : (a == 1 ? 2 + b : 5)) : (a + b);
            kk = cadd<T>(kk, cscale<T>(prod[ab * g.nspec + idx], (a == b ? T(1) : T(2)) * k[a] * k[b]));
          }
        v = csub<T>(v, cscale<T>(kk, rho));
      }
      v = cscale<T>(v, T(1) / k2);
    }
    out[idx] = v;
  }
}

// The same update for FP64 mode in double-float arithmetic: GB300 executes FP64 at a small
// fraction of its FP32 rate, and this kernel is arithmetic-bound in FP64. Inputs and outputs
// stay double; each value is split exactly into hi + lo floats on load and rejoined on store.
// Reciprocals take one Newton step from the float reciprocal (error about 2^-46).
__device__ __forceinline__ dd dd_rcp(dd a) {
  const dd r(__frcp_rn(a.hi));
  return r + r * (dd(1.0f) - a * r);
}
// Spectra are split into double-float pairs on load and joined on store with integer and FP32
// operations (dd_from_double, dd_to_double).
__device__ __forceinline__ double join_dd(dd a) { return dd_to_double(a); }

struct DDc { dd x, y; };
__device__ __forceinline__ DDc ddc(double2 v) { return {dd_from_double(v.x), dd_from_double(v.y)}; }

template <int D, bool PAIRS>
struct KNsUpdateDD {
  static constexpr int kThreads = 256, kMinBlocks = 0;
  static constexpr bool kAnyGrid = true;
  // prod_: the product coefficients as double2, or as double-float pairs (dd2) when PAIRS
  __device__ static void run(SpecGeom g, dd kunit, dd inv_rho, dd mu_dt_over_rho, dd dt, bool half, Body fb,
                             const void* __restrict__ prod_, const double2* __restrict__ f,
                             const double2* __restrict__ base, double2* __restrict__ out) {
  // 32-bit mode indices (fewer than 2^31 modes at every supported size)
  const unsigned nspec = (unsigned)g.nspec, hh = (unsigned)g.h, NN = (unsigned)g.N;
  for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nspec; idx += gridDim.x * blockDim.x) {
    const unsigned r = idx / hh;
    const int ix = (int)(idx - r * hh);
    const int iy = (D == 3) ? (int)(r % NN) : (int)r, iz = (D == 3) ? (int)(r / NN) : 0;
    const bool ok = !(iy == g.N / 2 || (D == 3 && iz == g.N / 2));
    const int my = iy < g.N / 2 ? iy : iy - g.N, mz = iz < g.N / 2 ? iz : iz - g.N;
    constexpr int d = D;
    const dd k[3] = {kunit * dd((float)ix), kunit * dd((float)my), kunit * dd((float)mz)};
    dd k2 = k[0] * k[0] + k[1] * k[1];
    if (d == 3) k2 = k2 + k[2] * k[2];
    DDc P[3];
    for (int a = 0; a < d; ++a) {
      dd sx(0.0f), sy(0.0f);
      for (int b = 0; b < d; ++b) {
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        const int ab = (d == 3) ? (lo == 0 ? hi : (lo == 1 ? 2 + hi : 5)) : (lo + hi);
        DDc pv;
        if constexpr (PAIRS) {
          const dd2 q = static_cast<const dd2*>(prod_)[ab * g.nspec + idx];
          pv = {q.x, q.y};
        } else {
          pv = ddc(static_cast<const double2*>(prod_)[ab * g.nspec + idx]);
        }
        sx = sx + pv.x * k[b];
        sy = sy + pv.y * k[b];
      }
      double2 fv = f[a * g.nspec + idx];
      if (idx == 0) fv.x += fb.f[a];
      const DDc fa = ddc(fv);
      P[a] = {fa.x * inv_rho + sy, fa.y * inv_rho - sx};  // f/rho - i s
    }
    dd kPx(0.0f), kPy(0.0f);
    for (int a = 0; a < d; ++a) { kPx = kPx + P[a].x * k[a]; kPy = kPy + P[a].y * k[a]; }
    const dd ik2 = (k2.hi > 0.0f) ? dd_rcp(k2) : dd(1.0f);
    const dd lam = mu_dt_over_rho * k2;
    const dd den = dd_rcp(dd(1.0f) + dd(0.5f) * lam);
    const dd cx = kPx * ik2, cy = kPy * ik2;
    const dd hdt = dd(0.5f) * dt, keep = dd(1.0f) - dd(0.5f) * lam;
    for (int a = 0; a < d; ++a) {
      double2 v = make_double2(0.0, 0.0);
      if (ok) {
        const dd qx = P[a].x - k[a] * cx, qy = P[a].y - k[a] * cy;
        const DDc bv = ddc(base[a * g.nspec + idx]);
        dd vx, vy;
        if (half) { vx = (qx * hdt + bv.x) * den; vy = (qy * hdt + bv.y) * den; }
        else { vx = (qx * dt + bv.x * keep) * den; vy = (qy * dt + bv.y * keep) * den; }
        v = make_double2(join_dd(vx), join_dd(vy));
      }
      out[a * g.nspec + idx] = v;
    }
  }
  }
};

// out_a = i k_b in_a on the half spectrum (the unpaired mode -N/2 set to zero)
template <typename T>
__global__ void k_mul_ik(SpecGeom g, int b, const C<T>* __restrict__ in, C<T>* __restrict__ out) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nspec;
       idx += (long long)gridDim.x * blockDim.x) {
    T k[3];
    const bool ok = decode_mode<T>(g, idx, k);
    for (int a = 0; a < g.d; ++a) {
      C<T> v = mk<T>(T(0), T(0));
      if (ok) v = cmul_i<T>(cscale<T>(in[a * g.nspec + idx], k[b]));
      out[a * g.nspec + idx] = v;
    }
  }
}

static unsigned grid_for(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  if (b > 65535LL * 8) b = 65535LL * 8;
  if (b < 1) b = 1;
  return (unsigned)b;
}

template <typename T>
void launch_stokeslet(const Plan& p, const C<T>* fhat, C<T>* uhat, cudaStream_t st) {
  const SpecGeom g = sgeom(p);
  launch<KStokeslet<T>>(grid_for(g.nspec), 256, 0, st, g, (T)(1.0 / p.mu), fhat, uhat);
}

template <typename T>
void launch_pressure(const Plan& p, const C<T>* prod, const C<T>* fhat, C<T>* phat, cudaStream_t st) {
  const SpecGeom g = sgeom(p);
  k_pressure<T><<<grid_for(g.nspec), 256, 0, st>>>(g, (T)p.rho, prod, fhat, phat);
}

template <typename T>
void launch_ns_update(const Plan& p, const void* ktab, const void* prod, bool prod_pairs, const C<T>* fhat,
                      const C<T>* ubase, C<T>* out, bool half, cudaStream_t st) {
  const SpecGeom g = sgeom(p);
  const Body fb = {{p.fbody[0], p.fbody[1], p.fbody[2]}};
  if constexpr (std::is_same<T, double>::value) {
    if (!p.native_fp64) {
      auto run = [&](auto k) {
        using K = typename decltype(k)::type;
        // blocks of 128 threads: at N = 64 the 131072 modes make 1024 blocks, six or seven an SM,
        // where blocks of 256 left a 0.84-wave grid with three or four an SM
        launch<K>(grid_for(g.nspec, 128), 128, 0, st, g, dd(g.kunit), dd(1.0 / p.rho), dd(p.mu * p.dt / p.rho), dd(p.dt),
                  half, fb, prod, (const double2*)fhat, (const double2*)ubase, (double2*)out);
      };
      if (p.d == 3) {
        if (prod_pairs) run(type_tag<KNsUpdateDD<3, true>>());
        else run(type_tag<KNsUpdateDD<3, false>>());
      } else {
        if (prod_pairs) run(type_tag<KNsUpdateDD<2, true>>());
        else run(type_tag<KNsUpdateDD<2, false>>());
      }
      return;
    }
  }
  if (prod_pairs) {
    std::fprintf(stderr, "fsib: double-float product pairs reach a non double-float update\n");
    std::abort();
  }
  auto run = [&](auto k) {
    using K = typename decltype(k)::type;
    launch<K>(grid_for(g.nspec), 256, 0, st, g, (const T*)ktab, (T)(1.0 / p.rho), (T)(p.mu * p.dt / p.rho), (T)p.dt,
              half, fb, (const C<T>*)prod, fhat, ubase, out);
  };
  if (p.d == 3) run(type_tag<KNsUpdate<T, 3>>());
  else run(type_tag<KNsUpdate<T, 2>>());
}

template <typename T>
void launch_mul_ik(const Plan& p, int b, const C<T>* in, C<T>* out, cudaStream_t st) {
  const SpecGeom g = sgeom(p);
  k_mul_ik<T><<<grid_for(g.nspec), 256, 0, st>>>(g, b, in, out);
}
template void launch_mul_ik<float>(const Plan&, int, const C<float>*, C<float>*, cudaStream_t);
template void launch_mul_ik<double>(const Plan&, int, const C<double>*, C<double>*, cudaStream_t);

template void launch_stokeslet<float>(const Plan&, const C<float>*, C<float>*, cudaStream_t);
template void launch_stokeslet<double>(const Plan&, const C<double>*, C<double>*, cudaStream_t);
template void launch_pressure<float>(const Plan&, const C<float>*, const C<float>*, C<float>*, cudaStream_t);
template void launch_pressure<double>(const Plan&, const C<double>*, const C<double>*, C<double>*, cudaStream_t);
template void launch_ns_update<float>(const Plan&, const void*, const void*, bool, const C<float>*, const C<float>*,
                                      C<float>*, bool, cudaStream_t);
template void launch_ns_update<double>(const Plan&, const void*, const void*, bool, const C<double>*,
                                       const C<double>*, C<double>*, bool, cudaStream_t);

}  // namespace fsib
