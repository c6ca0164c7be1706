// Fourier-space fluid solves on the half spectrum (Secs. 3.1-3.3, 6.1).
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
  const int ix = (int)(idx % g.h);
  const long long r = idx / g.h;
  const int iy = (int)(r % g.N);
  const int iz = (g.d == 3) ? (int)(r / g.N) : 0;
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
__global__ void k_stokeslet(SpecGeom g, T inv_mu, const C<T>* __restrict__ f, C<T>* __restrict__ u) {
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

// NS substep (Eqs. spatial_2, spatial_3 with V of Algorithm 2):
//   s_a = sum_b i k_b p_ab (divergence form of the dealiased nonlinear term),
//   P = f/rho - s, Q = P - k (k.P)/|k|^2 (|k|^2 := 1 at k = 0), lam = mu dt |k|^2 / rho,
//   half: out = (dt/2 Q + base)/(1 + lam/2); full: out = (dt Q + (1 - lam/2) base)/(1 + lam/2).
// A uniform body force density fb (Sec. 5.2.2) is the coefficient at k = 0 and is added there.
struct Body { double f[3]; };

template <typename T>
__global__ void k_ns_update(SpecGeom g, T inv_rho, T mu_dt_over_rho, T dt, bool half, Body fb,
                            const C<T>* __restrict__ prod, const C<T>* __restrict__ f,
                            const C<T>* __restrict__ base, C<T>* __restrict__ out) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nspec;
       idx += (long long)gridDim.x * blockDim.x) {
    T k[3];
    const bool ok = decode_mode<T>(g, idx, k);
    const int d = g.d;
    const T k2 = k[0] * k[0] + k[1] * k[1] + (d == 3 ? k[2] * k[2] : T(0));
    C<T> P[3];
    for (int a = 0; a < d; ++a) {
      C<T> s = mk<T>(T(0), T(0));
      for (int b = 0; b < d; ++b) {
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        const int ab = (d == 3) ? (lo == 0 ? hi : (lo == 1 ? 2 + hi : 5)) : (lo + hi);
        s = cadd<T>(s, cscale<T>(prod[ab * g.nspec + idx], k[b]));
      }
      s = cmul_i<T>(s);
      C<T> fa = f[a * g.nspec + idx];
      if (idx == 0) fa.x += (T)fb.f[a];
      P[a] = csub<T>(cscale<T>(fa, inv_rho), s);
    }
    C<T> kP = mk<T>(T(0), T(0));
    for (int a = 0; a < d; ++a) kP = cadd<T>(kP, cscale<T>(P[a], k[a]));
    const T ik2 = (k2 > T(0)) ? T(1) / k2 : T(1);
    const T lam = mu_dt_over_rho * k2;
    const T den = T(1) / (T(1) + T(0.5) * lam);
    for (int a = 0; a < d; ++a) {
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

static unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 65535LL * 8) b = 65535LL * 8;
  if (b < 1) b = 1;
  return (unsigned)b;
}

template <typename T>
void launch_stokeslet(const Plan& p, const C<T>* fhat, C<T>* uhat, cudaStream_t st) {
  const SpecGeom g = sgeom(p);
  k_stokeslet<T><<<grid_for(g.nspec), 256, 0, st>>>(g, (T)(1.0 / p.mu), fhat, uhat);
}

template <typename T>
void launch_pressure(const Plan& p, const C<T>* prod, const C<T>* fhat, C<T>* phat, cudaStream_t st) {
  const SpecGeom g = sgeom(p);
  k_pressure<T><<<grid_for(g.nspec), 256, 0, st>>>(g, (T)p.rho, prod, fhat, phat);
}

template <typename T>
void launch_ns_update(const Plan& p, const C<T>* prod, const C<T>* fhat, const C<T>* ubase,
                      C<T>* out, bool half, cudaStream_t st) {
  const SpecGeom g = sgeom(p);
  const Body fb = {{p.fbody[0], p.fbody[1], p.fbody[2]}};
  k_ns_update<T><<<grid_for(g.nspec), 256, 0, st>>>(g, (T)(1.0 / p.rho), (T)(p.mu * p.dt / p.rho),
                                                     (T)p.dt, half, fb, prod, fhat, ubase, out);
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
template void launch_ns_update<float>(const Plan&, const C<float>*, const C<float>*, const C<float>*,
                                      C<float>*, bool, cudaStream_t);
template void launch_ns_update<double>(const Plan&, const C<double>*, const C<double>*, const C<double>*,
                                       C<double>*, bool, cudaStream_t);

}  // namespace fsib
