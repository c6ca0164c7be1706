// C ABI of the FSIB library: planning, workspaces, staging of host arrays, and the
// orchestration of the transforms into spread / interp / fluid update / time step.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <unordered_set>
#include <string>
#include <type_traits>
#include <vector>

#include "fsib_internal.cuh"

using namespace fsib;

#define FSIB_VERSION "0.1.0"

struct fsib_plan {
  Plan p;
  Workspace ws;
  cudaStream_t user = nullptr;
  cudaStream_t own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaStream_t side = nullptr;                        // second branch of a Navier-Stokes step
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fork2 = nullptr, ev_join2 = nullptr;
  cudaEvent_t ev_fork3 = nullptr, ev_join3 = nullptr;
  cudaEvent_t ev_copy = nullptr;  // end of the copy of u-hat to host inside a step
  std::string err;
  bool ready = false;  // workspaces allocated for the current plan
  // per-launch-site profiler
  struct Site { std::string name; double total_ms = 0; int launches = 0; double bytes = 0, flops = 0; };
  struct Pending { int site; cudaEvent_t a, b; };
  bool prof_on = false;
  std::vector<Site> sites;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  // captured step graph
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[4] = {nullptr, nullptr, nullptr, nullptr};
  int graph_kernels = 0;
  unsigned long long gen = 0;  // bumped whenever the work of a step changes (batches re-record then)
};

// The step's work changed (plan, launch shapes, force model): drop the captured graph.
static void invalidate_graph(fsib_plan* h) {
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  ++h->gen;
}

static std::string g_create_err;

namespace fsib {

int check_last(const char* where) {
  (void)where;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FSIB_OK : FSIB_ECUDA;
}

size_t smem_optin() {
  static const int optin = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      v = 48 * 1024;
    }
    return v;
  }();
  return (size_t)optin;
}

Recorder*& recorder() {
  static thread_local Recorder* r = nullptr;
  return r;
}

void raise_smem_limit(const void* kernel) {
  static std::mutex mu;
  static std::unordered_set<const void*> done;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(kernel)) return;
  const int optin = (int)smem_optin();
  // the opt-in limit covers static and dynamic shared memory together
  cudaFuncAttributes fa;
  size_t stat = 0;
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) stat = fa.sharedSizeBytes;
  const int dyn = optin - (int)stat;
  if (dyn > 0 && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess)
    cudaGetLastError();
  done.insert(kernel);
}

}  // namespace fsib

// ---------------------------------------------------------------------------
// Planning
// ---------------------------------------------------------------------------
static bool is_smooth(int n) {
  for (int q : {2, 3})
    while (n % q == 0) n /= q;
  return n == 1;
}
static int smooth_even_at_least(int n) {
  if (n < 2) n = 2;
  while (!(n % 2 == 0 && is_smooth(n))) ++n;
  return n;
}

static void make_fftlen(FftLen& f, int n, int tw_off) {
  f.n = n;
  f.tw_off = tw_off;
  f.nstages = 0;
  int m = n;
  while (m % 4 == 0) { f.radix[f.nstages++] = 4; m /= 4; }
  while (m % 2 == 0) { f.radix[f.nstages++] = 2; m /= 2; }
  while (m % 3 == 0) { f.radix[f.nstages++] = 3; m /= 3; }
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n).
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wq) {
  x.assign(n, 0.0);
  wq.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double pp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
      }
      const double pn = (n == 1) ? z : p1;
      const double pnm1 = (n == 1) ? 1.0 : p0;
      pp = n * (z * pn - pnm1) / (z * z - 1.0);
      const double dz = pn / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z; x[n - 1 - i] = z;
    wq[i] = wq[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

// Fourier transform of the spreading kernel along one axis, in physical units:
// Psi(k) = int phi(2x/(w h)) exp(-i k x) dx = (w h/2) int_{-1}^{1} phi(z) cos(k w h z/2) dz.
static double psi_hat(double k, int w, double beta, double hf, const std::vector<double>& zq,
                      const std::vector<double>& wq) {
  const double a = 0.5 * w * hf;
  double s = 0;
  for (size_t i = 0; i < zq.size(); ++i) {
    const double z = zq[i];
    const double ph = std::exp(beta * (std::sqrt(std::max(0.0, 1.0 - z * z)) - 1.0));
    s += wq[i] * ph * std::cos(k * a * z);
  }
  return a * s;
}

static int plan_sizes(Plan& p, std::string& err) {
  const double pi = 3.14159265358979323846;
  int w = p.width_opt;
  if (w <= 0) w = (int)std::ceil(-std::log(p.tol) / (pi * std::sqrt(1.0 - 1.0 / p.sigma)));
  w = std::min(16, std::max(2, w));
  p.w = w;
  p.beta = 0.97 * pi * w * (1.0 - 1.0 / (2.0 * p.sigma));
  p.nf = smooth_even_at_least(std::max((int)std::ceil(p.sigma * p.N - 1e-9), 2 * w));
  while (p.nf % 8) p.nf = smooth_even_at_least(p.nf + 1);  // boxes of 8 cells tile the grid
  p.Nt = smooth_even_at_least((3 * p.N + 1) / 2);
  const int maxfft = (p.d == 2) ? kMaxFFT2 : kMaxFFT3;
  if (p.nf > maxfft || p.Nt > maxfft) {
    err = "fine or dealiasing grid exceeds the supported FFT length " + std::to_string(maxfft) + " (" +
          std::to_string(p.d) + "D)";
    return FSIB_EUNSUPPORTED;
  }
  int b = p.bin_opt;
  const bool gather = !(p.prec == FSIB_FP64 && p.native_fp64);
  if (gather) {
    if (p.d == 2 && b <= 0) {
      // 2D boxes: the largest side (32, 16, 8) that still gives one box per SM, so that a
      // small grid spreads over the whole GPU (one block per box)
      int dev = 0, sms = 1;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) { cudaGetLastError(); sms = 1; }
      b = 32;
      while (b > 8 && (long long)(p.nf / b) * (p.nf / b) < sms) b /= 2;
    }
    b = (p.d == 2) ? b : 8;  // 3D gather boxes are 8^3 (one run of 8 cells per task)
    if (p.d == 2) { b = std::max(8, std::min(32, b)); b = (b / 8) * 8; }
  } else if (b <= 0) {
    if (p.d == 2) b = 32;
    else b = (p.prec == FSIB_FP64 && w > 8) ? 4 : 8;
  }
  while (b > 8 && p.nf % b) b -= 8;
  while (b > 1 && p.nf % b) b /= 2;
  for (int a = 0; a < 3; ++a) { p.bins[a] = (a < p.d) ? b : 1; p.nbin[a] = (a < p.d) ? p.nf / b : 1; }
  p.nbins = 1;
  for (int a = 0; a < p.d; ++a) p.nbins *= p.nbin[a];
  make_fftlen(p.fl_nf, p.nf, 0);
  make_fftlen(p.fl_nt, p.Nt, p.nf);
  p.fl_nf.tile_p = p.fl_nt.tile_p = p.fft_p;
  p.fl_nf.rows_q = p.fl_nt.rows_q = p.fft_q;
  return FSIB_OK;
}

// ---------------------------------------------------------------------------
// Profiler: CUDA events around a launch site (only while profiling is enabled)
// ---------------------------------------------------------------------------
struct Prof {
  fsib_plan* h;
  int site = -1;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st;
  const char* prev_site = nullptr;  // recording: the enclosing site label, restored on exit
  Prof(fsib_plan* hh, const char* name, double bytes, double flops, cudaStream_t s) : h(hh), st(s) {
    if (Recorder* r = recorder()) {  // recording a batch member's step: label the operations
      prev_site = r->site;
      r->site = name;
      return;
    }
    if (!h->prof_on) return;
    for (size_t i = 0; i < h->sites.size(); ++i)
      if (h->sites[i].name == name) { site = (int)i; break; }
    if (site < 0) {
      fsib_plan::Site x;
      x.name = name;
      h->sites.push_back(x);
      site = (int)h->sites.size() - 1;
    }
    h->sites[site].bytes = bytes;
    h->sites[site].flops = flops;
    for (cudaEvent_t* e : {&a, &b}) {
      if (!h->pool.empty()) { *e = h->pool.back(); h->pool.pop_back(); }
      else cudaEventCreate(e);
    }
    cudaEventRecord(a, st);
  }
  ~Prof() {
    if (prev_site) {
      if (Recorder* r = recorder()) r->site = prev_site;
      return;
    }
    if (site < 0) return;
    cudaEventRecord(b, st);
    h->pending.push_back({site, a, b});
  }
};

static void prof_flush(fsib_plan* h) {
  if (h->pending.empty()) return;
  cudaStreamSynchronize(h->own);
  for (auto& q : h->pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      h->sites[q.site].total_ms += ms;
      h->sites[q.site].launches += 1;
    }
    h->pool.push_back(q.a);
    h->pool.push_back(q.b);
  }
  h->pending.clear();
  cudaGetLastError();
}

static double fft_flops(double lines, int n) { return lines * 5.0 * n * std::log2((double)n); }

// ---------------------------------------------------------------------------
// Workspaces
// ---------------------------------------------------------------------------
static void free_ws(Workspace& ws) {
  void* ptrs[] = {ws.tw, ws.dline, ws.dplane, ws.grid, ws.grid2, ws.s1, ws.s2, ws.s3, ws.s4, ws.fhat, ws.uhalf, ws.bin_of,
                  ws.rank, ws.counts, ws.offsets, ws.occ, ws.nocc, ws.perm, ws.i0, ws.delta, ws.Xh,
                  ws.cw, ws.Uh, ws.omega_ones, ws.red, ws.flag, ws.wts, ws.cwp, ws.ktab,
                  ws.box_ns, ws.box_np, ws.box_so, ws.box_po, ws.box_item, ws.box_sched, ws.box_work, ws.box_done,
                  ws.part, ws.band, ws.band_dil};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  ws.tw = ws.dline = ws.dplane = ws.grid = ws.grid2 = ws.s1 = ws.s2 = ws.s3 = ws.s4 = ws.fhat = ws.uhalf = nullptr;
  ws.bin_of = ws.rank = ws.counts = ws.offsets = ws.occ = ws.nocc = ws.perm = ws.i0 = nullptr;
  ws.delta = nullptr;
  ws.Xh = ws.cw = ws.Uh = ws.omega_ones = ws.red = nullptr;
  ws.flag = nullptr;
  ws.wts = ws.cwp = ws.ktab = nullptr;
  ws.box_ns = ws.box_np = ws.box_so = ws.box_po = ws.box_item = ws.box_sched = ws.box_work = ws.box_done = nullptr;
  ws.part = nullptr;
  ws.band = ws.band_dil = nullptr;
  void* adj[] = {ws.adj_spec, ws.adj_pts, ws.adj_ckpt, ws.adj_part, ws.adj_sig};
  for (void* q : adj)
    if (q) cudaFree(q);
  ws.adj_spec = nullptr; ws.adj_pts = ws.adj_ckpt = ws.adj_part = ws.adj_sig = nullptr;
  ws.adj_ckpt_bytes = 0;
  for (int i = 0; i < 4; ++i) {
    if (ws.stage[i]) cudaFree(ws.stage[i]);
    ws.stage[i] = nullptr; ws.stage_bytes[i] = 0;
  }
  if (ws.miss_host) cudaFreeHost(ws.miss_host);
  ws.miss_host = ws.miss_dev = nullptr;
}

static void free_mesh(Workspace& ws) {
  if (ws.csr_ptr) cudaFree(ws.csr_ptr);
  if (ws.csr_col) cudaFree(ws.csr_col);
  if (ws.csr_k) cudaFree(ws.csr_k);
  if (ws.tri) cudaFree(ws.tri);
  if (ws.inc_jk) cudaFree(ws.inc_jk);
  ws.csr_ptr = ws.csr_col = nullptr; ws.csr_k = nullptr; ws.tri = nullptr; ws.nnz = ws.ntri = 0;
  ws.inc_jk = nullptr;
}

template <typename P>
static int dmalloc(P** ptr, size_t bytes, size_t& total) {
  void* q = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&q, bytes) != cudaSuccess) { cudaGetLastError(); return FSIB_ENOMEM; }
  *ptr = reinterpret_cast<P*>(q);
  total += bytes;
  return FSIB_OK;
}

static size_t g_ws_bytes = 0;
static const int kMinSlice = 128;  // smallest spread slice the workspace is sized for

static int alloc_ws(fsib_plan* h) {
  Plan& p = h->p;
  Workspace& ws = h->ws;
  free_ws(ws);
  h->ready = false;
  invalidate_graph(h);
  const bool f64 = p.prec == FSIB_FP64;
  const size_t rs = f64 ? 8 : 4, cs = 2 * rs;
  const long long N = p.N, hh = p.N / 2, n = p.nf, Nt = p.Nt, d = p.d;
  const long long spec = d * hh * N * (d == 3 ? N : 1);
  long long s = 0;
  if (d == 3) {
    s = std::max({d * n * n * hh, d * n * N * hh, 3 * Nt * N * hh, 6 * Nt * Nt * hh, 6 * N * N * hh,
                  3 * Nt * Nt * hh, 6 * Nt * N * hh});
  } else {
    s = std::max({d * n * hh, 2 * Nt * hh, 3 * Nt * hh, 3 * N * hh});
  }
  const long long gcells = d * n * n * (d == 3 ? n : 1);
  size_t tot = 0;
  int rc = FSIB_OK;
  ws.spec_bytes = (size_t)spec * cs;
  ws.grid_bytes = (size_t)gcells * rs;
  ws.s1_bytes = ws.s2_bytes = (size_t)s * cs;
  const int ntw = p.nf + p.Nt;
  rc |= dmalloc(&ws.tw, (size_t)ntw * cs, tot);
  rc |= dmalloc(&ws.dline, (size_t)N * rs, tot);
  rc |= dmalloc(&ws.dplane, (size_t)(d == 3 ? N * hh : hh) * rs, tot);
  rc |= dmalloc(&ws.grid, ws.grid_bytes, tot);
  rc |= dmalloc(&ws.s1, ws.s1_bytes, tot);
  rc |= dmalloc(&ws.s2, ws.s2_bytes, tot);
  if (!p.stokes) {
    rc |= dmalloc(&ws.s3, ws.s1_bytes, tot);
    rc |= dmalloc(&ws.s4, ws.s1_bytes, tot);
    rc |= dmalloc(&ws.grid2, ws.grid_bytes, tot);
  }
  rc |= dmalloc(&ws.fhat, ws.spec_bytes, tot);
  rc |= dmalloc(&ws.uhalf, ws.spec_bytes, tot);
  rc |= dmalloc(&ws.bin_of, sizeof(int) * p.M, tot);
  rc |= dmalloc(&ws.rank, sizeof(int) * p.M, tot);
  rc |= dmalloc(&ws.counts, sizeof(int) * (size_t)p.nbins, tot);
  if (ws.counts && cudaMemset(ws.counts, 0, sizeof(int) * (size_t)p.nbins) != cudaSuccess) rc |= FSIB_ECUDA;
  rc |= dmalloc(&ws.offsets, sizeof(int) * (size_t)(p.nbins + 1), tot);
  rc |= dmalloc(&ws.occ, sizeof(int) * (size_t)p.nbins, tot);
  rc |= dmalloc(&ws.nocc, sizeof(int), tot);
  rc |= dmalloc(&ws.perm, sizeof(int) * p.M, tot);
  rc |= dmalloc(&ws.i0, sizeof(int) * d * p.M, tot);
  rc |= dmalloc(&ws.delta, rs * d * p.M, tot);
  rc |= dmalloc(&ws.Xh, sizeof(double) * d * p.M, tot);
  rc |= dmalloc(&ws.cw, sizeof(double) * d * p.M, tot);
  rc |= dmalloc(&ws.Uh, sizeof(double) * d * p.M, tot);
  ws.red_blocks = 2 * 152;
  rc |= dmalloc(&ws.red, sizeof(double) * (size_t)(ws.red_blocks + 1) * 10, tot);
  rc |= dmalloc(&ws.flag, sizeof(int) * 4, tot);
  rc |= dmalloc(&ws.wts, sizeof(double) * (size_t)p.M * d * p.w, tot);
  rc |= dmalloc(&ws.cwp, sizeof(double) * (size_t)p.M * d, tot);
  rc |= dmalloc(&ws.ktab, sizeof(double) * (size_t)p.N, tot);
  if (ws.ktab) {  // the same product the device formed per mode: (T)(kunit * m)
    const double kunit = 2.0 * 3.14159265358979323846 / p.L;
    std::vector<double> kd(p.N);
    std::vector<float> kf(p.N);
    for (int i = 0; i < p.N; ++i) {
      const int m = (i < p.N / 2) ? i : i - p.N;
      kd[i] = kunit * m;
      kf[i] = (float)(kunit * m);
    }
    const bool f32 = p.prec == FSIB_MIXED;
    if (cudaMemcpy(ws.ktab, f32 ? (const void*)kf.data() : (const void*)kd.data(),
                   (f32 ? sizeof(float) : sizeof(double)) * (size_t)p.N, cudaMemcpyHostToDevice) != cudaSuccess)
      rc |= FSIB_ECUDA;
  }
  rc |= dmalloc(&ws.box_ns, sizeof(int) * (size_t)p.nbins, tot);
  rc |= dmalloc(&ws.box_np, sizeof(int) * (size_t)p.nbins, tot);
  rc |= dmalloc(&ws.box_so, sizeof(int) * (size_t)(p.nbins + 1), tot);
  rc |= dmalloc(&ws.box_po, sizeof(int) * (size_t)(p.nbins + 1), tot);
  // slices: at most one per non-empty box plus one per kMinSlice candidates (<= 27 M candidates)
  const size_t nslice_cap = (size_t)std::min<long long>(p.nbins + 27 * (long long)p.M / kMinSlice + 64, 17LL * p.nbins);
  rc |= dmalloc(&ws.box_item, sizeof(int) * nslice_cap, tot);
  rc |= dmalloc(&ws.box_sched, sizeof(int) * nslice_cap, tot);
  rc |= dmalloc(&ws.box_work, sizeof(int) * 4, tot);
  rc |= dmalloc(&ws.box_done, sizeof(int) * (size_t)p.nbins, tot);
  rc |= dmalloc(&ws.band, (size_t)p.nbin[1] * (d == 3 ? p.nbin[2] : 1), tot);
  rc |= dmalloc(&ws.band_dil, (size_t)p.nbin[1] * (d == 3 ? p.nbin[2] : 1), tot);
  // partial slots: boxes with K > 1 hold K slots, K <= 2 cand/256; sum cand <= 27 M
  // (and at most 16 per box: dense point sets get larger slices)
  ws.part_slots = (d == 3) ? (size_t)std::min<long long>(2 * 27 * (long long)p.M / kMinSlice + 64, 16LL * p.nbins) : 1;
  rc |= dmalloc(&ws.part, (d == 3) ? sizeof(double) * 3 * 512 * ws.part_slots : gather2d_part_bytes(p), tot);
  // the 2D gather's completion counters return to zero after each use; they start at zero
  if (ws.box_done && cudaMemset(ws.box_done, 0, sizeof(int) * (size_t)p.nbins) != cudaSuccess) rc |= FSIB_ECUDA;
  if (cudaHostAlloc((void**)&ws.miss_host, sizeof(unsigned int), cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    ws.miss_host = nullptr;
    rc |= FSIB_ENOMEM;
  } else {
    *ws.miss_host = 0u;
    if (cudaHostGetDevicePointer((void**)&ws.miss_dev, ws.miss_host, 0) != cudaSuccess) {
      cudaGetLastError();
      rc |= FSIB_ENOMEM;
    }
  }
  if (rc != FSIB_OK) { free_ws(ws); h->err = "device allocation failed"; return FSIB_ENOMEM; }
  g_ws_bytes = tot;

  // twiddles exp(-2 pi i j/n) for the fine and dealiasing lengths
  const double pi = 3.14159265358979323846;
  std::vector<double> twd(2 * (size_t)ntw);
  auto fill = [&](int nn, int off) {
    for (int j = 0; j < nn; ++j) {
      const double ang = 2.0 * pi * (double)j / (double)nn;
      twd[2 * (off + j)] = std::cos(ang);
      twd[2 * (off + j) + 1] = -std::sin(ang);
    }
  };
  fill(p.nf, 0);
  fill(p.Nt, p.nf);
  // deconvolution: D[i] = h_f / Psi(k_i) per axis, FFT order, the unpaired mode -N/2 -> 0
  std::vector<double> zq, wq;
  gauss_legendre(std::max(64, 4 * p.w + 64), zq, wq);
  const double hf = p.L / p.nf;
  std::vector<double> D(N), Dp(d == 3 ? N * hh : hh);
  for (long long i = 0; i < N; ++i) {
    const long long m = (i < N / 2) ? i : i - N;
    D[i] = (i == N / 2) ? 0.0 : hf / psi_hat(2.0 * pi * m / p.L, p.w, p.beta, hf, zq, wq);
  }
  if (d == 3)
    for (long long iy = 0; iy < N; ++iy)
      for (long long ix = 0; ix < hh; ++ix) Dp[iy * hh + ix] = D[iy] * D[ix];
  else
    for (long long ix = 0; ix < hh; ++ix) Dp[ix] = D[ix];
  cudaError_t e = cudaSuccess;
  if (f64 && !p.native_fp64) {
    std::vector<dd> a(twd.begin(), twd.end()), b(D.begin(), D.end()), c(Dp.begin(), Dp.end());
    e = cudaMemcpy(ws.tw, a.data(), a.size() * sizeof(dd), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.dline, b.data(), b.size() * sizeof(dd), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.dplane, c.data(), c.size() * sizeof(dd), cudaMemcpyHostToDevice);
  } else if (f64) {
    e = cudaMemcpy(ws.tw, twd.data(), twd.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.dline, D.data(), D.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.dplane, Dp.data(), Dp.size() * 8, cudaMemcpyHostToDevice);
  } else {
    std::vector<float> a(twd.begin(), twd.end()), b(D.begin(), D.end()), c(Dp.begin(), Dp.end());
    e = cudaMemcpy(ws.tw, a.data(), a.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.dline, b.data(), b.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.dplane, c.data(), c.size() * 4, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) { h->err = std::string("table upload: ") + cudaGetErrorString(e); return FSIB_ECUDA; }
  h->ready = true;
  return FSIB_OK;
}

// Point side per arithmetic: gather spread / warp interp with per-point weight tables for
// the float and dd transforms; FP64 atomics kernels for native FP64.
template <typename TI>
static void spread_points(fsib_plan* h, const double* c, const double* omega, TI* grid, cudaStream_t st);
template <typename TI>
static void interp_points(fsib_plan* h, const TI* grid, double* U, cudaStream_t st, bool guarded = false);
// Row bands of the last gather binning (RowBands): the gather spread writes only those bands,
// and an interpolation that follows the same binning reads only those.
static bool uses_prep(const Plan& p);
static RowBands row_bands(const Plan& p, const Workspace& ws, bool dilated = false) {
  RowBands rb;
  if (!uses_prep(p) || !ws.band || !ws.band_dil) return rb;
  rb.flag = dilated ? ws.band_dil : ws.band;
  rb.n = p.nf;
  rb.b = p.bins[1];
  rb.nby = p.nbin[1];
  rb.d3 = (p.d == 3);
  return rb;
}

// The y passes of a 3D grid skip the z-slabs that no window reaches (see ZSkip).
static ZSkip z_skip(const Plan& p, const Workspace& ws, bool dilated, bool zero) {
  ZSkip zs;
  const RowBands rb = row_bands(p, ws, dilated);
  if (!rb.flag || p.d != 3) return zs;
  zs.flag = rb.flag;
  zs.outer = p.nf;
  zs.b = p.bins[2];
  zs.nby = p.nbin[1];
  zs.zero = zero;
  return zs;
}

template <typename TI>
static void rows_r2c_first(const Plan& p, Workspace& ws, const TI* grid, C<TI>* out, long long nrows,
                           const C<TI>* tw, cudaStream_t st) {
  launch_fft_rows_r2c<TI>(grid, out, nrows, p.N, p.fl_nf, tw, st, row_bands(p, ws));
}

// ---------------------------------------------------------------------------
// Transform sequences. TI is the transform arithmetic (float in mixed mode; dd,
// or double with the "native_fp64" option, in FP64 mode); TA is the element type
// of the spectral arrays at the API (float or double).
// ---------------------------------------------------------------------------
template <typename TI, typename TA>
static void forward_fine(fsib_plan* h, const TI* grid, C<TA>* out, cudaStream_t st) {
  const Plan& p = h->p;
  Workspace& ws = h->ws;
  const int N = p.N, hh = N / 2, n = p.nf, d = p.d;
  const C<TI>* tw = (const C<TI>*)ws.tw;
  C<TI>* s1 = (C<TI>*)ws.s1;
  C<TI>* s2 = (C<TI>*)ws.s2;
  Mult<TI> none;
  Mult<TI> dec;
  dec.scale = (TI)std::pow(p.L, -d);
  dec.dline = (const TI*)ws.dline;
  dec.dplane = (const TI*)ws.dplane;
  const double rs = sizeof(TI), cs = 2.0 * sizeof(TI);
  if (d == 3) {
    { Prof pr(h, "t1.rows_r2c", (double)d * n * n * n * rs + (double)d * n * n * hh * cs, fft_flops(0.5 * d * n * n, n), st);
      rows_r2c_first<TI>(p, ws, grid, s1, (long long)d * n * n, tw, st); }
    { Prof pr(h, "t1.fy_strided", (double)d * n * hh * (n + N) * cs, fft_flops((double)d * n * hh, n), st);
      launch_fft_strided<TI>(s1, s2, d, n, hh, N, p.fl_nf, false, none, tw, st, z_skip(p, ws, false, true)); }
    { Prof pr(h, "t1.fz_strided_deconv", (double)d * N * hh * (n + N) * cs, fft_flops((double)d * N * hh, n), st);
      launch_fft_strided<TI, TI, TA>(s2, out, d, 1, N * hh, N, p.fl_nf, false, dec, tw, st); }
  } else {
    { Prof pr(h, "t1.rows_r2c", (double)d * n * n * rs + (double)d * n * hh * cs, fft_flops(0.5 * d * n, n), st);
      rows_r2c_first<TI>(p, ws, grid, s1, (long long)d * n, tw, st); }
    { Prof pr(h, "t1.fy_strided_deconv", (double)d * hh * (n + N) * cs, fft_flops((double)d * hh, n), st);
      launch_fft_strided<TI, TI, TA>(s1, out, d, 1, hh, N, p.fl_nf, false, dec, tw, st); }
  }
}

template <typename TI, typename TA>
// sa, sb: scratch pair (default S1, S2).
// banded: the grid feeds an interpolation at the points of the last binning, so the rows that
// none of their windows reaches are not computed (1: those bands; 2: the widened bands of the
// last binning that recorded them, for points that have moved by less than a box since).
static void inverse_fine(fsib_plan* h, const C<TA>* in, TI* grid, cudaStream_t st, void* sa = nullptr,
                         void* sb = nullptr, int banded = 0) {
  const Plan& p = h->p;
  Workspace& ws = h->ws;
  const int N = p.N, hh = N / 2, n = p.nf, d = p.d;
  const C<TI>* tw = (const C<TI>*)ws.tw;
  C<TI>* s1 = (C<TI>*)(sa ? sa : ws.s1);
  C<TI>* s2 = (C<TI>*)(sb ? sb : ws.s2);
  Mult<TI> none;
  Mult<TI> dec;
  dec.dline = (const TI*)ws.dline;
  dec.dplane = (const TI*)ws.dplane;
  const double rs = sizeof(TI), cs = 2.0 * sizeof(TI);
  if (d == 3) {
    { Prof pr(h, "t2.iz_strided_deconv", (double)d * N * hh * (n + N) * cs, fft_flops((double)d * N * hh, n), st);
      launch_fft_strided<TI, TA, TI>(in, s1, d, 1, N * hh, N, p.fl_nf, true, dec, tw, st); }
    { Prof pr(h, "t2.iy_strided", (double)d * n * hh * (n + N) * cs, fft_flops((double)d * n * hh, n), st);
      launch_fft_strided<TI>(s1, s2, d, n, hh, N, p.fl_nf, true, none, tw, st,
                             banded ? z_skip(p, ws, banded == 2, false) : ZSkip()); }
    { Prof pr(h, "t2.ix_rows_c2r", (double)d * n * n * n * rs + (double)d * n * n * hh * cs, fft_flops(0.5 * d * n * n, n), st);
      launch_fft_rows_c2r<TI>(s2, grid, (long long)d * n * n, N, p.fl_nf, tw, st,
                              banded ? row_bands(p, ws, banded == 2) : RowBands()); }
  } else {
    { Prof pr(h, "t2.iy_strided_deconv", (double)d * hh * (n + N) * cs, fft_flops((double)d * hh, n), st);
      launch_fft_strided<TI, TA, TI>(in, s2, d, 1, hh, N, p.fl_nf, true, dec, tw, st); }
    { Prof pr(h, "t2.ix_rows_c2r", (double)d * n * n * rs + (double)d * n * hh * cs, fft_flops(0.5 * d * n, n), st);
      launch_fft_rows_c2r<TI>(s2, grid, (long long)d * n, N, p.fl_nf, tw, st,
                              banded ? row_bands(p, ws, banded == 2) : RowBands()); }
  }
}

// Fourier coefficients on K_N of the products u_a u_b (three-halves rule); returns the buffer. It
// holds C<TA> values, or with pairs and double-float transforms the double-float pairs themselves
// (the Navier-Stokes update reads those without a join and a split per value).
template <typename TI, typename TA>
static const void* products(fsib_plan* h, const C<TA>* u, cudaStream_t st, void* scratch1, void* scratch2,
                            bool pairs = false) {
  const bool keep = pairs && std::is_same<TI, dd>::value;
  const Plan& p = h->p;
  Workspace& ws = h->ws;
  const int N = p.N, hh = N / 2, nt = p.Nt, d = p.d;
  const C<TI>* tw = (const C<TI>*)ws.tw;
  C<TI>* s1 = (C<TI>*)scratch1;
  C<TI>* s2 = (C<TI>*)scratch2;
  Mult<TI> none;
  Mult<TI> sc;
  const double cs = 2.0 * sizeof(TI);
  if (d == 3) {
    sc.scale = (TI)(1.0 / ((double)nt * nt * nt));
    { Prof pr(h, "nl.iz_strided", 3.0 * N * hh * (N + nt) * cs, fft_flops(3.0 * N * hh, nt), st);
      launch_fft_strided<TI, TA, TI>(u, s1, 3, 1, N * hh, N, p.fl_nt, true, none, tw, st); }
    { Prof pr(h, "nl.iy_strided", 3.0 * nt * hh * (N + nt) * cs, fft_flops(3.0 * nt * hh, nt), st);
      launch_fft_strided<TI>(s1, s2, 3, nt, hh, N, p.fl_nt, true, none, tw, st); }
    { Prof pr(h, "nl.rows_product", 9.0 * nt * nt * hh * cs, fft_flops(0.5 * nt * nt * 9.0, nt), st);
      launch_rows_product<TI>(s2, s1, 3, (long long)nt * nt, N, p.fl_nt, tw, st); }
    { Prof pr(h, "nl.fy_strided", 6.0 * nt * hh * (N + nt) * cs, fft_flops(6.0 * nt * hh, nt), st);
      launch_fft_strided<TI>(s1, s2, 6, nt, hh, N, p.fl_nt, false, none, tw, st); }
    { Prof pr(h, "nl.fz_strided", 6.0 * N * hh * (N + nt) * cs, fft_flops(6.0 * N * hh, nt), st);
      if (keep) launch_fft_strided<TI>(s2, s1, 6, 1, N * hh, N, p.fl_nt, false, sc, tw, st);
      else launch_fft_strided<TI, TI, TA>(s2, (C<TA>*)s1, 6, 1, N * hh, N, p.fl_nt, false, sc, tw, st); }
    return s1;
  } else {
    sc.scale = (TI)(1.0 / ((double)nt * nt));
    { Prof pr(h, "nl.iy_strided", 2.0 * hh * (N + nt) * cs, fft_flops(2.0 * hh, nt), st);
      launch_fft_strided<TI, TA, TI>(u, s2, 2, 1, hh, N, p.fl_nt, true, none, tw, st); }
    { Prof pr(h, "nl.rows_product", 5.0 * nt * hh * cs, fft_flops(0.5 * nt * 5.0, nt), st);
      launch_rows_product<TI>(s2, s1, 2, (long long)nt, N, p.fl_nt, tw, st); }
    { Prof pr(h, "nl.fy_strided", 3.0 * hh * (N + nt) * cs, fft_flops(3.0 * hh, nt), st);
      if (keep) launch_fft_strided<TI>(s1, s2, 3, 1, hh, N, p.fl_nt, false, sc, tw, st);
      else launch_fft_strided<TI, TI, TA>(s1, (C<TA>*)s2, 3, 1, hh, N, p.fl_nt, false, sc, tw, st); }
    return s2;
  }
}

static bool uses_prep(const Plan& p) { return !(p.prec == FSIB_FP64 && p.native_fp64); }

// Sort the points into bins; for the gather kernels also evaluate their kernel weights
// (and, when c is given, their weighted forces) once per sort.
static void do_bin(fsib_plan* h, const double* X, cudaStream_t st, const double* c = nullptr,
                   const double* omega = nullptr, bool dilate = false) {
  const Plan& p = h->p;
  const double rs = (p.prec == FSIB_FP64) ? 8.0 : 4.0;
  {
    Prof pr(h, "sort", 2.0 * p.d * p.M * 8.0 + 4.0 * p.M * 8.0 + p.d * p.M * (4.0 + rs) + 12.0 * p.nbins, 0.0, st);
    launch_bin_points(p, h->ws, X, st, !uses_prep(p), dilate);  // the gather needs no occupied-bin list
  }
  if (!uses_prep(p)) return;
  const double ts = (p.prec == FSIB_FP64) ? 8.0 : 4.0;
  Prof pr(h, "point_weights", (double)p.M * p.d * (p.w * ts + rs + (c ? 8.0 + ts : 0.0)), 0.0, st);
  if (p.prec == FSIB_FP64) launch_point_prep<dd>(p, h->ws, c, omega, st);
  else launch_point_prep<float>(p, h->ws, c, omega, st);
}

// Algorithmic flops of one spread or interp launch: for every cell of every point's
// window, the weight product (d - 1 multiplications) and d multiply-adds (2 flops each).
static double point_flops(const Plan& p) {
  return (double)p.M * std::pow((double)p.w, p.d) * (3.0 * p.d - 1.0);
}

static double point_bytes(const Plan& p) {
  return (double)p.M * (4.0 + p.d * (4.0 + (p.prec == FSIB_FP64 ? 8.0 : 4.0) + 8.0));
}

template <typename TI>
static void spread_points(fsib_plan* h, const double* c, const double* omega, TI* grid, cudaStream_t st) {
  Prof pr(h, "spread", point_bytes(h->p) + (double)h->ws.grid_bytes, point_flops(h->p), st);
  launch_spread_gather<TI>(h->p, h->ws, grid, st);
}
template <>
void spread_points<double>(fsib_plan* h, const double* c, const double* omega, double* grid, cudaStream_t st) {
  { Prof pr(h, "zero_grid", (double)h->ws.grid_bytes, 0.0, st);
    memset_async(h->ws.grid, 0, h->ws.grid_bytes, st); }
  Prof pr(h, "spread", point_bytes(h->p) + (double)h->ws.grid_bytes, point_flops(h->p), st);
  launch_spread<double>(h->p, h->ws, c, omega, grid, st);
}
// guarded: the grid holds only the widened bands of an earlier binning (inverse_fine mode 2);
// a point whose window leaves them gets NaN and raises the handle's miss flag, which the next
// fsib_step, fsib_interp or fsib_invariants turns into FSIB_ENONFINITE (take_miss).
template <typename TI>
static void interp_points(fsib_plan* h, const TI* grid, double* U, cudaStream_t st, bool guarded) {
  Prof pr(h, "interp", point_bytes(h->p) + (double)h->ws.grid_bytes, point_flops(h->p), st);
  launch_interp_warp<TI>(h->p, h->ws, grid, U, st, guarded ? h->ws.band_dil : nullptr,
                         guarded ? h->ws.miss_dev : nullptr);
}
template <>
void interp_points<double>(fsib_plan* h, const double* grid, double* U, cudaStream_t st, bool) {
  Prof pr(h, "interp", point_bytes(h->p) + (double)h->ws.grid_bytes, point_flops(h->p), st);
  launch_interp<double>(h->p, h->ws, grid, U, st);
}

template <typename TI, typename TA>
static void do_spread(fsib_plan* h, const double* X, const double* c, const double* omega, C<TA>* fhat,
                      cudaStream_t st, bool dilate = false) {
  do_bin(h, X, st, c, omega, dilate);
  spread_points<TI>(h, c, omega, (TI*)h->ws.grid, st);
  forward_fine<TI, TA>(h, (const TI*)h->ws.grid, fhat, st);
}

// interp at the points of the last binning
template <typename TI, typename TA>
static void do_interp_sorted(fsib_plan* h, const C<TA>* uhat, double* U, cudaStream_t st, bool banded = false) {
  inverse_fine<TI, TA>(h, uhat, (TI*)h->ws.grid, st, nullptr, nullptr, banded ? 1 : 0);
  interp_points<TI>(h, (const TI*)h->ws.grid, U, st);
}

template <typename TA>
static void do_stokeslet(fsib_plan* h, const C<TA>* fhat, C<TA>* u, cudaStream_t st) {
  Prof pr(h, "stokeslet", 2.0 * (double)h->ws.spec_bytes, 0.0, st);
  launch_stokeslet<TA>(h->p, fhat, u, st);
}

template <typename TI, typename TA>
// P0: the product coefficients of u^m when they were computed beforehand (see do_step), as
// products() returns them with pairs = true.
static void do_fluid(fsib_plan* h, const C<TA>* fhat, C<TA>* u, C<TA>* uhalf, cudaStream_t st,
                     const void* P0 = nullptr) {
  constexpr bool kPairs = std::is_same<TI, dd>::value;  // products kept as double-float pairs
  if (h->p.stokes) {
    do_stokeslet<TA>(h, fhat, u, st);
    return;
  }
  const int d = h->p.d, np = d * (d + 1) / 2;
  const double ub = (double)h->ws.spec_bytes / d * (np + 3 * d);
  const void* P = P0 ? P0 : products<TI, TA>(h, u, st, h->ws.s1, h->ws.s2, true);
  { Prof pr(h, "ns_update", ub, 0.0, st);
    launch_ns_update<TA>(h->p, h->ws.ktab, P, kPairs, fhat, u, uhalf, true, st); }
  P = products<TI, TA>(h, uhalf, st, h->ws.s1, h->ws.s2, true);
  { Prof pr(h, "ns_update", ub, 0.0, st);
    launch_ns_update<TA>(h->p, h->ws.ktab, P, kPairs, fhat, u, u, false, st); }
}

template <typename TI, typename TA>
static void do_pressure(fsib_plan* h, const C<TA>* fhat, const C<TA>* u, C<TA>* phat, cudaStream_t st) {
  const C<TA>* P = (!h->p.stokes && u) ? (const C<TA>*)products<TI, TA>(h, u, st, h->ws.s1, h->ws.s2) : nullptr;
  launch_pressure<TA>(h->p, P, fhat, phat, st);
}

static void do_axpy(fsib_plan* h, double* y, const double* x, const double* v, double a, cudaStream_t st) {
  const long long dm = (long long)h->p.d * h->p.M;
  Prof pr(h, "positions", 24.0 * dm, 0.0, st);
  launch_axpy(y, x, v, a, dm, st);
}

static void do_force(fsib_plan* h, const double* X, double* c, cudaStream_t st) {
  const Plan& p = h->p;
  Prof pr(h, "force", 16.0 * p.d * p.M + 12.0 * h->ws.nnz + 4.0 * p.M, 0.0, st);
  launch_force(p, h->ws, X, c, st);
}

// One time step on device arrays (Algorithm 1, or the quasi-static Stokes midpoint rule).
// u_in / u_out (Navier-Stokes, pinned host memory, or NULL): u-hat^m is copied in from u_in
// at the head of the second stream's branch, so the copy overlaps the force, sort and type-1
// NUFFT, and u-hat^{m+1} is copied out to u_out on the second stream beside the interps.
template <typename TI, typename TA>
static void do_step(fsib_plan* h, double* X, C<TA>* uhat, double* U, cudaStream_t st,
                    const void* u_in = nullptr, void* u_out = nullptr) {
  const Plan& p = h->p;
  Workspace& ws = h->ws;
  const long long dm = (long long)p.d * p.M;
  C<TA>* fhat = (C<TA>*)ws.fhat;
  C<TA>* uh = (C<TA>*)ws.uhalf;
  if (!p.stokes) {
    // The nonlinear term of u^m does not depend on the boundary: its transforms run on a
    // second stream (own scratch s3, s4) while the force and the type-1 NUFFT run here.
    // While the profiler times launch sites, the branch runs in line so that no two sites overlap.
    const bool fork = !h->prof_on && !recorder();
    cudaStream_t sb = fork ? h->side : st;
    if (fork) {
      cudaEventRecord(h->ev_fork, st);
      cudaStreamWaitEvent(h->side, h->ev_fork, 0);
    }
    if (u_in) cudaMemcpyAsync(uhat, u_in, ws.spec_bytes, cudaMemcpyHostToDevice, sb);
    constexpr bool kPairs = std::is_same<TI, dd>::value;  // products kept as double-float pairs
    const void* P0 = products<TI, TA>(h, uhat, sb, ws.s3, ws.s4, true);
    if (fork) cudaEventRecord(h->ev_join, h->side);
    do_axpy(h, ws.Xh, X, U, 0.5 * p.dt, st);                    // Eq. spatial_1
    do_force(h, ws.Xh, ws.cw, st);                               // F^{m+1/2}
    do_spread<TI, TA>(h, ws.Xh, ws.cw, nullptr, fhat, st, true); // type-1 NUFFT; widened bands for U^{m+1}
    if (fork) cudaStreamWaitEvent(st, h->ev_join, 0);
    // Eqs. spatial_2, spatial_3. The type-2 prep of u^{m+1/2} needs only the half step: it runs
    // on the second stream (scratch S3/S4, fine grid) beside the second nonlinear term and the
    // full step; the type-2 prep of u^{m+1} follows it there (second fine grid), beside the
    // U^{m+1/2} interp and the re-sort.
    const double ub = (double)ws.spec_bytes / p.d * (p.d * (p.d + 1) / 2 + 3 * p.d);
    { Prof pr(h, "ns_update", ub, 0.0, st);
      launch_ns_update<TA>(p, ws.ktab, P0, kPairs, fhat, uhat, uh, true, st); }
    if (fork) {
      cudaEventRecord(h->ev_fork3, st);
      cudaStreamWaitEvent(h->side, h->ev_fork3, 0);
    }
    inverse_fine<TI, TA>(h, uh, (TI*)ws.grid, sb, ws.s3, ws.s4, 1);  // binning of X^{m+1/2}
    if (fork) cudaEventRecord(h->ev_join3, h->side);
    const void* P1 = products<TI, TA>(h, uh, st, ws.s1, ws.s2, true);
    { Prof pr(h, "ns_update", ub, 0.0, st);
      launch_ns_update<TA>(p, ws.ktab, P1, kPairs, fhat, uhat, uhat, false, st); }
    if (fork) {
      cudaEventRecord(h->ev_fork2, st);
      cudaStreamWaitEvent(h->side, h->ev_fork2, 0);
    }
    inverse_fine<TI, TA>(h, uhat, (TI*)ws.grid2, sb, ws.s3, ws.s4, 2);  // widened bands of X^{m+1/2}
    if (fork) {
      cudaEventRecord(h->ev_join2, h->side);
      cudaStreamWaitEvent(st, h->ev_join3, 0);
    }
    if (u_out) {  // after the join point: the final interp does not wait for the copy
      cudaMemcpyAsync(u_out, uhat, ws.spec_bytes, cudaMemcpyDeviceToHost, sb);
      if (fork) cudaEventRecord(h->ev_copy, h->side);
    }
    interp_points<TI>(h, (const TI*)ws.grid, ws.Uh, st);         // U^{m+1/2} at X^{m+1/2}
    do_axpy(h, X, X, ws.Uh, p.dt, st);                           // Eq. spatial_4
    do_bin(h, X, st);
    if (fork) cudaStreamWaitEvent(st, h->ev_join2, 0);
    interp_points<TI>(h, (const TI*)ws.grid2, U, st, true);      // U^{m+1} at X^{m+1}
    if (u_out && fork) cudaStreamWaitEvent(st, h->ev_copy, 0);
  } else {
    // U(X^m)
    do_force(h, X, ws.cw, st);
    do_spread<TI, TA>(h, X, ws.cw, nullptr, fhat, st);
    do_stokeslet<TA>(h, fhat, uh, st);
    do_interp_sorted<TI, TA>(h, uh, ws.Uh, st, true);
    do_axpy(h, ws.Xh, X, ws.Uh, 0.5 * p.dt, st);
    // U(X^{m+1/2})
    do_force(h, ws.Xh, ws.cw, st);
    do_spread<TI, TA>(h, ws.Xh, ws.cw, nullptr, fhat, st);
    do_stokeslet<TA>(h, fhat, uh, st);
    do_interp_sorted<TI, TA>(h, uh, ws.Uh, st, true);
    do_axpy(h, X, X, ws.Uh, p.dt, st);
    if (U) memcpy_async(U, ws.Uh, sizeof(double) * dm, cudaMemcpyDeviceToDevice, st);
    if (uhat) memcpy_async(uhat, uh, ws.spec_bytes, cudaMemcpyDeviceToDevice, st);
  }
}

// Run f<TI, TA> for the handle's arithmetic.
#define FSIB_DISPATCH(h, CALL_F, CALL_DD, CALL_D) \
  do {                                            \
    if ((h)->p.prec == FSIB_MIXED) { CALL_F; }    \
    else if ((h)->p.native_fp64) { CALL_D; }      \
    else { CALL_DD; }                             \
  } while (0)

// ---------------------------------------------------------------------------
// Entry helpers
// ---------------------------------------------------------------------------
static int fail(fsib_plan* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

static bool is_pinned_host(const void* q) {
  cudaPointerAttributes a;
  if (!q || cudaPointerGetAttributes(&a, q) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeHost;
}

static bool is_device_ptr(const void* q) {
  if (!q) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, q) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Begin a call: order the own stream after the user's stream.
static int begin(fsib_plan* h) {
  if (!h) return FSIB_EINVAL;
  if (!h->ready) return fail(h, FSIB_ESTATE, "workspaces not allocated");
  h->err.clear();
  if (cudaEventRecord(h->ev_in, h->user) != cudaSuccess) return fail(h, FSIB_ECUDA, "event record failed");
  if (cudaStreamWaitEvent(h->own, h->ev_in, 0) != cudaSuccess) return fail(h, FSIB_ECUDA, "stream wait failed");
  return FSIB_OK;
}

// Report (once) a velocity that a finished step could not interpolate: a point moved more than
// one box of the fine grid in half a step, beyond the rows computed for U^{m+1}. The flag lives
// in mapped host memory, so this reads it without a synchronisation; a step still running on
// the GPU is reported by a later call.
static int take_miss(fsib_plan* h) {
  volatile unsigned int* f = h->ws.miss_host;
  if (!f || *f == 0u) return FSIB_OK;
  *f = 0u;
  return fail(h, FSIB_ENONFINITE,
              "U^{m+1} is NaN at points that moved more than one box (8 fine cells) in half a step; "
              "the time step is far beyond a stable one");
}

static int finish(fsib_plan* h, bool sync) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, FSIB_ECUDA, std::string("CUDA: ") + cudaGetErrorString(e));
  if (cudaEventRecord(h->ev_out, h->own) != cudaSuccess) return fail(h, FSIB_ECUDA, "event record failed");
  if (cudaStreamWaitEvent(h->user, h->ev_out, 0) != cudaSuccess) return fail(h, FSIB_ECUDA, "stream wait failed");
  if (sync) {
    e = cudaStreamSynchronize(h->own);
    if (e != cudaSuccess) return fail(h, FSIB_ECUDA, std::string("CUDA: ") + cudaGetErrorString(e));
  }
  return FSIB_OK;
}

// Device view of an argument: the pointer itself, or a staging buffer (copied in if `in`).
struct Arg {
  void* dev = nullptr;
  void* host = nullptr;
  size_t bytes = 0;
};

static int stage(fsib_plan* h, int slot, const void* q, size_t bytes, bool in, Arg& a) {
  a.bytes = bytes;
  if (!q) { a.dev = nullptr; return FSIB_OK; }
  if (is_device_ptr(q)) { a.dev = const_cast<void*>(q); return FSIB_OK; }
  Workspace& ws = h->ws;
  if (ws.stage_bytes[slot] < bytes) {
    if (ws.stage[slot]) cudaFree(ws.stage[slot]);
    ws.stage[slot] = nullptr;
    ws.stage_bytes[slot] = 0;
    if (cudaMalloc(&ws.stage[slot], bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, FSIB_ENOMEM, "staging allocation failed");
    }
    ws.stage_bytes[slot] = bytes;
  }
  a.dev = ws.stage[slot];
  a.host = const_cast<void*>(q);
  if (in && cudaMemcpyAsync(a.dev, q, bytes, cudaMemcpyHostToDevice, h->own) != cudaSuccess)
    return fail(h, FSIB_ECUDA, "host-to-device copy failed");
  return FSIB_OK;
}

static int unstage(fsib_plan* h, const Arg& a) {
  if (a.host && a.dev && cudaMemcpyAsync(a.host, a.dev, a.bytes, cudaMemcpyDeviceToHost, h->own) != cudaSuccess)
    return fail(h, FSIB_ECUDA, "device-to-host copy failed");
  return FSIB_OK;
}

static size_t spec_bytes(const fsib_plan* h) { return h->ws.spec_bytes; }
static size_t pts_bytes(const fsib_plan* h) { return sizeof(double) * (size_t)h->p.d * h->p.M; }

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* fsib_version(void) { return FSIB_VERSION; }

const char* fsib_last_error(fsib_t h) { return h ? h->err.c_str() : g_create_err.c_str(); }

int fsib_create(fsib_t* out, int N, int d, int M, double mu, double rho, double dt, double tol) {
  g_create_err.clear();
  if (!out) { g_create_err = "out is NULL"; return FSIB_EINVAL; }
  *out = nullptr;
  if (d != 2 && d != 3) { g_create_err = "d must be 2 or 3"; return FSIB_EINVAL; }
  if (N < 4 || N > 1024 || (N % 2)) { g_create_err = "N must be even, 4 <= N <= 1024"; return FSIB_EINVAL; }
  if (M < 1) { g_create_err = "M must be >= 1"; return FSIB_EINVAL; }
  if (!(mu > 0) || !(dt > 0) || !std::isfinite(mu) || !std::isfinite(dt) || !std::isfinite(rho)) {
    g_create_err = "mu and dt must be positive and finite";
    return FSIB_EINVAL;
  }
  if (!(tol >= 1e-14 && tol <= 1e-2)) { g_create_err = "tol must be in [1e-14, 1e-2]"; return FSIB_EINVAL; }
  fsib_plan* h = new fsib_plan();
  Plan& p = h->p;
  p.d = d; p.N = N; p.M = M; p.mu = mu; p.rho = rho; p.dt = dt; p.tol = tol;
  p.stokes = !(rho > 0);
  int rc = plan_sizes(p, h->err);
  if (rc != FSIB_OK) { g_create_err = h->err; delete h; return rc; }
  if (cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork2, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join2, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork3, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join3, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_copy, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    g_create_err = "CUDA stream/event creation failed (no device?)";
    fsib_destroy(h);  // releases the streams and events created before the failure
    return FSIB_ECUDA;
  }
  rc = alloc_ws(h);
  if (rc != FSIB_OK) {
    g_create_err = h->err;
    fsib_destroy(h);
    return rc;
  }
  *out = h;
  return FSIB_OK;
}

int fsib_destroy(fsib_t h) {
  if (!h) return FSIB_OK;
  if (h->own) cudaStreamSynchronize(h->own);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  prof_flush(h);
  for (auto e : h->pool) cudaEventDestroy(e);
  free_ws(h->ws);
  free_mesh(h->ws);
  if (h->ws.target) cudaFree(h->ws.target);
  if (h->side) cudaStreamSynchronize(h->side);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_fork2) cudaEventDestroy(h->ev_fork2);
  if (h->ev_join2) cudaEventDestroy(h->ev_join2);
  if (h->ev_fork3) cudaEventDestroy(h->ev_fork3);
  if (h->ev_join3) cudaEventDestroy(h->ev_join3);
  if (h->ev_copy) cudaEventDestroy(h->ev_copy);
  if (h->own) cudaStreamDestroy(h->own);
  if (h->side) cudaStreamDestroy(h->side);
  delete h;
  return FSIB_OK;
}

int fsib_set_stream(fsib_t h, void* stream) {
  if (!h) return FSIB_EINVAL;
  h->user = (cudaStream_t)stream;
  return FSIB_OK;
}

int fsib_set_option(fsib_t h, const char* key, double v) {
  if (!h || !key) return FSIB_EINVAL;
  Plan q = h->p;
  std::string k(key);
  if (k == "precision") {
    if (v != 0 && v != 1) return fail(h, FSIB_EINVAL, "precision must be 0 or 1");
    q.prec = (int)v;
  } else if (k == "sigma") {
    if (!(v >= 1.5 && v <= 3.0)) return fail(h, FSIB_EINVAL, "sigma must be in [1.5, 3]");
    q.sigma = v;
  } else if (k == "width") {
    if (!(v == 0 || (v >= 2 && v <= 16))) return fail(h, FSIB_EINVAL, "width must be 0 or in [2, 16]");
    q.width_opt = (int)v;
  } else if (k == "bin") {
    if (!(v == 0 || (v >= 4 && v <= 64))) return fail(h, FSIB_EINVAL, "bin must be 0 or in [4, 64]");
    q.bin_opt = (int)v;
  } else if (k == "fft_tile") {
    if (!(v == 4 || v == 8 || v == 16)) return fail(h, FSIB_EINVAL, "fft_tile must be 4, 8 or 16");
    h->p.fft_p = (int)v;
    h->p.fl_nf.tile_p = h->p.fl_nt.tile_p = (int)v;
    invalidate_graph(h);
    return FSIB_OK;
  } else if (k == "fft_rows") {
    if (!(v == 2 || v == 4 || v == 8)) return fail(h, FSIB_EINVAL, "fft_rows must be 2, 4 or 8");
    h->p.fft_q = (int)v;
    h->p.fl_nf.rows_q = h->p.fl_nt.rows_q = (int)v;
    invalidate_graph(h);
    return FSIB_OK;
  } else if (k == "spread_slice") {
    if (!(v >= kMinSlice && v <= 4096)) return fail(h, FSIB_EINVAL, "spread_slice must be in [128, 4096]");
    h->p.slice = (int)v;
    invalidate_graph(h);
    return FSIB_OK;
  } else if (k == "spread_sum") {
    if (!(v == 0 || v == 1 || v == 2)) return fail(h, FSIB_EINVAL, "spread_sum must be 0, 1 or 2");
    h->p.spread_sum = (int)v;
    invalidate_graph(h);
    return FSIB_OK;
  } else if (k == "native_fp64") {
    q.native_fp64 = (v != 0);
  } else if (k == "graph") {
    h->p.use_graph = (v != 0);
    return FSIB_OK;
  } else if (k == "check_finite") {
    h->p.check_finite = (v != 0);
    return FSIB_OK;
  } else {
    return fail(h, FSIB_EINVAL, "unknown option key: " + k);
  }
  std::string err;
  int rc = plan_sizes(q, err);
  if (rc != FSIB_OK) return fail(h, rc, err);
  cudaStreamSynchronize(h->own);
  h->p = q;
  return alloc_ws(h);
}

int fsib_get_info(fsib_t h, const char* key, double* value) {
  if (!h || !key || !value) return FSIB_EINVAL;
  std::string k(key);
  const Plan& p = h->p;
  if (k == "nf") *value = p.nf;
  else if (k == "width") *value = p.w;
  else if (k == "beta") *value = p.beta;
  else if (k == "Nt") *value = p.Nt;
  else if (k == "precision") *value = p.prec;
  else if (k == "bin") *value = p.bins[0];
  else if (k == "sigma") *value = p.sigma;
  else if (k == "native_fp64") *value = p.native_fp64;
  else if (k == "fft_tile") *value = p.fft_p;
  else if (k == "fft_rows") *value = p.fft_q;
  else if (k == "spread_slice") *value = p.slice;
  else if (k == "spread_sum") *value = p.spread_sum;
  else if (k == "workspace_bytes") *value = (double)g_ws_bytes;
  else if (k == "launches_per_step") *value = h->graph_kernels;
  else return fail(h, FSIB_EINVAL, "unknown info key: " + k);
  return FSIB_OK;
}

int fsib_set_force_curve(fsib_t h, double K) {
  if (!h) return FSIB_EINVAL;
  if (h->p.d != 2) return fail(h, FSIB_EINVAL, "curve force needs d = 2");
  if (!std::isfinite(K)) return fail(h, FSIB_EINVAL, "K must be finite");
  h->ws.force_kind = 1;
  h->ws.curve_K = K;
  h->ws.stiffness = K;
  invalidate_graph(h);
  return FSIB_OK;
}

int fsib_set_force_mesh(fsib_t h, const int* tri, int ntri, const double* Xref, double sigma) {
  if (!h || !tri || !Xref || ntri < 1) return FSIB_EINVAL;
  if (h->p.d != 3) return fail(h, FSIB_EINVAL, "mesh force needs d = 3");
  const int M = h->p.M;
  // connectivity on the host (integer work): undirected edges -> CSR adjacency
  std::vector<int> t(3 * (size_t)ntri);
  if (is_device_ptr(tri)) {
    if (cudaMemcpy(t.data(), tri, t.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(h, FSIB_ECUDA, "copy of tri failed");
  } else {
    std::memcpy(t.data(), tri, t.size() * sizeof(int));
  }
  std::vector<std::vector<int>> adj(M);
  for (int q = 0; q < ntri; ++q) {
    for (int e = 0; e < 3; ++e) {
      const int a = t[3 * q + e], b = t[3 * q + (e + 1) % 3];
      if (a < 0 || a >= M || b < 0 || b >= M || a == b) return fail(h, FSIB_EINVAL, "bad triangle index");
      adj[a].push_back(b);
      adj[b].push_back(a);
    }
  }
  std::vector<int> ptr(M + 1, 0), col;
  for (int i = 0; i < M; ++i) {
    auto& v = adj[i];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    ptr[i + 1] = ptr[i] + (int)v.size();
    col.insert(col.end(), v.begin(), v.end());
  }
  Workspace& ws = h->ws;
  free_mesh(ws);
  size_t tot = 0;
  int rc = FSIB_OK;
  ws.nnz = (int)col.size();
  ws.ntri = ntri;
  rc |= dmalloc(&ws.csr_ptr, sizeof(int) * (M + 1), tot);
  rc |= dmalloc(&ws.csr_col, sizeof(int) * std::max<size_t>(1, col.size()), tot);
  rc |= dmalloc(&ws.csr_k, sizeof(double) * std::max<size_t>(1, col.size()), tot);
  rc |= dmalloc(&ws.tri, sizeof(int) * t.size(), tot);
  if (rc != FSIB_OK) { free_mesh(ws); return fail(h, FSIB_ENOMEM, "mesh allocation failed"); }
  cudaMemcpy(ws.csr_ptr, ptr.data(), sizeof(int) * (M + 1), cudaMemcpyHostToDevice);
  cudaMemcpy(ws.csr_col, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(ws.tri, t.data(), sizeof(int) * t.size(), cudaMemcpyHostToDevice);
  if ((rc = begin(h)) != FSIB_OK) return rc;
  Arg xr;
  if ((rc = stage(h, 0, Xref, sizeof(double) * 3 * (size_t)M, true, xr)) != FSIB_OK) return rc;
  launch_mesh_stiffness((const double*)xr.dev, ws.tri, ntri, M, sigma, ws.csr_ptr, ws.csr_col, ws.csr_k,
                        ws.nnz, h->own);
  ws.force_kind = 2;
  ws.stiffness = sigma;
  invalidate_graph(h);
  return finish(h, true);
}

int fsib_set_force_tension(fsib_t h, const int* tri, int ntri, double gamma) {
  if (!h || !tri || ntri < 1) return FSIB_EINVAL;
  if (h->p.d != 3) return fail(h, FSIB_EINVAL, "surface tension needs d = 3");
  if (!std::isfinite(gamma)) return fail(h, FSIB_EINVAL, "gamma must be finite");
  const int M = h->p.M;
  std::vector<int> t(3 * (size_t)ntri);
  if (is_device_ptr(tri)) {
    if (cudaMemcpy(t.data(), tri, t.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(h, FSIB_ECUDA, "copy of tri failed");
  } else {
    std::memcpy(t.data(), tri, t.size() * sizeof(int));
  }
  // incidence (integer work on the host): for node i, the other two vertices of each of its
  // triangles in the triangle's counter-clockwise order starting at i
  std::vector<int> ptr(M + 1, 0);
  for (size_t q = 0; q < t.size(); ++q) {
    const int a = t[q];
    if (a < 0 || a >= M) return fail(h, FSIB_EINVAL, "bad triangle index");
    ptr[a + 1]++;
  }
  for (int q = 0; q < ntri; ++q)
    if (t[3 * q] == t[3 * q + 1] || t[3 * q + 1] == t[3 * q + 2] || t[3 * q] == t[3 * q + 2])
      return fail(h, FSIB_EINVAL, "degenerate triangle");
  for (int i = 0; i < M; ++i) ptr[i + 1] += ptr[i];
  std::vector<int2> inc(3 * (size_t)ntri);
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (int q = 0; q < ntri; ++q)
    for (int r = 0; r < 3; ++r) {
      const int i = t[3 * q + r], j = t[3 * q + (r + 1) % 3], k = t[3 * q + (r + 2) % 3];
      inc[fill[i]++] = make_int2(j, k);
    }
  Workspace& ws = h->ws;
  free_mesh(ws);
  size_t tot = 0;
  int rc = FSIB_OK;
  ws.ntri = ntri;
  rc |= dmalloc(&ws.csr_ptr, sizeof(int) * (M + 1), tot);
  rc |= dmalloc(&ws.inc_jk, sizeof(int2) * inc.size(), tot);
  rc |= dmalloc(&ws.tri, sizeof(int) * t.size(), tot);
  if (rc != FSIB_OK) { free_mesh(ws); return fail(h, FSIB_ENOMEM, "mesh allocation failed"); }
  if (cudaMemcpy(ws.csr_ptr, ptr.data(), sizeof(int) * (M + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ws.inc_jk, inc.data(), sizeof(int2) * inc.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ws.tri, t.data(), sizeof(int) * t.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(h, FSIB_ECUDA, "copy of the incidence failed");
  ws.force_kind = 4;
  ws.stiffness = gamma;
  invalidate_graph(h);
  return FSIB_OK;
}

int fsib_set_force_target(fsib_t h, const double* Xtarget, double K, double omega) {
  if (!h || !Xtarget) return FSIB_EINVAL;
  if (!std::isfinite(K) || !std::isfinite(omega) || !(omega > 0.0))
    return fail(h, FSIB_EINVAL, "K must be finite and omega finite and > 0");
  Workspace& ws = h->ws;
  const size_t bytes = pts_bytes(h);
  if (!ws.target) {
    size_t tot = 0;
    if (dmalloc(&ws.target, bytes, tot) != FSIB_OK) return fail(h, FSIB_ENOMEM, "target allocation failed");
  }
  int rc = begin(h);
  if (rc != FSIB_OK) return rc;
  const cudaMemcpyKind kind = is_device_ptr(Xtarget) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cudaMemcpyAsync(ws.target, Xtarget, bytes, kind, h->own) != cudaSuccess)
    return fail(h, FSIB_ECUDA, "copy of the target points failed");
  ws.force_kind = 3;
  ws.target_wK = omega * K;
  ws.stiffness = K;
  invalidate_graph(h);
  return finish(h, true);
}

int fsib_set_body_force(fsib_t h, const double* f) {
  if (!h || !f) return FSIB_EINVAL;
  if (h->p.stokes) return fail(h, FSIB_EUNSUPPORTED, "a body force needs the Navier-Stokes stepper (rho > 0)");
  for (int a = 0; a < h->p.d; ++a)
    if (!std::isfinite(f[a])) return fail(h, FSIB_EINVAL, "body force must be finite");
  for (int a = 0; a < 3; ++a) h->p.fbody[a] = (a < h->p.d) ? f[a] : 0.0;
  invalidate_graph(h);
  return FSIB_OK;
}

int fsib_band_flux(fsib_t h, const void* uhat, int comp, int axis, double y0, double y1, double* flux) {
  int rc = begin(h);
  if (rc != FSIB_OK) return rc;
  if (!uhat || !flux) return fail(h, FSIB_EINVAL, "NULL array");
  if (comp < 0 || comp >= h->p.d || axis < 0 || axis >= h->p.d)
    return fail(h, FSIB_EINVAL, "comp and axis must lie in [0, d)");
  if (!std::isfinite(y0) || !std::isfinite(y1)) return fail(h, FSIB_EINVAL, "band limits must be finite");
  Arg au;
  if ((rc = stage(h, 3, uhat, spec_bytes(h), true, au)) != FSIB_OK) return rc;
  if (h->p.prec == FSIB_FP64)
    rc = run_band_flux<double>(h->p, h->ws, (const C<double>*)au.dev, comp, axis, y0, y1, flux, h->own);
  else
    rc = run_band_flux<float>(h->p, h->ws, (const C<float>*)au.dev, comp, axis, y0, y1, flux, h->own);
  const int rc2 = finish(h, true);
  if (rc == FSIB_ENONFINITE) return fail(h, rc, "non-finite flux");
  if (rc != FSIB_OK) return fail(h, rc, "flux reduction failed");
  return rc2;
}

int fsib_force(fsib_t h, const double* X, double* c) {
  int rc = begin(h);
  if (rc != FSIB_OK) return rc;
  if (!X || !c) return fail(h, FSIB_EINVAL, "NULL array");
  if (!h->ws.force_kind) return fail(h, FSIB_ESTATE, "no force model set");
  Arg ax, ac;
  if ((rc = stage(h, 0, X, pts_bytes(h), true, ax)) != FSIB_OK) return rc;
  if ((rc = stage(h, 1, c, pts_bytes(h), false, ac)) != FSIB_OK) return rc;
  do_force(h, (const double*)ax.dev, (double*)ac.dev, h->own);
  if ((rc = unstage(h, ac)) != FSIB_OK) return rc;
  return finish(h, ac.host != nullptr);
}

int fsib_spread(fsib_t h, const double* X, const double* F, const double* omega, void* fhat) {
  int rc = begin(h);
  if (rc != FSIB_OK) return rc;
  if (!X || !F || !fhat) return fail(h, FSIB_EINVAL, "NULL array");
  Arg ax, af, ao, ah;
  if ((rc = stage(h, 0, X, pts_bytes(h), true, ax)) != FSIB_OK) return rc;
  if ((rc = stage(h, 1, F, pts_bytes(h), true, af)) != FSIB_OK) return rc;
  if ((rc = stage(h, 2, omega, sizeof(double) * h->p.M, true, ao)) != FSIB_OK) return rc;
  if ((rc = stage(h, 3, fhat, spec_bytes(h), false, ah)) != FSIB_OK) return rc;
  const double *xd = (const double*)ax.dev, *fd = (const double*)af.dev, *od = (const double*)ao.dev;
  FSIB_DISPATCH(h, (do_spread<float, float>(h, xd, fd, od, (C<float>*)ah.dev, h->own)),
                (do_spread<dd, double>(h, xd, fd, od, (C<double>*)ah.dev, h->own)),
                (do_spread<double, double>(h, xd, fd, od, (C<double>*)ah.dev, h->own)));
  if ((rc = unstage(h, ah)) != FSIB_OK) return rc;
  return finish(h, ah.host != nullptr);
}

int fsib_interp(fsib_t h, const void* uhat, const double* X, double* U) {
  int rc = begin(h);
  if (rc != FSIB_OK) return rc;
  if ((rc = take_miss(h)) != FSIB_OK) return rc;
  if (!X || !U || !uhat) return fail(h, FSIB_EINVAL, "NULL array");
  Arg ax, au, ah;
  if ((rc = stage(h, 0, X, pts_bytes(h), true, ax)) != FSIB_OK) return rc;
  if ((rc = stage(h, 3, uhat, spec_bytes(h), true, ah)) != FSIB_OK) return rc;
  if ((rc = stage(h, 1, U, pts_bytes(h), false, au)) != FSIB_OK) return rc;
  do_bin(h, (const double*)ax.dev, h->own);
  FSIB_DISPATCH(h, (do_interp_sorted<float, float>(h, (const C<float>*)ah.dev, (double*)au.dev, h->own, true)),
                (do_interp_sorted<dd, double>(h, (const C<double>*)ah.dev, (double*)au.dev, h->own, true)),
                (do_interp_sorted<double, double>(h, (const C<double>*)ah.dev, (double*)au.dev, h->own, true)));
  if ((rc = unstage(h, au)) != FSIB_OK) return rc;
  return finish(h, au.host != nullptr);
}

int fsib_fluid_step(fsib_t h, const void* fhat, void* uhat, void* uhat_half) {
  int rc = begin(h);
  if (rc != FSIB_OK) return rc;
  if (!fhat || !uhat) return fail(h, FSIB_EINVAL, "NULL array");
  Arg af, au, ah;
  if ((rc = stage(h, 0, fhat, spec_bytes(h), true, af)) != FSIB_OK) return rc;
  if ((rc = stage(h, 1, uhat, spec_bytes(h), !h->p.stokes, au)) != FSIB_OK) return rc;
  if ((rc = stage(h, 2, uhat_half, spec_bytes(h), false, ah)) != FSIB_OK) return rc;
  void* half = ah.dev ? ah.dev : h->ws.uhalf;
  FSIB_DISPATCH(h, (do_fluid<float, float>(h, (const C<float>*)af.dev, (C<float>*)au.dev, (C<float>*)half, h->own)),
                (do_fluid<dd, double>(h, (const C<double>*)af.dev, (C<double>*)au.dev, (C<double>*)half, h->own)),
                (do_fluid<double, double>(h, (const C<double>*)af.dev, (C<double>*)au.dev, (C<double>*)half, h->own)));
  if ((rc = unstage(h, au)) != FSIB_OK) return rc;
  if (!h->p.stokes && (rc = unstage(h, ah)) != FSIB_OK) return rc;
  return finish(h, au.host != nullptr || ah.host != nullptr);
}

int fsib_pressure(fsib_t h, const void* fhat, const void* uhat, void* phat) {
  int rc = begin(h);
  if (rc != FSIB_OK) return rc;
  if (!fhat || !phat) return fail(h, FSIB_EINVAL, "NULL array");
  Arg af, au, ap;
  if ((rc = stage(h, 0, fhat, spec_bytes(h), true, af)) != FSIB_OK) return rc;
  if ((rc = stage(h, 1, uhat, spec_bytes(h), true, au)) != FSIB_OK) return rc;
  if ((rc = stage(h, 2, phat, spec_bytes(h) / h->p.d, false, ap)) != FSIB_OK) return rc;
  FSIB_DISPATCH(h, (do_pressure<float, float>(h, (const C<float>*)af.dev, (const C<float>*)au.dev, (C<float>*)ap.dev, h->own)),
                (do_pressure<dd, double>(h, (const C<double>*)af.dev, (const C<double>*)au.dev, (C<double>*)ap.dev, h->own)),
                (do_pressure<double, double>(h, (const C<double>*)af.dev, (const C<double>*)au.dev, (C<double>*)ap.dev, h->own)));
  if ((rc = unstage(h, ap)) != FSIB_OK) return rc;
  return finish(h, ap.host != nullptr);
}

static int count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
  int k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

int fsib_step(fsib_t h, double* X, void* uhat, double* U, int nsteps) {
  int rc = begin(h);
  if (rc != FSIB_OK) return rc;
  if ((rc = take_miss(h)) != FSIB_OK) return rc;
  if (!X) return fail(h, FSIB_EINVAL, "X is NULL");
  if (nsteps < 0) return fail(h, FSIB_EINVAL, "nsteps < 0");
  if (!h->ws.force_kind) return fail(h, FSIB_ESTATE, "no force model set");
  const bool ns = !h->p.stokes;
  if (ns && (!uhat || !U)) return fail(h, FSIB_EINVAL, "Navier-Stokes step needs uhat and U");
  // A single Navier-Stokes step on a pinned host u-hat copies it inside the step (see do_step),
  // overlapped with work that does not read it; otherwise host arrays are staged around it.
  const bool u_inside = ns && nsteps == 1 && !is_device_ptr(uhat) && is_pinned_host(uhat);
  Arg ax, au, aU;
  if ((rc = stage(h, 0, X, pts_bytes(h), true, ax)) != FSIB_OK) return rc;
  if ((rc = stage(h, 3, uhat, spec_bytes(h), ns && !u_inside, au)) != FSIB_OK) return rc;
  if ((rc = stage(h, 1, U, pts_bytes(h), ns, aU)) != FSIB_OK) return rc;
  const void* u_in = u_inside ? au.host : nullptr;
  void* u_out = u_inside ? au.host : nullptr;
  const bool f64 = h->p.prec == FSIB_FP64;
  auto enqueue = [&](cudaStream_t st) {
    FSIB_DISPATCH(h, (do_step<float, float>(h, (double*)ax.dev, (C<float>*)au.dev, (double*)aU.dev, st, u_in, u_out)),
                  (do_step<dd, double>(h, (double*)ax.dev, (C<double>*)au.dev, (double*)aU.dev, st, u_in, u_out)),
                  (do_step<double, double>(h, (double*)ax.dev, (C<double>*)au.dev, (double*)aU.dev, st, u_in, u_out)));
  };
  if (nsteps > 0) {
    if (h->p.use_graph && !h->prof_on) {
      const void* key[4] = {ax.dev, au.dev, aU.dev, u_in};
      if (!h->gexec || std::memcmp(key, h->gkey, sizeof(key)) != 0) {
        if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(h->own, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
          return fail(h, FSIB_ECUDA, "stream capture failed to start");
        enqueue(h->own);
        cudaError_t e = cudaStreamEndCapture(h->own, &g);
        if (e != cudaSuccess || !g) return fail(h, FSIB_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
        h->graph_kernels = count_kernel_nodes(g);
        e = cudaGraphInstantiate(&h->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { h->gexec = nullptr; return fail(h, FSIB_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e)); }
        std::memcpy(h->gkey, key, sizeof(key));
      }
      for (int s = 0; s < nsteps; ++s)
        if (cudaGraphLaunch(h->gexec, h->own) != cudaSuccess) return fail(h, FSIB_ECUDA, "graph launch failed");
    } else {
      for (int s = 0; s < nsteps; ++s) enqueue(h->own);
    }
  }
  if ((rc = unstage(h, ax)) != FSIB_OK) return rc;
  if (!u_inside && (rc = unstage(h, au)) != FSIB_OK) return rc;
  if ((rc = unstage(h, aU)) != FSIB_OK) return rc;
  const bool host = ax.host || au.host || aU.host;
  rc = finish(h, host || h->p.check_finite);
  if (rc != FSIB_OK) return rc;
  if (host || h->p.check_finite) {
    if ((rc = take_miss(h)) != FSIB_OK) return rc;  // the steps have finished: report at once
  }
  if (h->p.check_finite) {
    double inv[6];
    const int r2 = f64 ? run_invariants<double>(h->p, h->ws, (const double*)ax.dev, nullptr, inv, h->own)
                       : run_invariants<float>(h->p, h->ws, (const double*)ax.dev, nullptr, inv, h->own);
    if (r2 == FSIB_ENONFINITE) return fail(h, FSIB_ENONFINITE, "non-finite positions after the step");
    if (r2 != FSIB_OK) return fail(h, r2, "finite check failed");
  }
  return FSIB_OK;
}

int fsib_invariants(fsib_t h, const double* X, const void* uhat, double out[6]) {
  int rc = begin(h);
  if (rc != FSIB_OK) return rc;
  if ((rc = take_miss(h)) != FSIB_OK) return rc;
  if (!X || !out) return fail(h, FSIB_EINVAL, "NULL array");
  if (h->p.d == 3 && h->ws.force_kind != 3 && !h->ws.tri)
    return fail(h, FSIB_ESTATE, "3D invariants need the mesh (fsib_set_force_mesh)");
  Arg ax, au;
  if ((rc = stage(h, 0, X, pts_bytes(h), true, ax)) != FSIB_OK) return rc;
  if ((rc = stage(h, 3, uhat, spec_bytes(h), true, au)) != FSIB_OK) return rc;
  if (h->p.prec == FSIB_FP64)
    rc = run_invariants<double>(h->p, h->ws, (const double*)ax.dev, (const C<double>*)au.dev, out, h->own);
  else
    rc = run_invariants<float>(h->p, h->ws, (const double*)ax.dev, (const C<float>*)au.dev, out, h->own);
  const int rc2 = finish(h, true);
  if (rc2 == FSIB_OK && rc == FSIB_OK) {
    const int rc3 = take_miss(h);  // a step that finished during this call
    if (rc3 != FSIB_OK) return rc3;
  }
  if (rc == FSIB_ENONFINITE) return fail(h, rc, "non-finite values in X or uhat");
  if (rc != FSIB_OK) return fail(h, rc, "invariant reduction failed");
  return rc2;
}

int fsib_profile_enable(fsib_t h, int on) {
  if (!h) return FSIB_EINVAL;
  prof_flush(h);
  h->prof_on = (on != 0);
  return FSIB_OK;
}

int fsib_profile_reset(fsib_t h) {
  if (!h) return FSIB_EINVAL;
  prof_flush(h);
  h->sites.clear();
  return FSIB_OK;
}

int fsib_profile_count(fsib_t h) {
  if (!h) return FSIB_EINVAL;
  prof_flush(h);
  return (int)h->sites.size();
}

int fsib_profile_entry(fsib_t h, int i, char* name, int name_len, double* total_ms, int* launches,
                       double* bytes_per_launch, double* flops_per_launch) {
  if (!h) return FSIB_EINVAL;
  prof_flush(h);
  if (i < 0 || i >= (int)h->sites.size()) return fail(h, FSIB_EINVAL, "profile index out of range");
  const auto& s = h->sites[i];
  if (name && name_len > 0) {
    std::strncpy(name, s.name.c_str(), (size_t)name_len - 1);
    name[name_len - 1] = 0;
  }
  if (total_ms) *total_ms = s.total_ms;
  if (launches) *launches = s.launches;
  if (bytes_per_launch) *bytes_per_launch = s.bytes;
  if (flops_per_launch) *flops_per_launch = s.flops;
  return FSIB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Type-1 spread that allocates nothing (fsib_spread_static).
//
// Some callers cannot call cudaMalloc: code that runs inside a host framework
// whose caching allocator owns all device memory and forbids raw allocations,
// and latency-critical loops where cudaMalloc's implicit device-wide
// synchronisation is not acceptable. For them the whole scratch of one type-1
// transform (fine grid, FFT intermediates, point sort, twiddle and
// deconvolution tables) lives in the file-scope array below, which every GPU
// that loads the library holds until the process exits. The caller passes only
// its inputs and output. All calls share this array: two calls that overlap on
// the GPU (different streams, or different host threads) race on it.
// ---------------------------------------------------------------------------
#define FSIB_STATIC_SCRATCH_BYTES (64ull << 20)

static __device__ __align__(256) unsigned char g_static_scratch[FSIB_STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch per device. In host code the symbol name is
// only a host-side stand-in, so the address must come from cudaGetSymbolAddress
// with the device current. The address is looked up again on every call made
// outside stream capture: after a device reset the module is loaded anew and the
// array may sit elsewhere (its contents, the cached tables included, are gone).
static std::mutex g_static_mu;
static void* g_static_addr[64] = {nullptr};

// Twiddle and deconvolution tables last uploaded into each device's scratch, by the
// sizes that fix them. A call with the same sizes uploads nothing, so it can run under
// stream capture; the tables sit at the start of the scratch, at offsets fixed by
// (n_f, N, precision) alone.
struct StaticTables {
  void* base = nullptr;
  int N = 0, d = 0, nf = 0, w = 0, prec = -1;
  double beta = 0.0;
};
static StaticTables g_static_tab[64];

static int static_scratch_base(void** out, int* dev_out, bool capturing, std::string& err) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    err = "no current CUDA device";
    return FSIB_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (capturing) {
    if (!g_static_addr[dev]) {
      err = "the first fsib_spread_static call on a device must come before any stream capture";
      return FSIB_EINVAL;
    }
  } else {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      err = std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e);
      return FSIB_ECUDA;
    }
    if (p != g_static_addr[dev]) g_static_tab[dev] = StaticTables();  // a new module: no tables yet
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  *dev_out = dev;
  return FSIB_OK;
}

static thread_local std::string g_static_err;

// Carve 256-byte aligned pieces out of [base, base + cap).
struct Carver {
  unsigned char* base;
  size_t used = 0;
  template <typename P>
  P* take(size_t bytes) {
    used = (used + 255) & ~size_t(255);
    P* q = reinterpret_cast<P*>(base ? base + used : nullptr);
    used += bytes ? bytes : 16;
    return q;
  }
};

template <typename T>
static int spread_static_impl(const Plan& p, const double* X, const double* F, const double* omega,
                              void* fhat, cudaStream_t st) {
  const long long N = p.N, hh = p.N / 2, n = p.nf, d = p.d;
  const size_t rs = sizeof(T), cs = 2 * sizeof(T);
  const long long gcells = d * n * n * (d == 3 ? n : 1);
  const long long s1n = (d == 3) ? d * n * n * hh : d * n * hh;
  const long long s2n = (d == 3) ? d * n * N * hh : 1;
  const long long dpn = (d == 3) ? N * hh : hh;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    g_static_err = "cudaStreamIsCapturing failed on the given stream";
    return FSIB_ECUDA;
  }
  const bool capturing = cap != cudaStreamCaptureStatusNone;

  // Layout pass (base = null) to size the request, then the real carve. The tables come
  // first, so their offsets depend on (n_f, N, precision) only.
  Workspace ws;
  size_t need = 0;
  unsigned char* base = nullptr;
  int dev = 0;
  for (int pass = 0; pass < 2; ++pass) {
    Carver c{base};
    ws.tw = c.take<void>((size_t)n * cs);
    ws.dline = c.take<void>((size_t)N * rs);
    ws.dplane = c.take<void>((size_t)dpn * rs);
    ws.grid = c.take<void>((size_t)gcells * rs);
    ws.grid_bytes = (size_t)gcells * rs;
    ws.s1 = c.take<void>((size_t)s1n * cs);
    ws.s2 = c.take<void>((size_t)s2n * cs);
    ws.bin_of = c.take<int>(sizeof(int) * p.M);
    ws.rank = c.take<int>(sizeof(int) * p.M);
    ws.perm = c.take<int>(sizeof(int) * p.M);
    ws.i0 = c.take<int>(sizeof(int) * d * p.M);
    ws.delta = c.take<void>(rs * d * p.M);
    ws.counts = c.take<int>(sizeof(int) * (size_t)p.nbins);
    ws.offsets = c.take<int>(sizeof(int) * (size_t)(p.nbins + 1));
    ws.occ = c.take<int>(sizeof(int) * (size_t)p.nbins);
    ws.nocc = c.take<int>(sizeof(int));
    need = c.used;
    if (pass == 0) {
      if (need > FSIB_STATIC_SCRATCH_BYTES) {
        g_static_err = "problem needs " + std::to_string(need) + " bytes of scratch; the static scratch holds " +
                       std::to_string((unsigned long long)FSIB_STATIC_SCRATCH_BYTES) + " bytes";
        return FSIB_EINVAL;
      }
      void* b = nullptr;
      const int rc = static_scratch_base(&b, &dev, capturing, g_static_err);
      if (rc != FSIB_OK) return rc;
      base = static_cast<unsigned char*>(b);
    }
  }

  // Twiddles of the fine grid and per-axis deconvolution: uploaded once per device and sizes.
  bool have;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    const StaticTables& t = g_static_tab[dev];
    have = t.base == base && t.N == p.N && t.d == p.d && t.nf == p.nf && t.w == p.w && t.beta == p.beta &&
           t.prec == p.prec;
  }
  cudaError_t e = cudaSuccess;
  if (!have) {
    if (capturing) {
      g_static_err = "the tables for these sizes are not in the static scratch: make one call with the same "
                     "N, d, tol and precision outside stream capture first";
      return FSIB_EINVAL;
    }
    const double pi = 3.14159265358979323846;
    std::vector<T> tw(2 * (size_t)n), D(N), Dp(dpn);
    for (long long j = 0; j < n; ++j) {
      const double ang = 2.0 * pi * (double)j / (double)n;
      tw[2 * j] = (T)std::cos(ang);
      tw[2 * j + 1] = (T)(-std::sin(ang));
    }
    std::vector<double> zq, wq, Dd(N);
    gauss_legendre(std::max(64, 4 * p.w + 64), zq, wq);
    const double hf = p.L / p.nf;
    for (long long i = 0; i < N; ++i) {
      const long long m = (i < N / 2) ? i : i - N;
      Dd[i] = (i == N / 2) ? 0.0 : hf / psi_hat(2.0 * pi * m / p.L, p.w, p.beta, hf, zq, wq);
      D[i] = (T)Dd[i];
    }
    for (long long q = 0; q < dpn; ++q) Dp[q] = (T)((d == 3) ? Dd[q / hh] * Dd[q % hh] : Dd[q]);
    // the host vectors die with this scope: the copies complete before it ends
    e = cudaMemcpyAsync(ws.tw, tw.data(), tw.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ws.dline, D.data(), D.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ws.dplane, Dp.data(), Dp.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      g_static_err = std::string("table upload: ") + cudaGetErrorString(e);
      return FSIB_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticTables& t = g_static_tab[dev];
    t.base = base; t.N = p.N; t.d = p.d; t.nf = p.nf; t.w = p.w; t.beta = p.beta; t.prec = p.prec;
  }
  // The scratch keeps the previous call's contents: zero what must start at zero
  // (the grid accumulates spread contributions; the bin counts start at zero).
  e = cudaMemsetAsync(ws.grid, 0, ws.grid_bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws.counts, 0, sizeof(int) * (size_t)p.nbins, st);  // the binning counts into it
  if (e != cudaSuccess) {
    cudaGetLastError();
    g_static_err = std::string("scratch clear: ") + cudaGetErrorString(e);
    return FSIB_ECUDA;
  }

  launch_bin_points(p, ws, X, st);
  launch_spread<T>(p, ws, F, omega, (T*)ws.grid, st);
  const C<T>* twc = (const C<T>*)ws.tw;
  C<T>* s1 = (C<T>*)ws.s1;
  C<T>* s2 = (C<T>*)ws.s2;
  Mult<T> none, dec;
  dec.scale = (T)std::pow(p.L, -(double)d);
  dec.dline = (const T*)ws.dline;
  dec.dplane = (const T*)ws.dplane;
  if (d == 3) {
    launch_fft_rows_r2c<T>((const T*)ws.grid, s1, d * n * n, p.N, p.fl_nf, twc, st);
    launch_fft_strided<T>(s1, s2, (int)d, (int)n, (int)hh, p.N, p.fl_nf, false, none, twc, st);
    launch_fft_strided<T>(s2, (C<T>*)fhat, (int)d, 1, (int)(N * hh), p.N, p.fl_nf, false, dec, twc, st);
  } else {
    launch_fft_rows_r2c<T>((const T*)ws.grid, s1, d * n, p.N, p.fl_nf, twc, st);
    launch_fft_strided<T>(s1, (C<T>*)fhat, (int)d, 1, (int)hh, p.N, p.fl_nf, false, dec, twc, st);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_static_err = std::string("CUDA: ") + cudaGetErrorString(e);
    return FSIB_ECUDA;
  }
  return FSIB_OK;
}

extern "C" {

int fsib_spread_static(int N, int d, int M, double tol, int precision, const double* X, const double* F,
                       const double* omega, void* fhat, void* stream) {
  g_static_err.clear();
  if ((d != 2 && d != 3) || N < 4 || N > 1024 || (N % 2) || M < 1 || !(tol >= 1e-14 && tol <= 1e-2) ||
      (precision != FSIB_FP64 && precision != FSIB_MIXED)) {
    g_static_err = "bad N, d, M, tol or precision";
    return FSIB_EINVAL;
  }
  if (!X || !F || !fhat) { g_static_err = "NULL array"; return FSIB_EINVAL; }
  if (!is_device_ptr(X) || !is_device_ptr(F) || !is_device_ptr(fhat) || (omega && !is_device_ptr(omega))) {
    g_static_err = "fsib_spread_static takes device arrays only";
    return FSIB_EINVAL;
  }
  Plan p;
  p.d = d; p.N = N; p.M = M; p.tol = tol; p.prec = precision;
  std::string err;
  int rc = plan_sizes(p, err);
  if (rc != FSIB_OK) { g_static_err = err; return rc; }
  cudaStream_t st = (cudaStream_t)stream;
  rc = (precision == FSIB_FP64) ? spread_static_impl<double>(p, X, F, omega, fhat, st)
                                : spread_static_impl<float>(p, X, F, omega, fhat, st);
  return rc;
}

const char* fsib_static_last_error(void) { return g_static_err.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner: picks the launch shapes (strided-tile lines, row pairs per CTA, spread
// slice size) that minimise the measured time of one step, by coordinate descent
// over the candidate values, timing direct launches on copies of the caller's state.
// ---------------------------------------------------------------------------
static int time_steps(fsib_plan* h, double* X, void* u, double* U, const double* X0, const void* u0,
                      const double* U0, int reps, float* ms_out) {
  const Plan& p = h->p;
  const size_t xb = pts_bytes(h), ub = spec_bytes(h);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto one = [&]() {
    FSIB_DISPATCH(h, (do_step<float, float>(h, X, (C<float>*)u, U, h->own)),
                  (do_step<dd, double>(h, X, (C<double>*)u, U, h->own)),
                  (do_step<double, double>(h, X, (C<double>*)u, U, h->own)));
  };
  cudaMemcpyAsync(X, X0, xb, cudaMemcpyDeviceToDevice, h->own);
  if (u0) cudaMemcpyAsync(u, u0, ub, cudaMemcpyDeviceToDevice, h->own);
  if (U0) cudaMemcpyAsync(U, U0, xb, cudaMemcpyDeviceToDevice, h->own);
  one();  // warm-up
  cudaEventRecord(e0, h->own);
  for (int r = 0; r < reps; ++r) one();
  cudaEventRecord(e1, h->own);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  (void)p;
  if (e != cudaSuccess) return FSIB_ECUDA;
  *ms_out = ms / reps;
  return FSIB_OK;
}

extern "C" int fsib_autotune(fsib_t h, const double* X, const void* uhat, const double* U) {
  int rc = begin(h);
  if (rc != FSIB_OK) return rc;
  if (!X) return fail(h, FSIB_EINVAL, "X is NULL");
  if (!h->ws.force_kind) return fail(h, FSIB_ESTATE, "no force model set");
  const bool ns = !h->p.stokes;
  if (ns && (!uhat || !U)) return fail(h, FSIB_EINVAL, "Navier-Stokes autotuning needs uhat and U");
  Arg ax, au, aU;
  if ((rc = stage(h, 0, X, pts_bytes(h), true, ax)) != FSIB_OK) return rc;
  if ((rc = stage(h, 3, uhat, spec_bytes(h), true, au)) != FSIB_OK) return rc;
  if ((rc = stage(h, 1, U, pts_bytes(h), true, aU)) != FSIB_OK) return rc;
  double *tX = nullptr, *tU = nullptr;
  void* tu = nullptr;
  size_t tot = 0;
  rc |= dmalloc(&tX, pts_bytes(h), tot);
  rc |= dmalloc(&tU, pts_bytes(h), tot);
  rc |= dmalloc(&tu, spec_bytes(h), tot);
  if (rc != FSIB_OK) { cudaFree(tX); cudaFree(tU); cudaFree(tu); return fail(h, FSIB_ENOMEM, "autotune allocation"); }
  struct Knob { const char* key; int vals[3]; };
  const Knob knobs[3] = {{"fft_tile", {4, 8, 16}}, {"fft_rows", {2, 4, 8}}, {"spread_slice", {128, 256, 512}}};
  const int nk = (h->p.d == 3) ? 3 : 2;
  for (int k = 0; k < nk && rc == FSIB_OK; ++k) {
    double cur = 0;
    fsib_get_info(h, knobs[k].key, &cur);
    float best = 1e30f;
    int bestv = (int)cur;
    for (int v : knobs[k].vals) {
      if ((rc = fsib_set_option(h, knobs[k].key, v)) != FSIB_OK) break;
      float ms = 0;
      rc = time_steps(h, tX, tu, tU, (const double*)ax.dev, au.dev, (const double*)aU.dev, 3, &ms);
      if (rc != FSIB_OK) break;
      if (ms < best) { best = ms; bestv = v; }
    }
    if (rc == FSIB_OK) rc = fsib_set_option(h, knobs[k].key, bestv);
  }
  cudaStreamSynchronize(h->own);
  cudaFree(tX);
  cudaFree(tU);
  cudaFree(tu);
  if (rc != FSIB_OK) return fail(h, rc, "autotune failed: " + h->err);
  return finish(h, true);
}

// ---------------------------------------------------------------------------
// Batches of independent problems. Every member is a full handle; one captured CUDA
// graph advances all of them, with one branch per member (forked from and joined
// into the batch stream), so the members' kernels run concurrently.
// ---------------------------------------------------------------------------
struct fsib_batch {
  std::vector<fsib_plan*> m;
  cudaStream_t user = nullptr, own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t gexec = nullptr;
  std::vector<const void*> gkey;
  std::vector<unsigned long long> ggen;  // members' step generations the graph was built from
  int graph_kernels = 0;
  int merge = 1;                     // 1: one launch per phase over the members (default); 0: branches
  int group_max = 0;                 // largest merged group (0: no limit); larger classes are split
  int groups = 0;                    // member groups of the merged graph (concurrent branches)
  std::vector<cudaStream_t> gs;      // capture streams of the groups
  std::vector<cudaEvent_t> gjoin;
  std::string err;
};

static int bfail(fsib_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

// Merged batch step (option "merge" = 1). Each member's step is recorded by the launch layer
// (launch.cuh) in program order, its operations labelled by launch site. Members whose site
// sequences agree (same dimension, kind of flow and arithmetic) form a group; the group's schedule
// walks the sites in order and, inside a site, takes the r-th operation of every member at once:
// kernels with the same functor, block and shared memory, and the same grid unless the kernel is
// correct for any grid, become one k_multi launch over those members (blockIdx.y = member, grid
// = the largest asked for, the members' parameters in the launch's parameter space; at most
// kMaxMerge members a launch); other operations run per member. The groups are concurrent
// branches of the captured graph; a group lists its members by decreasing M, so that the largest
// problems' blocks start first.
struct BatchItem {
  bool merged = false;
  std::vector<const RecOp*> ops;  // one per member taking part
  dim3 grid;                      // merged: x = the largest grid asked for, y = members
};

static bool merges_with(const RecOp& a, const RecOp& b) {
  return a.kind == RecOp::kKernel && b.kind == RecOp::kKernel && a.emit && a.id == b.id &&
         a.block.x == b.block.x && a.block.y == b.block.y && a.block.z == b.block.z && a.smem == b.smem &&
         a.grid.y == 1 && a.grid.z == 1 && b.grid.y == 1 && b.grid.z == 1 && (a.any_grid || a.grid.x == b.grid.x);
}

static int batch_capture_merged(fsib_batch* b, double* const* X, void* const* uhat, double* const* U,
                                cudaGraph_t* graph) {
  const size_t n = b->m.size();
  std::vector<Recorder> rec(n);
  for (size_t i = 0; i < n; ++i) {
    fsib_plan* h = b->m[i];
    void* u = uhat ? uhat[i] : nullptr;
    double* Ui = U ? U[i] : nullptr;
    recorder() = &rec[i];
    FSIB_DISPATCH(h, (do_step<float, float>(h, X[i], (C<float>*)u, Ui, b->own)),
                  (do_step<dd, double>(h, X[i], (C<double>*)u, Ui, b->own)),
                  (do_step<double, double>(h, X[i], (C<double>*)u, Ui, b->own)));
    recorder() = nullptr;
  }
  // segments: runs of operations with the same site label
  struct Seg { std::string label; size_t lo, hi; };
  std::vector<std::vector<Seg>> segs(n);
  std::vector<std::string> keys(n);
  for (size_t i = 0; i < n; ++i) {
    const std::vector<RecOp>& ops = rec[i].ops;
    for (size_t k = 0; k < ops.size(); ++k) {
      if (segs[i].empty() || segs[i].back().label != ops[k].site) segs[i].push_back({ops[k].site, k, k});
      segs[i].back().hi = k + 1;
    }
    // one group per grid shape: its members' operations line up one to one (they differ in M
    // only), and the groups, each a chain of merged launches, run concurrently
    const Plan& p = b->m[i]->p;
    keys[i] = std::to_string(p.d) + " " + std::to_string(p.N) + " " + std::to_string(p.nf) + " " +
              std::to_string(p.Nt) + "\n";
    for (const Seg& sg : segs[i]) keys[i] += sg.label + "\n";
  }
  std::vector<std::vector<size_t>> classes;
  std::vector<std::string> ckeys;
  for (size_t i = 0; i < n; ++i) {
    size_t g = 0;
    while (g < ckeys.size() && ckeys[g] != keys[i]) ++g;
    if (g == ckeys.size()) { ckeys.push_back(keys[i]); classes.emplace_back(); }
    classes[g].push_back(i);
  }
  // A class larger than group_max is split into balanced groups (members dealt out by size), so
  // that no single chain of launches holds most of the work.
  std::vector<std::vector<size_t>> groups;
  for (std::vector<size_t>& c : classes) {
    const size_t cap = b->group_max > 0 ? (size_t)b->group_max : c.size();
    const size_t nsub = (c.size() + cap - 1) / cap;
    std::stable_sort(c.begin(), c.end(), [&](size_t x, size_t y) { return b->m[x]->p.M > b->m[y]->p.M; });
    std::vector<std::vector<size_t>> sub(nsub);
    for (size_t j = 0; j < c.size(); ++j) sub[j % nsub].push_back(c[j]);
    for (auto& g : sub) groups.push_back(std::move(g));
  }
  std::vector<std::vector<BatchItem>> sched(groups.size());
  for (size_t g = 0; g < groups.size(); ++g) {
    const std::vector<size_t>& mem = groups[g];
    const size_t nseg = segs[mem[0]].size();
    for (size_t sgi = 0; sgi < nseg; ++sgi) {
      size_t R = 0;
      for (size_t i : mem) R = std::max(R, segs[i][sgi].hi - segs[i][sgi].lo);
      for (size_t r = 0; r < R; ++r) {
        std::vector<BatchItem> items;
        for (size_t i : mem) {
          const Seg& sg = segs[i][sgi];
          if (sg.lo + r >= sg.hi) continue;
          const RecOp* op = &rec[i].ops[sg.lo + r];
          BatchItem* into = nullptr;
          for (BatchItem& it : items)
            if (it.ops.size() < (size_t)kMaxMerge && merges_with(*it.ops[0], *op)) { into = &it; break; }
          if (!into) { items.emplace_back(); into = &items.back(); }
          into->ops.push_back(op);
        }
        for (BatchItem& it : items) {
          const RecOp& op0 = *it.ops[0];
          it.merged = it.ops.size() > 1 && op0.emit != nullptr;
          if (it.merged) {
            unsigned gx = 1;
            for (const RecOp* o : it.ops) gx = std::max(gx, o->grid.x);
            it.grid = dim3(gx, (unsigned)it.ops.size(), 1);
          }
          sched[g].push_back(std::move(it));
        }
      }
    }
  }
  while (b->gs.size() < groups.size()) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      return bfail(b, FSIB_ECUDA, "CUDA stream/event creation failed");
    b->gs.push_back(st);
    b->gjoin.push_back(ev);
  }
  if (cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return bfail(b, FSIB_ECUDA, "stream capture failed to start");
  cudaEventRecord(b->fork, b->own);
  for (size_t g = 0; g < groups.size(); ++g) {
    cudaStream_t st = b->gs[g];
    cudaStreamWaitEvent(st, b->fork, 0);
    for (const BatchItem& it : sched[g]) {
      if (it.merged) {
        const RecOp& o = *it.ops[0];
        const void* packs[kMaxMerge];
        for (size_t j = 0; j < it.ops.size(); ++j) packs[j] = it.ops[j]->pack.data();
        o.emit(it.grid, o.block, o.smem, st, packs);
        continue;
      }
      for (const RecOp* o : it.ops) {
        if (o->kind == RecOp::kKernel) o->emit_one(o->grid, o->block, o->smem, st, o->pack.data());
        else if (o->kind == RecOp::kMemset) cudaMemsetAsync(o->dst, o->value, o->bytes, st);
        else cudaMemcpyAsync(o->dst, o->src, o->bytes, o->ckind, st);
      }
    }
    cudaEventRecord(b->gjoin[g], st);
    cudaStreamWaitEvent(b->own, b->gjoin[g], 0);
  }
  const cudaError_t e = cudaStreamEndCapture(b->own, graph);
  if (e != cudaSuccess || !*graph) return bfail(b, FSIB_ECUDA, std::string("batch capture: ") + cudaGetErrorString(e));
  b->groups = (int)groups.size();
  return FSIB_OK;
}


extern "C" {

int fsib_batch_destroy(fsib_batch* b) {
  if (!b) return FSIB_OK;
  if (b->own) cudaStreamSynchronize(b->own);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (auto st : b->gs) cudaStreamDestroy(st);
  for (auto e : b->gjoin) cudaEventDestroy(e);
  for (auto* h : b->m) fsib_destroy(h);
  for (auto e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->own) cudaStreamDestroy(b->own);
  delete b;
  return FSIB_OK;
}

int fsib_batch_create(fsib_batch** out, int nprob, const int* N, const int* d, const int* M, const double* mu,
                      const double* rho, const double* dt, const double* tol, int precision) {
  g_create_err.clear();
  if (!out || nprob < 1 || !N || !d || !M || !mu || !rho || !dt || !tol ||
      (precision != FSIB_FP64 && precision != FSIB_MIXED)) {
    g_create_err = "bad batch arguments";
    return FSIB_EINVAL;
  }
  *out = nullptr;
  fsib_batch* b = new fsib_batch();
  if (cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    g_create_err = "CUDA stream/event creation failed";
    fsib_batch_destroy(b);
    return FSIB_ECUDA;
  }
  for (int i = 0; i < nprob; ++i) {
    fsib_plan* h = nullptr;
    int rc = fsib_create(&h, N[i], d[i], M[i], mu[i], rho[i], dt[i], tol[i]);
    if (rc == FSIB_OK && precision == FSIB_MIXED) rc = fsib_set_option(h, "precision", 1);
    if (rc != FSIB_OK) {
      g_create_err = "member " + std::to_string(i) + ": " + (h ? h->err : g_create_err);
      if (h) fsib_destroy(h);
      fsib_batch_destroy(b);
      return rc;
    }
    b->m.push_back(h);
    cudaEvent_t e;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    b->join.push_back(e);
  }
  *out = b;
  return FSIB_OK;
}

int fsib_batch_member(fsib_batch* b, int i, fsib_t* h) {
  if (!b || !h || i < 0 || i >= (int)b->m.size()) return FSIB_EINVAL;
  *h = b->m[i];
  return FSIB_OK;
}

int fsib_batch_set_stream(fsib_batch* b, void* stream) {
  if (!b) return FSIB_EINVAL;
  b->user = (cudaStream_t)stream;
  return FSIB_OK;
}

const char* fsib_batch_last_error(fsib_batch* b) { return b ? b->err.c_str() : g_create_err.c_str(); }

int fsib_batch_info(fsib_batch* b, const char* key, double* value) {
  if (!b || !key || !value) return FSIB_EINVAL;
  const std::string k(key);
  if (k == "nprob") *value = (double)b->m.size();
  else if (k == "launches_per_step") *value = b->graph_kernels;
  else if (k == "merge") *value = b->merge;
  else if (k == "group_max") *value = b->group_max;
  else if (k == "groups") *value = b->groups;
  else return bfail(b, FSIB_EINVAL, "unknown info key: " + k);
  return FSIB_OK;
}

int fsib_batch_set_option(fsib_batch* b, const char* key, double value) {
  if (!b || !key) return FSIB_EINVAL;
  const std::string k(key);
  if (k == "merge") {
    if (value != 0 && value != 1) return bfail(b, FSIB_EINVAL, "merge must be 0 or 1");
    b->merge = (int)value;
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    return FSIB_OK;
  }
  if (k == "group_max") {
    if (!(value >= 0 && value <= 65535) || value != (double)(int)value)
      return bfail(b, FSIB_EINVAL, "group_max must be an integer in [0, 65535]");
    b->group_max = (int)value;
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    return FSIB_OK;
  }
  return bfail(b, FSIB_EINVAL, "unknown batch option key: " + k);
}

int fsib_batch_autotune(fsib_batch* b, double* const* X, void* const* uhat, double* const* U) {
  if (!b || !X) return FSIB_EINVAL;
  for (size_t i = 0; i < b->m.size(); ++i) {
    const int rc = fsib_autotune(b->m[i], X[i], uhat ? uhat[i] : nullptr, U ? U[i] : nullptr);
    if (rc != FSIB_OK) return bfail(b, rc, "member " + std::to_string(i) + ": " + b->m[i]->err);
  }
  if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
  return FSIB_OK;
}

int fsib_batch_step(fsib_batch* b, double* const* X, void* const* uhat, double* const* U, int nsteps) {
  if (!b || !X || nsteps < 0) return FSIB_EINVAL;
  b->err.clear();
  const size_t n = b->m.size();
  std::vector<const void*> key;
  for (size_t i = 0; i < n; ++i) {
    fsib_plan* h = b->m[i];
    const bool ns = !h->p.stokes;
    void* u = uhat ? uhat[i] : nullptr;
    double* Ui = U ? U[i] : nullptr;
    if (!X[i] || !is_device_ptr(X[i]) || (u && !is_device_ptr(u)) || (Ui && !is_device_ptr(Ui)))
      return bfail(b, FSIB_EINVAL, "fsib_batch_step takes device arrays (member " + std::to_string(i) + ")");
    if (ns && (!u || !Ui)) return bfail(b, FSIB_EINVAL, "Navier-Stokes member needs uhat and U");
    if (!h->ws.force_kind) return bfail(b, FSIB_ESTATE, "member " + std::to_string(i) + " has no force model");
    key.push_back(X[i]); key.push_back(u); key.push_back(Ui);
  }
  std::vector<unsigned long long> gen;
  for (size_t i = 0; i < n; ++i) gen.push_back(b->m[i]->gen);
  if (cudaEventRecord(b->ev_in, b->user) != cudaSuccess || cudaStreamWaitEvent(b->own, b->ev_in, 0) != cudaSuccess)
    return bfail(b, FSIB_ECUDA, "stream ordering failed");
  if (!b->gexec || key != b->gkey || gen != b->ggen) {
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    cudaGraph_t g = nullptr;
    if (b->merge) {
      const int rc = batch_capture_merged(b, X, uhat, U, &g);
      if (rc != FSIB_OK) return rc;
    } else {
      if (cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bfail(b, FSIB_ECUDA, "stream capture failed to start");
      cudaEventRecord(b->fork, b->own);
      for (size_t i = 0; i < n; ++i) {
        fsib_plan* h = b->m[i];
        cudaStreamWaitEvent(h->own, b->fork, 0);
        void* u = uhat ? uhat[i] : nullptr;
        double* Ui = U ? U[i] : nullptr;
        FSIB_DISPATCH(h, (do_step<float, float>(h, X[i], (C<float>*)u, Ui, h->own)),
                      (do_step<dd, double>(h, X[i], (C<double>*)u, Ui, h->own)),
                      (do_step<double, double>(h, X[i], (C<double>*)u, Ui, h->own)));
        cudaEventRecord(b->join[i], h->own);
        cudaStreamWaitEvent(b->own, b->join[i], 0);
      }
      cudaError_t e = cudaStreamEndCapture(b->own, &g);
      if (e != cudaSuccess || !g) return bfail(b, FSIB_ECUDA, std::string("batch capture: ") + cudaGetErrorString(e));
      b->groups = (int)n;
    }
    cudaError_t e = cudaSuccess;
    b->graph_kernels = count_kernel_nodes(g);
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->gexec = nullptr; return bfail(b, FSIB_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e)); }
    b->gkey = key;
    b->ggen = gen;
  }
  for (int s = 0; s < nsteps; ++s)
    if (cudaGraphLaunch(b->gexec, b->own) != cudaSuccess) return bfail(b, FSIB_ECUDA, "graph launch failed");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(b, FSIB_ECUDA, std::string("CUDA: ") + cudaGetErrorString(e));
  if (cudaEventRecord(b->ev_out, b->own) != cudaSuccess || cudaStreamWaitEvent(b->user, b->ev_out, 0) != cudaSuccess)
    return bfail(b, FSIB_ECUDA, "stream ordering failed");
  return FSIB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Reverse mode of the quasi-static Stokes stepper (see include/fsib.h):
//   velocity VJP:  J^T lam = (grad u)^T lam + (grad w)^T c + c(w),  d/dsigma: sum w.c / sigma,
//   where u is the flow of the forces c(X) and w the flow of lam used as forces;
//   step VJP for X1 = X + dt U(X + dt/2 U(X)):  a = dt J(X_half)^T lam1,
//   lam0 = lam1 + a + dt/2 J(X)^T a.
// The forward states are recomputed from checkpoints, one segment at a time.
// ---------------------------------------------------------------------------
static int ensure_adjoint(fsib_plan* h, int K, int ckpt) {
  Workspace& ws = h->ws;
  const Plan& p = h->p;
  const size_t dm = (size_t)p.d * p.M;
  size_t tot = 0;
  int rc = FSIB_OK;
  if (!ws.adj_spec) rc |= dmalloc(&ws.adj_spec, 3 * ws.spec_bytes, tot);
  if (!ws.adj_pts) rc |= dmalloc(&ws.adj_pts, sizeof(double) * (2 * (size_t)p.d * dm + 10 * dm), tot);
  if (!ws.adj_part) rc |= dmalloc(&ws.adj_part, sizeof(double) * 2 * 152 * 4, tot);
  if (!ws.adj_sig) rc |= dmalloc(&ws.adj_sig, sizeof(double) * 2, tot);
  const int nck = (K + ckpt - 1) / ckpt;
  const size_t need = sizeof(double) * dm * (size_t)(nck + ckpt + 1);
  if (ws.adj_ckpt_bytes < need) {
    if (ws.adj_ckpt) cudaFree(ws.adj_ckpt);
    ws.adj_ckpt = nullptr;
    ws.adj_ckpt_bytes = 0;
    rc |= dmalloc(&ws.adj_ckpt, need, tot);
    if (rc == FSIB_OK) ws.adj_ckpt_bytes = need;
  }
  return rc == FSIB_OK ? FSIB_OK : FSIB_ENOMEM;
}

struct AdjBufs {
  double *Gu, *Gw, *w, *fw, *c, *a, *Uxm, *Xh;
};
static AdjBufs adj_bufs(fsib_plan* h) {
  const size_t dm = (size_t)h->p.d * h->p.M;
  double* b = h->ws.adj_pts;
  AdjBufs r;
  r.Gu = b; b += (size_t)h->p.d * dm;
  r.Gw = b; b += (size_t)h->p.d * dm;
  r.w = b; b += dm;
  r.fw = b; b += dm;
  r.c = b; b += dm;
  r.a = b; b += dm;
  r.Uxm = b; b += dm;
  r.Xh = b;
  return r;
}

// G[b][a][j] = d u_a / d x_b at the points of the last binning.
template <typename TI, typename TA>
static void do_interp_grad(fsib_plan* h, const C<TA>* u, double* G, cudaStream_t st) {
  const Plan& p = h->p;
  C<TA>* tmp = (C<TA>*)((char*)h->ws.adj_spec + 2 * h->ws.spec_bytes);
  for (int b = 0; b < p.d; ++b) {
    { Prof pr(h, "mul_ik", 2.0 * (double)h->ws.spec_bytes, 0.0, st);
      launch_mul_ik<TA>(p, b, u, tmp, st); }
    do_interp_sorted<TI, TA>(h, tmp, G + (size_t)b * p.d * p.M, st);
  }
}

// gX += s J(X)^T lam; sigma accumulator += s lam . dU/dsigma
template <typename TI, typename TA>
static void do_vjp(fsib_plan* h, const double* X, const double* lam, double s, double* gX, cudaStream_t st) {
  const Plan& p = h->p;
  Workspace& ws = h->ws;
  AdjBufs B = adj_bufs(h);
  C<TA>* uA = (C<TA>*)ws.adj_spec;
  C<TA>* wB = (C<TA>*)((char*)ws.adj_spec + ws.spec_bytes);
  C<TA>* fhat = (C<TA>*)ws.fhat;
  do_force(h, X, B.c, st);
  do_spread<TI, TA>(h, X, B.c, nullptr, fhat, st);
  do_stokeslet<TA>(h, fhat, uA, st);
  do_interp_grad<TI, TA>(h, uA, B.Gu, st);
  do_spread<TI, TA>(h, X, lam, nullptr, fhat, st);
  do_stokeslet<TA>(h, fhat, wB, st);
  do_interp_sorted<TI, TA>(h, wB, B.w, st);
  do_interp_grad<TI, TA>(h, wB, B.Gw, st);
  do_force(h, B.w, B.fw, st);
  Prof pr(h, "vjp_combine", 8.0 * p.M * (2.0 * p.d * p.d + 6.0 * p.d), 0.0, st);
  launch_vjp_combine(p.d, p.M, s, ws.stiffness, B.Gu, B.Gw, lam, B.c, B.fw, B.w, gX, ws.adj_part, 2 * 152, ws.adj_sig, st);
}

// lam <- reverse of one midpoint Stokes step taken from X
template <typename TI, typename TA>
static void do_step_vjp(fsib_plan* h, const double* X, double* lam, cudaStream_t st) {
  const Plan& p = h->p;
  AdjBufs B = adj_bufs(h);
  const long long dm = (long long)p.d * p.M;
  C<TA>* uA = (C<TA>*)h->ws.adj_spec;
  // recompute X_half = X + dt/2 U(X)
  do_force(h, X, B.c, st);
  do_spread<TI, TA>(h, X, B.c, nullptr, (C<TA>*)h->ws.fhat, st);
  do_stokeslet<TA>(h, (C<TA>*)h->ws.fhat, uA, st);
  do_interp_sorted<TI, TA>(h, uA, B.Uxm, st);
  do_axpy(h, B.Xh, X, B.Uxm, 0.5 * p.dt, st);
  cudaMemsetAsync(B.a, 0, sizeof(double) * dm, st);
  do_vjp<TI, TA>(h, B.Xh, lam, p.dt, B.a, st);          // a = dt J(X_half)^T lam
  do_axpy(h, lam, lam, B.a, 1.0, st);                   // lam += a
  do_vjp<TI, TA>(h, X, B.a, 0.5 * p.dt, lam, st);       // lam += dt/2 J(X)^T a
}

template <typename TI, typename TA>
static void do_adjoint(fsib_plan* h, const double* X0, int K, int ckpt, const double* dLdXK, double* dLdX0,
                       double* dLdsig, cudaStream_t st) {
  const Plan& p = h->p;
  const size_t dm = (size_t)p.d * p.M;
  const int nck = (K + ckpt - 1) / ckpt;
  double* ck = h->ws.adj_ckpt;                   // nck checkpoints
  double* seg = ck + (size_t)nck * dm;           // ckpt segment states
  double* Xw = seg + (size_t)ckpt * dm;          // working state (reuses the last segment slot region)
  (void)Xw;
  // forward sweep, keeping X at steps 0, ckpt, 2 ckpt, ...
  cudaMemcpyAsync(seg, X0, sizeof(double) * dm, cudaMemcpyDeviceToDevice, st);
  for (int m = 0; m < K; ++m) {
    if (m % ckpt == 0) cudaMemcpyAsync(ck + (size_t)(m / ckpt) * dm, seg, sizeof(double) * dm, cudaMemcpyDeviceToDevice, st);
    do_step<TI, TA>(h, seg, nullptr, nullptr, st);
  }
  // reverse sweep
  cudaMemcpyAsync(dLdX0, dLdXK, sizeof(double) * dm, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(h->ws.adj_sig, 0, sizeof(double), st);
  for (int s = nck - 1; s >= 0; --s) {
    const int start = s * ckpt, len = std::min(ckpt, K - start);
    cudaMemcpyAsync(seg, ck + (size_t)s * dm, sizeof(double) * dm, cudaMemcpyDeviceToDevice, st);
    for (int i = 1; i < len; ++i) {
      cudaMemcpyAsync(seg + (size_t)i * dm, seg + (size_t)(i - 1) * dm, sizeof(double) * dm, cudaMemcpyDeviceToDevice, st);
      do_step<TI, TA>(h, seg + (size_t)i * dm, nullptr, nullptr, st);
    }
    for (int i = len - 1; i >= 0; --i) do_step_vjp<TI, TA>(h, seg + (size_t)i * dm, dLdX0, st);
  }
  cudaMemcpyAsync(dLdsig, h->ws.adj_sig, sizeof(double), cudaMemcpyDeviceToDevice, st);
}

extern "C" {

int fsib_interp_grad(fsib_t h, const void* uhat, const double* X, double* G) {
  int rc = begin(h);
  if (rc != FSIB_OK) return rc;
  if (!uhat || !X || !G) return fail(h, FSIB_EINVAL, "NULL array");
  if ((rc = ensure_adjoint(h, 1, 1)) != FSIB_OK) return fail(h, rc, "adjoint workspace allocation failed");
  Arg ax, au, ag;
  if ((rc = stage(h, 0, X, pts_bytes(h), true, ax)) != FSIB_OK) return rc;
  if ((rc = stage(h, 3, uhat, spec_bytes(h), true, au)) != FSIB_OK) return rc;
  if ((rc = stage(h, 1, G, pts_bytes(h) * h->p.d, false, ag)) != FSIB_OK) return rc;
  do_bin(h, (const double*)ax.dev, h->own);
  FSIB_DISPATCH(h, (do_interp_grad<float, float>(h, (const C<float>*)au.dev, (double*)ag.dev, h->own)),
                (do_interp_grad<dd, double>(h, (const C<double>*)au.dev, (double*)ag.dev, h->own)),
                (do_interp_grad<double, double>(h, (const C<double>*)au.dev, (double*)ag.dev, h->own)));
  if ((rc = unstage(h, ag)) != FSIB_OK) return rc;
  return finish(h, ag.host != nullptr);
}

int fsib_step_adjoint(fsib_t h, const double* X0, int K, int ckpt_every, const double* dLdXK, double* dLdX0,
                      double* dLdsigma) {
  int rc = begin(h);
  if (rc != FSIB_OK) return rc;
  if (!X0 || !dLdXK || !dLdX0 || !dLdsigma) return fail(h, FSIB_EINVAL, "NULL array");
  if (!h->p.stokes) return fail(h, FSIB_EUNSUPPORTED, "the adjoint covers the quasi-static Stokes stepper");
  if (!h->ws.force_kind) return fail(h, FSIB_ESTATE, "no force model set");
  if (h->ws.force_kind >= 3) return fail(h, FSIB_EUNSUPPORTED, "the adjoint covers the curve and mesh force laws");
  if (K < 1 || ckpt_every < 1) return fail(h, FSIB_EINVAL, "K and ckpt_every must be >= 1");
  if (ckpt_every > K) ckpt_every = K;
  if ((rc = ensure_adjoint(h, K, ckpt_every)) != FSIB_OK) return fail(h, rc, "adjoint workspace allocation failed");
  Arg ax, al, ag, as;
  if ((rc = stage(h, 0, X0, pts_bytes(h), true, ax)) != FSIB_OK) return rc;
  if ((rc = stage(h, 1, dLdXK, pts_bytes(h), true, al)) != FSIB_OK) return rc;
  if ((rc = stage(h, 2, dLdX0, pts_bytes(h), false, ag)) != FSIB_OK) return rc;
  if ((rc = stage(h, 3, dLdsigma, sizeof(double), false, as)) != FSIB_OK) return rc;
  FSIB_DISPATCH(h,
    (do_adjoint<float, float>(h, (const double*)ax.dev, K, ckpt_every, (const double*)al.dev, (double*)ag.dev, (double*)as.dev, h->own)),
    (do_adjoint<dd, double>(h, (const double*)ax.dev, K, ckpt_every, (const double*)al.dev, (double*)ag.dev, (double*)as.dev, h->own)),
    (do_adjoint<double, double>(h, (const double*)ax.dev, K, ckpt_every, (const double*)al.dev, (double*)ag.dev, (double*)as.dev, h->own)));
  if ((rc = unstage(h, ag)) != FSIB_OK) return rc;
  if ((rc = unstage(h, as)) != FSIB_OK) return rc;
  return finish(h, ag.host != nullptr || as.host != nullptr);
}

}  // extern "C"
