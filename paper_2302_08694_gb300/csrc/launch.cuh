// Kernel launch layer.
//
// Every kernel of the library is a functor type K:
//   static constexpr int  kThreads, kMinBlocks;  // launch bounds (kMinBlocks 0: none)
//   static constexpr bool kAnyGrid;              // correct for any number of blocks (grid-stride
//                                                // loops or dynamic work claiming), so that one
//                                                // launch may serve problems that asked for
//                                                // different grids
//   __device__ static void run(P... params);     // the kernel body (one non-template overload)
// launch<K>(grid, block, smem, stream, args...) runs the body as k_single<K, P...>, one problem
// per launch. While a Recorder is installed on the calling host thread, launch<K>, memset_async
// and memcpy_async record the operation instead of enqueueing it; a batch uses the recordings of
// its members to run each phase of their steps as one k_multi<K, P...> launch, whose blockIdx.y
// selects the problem and whose parameter space holds every problem's parameters.
#pragma once
#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>
#include <utility>
#include <vector>

namespace fsib {

// The parameters of one launch in order: a tuple that device code unpacks into K::run.
template <class... A> struct Pack;
template <> struct Pack<> {
  template <class K, class... B> __device__ __forceinline__ void call(B... b) const { K::run(b...); }
  template <class F, class... B> void apply(F&& f, B... b) const { f(b...); }
};
template <class H, class... T> struct Pack<H, T...> {
  H h;
  Pack<T...> t;
  template <class K, class... B> __device__ __forceinline__ void call(B... b) const { t.template call<K>(b..., h); }
  template <class F, class... B> void apply(F&& f, B... b) const { t.apply(f, b..., h); }
};
template <class... A> struct PackMaker;
template <> struct PackMaker<> {
  static Pack<> make() { return Pack<>{}; }
};
template <class H, class... T> struct PackMaker<H, T...> {
  static Pack<H, T...> make(H h, T... t) {
    Pack<H, T...> p;
    p.h = h;
    p.t = PackMaker<T...>::make(t...);
    return p;
  }
};

// Programmatic dependent launch: every launch-layer kernel is launched with programmatic stream
// serialisation and waits, before its body runs, for the previous kernel of its stream to
// complete with its memory operations visible (griddepcontrol.wait). No kernel triggers early, so
// the next kernel's blocks become eligible as this kernel's blocks exit: its launch overlaps this
// kernel's last wave instead of following the whole grid, while every body still sees the memory
// effects of plain stream order. Triggering at block entry (launch_dependents) was slower: the
// waiting blocks then held SM slots that the running kernel's later waves needed.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <class K, class... P>
__global__ void __launch_bounds__(K::kThreads, K::kMinBlocks) k_single(P... p) {
  pdl_enter();
  K::run(p...);
}
// The parameters of up to kMaxMerge problems travel by value in the kernel's parameter space (the
// constant bank), indexed by blockIdx.y, so a merged kernel reads them as a single launch does.
constexpr int kMaxMerge = 16;
template <class PK> struct PackTable { PK p[kMaxMerge]; };
template <class K, class... P>
__global__ void __launch_bounds__(K::kThreads, K::kMinBlocks) k_multi(const PackTable<Pack<P...>> t) {
  pdl_enter();
  t.p[blockIdx.y].template call<K>();
}

// Launch with programmatic stream serialisation (see pdl_enter).
template <class... P, class... A>
inline void pdl_launch(void (*kern)(P...), dim3 g, dim3 b, size_t smem, cudaStream_t st, A&&... a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, std::forward<A>(a)...);
}

void raise_smem_limit(const void* kernel);

// A functor may declare kMerge = false: a batch then launches it once per problem instead of
// merging it (the kernel is not compiled a second time as k_multi).
template <class K, class = void> struct MergeOf { static constexpr bool value = true; };
template <class K> struct MergeOf<K, std::void_t<decltype(K::kMerge)>> { static constexpr bool value = K::kMerge; };

// One recorded stream operation.
struct RecOp {
  enum Kind { kKernel, kMemset, kMemcpy };
  Kind kind = kKernel;
  const char* site = "";   // launch site (profiling name) the operation belongs to
  // kernels
  const void* id = nullptr;  // kernel identity: operations with equal id, block and smem can merge
  // merged launch over grid.y <= kMaxMerge problems, packs[i] the pack of problem i on the host
  // (nullptr: the kernel does not merge)
  void (*emit)(dim3 grid, dim3 block, size_t smem, cudaStream_t st, const void* const* packs) = nullptr;
  // launch for one problem from the pack on the host
  void (*emit_one)(dim3 grid, dim3 block, size_t smem, cudaStream_t st, const void* pack) = nullptr;
  dim3 grid, block;
  size_t smem = 0;
  bool any_grid = false;
  std::vector<unsigned char> pack;  // the Pack<P...> of this launch
  size_t pack_align = 1;
  // memset / memcpy
  void* dst = nullptr;
  const void* src = nullptr;
  size_t bytes = 0;
  int value = 0;
  cudaMemcpyKind ckind = cudaMemcpyDeviceToDevice;
};

struct Recorder {
  std::vector<RecOp> ops;
  const char* site = "";
};

// The recorder of the calling host thread (nullptr: operations are enqueued).
Recorder*& recorder();

template <class K, class F> struct Launcher;
template <class K, class... P> struct Launcher<K, void (*)(P...)> {
  using PK = Pack<std::decay_t<P>...>;
  static const void* single() { return reinterpret_cast<const void*>(&k_single<K, std::decay_t<P>...>); }
  static const void* multi() { return reinterpret_cast<const void*>(&k_multi<K, std::decay_t<P>...>); }
  static void emit(dim3 g, dim3 b, size_t smem, cudaStream_t st, const void* const* packs) {
    if (smem > 48 * 1024) raise_smem_limit(multi());
    PackTable<PK> t;
    for (unsigned i = 0; i < g.y && i < (unsigned)kMaxMerge; ++i) std::memcpy(&t.p[i], packs[i], sizeof(PK));
    pdl_launch(&k_multi<K, std::decay_t<P>...>, g, b, smem, st, t);
  }
  static void emit_one(dim3 g, dim3 b, size_t smem, cudaStream_t st, const void* pack) {
    reinterpret_cast<const PK*>(pack)->apply(
        [&](auto... a) { pdl_launch(&k_single<K, std::decay_t<P>...>, g, b, smem, st, a...); });
  }
  template <class... A>
  static void go(dim3 g, dim3 b, size_t smem, cudaStream_t st, A&&... a) {
    static_assert(sizeof...(A) == sizeof...(P), "launch<K>: wrong number of kernel arguments");
    if (Recorder* r = recorder()) {
      const PK pk = PackMaker<std::decay_t<P>...>::make(std::decay_t<P>(std::forward<A>(a))...);
      RecOp op;
      op.kind = RecOp::kKernel;
      op.site = r->site;
      if constexpr (MergeOf<K>::value) {
        op.id = multi();
        op.emit = &emit;
      } else {
        op.id = single();
      }
      op.emit_one = &emit_one;
      op.grid = g;
      op.block = b;
      op.smem = smem;
      op.any_grid = K::kAnyGrid;
      op.pack.resize(sizeof(PK));
      std::memcpy(op.pack.data(), &pk, sizeof(PK));
      op.pack_align = alignof(PK);
      r->ops.push_back(std::move(op));
      return;
    }
    pdl_launch(&k_single<K, std::decay_t<P>...>, g, b, smem, st, std::decay_t<P>(std::forward<A>(a))...);
  }
};

template <class K, class... A>
inline void launch(dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... a) {
  Launcher<K, decltype(&K::run)>::go(grid, block, smem, st, std::forward<A>(a)...);
}
// A value that carries a type (to pick a kernel functor at run time inside a generic lambda).
template <class K> struct type_tag { using type = K; };

// The kernel that launch<K> runs for one problem (occupancy queries, function attributes).
template <class K>
inline const void* kernel_ptr() {
  return Launcher<K, decltype(&K::run)>::single();
}

inline cudaError_t memset_async(void* p, int v, size_t n, cudaStream_t st) {
  if (Recorder* r = recorder()) {
    RecOp op;
    op.kind = RecOp::kMemset;
    op.site = r->site;
    op.dst = p;
    op.value = v;
    op.bytes = n;
    r->ops.push_back(std::move(op));
    return cudaSuccess;
  }
  return cudaMemsetAsync(p, v, n, st);
}

inline cudaError_t memcpy_async(void* dst, const void* src, size_t n, cudaMemcpyKind kind, cudaStream_t st) {
  if (Recorder* r = recorder()) {
    RecOp op;
    op.kind = RecOp::kMemcpy;
    op.site = r->site;
    op.dst = dst;
    op.src = src;
    op.bytes = n;
    op.ckind = kind;
    r->ops.push_back(std::move(op));
    return cudaSuccess;
  }
  return cudaMemcpyAsync(dst, src, n, kind, st);
}

}  // namespace fsib
